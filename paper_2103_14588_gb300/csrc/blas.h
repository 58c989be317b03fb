// Internal launchers of the GMRES vector kernels (blas.cu).
#pragma once

#include "internal.h"

#define DST_MAX_VEC 64            // basis vectors one projection / update handles
#define DST_MAX_RED_BLOCKS 608    // CTAs of a reduction pass (4 per SM)
#define DST_MAX_DEVICES 64        // device ordinals the static-scratch entry point tracks

int dst_reduction_blocks(int64_t n);
int dst_projection_blocks(int64_t n);
int dst_k_project(int64_t n, int nvec, const double2 *V, const double2 *w, double2 *h, double2 *partials,
                  int nblk, cudaStream_t s, double *wnrm2 = nullptr, double *wnrm_partials = nullptr,
                  const double *gate = nullptr);
int dst_k_update(int64_t n, int nvec, const double2 *V, const double2 *h, double2 *w, double *nrm2,
                 double *partials, int nblk, cudaStream_t s, const double *gate = nullptr, double *counter = nullptr);
int dst_k_nrm2(int64_t n, const double2 *x, double *nrm2, double *partials, int nblk, cudaStream_t s);
int dst_k_residual(int64_t n, const double2 *b, const double2 *y, double2 *r, double *nrm2, double *partials,
                   int nblk, cudaStream_t s);
int dst_k_scale(int64_t n, const double2 *src, double2 *dst, const double *nrm2, double scale, cudaStream_t s);
int dst_k_cast_64_32(int64_t n, const double2 *src, float2 *dst, cudaStream_t s);
int dst_k_cast_32_64(int64_t n, const float2 *src, double2 *dst, cudaStream_t s);
int dst_k_axpy1(int64_t n, const double2 *d, double2 *x, cudaStream_t s);
int dst_k_sub_f32(int64_t n, const float2 *v, const float2 *a, float2 *r, cudaStream_t s);   // r = v - a
int dst_k_add_f32(int64_t n, const float2 *a, float2 *z, cudaStream_t s);                     // z += a
int dst_k_reduce_partials(int nblk, int nvec, const double2 *partials, double2 *out, cudaStream_t s,
                          const double *gate = nullptr);
int dst_k_reduce_real(int nblk, const double *partials, double *out, cudaStream_t s, const double *gate = nullptr,
                      double *counter = nullptr);

// double-FP32 (df32) Arnoldi kernels (blas_df.cu); a df32 vector of n complex
// entries is float2 hi[n] followed by float2 lo[n].  The projection and the
// update reduce across CTAs inside the kernel (last CTA to take a ticket);
// ticket points to a zero-initialised counter that the kernel leaves at zero.
// vlo = false: every vector (basis and w) is the hi plane alone, n float2,
// and w_hi_only must be true.
int dst_k_project_df(int64_t n, int nvec, const float2 *V, const float2 *w, bool w_hi_only, double2 *h,
                     double2 *partials, int nblk, cudaStream_t s, double *wnrm2, double *wnrm_partials,
                     const double *gate, unsigned *ticket, bool vlo = true);
int dst_k_update_df(int64_t n, int nvec, const float2 *V, const double2 *h, float2 *w, bool w_hi_only, double *nrm2,
                    double *partials, int nblk, cudaStream_t s, const double *gate, double *counter,
                    unsigned *ticket, bool vlo = true);
int dst_k_scale_df(int64_t n, float2 *v, const double *nrm2, cudaStream_t s, bool vlo = true);
// projection on the FP32-stored basis fed by bulk asynchronous copies (two
// CTAs per SM, 96 KB shared memory each); partials holds nblk x (nvec + 1) double2; a
// failed (timed-out) copy wait sets *err = 1.
int dst_tma_projection_blocks(int64_t n);
int dst_k_project_tma(int64_t n, int nvec, const float2 *V, const float2 *w, double2 *h, double2 *partials, int nblk,
                      cudaStream_t s, double *wnrm2, const double *gate, unsigned *ticket, double *err);
// the update w -= V h (FP32-stored basis) with the basis fed by the same bulk
// copies; partials: nblk doubles; gate / counter as in dst_k_update_df.
int dst_k_update_tma(int64_t n, int nvec, const float2 *V, const double2 *h, float2 *w, double *nrm2,
                     double *partials, int nblk, cudaStream_t s, const double *gate, double *counter,
                     unsigned *ticket, double *err);
// x += V y (FP32-stored basis, k vectors) with the basis fed by the same bulk copies;
// the per-entry arithmetic of dst_k_combine_df.  A failed wait sets *err = 1.
int dst_k_combine_tma(int64_t n, int k, const float2 *V, const double2 *y, double2 *x, int nblk, cudaStream_t s,
                      double *err);
int dst_k_split_f64_df(int64_t n, const double2 *src, const double *nrm2, float2 *dst, cudaStream_t s,
                       bool vlo = true);
int dst_k_combine_df(int64_t n, int k, const float2 *V, const double2 *y, double2 *x, cudaStream_t s,
                     bool vlo = true);

// BiCGSTAB steps (blas.cu); sc = double2[8] device scalars (see blas.cu)
int dst_k_bicg_scalar(int mode, double2 *sc, cudaStream_t s);
int dst_k_bicg_p(int64_t n, const double2 *r, const double2 *v, double2 *p, const double2 *sc, cudaStream_t s);
int dst_k_bicg_s(int64_t n, const double2 *r, const double2 *v, double2 *sv, const double2 *sc, cudaStream_t s);
int dst_k_bicg_xr(int64_t n, double2 *x, const double2 *p, const double2 *sv, const double2 *t, double2 *r,
                  const double2 *sc, double *nrm2, double *partials, int nblk, cudaStream_t s);
