// Internal launchers of the GMRES vector kernels (blas.cu).
#pragma once

#include "internal.h"

#define DST_MAX_VEC 64            // basis vectors one projection / update handles
#define DST_MAX_RED_BLOCKS 1216   // CTAs of a reduction pass (8 per SM)
#define DST_MAX_DEVICES 64        // device ordinals the static-scratch entry point tracks

int dst_reduction_blocks(int64_t n);
int dst_k_project(int64_t n, int nvec, const double2 *V, const double2 *w, double2 *h, double2 *partials,
                  int nblk, cudaStream_t s);
int dst_k_update(int64_t n, int nvec, const double2 *V, const double2 *h, double2 *w, double *nrm2,
                 double *partials, int nblk, cudaStream_t s);
int dst_k_nrm2(int64_t n, const double2 *x, double *nrm2, double *partials, int nblk, cudaStream_t s);
int dst_k_residual(int64_t n, const double2 *b, const double2 *y, double2 *r, double *nrm2, double *partials,
                   int nblk, cudaStream_t s);
int dst_k_scale(int64_t n, const double2 *src, double2 *dst, const double *nrm2, double scale, cudaStream_t s);
int dst_k_cast_64_32(int64_t n, const double2 *src, float2 *dst, cudaStream_t s);
int dst_k_cast_32_64(int64_t n, const float2 *src, double2 *dst, cudaStream_t s);
int dst_k_axpy1(int64_t n, const double2 *d, double2 *x, cudaStream_t s);
