// Batched persistent solver: many independent meshes, one CTA per mesh, the
// whole mixed-precision GMRES of each mesh inside one kernel launch.
//
// A small mesh alone cannot fill the GPU: its vectors are a few MB, so every
// kernel of the one-mesh solver (dst_solve) is short and launch- or latency-
// bound, and the host synchronises once per GMRES cycle.  Here each CTA owns
// one mesh for the whole solve and runs, without leaving the kernel,
//   the FP64 residual r = b - A x (FP64 operator apply, Eq. 11),
//   one GMRES(m) cycle on the correction equation with the FP32 operator
//   apply, an FP32-stored basis, classical Gram-Schmidt with a DGKS second
//   pass in compensated FP32 arithmetic (df_arith.cuh) and FP64 Givens
//   rotations / least squares (Sec. 2.2),
//   x += V y in compensated arithmetic, FP64 accumulation,
// until the true FP64 residual meets the tolerance (the iterative refinement
// of the one-mesh mixed solve).  All reductions are CTA-local (no grid-wide
// synchronisation, no waits on other CTAs); every loop is bounded by the
// iteration and refinement caps.  Meshes of one spatial dimension share a
// launch (1+1: 256 threads per CTA, 2+1: 128, the operator-apply tiling of
// apply_pipe.cuh); the two launches run on two streams.
//
// One CTA streams a mesh's basis at a few GB/s only, so the persistent kernel
// takes small meshes (opts->batch_cta_max unknowns at most); larger meshes
// run the single-mesh mixed solve, several at once from worker threads, each
// on its own stream, so that their short kernels overlap on the GPU.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstdint>
#include <vector>

#include "apply_pipe.cuh"
#include "blas.h"
#include "df_arith.cuh"

namespace dst {
namespace {

constexpr int BMAXV = DST_MAX_VEC;     // Gram-Schmidt coefficient buffers
constexpr int BMAXM = 32;              // restart length at most (Hessenberg in shared memory)

// Per-mesh descriptor (device memory).
struct BatchInst {
    OpParams p;                 // vmode 0: x-only weights (zero potential: weights +-m)
    int64_t n;                  // unknowns
    int64_t tiles_x, tiles_y, tiles, chunks;
    const double2 *b;           // right-hand side
    double2 *x;                 // solution (the caller's psi)
    double2 *r;                 // FP64 scratch: A x, then the residual
    float2 *V;                  // (m + 1) x n FP32 basis
    double *out;                // [0] steps, [1] cycles, [2] status, [3] ||r|| / ||b||, [4] estimate
};

struct BatchOpts {
    int m, max_iters, max_refine, use_initial_guess, ortho;
    double rtol, inner_rtol;
};

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 zscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double zabs(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

template <int D>
struct BatchShape {
    using S32 = PipeShape<D, 2, float>;
    using S64 = PipeShape<D, 2, double>;
    static constexpr int NT = S32::NTHR;
    static constexpr int NW = NT / 32;
    static constexpr int SMEM = S32::SMEM > S64::SMEM ? S32::SMEM : S64::SMEM;
    static_assert(S32::NTHR == S64::NTHR, "one thread count for both precisions");
};

// Sum of per-thread FP64 values over the CTA; every thread gets the result.
template <int NW>
__device__ __forceinline__ double cta_sum(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = dwarp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < NW; ++k) t += red[k];
    return t;
}

// Same for a df32 per-thread value.
template <int NW>
__device__ __forceinline__ double cta_sum_df(DfAcc a, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double v = dfwarp_sum(a);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < NW; ++k) t += red[k];
    return t;
}

template <int D>
__global__ void __launch_bounds__(BatchShape<D>::NT, 2)
batch_solve_kernel(const BatchInst *__restrict__ insts, BatchOpts o) {
    using BS = BatchShape<D>;
    constexpr int NT = BS::NT, NW = BS::NW;
    extern __shared__ __align__(16) char ring[];
    __shared__ double red[NW * 8];
    __shared__ double2 hcol[BMAXV];        // Gram-Schmidt coefficients of the current step
    __shared__ float4 hs[BMAXV];           // the same (or y) split into FP32 hi / lo
    __shared__ double ctl[8];              // values thread 0 decides for the CTA
    __shared__ double2 H[(BMAXM + 1) * BMAXM];    // Hessenberg of the cycle (row stride m)
    __shared__ double2 g[BMAXM + 1], sn[BMAXM];   // rotated right-hand side, Givens sines
    __shared__ double cs[BMAXM];                  // Givens cosines
    const BatchInst &I = insts[blockIdx.x];
    const int tid = threadIdx.x;
    const int64_t n = I.n, nu = n >> 1;    // entries; float4 units of two entries
    const int m = o.m;
    const int64_t ntc = I.tiles * I.chunks;

    auto apply32 = [&](const float2 *xin, float2 *yout) {
        for (int64_t tc = 0; tc < ntc; ++tc) {
            apply_pipe_tile<D, 2, float, false, false>(I.p, xin, yout, I.tiles_x, I.tiles_y, tc % I.tiles,
                                                        tc / I.tiles, ring);
            __syncthreads();
        }
    };
    auto apply64 = [&](const double2 *xin, double2 *yout) {
        for (int64_t tc = 0; tc < ntc; ++tc) {
            apply_pipe_tile<D, 2, double, false, false>(I.p, xin, yout, I.tiles_x, I.tiles_y, tc % I.tiles,
                                                         tc / I.tiles, ring);
            __syncthreads();
        }
    };
    // r = b - r (r holds A x on entry); returns ||r||^2
    auto residual = [&]() {
        double acc = 0.0;
        for (int64_t i = tid; i < n; i += NT) {
            const double2 bi = I.b[i], ai = I.r[i];
            const double2 ri = make_double2(bi.x - ai.x, bi.y - ai.y);
            I.r[i] = ri;
            acc = fma(ri.x, ri.x, fma(ri.y, ri.y, acc));
        }
        return cta_sum<NW>(acc, red);
    };
    // hcol[0..nv) = conj(V_j) w over the unit-norm FP32 basis; returns ||w||^2
    auto project = [&](const float2 *w, int nv) {
        const float4 *w4 = reinterpret_cast<const float4 *>(w);
        DfAcc wn;
        wn.zero();
        float sw = 0.f;
        for (int64_t u = tid; u < nu; u += NT) {
            const float4 a = w4[u];
            float p, e;
            p = a.x * a.x; e = fmaf(a.x, a.x, -p); wn.add(p, e);
            p = a.y * a.y; e = fmaf(a.y, a.y, -p); wn.add(p, e);
            p = a.z * a.z; e = fmaf(a.z, a.z, -p); wn.add(p, e);
            p = a.w * a.w; e = fmaf(a.w, a.w, -p); wn.add(p, e);
            sw += (fabsf(a.x) + fabsf(a.y)) + (fabsf(a.z) + fabsf(a.w));
        }
        const float sigma = anchor_above(sw);
        for (int j0 = 0; j0 < nv; j0 += 4) {
            const int gv = nv - j0 < 4 ? nv - j0 : 4;
            AnAcc re[4], im[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { re[q].init(sigma); im[q].init(sigma); }
            for (int64_t u = tid; u < nu; u += NT) {
                const float4 a = w4[u];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (q < gv) {
                        const float4 v = reinterpret_cast<const float4 *>(I.V + (size_t)(j0 + q) * n)[u];
                        cdot_an(v.x, v.y, a.x, a.y, re[q], im[q]);
                        cdot_an(v.z, v.w, a.z, a.w, re[q], im[q]);
                    }
                }
            }
            const int lane = tid & 31, warp = tid >> 5;
            double sv[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                DfAcc r_, i_;
                r_.hi = re[q].hi - sigma; r_.lo = re[q].lo;
                i_.hi = im[q].hi - sigma; i_.lo = im[q].lo;
                sv[2 * q] = dfwarp_sum(r_);
                sv[2 * q + 1] = dfwarp_sum(i_);
            }
            __syncthreads();
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < 8; ++k) red[warp * 8 + k] = sv[k];
            __syncthreads();
            if (tid < 2 * gv) {
                double t = 0.0;
                for (int k = 0; k < NW; ++k) t += red[k * 8 + tid];
                reinterpret_cast<double *>(hcol + j0)[tid] = t;
            }
            __syncthreads();
        }
        return cta_sum_df<NW>(wn, red);
    };
    // w -= sum_j V_j c_j, c = hcol[0..nv) (or the given coefficients), rounded to FP32; returns ||w||^2
    auto update = [&](float2 *w, int nv) {
        if (tid < nv) {
            const double2 c = hcol[tid];
            const float rh = (float)c.x, ih = (float)c.y;
            hs[tid] = make_float4(rh, (float)(c.x - (double)rh), ih, (float)(c.y - (double)ih));
        }
        if (tid == 0) {
            double t = 0.0;
            for (int j = 0; j < nv; ++j) t += fabs(hcol[j].x) + fabs(hcol[j].y);
            ctl[7] = t;
        }
        __syncthreads();
        const float h1 = (float)ctl[7];
        float4 *w4 = reinterpret_cast<float4 *>(w);
        DfAcc nr;
        nr.zero();
        for (int64_t u = tid; u < nu; u += NT) {
            const float4 a = w4[u];
            const float sigma =
                anchor_above(fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))) + h1);
            AnAcc ar0, ai0, ar1, ai1;
            ar0.init(sigma); ai0.init(sigma); ar1.init(sigma); ai1.init(sigma);
            ar0.add(a.x); ai0.add(a.y); ar1.add(a.z); ai1.add(a.w);
            for (int j0 = 0; j0 < nv; j0 += 4) {       // four basis vectors in flight
                float4 v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    v[q] = j0 + q < nv ? reinterpret_cast<const float4 *>(I.V + (size_t)(j0 + q) * n)[u]
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (j0 + q < nv) {
                        const float4 c = hs[j0 + q];
                        caxpy_an(v[q].x, v[q].y, c, ar0, ai0);
                        caxpy_an(v[q].z, v[q].w, c, ar1, ai1);
                    }
                }
            }
            const float4 q = make_float4((ar0.hi - sigma) + ar0.lo, (ai0.hi - sigma) + ai0.lo,
                                         (ar1.hi - sigma) + ar1.lo, (ai1.hi - sigma) + ai1.lo);
            w4[u] = q;
            float p, e;
            p = q.x * q.x; e = fmaf(q.x, q.x, -p); nr.add(p, e);
            p = q.y * q.y; e = fmaf(q.y, q.y, -p); nr.add(p, e);
            p = q.z * q.z; e = fmaf(q.z, q.z, -p); nr.add(p, e);
            p = q.w * q.w; e = fmaf(q.w, q.w, -p); nr.add(p, e);
        }
        return cta_sum_df<NW>(nr, red);
    };
    // w *= 1 / sqrt(nrm2), rounded to FP32 once
    auto scale = [&](float2 *w, double nrm2) {
        const double sd = 1.0 / sqrt(nrm2);
        const float sh = (float)sd, sl = (float)(sd - (double)sh);
        for (int64_t i = tid; i < n; i += NT) {
            const float2 a = w[i];
            float p, e;
            float2 q;
            p = a.x * sh; e = fmaf(a.x, sh, -p); e = fmaf(a.x, sl, e); q.x = p + e;
            p = a.y * sh; e = fmaf(a.y, sh, -p); e = fmaf(a.y, sl, e); q.y = p + e;
            w[i] = q;
        }
        __syncthreads();
    };

    // ---- the solve ---------------------------------------------------------
    if (!o.use_initial_guess)
        for (int64_t i = tid; i < n; i += NT) I.x[i] = make_double2(0.0, 0.0);
    double bacc = 0.0;
    for (int64_t i = tid; i < n; i += NT) bacc = fma(I.b[i].x, I.b[i].x, fma(I.b[i].y, I.b[i].y, bacc));
    const double bnorm = sqrt(cta_sum<NW>(bacc, red));
    const double tol = o.rtol * bnorm;
    int steps = 0, cycles = 0, status = DST_NOT_CONVERGED;
    double rnorm = 0.0, est = 0.0;
    if (!(bnorm > 0.0)) {       // b = 0 (or NaN): x = 0 is the solution
        for (int64_t i = tid; i < n; i += NT) I.x[i] = make_double2(0.0, 0.0);
        status = bnorm == 0.0 ? DST_OK : DST_ERR_NAN;
    } else {
        for (;;) {
            __syncthreads();
            apply64(I.x, I.r);
            rnorm = sqrt(residual());
            if (!isfinite(rnorm)) { status = DST_ERR_NAN; break; }
            if (rnorm <= tol) { status = DST_OK; break; }
            if (cycles >= o.max_refine || steps >= o.max_iters) break;
            // V_0 = r / ||r|| in FP32
            const double inv = 1.0 / rnorm;
            for (int64_t i = tid; i < n; i += NT) {
                const double2 ri = I.r[i];
                I.V[i] = make_float2((float)(ri.x * inv), (float)(ri.y * inv));
            }
            if (tid == 0) {
                for (int i = 0; i <= m; ++i) g[i] = make_double2(0.0, 0.0);
                g[0] = make_double2(rnorm, 0.0);
            }
            __syncthreads();
            const double itol = fmax(o.inner_rtol * rnorm, 0.5 * tol);
            int k = 0;
            for (int j = 0; j < m && steps < o.max_iters; ++j) {
                float2 *wv = I.V + (size_t)(j + 1) * n;
                apply32(I.V + (size_t)j * n, wv);
                const int nv = j + 1;
                const double before = project(wv, nv);
                double after = update(wv, nv);
                // column in FP64; second pass when the DGKS test asks (or always)
                __shared__ double2 col[BMAXV];
                if (tid < nv) col[tid] = hcol[tid];
                __syncthreads();
                if (o.ortho == 1 || (o.ortho == 0 && after < 0.5 * before)) {
                    project(wv, nv);
                    after = update(wv, nv);
                    if (tid < nv) col[tid] = zadd(col[tid], hcol[tid]);
                }
                __syncthreads();
                if (tid == 0) {
                    // Givens rotations (thread 0, FP64)
                    const double hn = sqrt(after);
                    double colsq = 0.0;
                    for (int i = 0; i < nv; ++i) {
                        H[(size_t)i * m + j] = col[i];
                        colsq += col[i].x * col[i].x + col[i].y * col[i].y;
                    }
                    H[(size_t)(j + 1) * m + j] = make_double2(hn, 0.0);
                    for (int i = 0; i < j; ++i) {
                        const double2 hij = H[(size_t)i * m + j], hi1 = H[(size_t)(i + 1) * m + j];
                        const double c = cs[i];
                        const double2 s = sn[i];
                        H[(size_t)i * m + j] = zadd(zscale(c, hij), zmul(s, hi1));
                        H[(size_t)(i + 1) * m + j] = zadd(zscale(-1.0, zmul(zconj(s), hij)), zscale(c, hi1));
                    }
                    const double2 a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
                    double c;
                    double2 s;
                    const double aa = zabs(a), ab = zabs(bb);
                    if (ab == 0.0) { c = 1.0; s = make_double2(0.0, 0.0); }
                    else if (aa == 0.0) { c = 0.0; s = make_double2(1.0, 0.0); }
                    else {
                        const double rho = sqrt(aa * aa + ab * ab);
                        c = aa / rho;
                        s = zscale(1.0 / rho, zmul(zscale(1.0 / aa, a), zconj(bb)));
                    }
                    cs[j] = c;
                    sn[j] = s;
                    H[(size_t)j * m + j] = zadd(zscale(c, a), zmul(s, bb));
                    H[(size_t)(j + 1) * m + j] = make_double2(0.0, 0.0);
                    g[j + 1] = zscale(-1.0, zmul(zconj(s), g[j]));
                    g[j] = zscale(c, g[j]);
                    const double res = zabs(g[j + 1]);
                    const bool finite = isfinite(hn) && isfinite(colsq);
                    const bool brk = hn <= 1e-14 * sqrt(colsq + hn * hn);
                    ctl[0] = res;
                    ctl[1] = finite ? 1.0 : 0.0;
                    ctl[2] = (brk || res <= itol) ? 1.0 : 0.0;
                    ctl[3] = hn * hn;
                }
                __syncthreads();
                est = ctl[0];
                ++steps;
                k = j + 1;
                if (ctl[1] == 0.0) { status = DST_ERR_NAN; break; }
                if (ctl[2] != 0.0) break;
                scale(wv, ctl[3]);
            }
            if (status == DST_ERR_NAN) break;
            // y = R^-1 g (thread 0), then x += V y
            if (tid == 0) {
                for (int i = k - 1; i >= 0; --i) {
                    double2 acc = g[i];
                    for (int l = i + 1; l < k; ++l) acc = zsub(acc, zmul(H[(size_t)i * m + l], hcol[l]));
                    hcol[i] = zdiv(acc, H[(size_t)i * m + i]);
                }
            }
            __syncthreads();
            if (tid < k) {
                const double2 c = hcol[tid];
                const float rh = (float)(-c.x), ih = (float)(-c.y);
                hs[tid] = make_float4(rh, (float)(-c.x - (double)rh), ih, (float)(-c.y - (double)ih));
            }
            __syncthreads();
            for (int64_t i = tid; i < n; i += NT) {
                DfAcc ar, ai;
                ar.zero();
                ai.zero();
                for (int j0 = 0; j0 < k; j0 += 4) {        // four basis vectors in flight
                    float2 v[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        v[q] = j0 + q < k ? I.V[(size_t)(j0 + q) * n + i] : make_float2(0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (j0 + q < k) caxpy_sub<false>(v[q].x, v[q].y, 0.f, 0.f, hs[j0 + q], ar, ai);   // acc -= v (-y)
                }
                double2 xi = I.x[i];
                xi.x += ar.value();
                xi.y += ai.value();
                I.x[i] = xi;
            }
            ++cycles;
        }
    }
    if (tid == 0) {
        I.out[0] = steps;
        I.out[1] = cycles;
        I.out[2] = status;
        I.out[3] = bnorm > 0.0 ? rnorm / bnorm : 0.0;
        I.out[4] = bnorm > 0.0 ? est / bnorm : 0.0;
    }
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

template <int D>
int launch_batch(const BatchInst *insts, int count, const BatchOpts &o, cudaStream_t s) {
    if (count <= 0) return DST_OK;
    using BS = BatchShape<D>;
    static bool configured[DST_MAX_DEVICES_APPLY] = {};
    int dev = 0;
    DST_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= DST_MAX_DEVICES_APPLY || !configured[dev]) {
        DST_CUDA_TRY(cudaFuncSetAttribute(batch_solve_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          BS::SMEM));
        if (dev >= 0 && dev < DST_MAX_DEVICES_APPLY) configured[dev] = true;
    }
    batch_solve_kernel<D><<<count, BS::NT, BS::SMEM, s>>>(insts, o);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

}  // namespace
}  // namespace dst

using namespace dst;

// Meshes up to this many unknowns go to the persistent one-CTA-per-mesh kernel
// when opts->batch_cta_max is negative (automatic).
constexpr int64_t BATCH_CTA_MAX_AUTO = 4096;
constexpr int BATCH_WORKERS = 16;          // concurrent single-mesh solves (one stream each)

static int solve_batch(int count, dst_mesh *const *meshes, const dst_solve_opts *opts, void *const *psi,
                       dst_solve_stats *stats, void *stream) {
    if (count <= 0 || !meshes || !opts || !psi || !stats) return DST_ERR_ARG;
    const dst_solve_opts &u = *opts;
    if (u.restart < 1 || u.restart > BMAXM || u.max_iters < 1 || u.max_refine < 1 || !(u.rtol > 0) ||
        !(u.inner_rtol > 0) || u.ortho < 0 || u.ortho > 2 || u.method != 0)
        return DST_ERR_ARG;
    int dev = 0;
    DST_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= DST_MAX_DEVICES_APPLY) return DST_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        const dst_mesh *mh = meshes[i];
        if (!mh || !psi[i]) return DST_ERR_ARG;
        if (mh->device != dev || (mh->d != 1 && mh->d != 2) || mh->v_general) {
            dst_internal_set_error_detail("dst_solve_batch: every mesh must be 1+1 or 2+1, on the current "
                                          "device, with an x-only potential");
            return DST_ERR_ARG;
        }
        if ((reinterpret_cast<uintptr_t>(psi[i]) & 15) != 0) return DST_ERR_ARG;
        if (!mh->d_psi0) return DST_ERR_STATE;
        for (int k = 0; k < i; ++k)
            if (meshes[k] == mh || psi[k] == psi[i]) return DST_ERR_ARG;    // each mesh / psi once
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t cta_max = u.batch_cta_max >= 0 ? u.batch_cta_max : BATCH_CTA_MAX_AUTO;
    auto t0 = std::chrono::steady_clock::now();
    std::vector<int> small, big;
    for (int i = 0; i < count; ++i) (meshes[i]->n_unknowns <= cta_max ? small : big).push_back(i);
    // largest first: the longest solves start earliest
    auto by_size = [&](int a, int c) { return meshes[a]->n_unknowns > meshes[c]->n_unknowns; };
    std::sort(small.begin(), small.end(), by_size);
    std::sort(big.begin(), big.end(), by_size);
    std::vector<int> rcs(count, DST_OK);
    const int cs_ = (int)small.size();
    // host memory of the small-mesh path, taken before any worker starts
    std::vector<BatchInst> packed;
    packed.reserve(cs_);
    std::vector<double> outs((size_t)cs_ * 8, 0.0);
    std::vector<std::thread> workers;
    const int nw = std::min<int>((int)big.size(), BATCH_WORKERS);
    workers.reserve(nw);
    cudaEvent_t start = nullptr;
    DST_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    cudaEventRecord(start, s);
    // large meshes: single-mesh mixed solves, BATCH_WORKERS at a time on their own streams
    std::atomic<int> next{0};
    auto worker = [&] {
        cudaSetDevice(dev);
        cudaStream_t ws = nullptr;
        if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
            for (int k = next++; k < (int)big.size(); k = next++) rcs[big[k]] = DST_ERR_CUDA;
            return;
        }
        cudaStreamWaitEvent(ws, start, 0);
        dst_solve_opts o1 = u;
        o1.mixed_precision = 1;
        o1.mixed_ortho = 2;
        o1.inner_cycles = 1;
        o1.profile = 0;
        for (int k = next++; k < (int)big.size(); k = next++) {
            const int i = big[k];
            rcs[i] = dst_solve(meshes[i], &o1, psi[i], &stats[i], ws);
        }
        cudaStreamDestroy(ws);
    };
    for (int w = 0; w < nw; ++w) {
        try {
            workers.emplace_back(worker);
        } catch (...) {
            break;      // fewer workers: those running take every large mesh between them
        }
    }
    int rc = DST_OK;
    // small meshes: one CTA each in the persistent kernel.  No exception leaves
    // this block while workers run (they use this frame's locals).
    char *wsb = nullptr;
    int c1 = 0;
    if (cs_ > 0) try {
        const int m = u.restart;
        std::vector<size_t> off(cs_);
        size_t total = align256(sizeof(BatchInst) * cs_);
        for (int k = 0; k < cs_; ++k) {
            const int64_t n = meshes[small[k]]->n_unknowns;
            off[k] = total;
            total += align256(sizeof(double2) * n) * 2 + align256(sizeof(float2) * n * (m + 1)) +
                     align256(sizeof(double) * 8);
        }
        if (cudaMallocAsync(reinterpret_cast<void **>(&wsb), total, s) != cudaSuccess) {
            cudaGetLastError();
            wsb = nullptr;
            rc = DST_ERR_OOM;
        }
        std::vector<int> o1, o2;
        for (int k = 0; k < cs_; ++k) (meshes[small[k]]->d == 1 ? o1 : o2).push_back(k);
        c1 = (int)o1.size();
        std::vector<int> order(o1);
        order.insert(order.end(), o2.begin(), o2.end());
        for (int q = 0; q < cs_ && rc == DST_OK; ++q) {
            const int k = order[q];
            dst_mesh *mh = meshes[small[k]];
            BatchInst b;
            b.p = dst_internal_params(mh);
            b.p.vmode = 0;                      // the weights +-m + V_e cover a zero potential too
            b.n = mh->n_unknowns;
            if (mh->d == 1) {
                b.tiles_x = (b.p.ax[0].n + PipeTile<1>::TX - 1) / PipeTile<1>::TX;
                b.tiles_y = 1;
                b.chunks = (b.p.nt + PipeTile<1>::TT - 1) / PipeTile<1>::TT;
            } else {
                b.tiles_x = (b.p.ax[0].n + PipeTile<2>::TX - 1) / PipeTile<2>::TX;
                b.tiles_y = (b.p.ax[1].n + PipeTile<2>::TY - 1) / PipeTile<2>::TY;
                b.chunks = (b.p.nt + PipeTile<2>::TT - 1) / PipeTile<2>::TT;
            }
            b.tiles = b.tiles_x * b.tiles_y;
            char *q2 = wsb + off[k];
            b.b = reinterpret_cast<double2 *>(q2);
            b.r = reinterpret_cast<double2 *>(q2 + align256(sizeof(double2) * b.n));
            q2 += align256(sizeof(double2) * b.n) * 2;
            b.V = reinterpret_cast<float2 *>(q2);
            q2 += align256(sizeof(float2) * b.n * (m + 1));
            b.out = reinterpret_cast<double *>(q2);
            b.x = static_cast<double2 *>(psi[small[k]]);
            rc = dst_internal_rhs(mh, const_cast<double2 *>(b.b), s);
            packed.push_back(b);
        }
        // small[order[q]] is the mesh of packed[q]
        std::vector<int> mesh_of(cs_);
        for (int q = 0; q < cs_; ++q) mesh_of[q] = small[order[q]];
        small = mesh_of;
        BatchInst *d_inst = reinterpret_cast<BatchInst *>(wsb);
        if (rc == DST_OK &&
            cudaMemcpyAsync(d_inst, packed.data(), sizeof(BatchInst) * cs_, cudaMemcpyHostToDevice, s) != cudaSuccess)
            rc = DST_ERR_CUDA;
        BatchOpts bo{m, u.max_iters, u.max_refine, u.use_initial_guess, u.ortho, u.rtol, u.inner_rtol};
        // one side stream per device for the 2+1 kernel, shared by concurrent calls
        static cudaStream_t side[DST_MAX_DEVICES_APPLY] = {};
        static std::mutex side_mu;
        const int c2 = cs_ - c1;
        if (rc == DST_OK && c1 > 0 && c2 > 0) {
            cudaEvent_t fork = nullptr, join = nullptr;
            {
                std::lock_guard<std::mutex> lk(side_mu);
                if (!side[dev] && cudaStreamCreateWithFlags(&side[dev], cudaStreamNonBlocking) != cudaSuccess) {
                    side[dev] = nullptr;
                    rc = DST_ERR_CUDA;
                }
            }
            if (rc == DST_OK && (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
                                 cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess))
                rc = DST_ERR_CUDA;
            if (rc == DST_OK) {
                cudaEventRecord(fork, s);
                cudaStreamWaitEvent(side[dev], fork, 0);
                rc = launch_batch<2>(d_inst + c1, c2, bo, side[dev]);
                cudaEventRecord(join, side[dev]);
                if (rc == DST_OK) rc = launch_batch<1>(d_inst, c1, bo, s);
                cudaStreamWaitEvent(s, join, 0);
            }
            if (fork) cudaEventDestroy(fork);
            if (join) cudaEventDestroy(join);
        } else if (rc == DST_OK) {
            rc = launch_batch<1>(d_inst, c1, bo, s);
            if (rc == DST_OK) rc = launch_batch<2>(d_inst + c1, c2, bo, s);
        }
        for (int q = 0; q < cs_ && rc == DST_OK; ++q)
            if (cudaMemcpyAsync(outs.data() + 8 * q, packed[q].out, sizeof(double) * 8, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess)
                rc = DST_ERR_CUDA;
    } catch (const std::exception &e) {
        dst_internal_set_exception_detail("dst_solve_batch", e.what());
        if (rc == DST_OK) rc = DST_ERR_OOM;
    } catch (...) {
        dst_internal_set_exception_detail("dst_solve_batch", "unknown C++ exception");
        if (rc == DST_OK) rc = DST_ERR_OOM;
    }
    if (workers.empty() && !big.empty()) worker();      // no thread could be started
    for (auto &t : workers) t.join();
    cudaError_t se = cudaStreamSynchronize(s);
    if (rc == DST_OK && se != cudaSuccess) rc = DST_ERR_CUDA;
    if (wsb) cudaFreeAsync(wsb, s);
    cudaEventDestroy(start);
    if (rc != DST_OK) return rc;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int worst = DST_OK;
    for (int q = 0; q < cs_; ++q) {
        const double *o = outs.data() + 8 * q;
        dst_solve_stats &st = stats[small[q]];
        st = dst_solve_stats{};
        st.iters = (int)o[0];
        st.restarts = (int)o[1];
        st.refinements = (int)o[1];
        st.status = (int)o[2];
        st.rel_resid_true = o[3];
        st.rel_resid_est = o[4];
        st.launches = 1;
    }
    for (int i = 0; i < count; ++i) {
        stats[i].seconds = secs;
        if (stats[i].status < 0 && (worst == DST_OK || stats[i].status < worst)) worst = stats[i].status;
        if (rcs[i] < 0 && (worst == DST_OK || rcs[i] < worst)) worst = rcs[i];
    }
    return worst;
}

extern "C" int dst_solve_batch(int count, dst_mesh *const *meshes, const dst_solve_opts *opts, void *const *psi,
                               dst_solve_stats *stats, void *stream) {
    return dst_internal_guard("dst_solve_batch",
                              [&] { return solve_batch(count, meshes, opts, psi, stats, stream); });
}
