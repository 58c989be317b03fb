// Vector kernels of restarted GMRES (Saad & Schultz 1986, the Krylov solver
// of Sec. 2.2): the classical Gram-Schmidt projection h = V^H w, the update
// w <- w - V h fused with ||w||^2, scaling, residuals and precision casts.
//
// Reductions are deterministic: each CTA owns a fixed contiguous slice of the
// vector, threads accumulate their elements in a fixed order, warps reduce by
// a fixed shuffle tree, CTAs write partials that a second kernel sums in CTA
// order.  All arithmetic of these kernels is FP64.
#include <mutex>

#include "blas.h"

namespace dst {

static constexpr int RED_THREADS = 256;
static constexpr int PROJ_GROUP = 8;     // basis vectors per register group

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of one double (result valid in thread 0); fixed order.
__device__ __forceinline__ double block_sum(double v, double *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
    return r;
}

// Second Gram-Schmidt pass gate evaluated on the device: nrm[0] = ||w||^2
// after the first pass, nrm[3] = ||A v_j||^2 before it (DGKS: reorthogonalise
// when ||w|| < ||A v_j|| / sqrt 2).  A null gate means "always run".
__device__ __forceinline__ bool dgks_skip(const double *gate) {
    return gate != nullptr && !(gate[0] < 0.5 * gate[3]);
}

__device__ __forceinline__ void slice(int64_t n, int64_t &b, int64_t &e) {
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    b = (int64_t)blockIdx.x * per;
    e = b + per < n ? b + per : n;
}

// partials[blk * nvec + j] = sum over the CTA's slice of conj(V_j) w, and
// (if wnrm_partials) partials of ||w||^2.  Threads accumulate PROJ_GROUP basis
// vectors at a time over their elements; each group is reduced across the warp
// by shuffles and parked in shared memory; one barrier at the end, then the
// warps' values are summed in warp order.
__global__ void __launch_bounds__(RED_THREADS)
project_partial_kernel(int64_t n, int nvec, const double2 *__restrict__ V, const double2 *__restrict__ w,
                       double2 *__restrict__ partials, double *__restrict__ wnrm_partials, const double *gate) {
    if (dgks_skip(gate)) return;
    constexpr int NW = RED_THREADS / 32;
    __shared__ double red[NW][2 * DST_MAX_VEC + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t b, e;
    slice(n, b, e);
    double wn = 0.0;
    for (int j0 = 0; j0 < nvec; j0 += PROJ_GROUP) {
        const int gv = nvec - j0 < PROJ_GROUP ? nvec - j0 : PROJ_GROUP;
        double ar[PROJ_GROUP], ai[PROJ_GROUP];
#pragma unroll
        for (int g = 0; g < PROJ_GROUP; ++g) { ar[g] = 0.0; ai[g] = 0.0; }
        for (int64_t i = b + threadIdx.x; i < e; i += RED_THREADS) {
            const double2 wi = w[i];
            if (j0 == 0) wn = fma(wi.x, wi.x, fma(wi.y, wi.y, wn));
#pragma unroll
            for (int g = 0; g < PROJ_GROUP; ++g) {
                if (g < gv) {
                    const double2 v = V[(int64_t)(j0 + g) * n + i];
                    ar[g] = fma(v.x, wi.x, fma(v.y, wi.y, ar[g]));
                    ai[g] = fma(v.x, wi.y, fma(-v.y, wi.x, ai[g]));
                }
            }
        }
#pragma unroll
        for (int g = 0; g < PROJ_GROUP; ++g) {
            if (g < gv) {
                const double sr = warp_sum(ar[g]), si = warp_sum(ai[g]);
                if (lane == 0) { red[warp][2 * (j0 + g)] = sr; red[warp][2 * (j0 + g) + 1] = si; }
            }
        }
    }
    wn = warp_sum(wn);
    if (lane == 0) red[warp][2 * DST_MAX_VEC] = wn;
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * nvec; q += RED_THREADS) {
        double s_ = 0.0;
#pragma unroll
        for (int k = 0; k < NW; ++k) s_ += red[k][q];
        reinterpret_cast<double *>(partials + (int64_t)blockIdx.x * nvec)[q] = s_;
    }
    if (wnrm_partials && threadIdx.x == 0) {
        double s_ = 0.0;
#pragma unroll
        for (int k = 0; k < NW; ++k) s_ += red[k][2 * DST_MAX_VEC];
        wnrm_partials[blockIdx.x] = s_;
    }
}

// out[j] = sum_blk partials[blk * nvec + j]   (one CTA per j)
__global__ void __launch_bounds__(RED_THREADS)
reduce_partials_kernel(int nblk, int nvec, const double2 *__restrict__ partials, double2 *__restrict__ out,
                       const double *gate) {
    __shared__ double sh[RED_THREADS / 32];
    const int j = blockIdx.x;
    if (dgks_skip(gate)) {
        if (threadIdx.x == 0) out[j] = make_double2(0.0, 0.0);
        return;
    }
    double sr = 0.0, si = 0.0;
    for (int k = threadIdx.x; k < nblk; k += RED_THREADS) {
        const double2 v = partials[(int64_t)k * nvec + j];
        sr += v.x;
        si += v.y;
    }
    sr = block_sum(sr, sh);
    si = block_sum(si, sh);
    if (threadIdx.x == 0) out[j] = make_double2(sr, si);
}

// w <- w - sum_j V_j h_j ; partial ||w||^2 per CTA.
__global__ void __launch_bounds__(RED_THREADS)
update_kernel(int64_t n, int nvec, const double2 *__restrict__ V, const double2 *__restrict__ h,
              double2 *__restrict__ w, double *__restrict__ nrm_partials, const double *gate) {
    if (dgks_skip(gate)) return;
    __shared__ double2 hs[DST_MAX_VEC];
    __shared__ double sh[RED_THREADS / 32];
    for (int j = threadIdx.x; j < nvec; j += RED_THREADS) hs[j] = h[j];
    __syncthreads();
    int64_t b, e;
    slice(n, b, e);
    double nr = 0.0;
    for (int64_t i = b + threadIdx.x; i < e; i += RED_THREADS) {
        double2 acc = w[i];
        for (int j = 0; j < nvec; ++j) {
            const double2 v = V[(int64_t)j * n + i];
            const double2 c = hs[j];
            acc.x = fma(-v.x, c.x, fma(v.y, c.y, acc.x));
            acc.y = fma(-v.x, c.y, fma(-v.y, c.x, acc.y));
        }
        w[i] = acc;
        nr = fma(acc.x, acc.x, fma(acc.y, acc.y, nr));
    }
    nr = block_sum(nr, sh);
    if (threadIdx.x == 0 && nrm_partials) nrm_partials[blockIdx.x] = nr;
}

__global__ void __launch_bounds__(RED_THREADS)
reduce_real_kernel(int nblk, const double *__restrict__ partials, double *out, const double *gate,
                   double *counter) {
    if (dgks_skip(gate)) return;
    __shared__ double sh[RED_THREADS / 32];
    double s = 0.0;
    for (int k = threadIdx.x; k < nblk; k += RED_THREADS) s += partials[k];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        *out = s;
        if (counter) *counter += 1.0;
    }
}

// ||x||^2 partials
__global__ void __launch_bounds__(RED_THREADS)
nrm2_partial_kernel(int64_t n, const double2 *__restrict__ x, double *__restrict__ partials) {
    __shared__ double sh[RED_THREADS / 32];
    int64_t b, e;
    slice(n, b, e);
    double s = 0.0;
    for (int64_t i = b + threadIdx.x; i < e; i += RED_THREADS) {
        const double2 v = x[i];
        s = fma(v.x, v.x, fma(v.y, v.y, s));
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// r = b - y ; ||r||^2 partials
__global__ void __launch_bounds__(RED_THREADS)
residual_kernel(int64_t n, const double2 *__restrict__ b_, const double2 *__restrict__ y, double2 *__restrict__ r,
                double *__restrict__ partials) {
    __shared__ double sh[RED_THREADS / 32];
    int64_t b, e;
    slice(n, b, e);
    double s = 0.0;
    for (int64_t i = b + threadIdx.x; i < e; i += RED_THREADS) {
        const double2 u = b_[i], v = y[i];
        const double2 d = make_double2(u.x - v.x, u.y - v.y);
        r[i] = d;
        s = fma(d.x, d.x, fma(d.y, d.y, s));
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// dst = src * (1/sqrt(*nrm2)) (or * scale when nrm2 is null)
__global__ void scale_kernel(int64_t n, const double2 *__restrict__ src, double2 *__restrict__ dst,
                             const double *__restrict__ nrm2, double scale) {
    __shared__ double s_sh;       // 1/sqrt once per CTA: FP64 division is slow here
    if (threadIdx.x == 0) s_sh = nrm2 ? 1.0 / sqrt(*nrm2) : scale;
    __syncthreads();
    const double s = s_sh;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = src[i];
        dst[i] = make_double2(v.x * s, v.y * s);
    }
}

__global__ void cast_64_32_kernel(int64_t n, const double2 *__restrict__ src, float2 *__restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = src[i];
        dst[i] = make_float2((float)v.x, (float)v.y);
    }
}

__global__ void cast_32_64_kernel(int64_t n, const float2 *__restrict__ src, double2 *__restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = src[i];
        dst[i] = make_double2((double)v.x, (double)v.y);
    }
}

// x += d
__global__ void axpy1_kernel(int64_t n, const double2 *__restrict__ d, double2 *__restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = x[i], b = d[i];
        x[i] = make_double2(a.x + b.x, a.y + b.y);
    }
}

// ---- BiCGSTAB (van der Vorst 1992) vector steps with device-resident scalars ----
// sc (double2[8]): 0 rho, 1 alpha, 2 omega, 3 beta, 4 (rhat, v), 5 (t, s), 6 (t, t) in .x, 7 (rhat, r)

__device__ __forceinline__ double2 cmulz(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cdivz(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// mode 0: beta = (rho_new / rho)(alpha / omega), rho = rho_new; 1: alpha = rho / (rhat, v);
// 2: omega = (t, s) / (t, t); 3: initialise rho = alpha = omega = 1
__global__ void bicg_scalar_kernel(int mode, double2 *sc) {
    if (threadIdx.x != 0) return;
    if (mode == 0) {
        sc[3] = cmulz(cdivz(sc[7], sc[0]), cdivz(sc[1], sc[2]));
        sc[0] = sc[7];
    } else if (mode == 1) {
        sc[1] = cdivz(sc[0], sc[4]);
    } else if (mode == 2) {
        sc[2] = make_double2(sc[5].x / sc[6].x, sc[5].y / sc[6].x);
    } else {
        sc[0] = sc[1] = sc[2] = make_double2(1.0, 0.0);
    }
}

// p = r + beta (p - omega v)
__global__ void bicg_p_kernel(int64_t n, const double2 *__restrict__ r, const double2 *__restrict__ v,
                              double2 *__restrict__ p, const double2 *__restrict__ sc) {
    const double2 beta = sc[3], omega = sc[2];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 ov = cmulz(omega, v[i]);
        const double2 d = make_double2(p[i].x - ov.x, p[i].y - ov.y);
        const double2 bd = cmulz(beta, d);
        p[i] = make_double2(r[i].x + bd.x, r[i].y + bd.y);
    }
}

// s = r - alpha v
__global__ void bicg_s_kernel(int64_t n, const double2 *__restrict__ r, const double2 *__restrict__ v,
                              double2 *__restrict__ s, const double2 *__restrict__ sc) {
    const double2 alpha = sc[1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 av = cmulz(alpha, v[i]);
        s[i] = make_double2(r[i].x - av.x, r[i].y - av.y);
    }
}

// x += alpha p + omega s; r = s - omega t; partials of ||r||^2 (CTA slices, fixed order)
__global__ void __launch_bounds__(RED_THREADS)
bicg_xr_kernel(int64_t n, double2 *__restrict__ x, const double2 *__restrict__ p, const double2 *__restrict__ s,
               const double2 *__restrict__ t, double2 *__restrict__ r, const double2 *__restrict__ sc,
               double *__restrict__ partials) {
    __shared__ double sh[RED_THREADS / 32];
    const double2 alpha = sc[1], omega = sc[2];
    int64_t b, e;
    slice(n, b, e);
    double acc = 0.0;
    for (int64_t i = b + threadIdx.x; i < e; i += RED_THREADS) {
        const double2 ap = cmulz(alpha, p[i]), os = cmulz(omega, s[i]), ot = cmulz(omega, t[i]);
        x[i] = make_double2(x[i].x + ap.x + os.x, x[i].y + ap.y + os.y);
        const double2 rr = make_double2(s[i].x - ot.x, s[i].y - ot.y);
        r[i] = rr;
        acc = fma(rr.x, rr.x, fma(rr.y, rr.y, acc));
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

}  // namespace dst

using namespace dst;

int dst_k_bicg_scalar(int mode, double2 *sc, cudaStream_t s) {
    bicg_scalar_kernel<<<1, 32, 0, s>>>(mode, sc);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_bicg_p(int64_t n, const double2 *r, const double2 *v, double2 *p, const double2 *sc, cudaStream_t s);
int dst_k_bicg_s(int64_t n, const double2 *r, const double2 *v, double2 *sv, const double2 *sc, cudaStream_t s);

int dst_k_bicg_xr(int64_t n, double2 *x, const double2 *p, const double2 *sv, const double2 *t, double2 *r,
                  const double2 *sc, double *nrm2, double *partials, int nblk, cudaStream_t s) {
    bicg_xr_kernel<<<nblk, RED_THREADS, 0, s>>>(n, x, p, sv, t, r, sc, partials);
    reduce_real_kernel<<<1, RED_THREADS, 0, s>>>(nblk, partials, nrm2, nullptr, nullptr);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

static unsigned stream_blocks(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

int dst_k_project(int64_t n, int nvec, const double2 *V, const double2 *w, double2 *h, double2 *partials,
                  int nblk, cudaStream_t s, double *wnrm2, double *wnrm_partials, const double *gate) {
    project_partial_kernel<<<nblk, RED_THREADS, 0, s>>>(n, nvec, V, w, partials, wnrm2 ? wnrm_partials : nullptr,
                                                        gate);
    reduce_partials_kernel<<<nvec, RED_THREADS, 0, s>>>(nblk, nvec, partials, h, gate);
    if (wnrm2) reduce_real_kernel<<<1, RED_THREADS, 0, s>>>(nblk, wnrm_partials, wnrm2, gate, nullptr);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_reduce_partials(int nblk, int nvec, const double2 *partials, double2 *out, cudaStream_t s,
                          const double *gate) {
    reduce_partials_kernel<<<nvec, RED_THREADS, 0, s>>>(nblk, nvec, partials, out, gate);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_reduce_real(int nblk, const double *partials, double *out, cudaStream_t s, const double *gate,
                      double *counter) {
    reduce_real_kernel<<<1, RED_THREADS, 0, s>>>(nblk, partials, out, gate, counter);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_update(int64_t n, int nvec, const double2 *V, const double2 *h, double2 *w, double *nrm2,
                 double *partials, int nblk, cudaStream_t s, const double *gate, double *counter) {
    update_kernel<<<nblk, RED_THREADS, 0, s>>>(n, nvec, V, h, w, nrm2 ? partials : nullptr, gate);
    if (nrm2) reduce_real_kernel<<<1, RED_THREADS, 0, s>>>(nblk, partials, nrm2, gate, counter);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_nrm2(int64_t n, const double2 *x, double *nrm2, double *partials, int nblk, cudaStream_t s) {
    nrm2_partial_kernel<<<nblk, RED_THREADS, 0, s>>>(n, x, partials);
    reduce_real_kernel<<<1, RED_THREADS, 0, s>>>(nblk, partials, nrm2, nullptr, nullptr);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_residual(int64_t n, const double2 *b, const double2 *y, double2 *r, double *nrm2, double *partials,
                   int nblk, cudaStream_t s) {
    residual_kernel<<<nblk, RED_THREADS, 0, s>>>(n, b, y, r, partials);
    reduce_real_kernel<<<1, RED_THREADS, 0, s>>>(nblk, partials, nrm2, nullptr, nullptr);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_scale(int64_t n, const double2 *src, double2 *dst, const double *nrm2, double scale, cudaStream_t s) {
    scale_kernel<<<stream_blocks(n), 256, 0, s>>>(n, src, dst, nrm2, scale);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_cast_64_32(int64_t n, const double2 *src, float2 *dst, cudaStream_t s) {
    cast_64_32_kernel<<<stream_blocks(n), 256, 0, s>>>(n, src, dst);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_cast_32_64(int64_t n, const float2 *src, double2 *dst, cudaStream_t s) {
    cast_32_64_kernel<<<stream_blocks(n), 256, 0, s>>>(n, src, dst);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_bicg_p(int64_t n, const double2 *r, const double2 *v, double2 *p, const double2 *sc, cudaStream_t s) {
    bicg_p_kernel<<<stream_blocks(n), 256, 0, s>>>(n, r, v, p, sc);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_bicg_s(int64_t n, const double2 *r, const double2 *v, double2 *sv, const double2 *sc, cudaStream_t s) {
    bicg_s_kernel<<<stream_blocks(n), 256, 0, s>>>(n, r, v, sv, sc);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

namespace {
// r = v - a (FP32 complex vectors)
__global__ void sub_f32_kernel(int64_t n, const float2 *__restrict__ v, const float2 *__restrict__ a,
                               float2 *__restrict__ r) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 x = v[i], y = a[i];
        r[i] = make_float2(x.x - y.x, x.y - y.y);
    }
}
// z += a
__global__ void add_f32_kernel(int64_t n, const float2 *__restrict__ a, float2 *__restrict__ z) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 x = z[i], y = a[i];
        z[i] = make_float2(x.x + y.x, x.y + y.y);
    }
}
}  // namespace

int dst_k_sub_f32(int64_t n, const float2 *v, const float2 *a, float2 *r, cudaStream_t s) {
    sub_f32_kernel<<<stream_blocks(n), 256, 0, s>>>(n, v, a, r);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_add_f32(int64_t n, const float2 *a, float2 *z, cudaStream_t s) {
    add_f32_kernel<<<stream_blocks(n), 256, 0, s>>>(n, a, z);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_axpy1(int64_t n, const double2 *d, double2 *x, cudaStream_t s) {
    axpy1_kernel<<<stream_blocks(n), 256, 0, s>>>(n, d, x);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_projection_blocks(int64_t n) {
    int64_t b = (n + 4095) / 4096;
    if (b > 456) b = 456;
    return (int)(b < 1 ? 1 : b);
}

int dst_reduction_blocks(int64_t n) {
    int64_t b = (n + 2047) / 2048;
    if (b > DST_MAX_RED_BLOCKS) b = DST_MAX_RED_BLOCKS;
    return (int)(b < 1 ? 1 : b);
}

// ---- projection without device allocation --------------------------------
//
// Scratch for callers that may not allocate device memory: the reduction
// partials live in a fixed file-scope device array instead of coming from the
// stream-ordered allocator.  Host code cannot pass the symbol itself (on the
// host it only names a shadow variable); its device address is looked up once
// per device with cudaGetSymbolAddress and cached.
#define DST_NOALLOC_PARTIALS ((size_t)1216 * DST_MAX_VEC)
static_assert(DST_NOALLOC_PARTIALS >= (size_t)DST_MAX_RED_BLOCKS * DST_MAX_VEC,
              "the static scratch must hold the partials of the largest reduction grid for 64 vectors");
static __device__ __align__(256) double2 g_noalloc_partials[DST_NOALLOC_PARTIALS];

static std::mutex g_noalloc_mutex;
static void *g_noalloc_addr[DST_MAX_DEVICES];

static int noalloc_scratch(void **out) {
    int dev = 0;
    DST_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= DST_MAX_DEVICES) {
        dst_internal_set_error_detail("dst_arnoldi_project_noalloc: device ordinal out of range");
        return DST_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        DST_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_partials));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return DST_OK;
}

extern "C" int dst_arnoldi_project_noalloc(int64_t n, int nvec, const void *V, const void *w, void *h,
                                           void *stream) {
    if (n < 1) {
        dst_internal_set_error_detail("dst_arnoldi_project_noalloc: n must be at least 1");
        return DST_ERR_ARG;
    }
    if (!V || !w || !h) {
        dst_internal_set_error_detail("dst_arnoldi_project_noalloc: V, w and h must be device pointers, not NULL");
        return DST_ERR_ARG;
    }
    if (nvec < 1 || nvec > DST_MAX_VEC) {
        dst_internal_set_error_detail("dst_arnoldi_project_noalloc: nvec must be 1..64 (the static scratch "
                                      "holds 1216 x 64 partial sums)");
        return DST_ERR_ARG;
    }
    const int nblk = dst_reduction_blocks(n);
    if ((size_t)nblk * (size_t)nvec > DST_NOALLOC_PARTIALS) {
        dst_internal_set_error_detail("dst_arnoldi_project_noalloc: partial sums exceed the static scratch");
        return DST_ERR_ARG;
    }
    void *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != DST_OK) return rc;
    return dst_k_project(n, nvec, (const double2 *)V, (const double2 *)w, (double2 *)h, (double2 *)scratch,
                         nblk, (cudaStream_t)stream);
}

// ---- C ABI wrappers -------------------------------------------------------

extern "C" int dst_arnoldi_project(int64_t n, int nvec, const void *V, const void *w, void *h, void *stream) {
    if (n < 1 || nvec < 1 || nvec > DST_MAX_VEC || !V || !w || !h) return DST_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int nblk = dst_reduction_blocks(n);
    void *partials = nullptr;
    if (cudaMallocAsync(&partials, sizeof(double2) * (size_t)nblk * nvec, s) != cudaSuccess) return DST_ERR_OOM;
    int rc = dst_k_project(n, nvec, (const double2 *)V, (const double2 *)w, (double2 *)h, (double2 *)partials, nblk, s);
    cudaError_t e = cudaFreeAsync(partials, s);
    if (rc != DST_OK) return rc;
    DST_CUDA_TRY(e);
    return DST_OK;
}

extern "C" int dst_arnoldi_update(int64_t n, int nvec, const void *V, const void *h, void *w, void *nrm2,
                                  void *stream) {
    if (n < 1 || nvec < 1 || nvec > DST_MAX_VEC || !V || !w || !h || !nrm2) return DST_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int nblk = dst_reduction_blocks(n);
    void *partials = nullptr;
    if (cudaMallocAsync(&partials, sizeof(double) * (size_t)nblk, s) != cudaSuccess) return DST_ERR_OOM;
    int rc = dst_k_update(n, nvec, (const double2 *)V, (const double2 *)h, (double2 *)w, (double *)nrm2,
                          (double *)partials, nblk, s);
    cudaError_t e = cudaFreeAsync(partials, s);
    if (rc != DST_OK) return rc;
    DST_CUDA_TRY(e);
    return DST_OK;
}
