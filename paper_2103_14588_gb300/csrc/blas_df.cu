// Arnoldi kernels in double-FP32 ("df32") arithmetic for the mixed-precision
// solve.
//
// GB300 executes FP64 at 1/64 of its FP32 rate, so classical Gram-Schmidt in
// native FP64 is bound by the FP64 pipe long before HBM.  These kernels keep
// the Krylov basis of the FP32-apply GMRES cycles as pairs of FP32 planes,
// value = hi + lo (|lo| <= ulp(hi)/2), which carry a 48-bit significand - the
// same 16 bytes per complex entry as FP64 - and do the inner products and
// updates with error-free transformations on the FP32 pipes:
//   TwoProd(a, b): p = a*b, e = fma(a, b, -p)            (exact product, Dekker/FMA)
//   TwoSum(a, b):  s = a+b, e = (a-(s-bb)) + (b-bb)       (exact sum, Knuth)
// A df32 product (ah + al)(bh + bl) is p + (e + ah*bl + al*bh); sums run in a
// (hi, lo) accumulator (the "double-single" arithmetic of Dekker 1971 and the
// compensated dot product of Ogita, Rump & Oishi 2005).  Per-thread partial
// sums are reduced across the warp in df32 (shuffles of hi and lo), converted
// to FP64 once per warp and summed across warps and CTAs in FP64, in a fixed
// order (deterministic).
//
// Layout of a df32 complex vector of n entries: float2 hi[n] followed by
// float2 lo[n] (re, im interleaved in each plane).  The hi plane alone is the
// vector rounded to FP32 - the input the FP32 operator apply reads directly.
//
// A basis may instead be stored as the hi plane alone (8 bytes per complex
// entry, half the traffic; VL = false in the templates, project_f32_kernel
// and update_f32_kernel): the stored vectors are FP32 numbers, but the
// products are still exact (TwoProd) and the sums compensated, so inner
// products and updates keep FP64-class accuracy with respect to the stored
// values; updated vectors are rounded to FP32 once.
#include <algorithm>

#include "blas.h"
#include "df_arith.cuh"
#include "tma.cuh"

namespace dst {

static constexpr int DF_THREADS = 256;
static constexpr int DF_GROUP = 4;

// Slices start at even entries so that two neighbouring complex entries of
// a plane form one aligned 16-byte (float4) load; n is even for every mesh
// (NC = 2 or 4 components per node).
__device__ __forceinline__ void df_slice2(int64_t n, int64_t &b, int64_t &e) {
    int64_t per = (n + gridDim.x - 1) / gridDim.x;
    per += per & 1;
    b = (int64_t)blockIdx.x * per;
    e = b + per < n ? b + per : n;
}

// acc += conj(v) w for one complex entry, df32 (v = vh + vl, w = ah + al);
// VL / WL: whether v / w carry a lo plane
template <bool VL, bool WL>
__device__ __forceinline__ void cdot_acc(float vhr, float vhi, float vlr, float vli, float ar, float ai, float alr,
                                         float ali, DfAcc &re, DfAcc &im) {
    float p1, e1, p2, e2;
    df_prod_t<VL, WL>(vhr, vlr, ar, alr, p1, e1);
    df_prod_t<VL, WL>(vhi, vli, ai, ali, p2, e2);
    re.add(p1, e1);
    re.add(p2, e2);
    df_prod_t<VL, WL>(vhr, vlr, ai, ali, p1, e1);
    df_prod_t<VL, WL>(vhi, vli, ar, alr, p2, e2);
    im.add(p1, e1);
    im.add(-p2, -e2);
}

// h_j partials = sum conj(V_j) w over the CTA's slice; ||w||^2 partials.
// w_hi_only: w's lo plane is taken as zero (a fresh FP32 apply output).
// Each thread takes two neighbouring entries per step (float4 loads of both
// planes) and DF_GROUP basis vectors per sweep over its slice.
// The last CTA to finish (atomic ticket) sums every CTA's partials in CTA
// order and writes h (and ||w||^2): a deterministic single-kernel reduction.
template <bool W_HI_ONLY>
__global__ void __launch_bounds__(DF_THREADS)
project_df_kernel(int64_t n, int nvec, const float2 *__restrict__ V, const float2 *__restrict__ w,
                  double2 *__restrict__ partials, double *__restrict__ wnrm_partials, const double *gate,
                  double2 *__restrict__ h, double *__restrict__ wnrm2, unsigned *__restrict__ ticket) {
    if (gate != nullptr && !(gate[0] < 0.5 * gate[3])) {           // DGKS: no second pass needed
        if (blockIdx.x == 0)
            for (int j = threadIdx.x; j < nvec; j += DF_THREADS) h[j] = make_double2(0.0, 0.0);
        return;
    }
    constexpr int NW = DF_THREADS / 32;
    __shared__ double red[NW][2 * DST_MAX_VEC + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t b, e;
    df_slice2(n, b, e);
    const float4 *wh = reinterpret_cast<const float4 *>(w), *wl = reinterpret_cast<const float4 *>(w + n);
    DfAcc wn;
    wn.zero();
    for (int j0 = 0; j0 < nvec; j0 += DF_GROUP) {
        const int gv = nvec - j0 < DF_GROUP ? nvec - j0 : DF_GROUP;
        DfAcc re[DF_GROUP], im[DF_GROUP];
#pragma unroll
        for (int g = 0; g < DF_GROUP; ++g) { re[g].zero(); im[g].zero(); }
        for (int64_t i = b + 2 * threadIdx.x; i < e; i += 2 * DF_THREADS) {
            const int64_t q = i >> 1;
            const float4 a = wh[q];
            const float4 al = W_HI_ONLY ? make_float4(0.f, 0.f, 0.f, 0.f) : wl[q];
            float4 vh[DF_GROUP], vl[DF_GROUP];
#pragma unroll
            for (int g = 0; g < DF_GROUP; ++g) {
                if (g < gv) {
                    const float4 *vj = reinterpret_cast<const float4 *>(V + (int64_t)(j0 + g) * 2 * n);
                    vh[g] = vj[q];
                    vl[g] = vj[(n >> 1) + q];
                }
            }
            if (j0 == 0) {
                float p, r;
                df_prod_t<!W_HI_ONLY, !W_HI_ONLY>(a.x, al.x, a.x, al.x, p, r); wn.add(p, r);
                df_prod_t<!W_HI_ONLY, !W_HI_ONLY>(a.y, al.y, a.y, al.y, p, r); wn.add(p, r);
                df_prod_t<!W_HI_ONLY, !W_HI_ONLY>(a.z, al.z, a.z, al.z, p, r); wn.add(p, r);
                df_prod_t<!W_HI_ONLY, !W_HI_ONLY>(a.w, al.w, a.w, al.w, p, r); wn.add(p, r);
            }
#pragma unroll
            for (int g = 0; g < DF_GROUP; ++g) {
                if (g < gv) {
                    cdot_acc<true, !W_HI_ONLY>(vh[g].x, vh[g].y, vl[g].x, vl[g].y, a.x, a.y, al.x, al.y, re[g], im[g]);
                    cdot_acc<true, !W_HI_ONLY>(vh[g].z, vh[g].w, vl[g].z, vl[g].w, a.z, a.w, al.z, al.w, re[g], im[g]);
                }
            }
        }
#pragma unroll
        for (int g = 0; g < DF_GROUP; ++g) {
            if (g < gv) {
                const double sr = dfwarp_sum(re[g]), si = dfwarp_sum(im[g]);
                if (lane == 0) { red[warp][2 * (j0 + g)] = sr; red[warp][2 * (j0 + g) + 1] = si; }
            }
        }
    }
    const double wsum = dfwarp_sum(wn);
    if (lane == 0) red[warp][2 * DST_MAX_VEC] = wsum;
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * nvec; q += DF_THREADS) {
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
    // last CTA: final reduction over CTAs in CTA order
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // one warp per value: lanes stride over the CTAs, then a fixed shuffle tree
    const double *pd = reinterpret_cast<const double *>(partials);
    for (int q = warp; q < 2 * nvec + 1; q += NW) {
        double s_ = 0.0;
        if (q < 2 * nvec) {
            for (unsigned k = lane; k < gridDim.x; k += 32) s_ += __ldcg(pd + (size_t)k * 2 * nvec + q);
        } else if (wnrm2) {
            for (unsigned k = lane; k < gridDim.x; k += 32) s_ += __ldcg(wnrm_partials + k);
        }
        s_ = dwarp_sum(s_);
        if (lane == 0) {
            if (q < 2 * nvec) reinterpret_cast<double *>(h)[q] = s_;
            else if (wnrm2) *wnrm2 = s_;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *ticket = 0u;
}

// w <- w - sum_j V_j h_j in df32 (h given in FP64, split per CTA), and
// partials of ||w||^2 after the update.  W_HI_ONLY: w's lo plane is read as
// zero.  Two neighbouring entries per thread step, as in the projection.
template <bool W_HI_ONLY>
__global__ void __launch_bounds__(DF_THREADS)
update_df_kernel(int64_t n, int nvec, const float2 *__restrict__ V, const double2 *__restrict__ h,
                 float2 *__restrict__ w, double *__restrict__ nrm_partials, const double *gate,
                 double *__restrict__ nrm2, double *__restrict__ counter, unsigned *__restrict__ ticket) {
    if (gate != nullptr && !(gate[0] < 0.5 * gate[3])) return;     // DGKS: no second pass needed
    constexpr int NW = DF_THREADS / 32;
    __shared__ float4 hs[DST_MAX_VEC];     // (re_hi, re_lo, im_hi, im_lo)
    __shared__ double red[NW];
    for (int j = threadIdx.x; j < nvec; j += DF_THREADS) {
        const double2 c = h[j];
        const float rh = (float)c.x, ih = (float)c.y;
        hs[j] = make_float4(rh, (float)(c.x - (double)rh), ih, (float)(c.y - (double)ih));
    }
    __syncthreads();
    int64_t b, e;
    df_slice2(n, b, e);
    float4 *wh = reinterpret_cast<float4 *>(w), *wl = reinterpret_cast<float4 *>(w + n);
    DfAcc nr;
    nr.zero();
    for (int64_t i = b + 2 * threadIdx.x; i < e; i += 2 * DF_THREADS) {
        const int64_t q = i >> 1;
        const float4 a = wh[q];
        const float4 al = W_HI_ONLY ? make_float4(0.f, 0.f, 0.f, 0.f) : wl[q];
        DfAcc ar0, ai0, ar1, ai1;
        ar0.hi = a.x; ar0.lo = al.x; ai0.hi = a.y; ai0.lo = al.y;
        ar1.hi = a.z; ar1.lo = al.z; ai1.hi = a.w; ai1.lo = al.w;
        // software pipelining: the planes of V_{j+1} are loaded before V_j is combined
        const float4 *v0 = reinterpret_cast<const float4 *>(V);
        float4 vh = v0[q], vl = v0[(n >> 1) + q];
        for (int j = 0; j < nvec; ++j) {
            float4 nh = vh, nl = vl;
            if (j + 1 < nvec) {
                const float4 *vn = reinterpret_cast<const float4 *>(V + (int64_t)(j + 1) * 2 * n);
                nh = vn[q];
                nl = vn[(n >> 1) + q];
            }
            const float4 c = hs[j];
            caxpy_sub(vh.x, vh.y, vl.x, vl.y, c, ar0, ai0);
            caxpy_sub(vh.z, vh.w, vl.z, vl.w, c, ar1, ai1);
            vh = nh;
            vl = nl;
        }
        renorm(ar0); renorm(ai0); renorm(ar1); renorm(ai1);
        wh[q] = make_float4(ar0.hi, ai0.hi, ar1.hi, ai1.hi);
        wl[q] = make_float4(ar0.lo, ai0.lo, ar1.lo, ai1.lo);
        float p, r;
        df_prod(ar0.hi, ar0.lo, ar0.hi, ar0.lo, p, r); nr.add(p, r);
        df_prod(ai0.hi, ai0.lo, ai0.hi, ai0.lo, p, r); nr.add(p, r);
        df_prod(ar1.hi, ar1.lo, ar1.hi, ar1.lo, p, r); nr.add(p, r);
        df_prod(ai1.hi, ai1.lo, ai1.hi, ai1.lo, p, r); nr.add(p, r);
    }
    const double s_ = dfwarp_sum(nr);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s_;
    __syncthreads();
    if (!nrm_partials) return;
    if (threadIdx.x == 0) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < NW; ++k) t += red[k];
        nrm_partials[blockIdx.x] = t;
    }
    // last CTA: ||w||^2 = sum over CTAs in CTA order (and bump the pass counter)
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    double t = 0.0;
    for (unsigned k = threadIdx.x; k < gridDim.x; k += 32) t += __ldcg(nrm_partials + k);
    t = dwarp_sum(t);
    if (threadIdx.x == 0) {
        *nrm2 = t;
        if (counter) *counter += 1.0;
        *ticket = 0u;
    }
}

// h_j = conj(V_j) w for an FP32-stored unit-norm basis and FP32 w, plus
// ||w||^2; same slices, grouping and last-CTA reduction as project_df_kernel.
__global__ void __launch_bounds__(DF_THREADS)
project_f32_kernel(int64_t n, int nvec, const float2 *__restrict__ V, const float2 *__restrict__ w,
                   double2 *__restrict__ partials, double *__restrict__ wnrm_partials, const double *gate,
                   double2 *__restrict__ h, double *__restrict__ wnrm2, unsigned *__restrict__ ticket) {
    if (gate != nullptr && !(gate[0] < 0.5 * gate[3])) {           // DGKS: no second pass needed
        if (blockIdx.x == 0)
            for (int j = threadIdx.x; j < nvec; j += DF_THREADS) h[j] = make_double2(0.0, 0.0);
        return;
    }
    constexpr int NW = DF_THREADS / 32;
    __shared__ double red[NW][2 * DST_MAX_VEC + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t b, e;
    df_slice2(n, b, e);
    const float4 *wh = reinterpret_cast<const float4 *>(w);
    // the thread's entries once: ||w||^2 and the bound sum |w| (every partial
    // sum of conj(v) w over these entries is at most that in magnitude)
    DfAcc wn;
    wn.zero();
    float sw = 0.f;
    for (int64_t i = b + 2 * threadIdx.x; i < e; i += 2 * DF_THREADS) {
        const float4 a = wh[i >> 1];
        float p, r;
        p = a.x * a.x; r = fmaf(a.x, a.x, -p); wn.add(p, r);
        p = a.y * a.y; r = fmaf(a.y, a.y, -p); wn.add(p, r);
        p = a.z * a.z; r = fmaf(a.z, a.z, -p); wn.add(p, r);
        p = a.w * a.w; r = fmaf(a.w, a.w, -p); wn.add(p, r);
        sw += (fabsf(a.x) + fabsf(a.y)) + (fabsf(a.z) + fabsf(a.w));
    }
    const float sigma = anchor_above(sw);
    const int64_t ub = b >> 1, ue = e >> 1;      // the slice in float4 units (two entries each)
    for (int j0 = 0; j0 < nvec; j0 += DF_GROUP) {
        const int gv = nvec - j0 < DF_GROUP ? nvec - j0 : DF_GROUP;
        AnAcc re[DF_GROUP], im[DF_GROUP];
#pragma unroll
        for (int g = 0; g < DF_GROUP; ++g) { re[g].init(sigma); im[g].init(sigma); }
        // two float4 units per thread and step, DF_THREADS apart
        for (int64_t u = ub + threadIdx.x; u < ue; u += 2 * DF_THREADS) {
            const int64_t u1 = u + DF_THREADS;
            const bool two = u1 < ue;
            const float4 a0 = wh[u];
            const float4 a1 = two ? wh[u1] : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 v0h[DF_GROUP], v1h[DF_GROUP];
#pragma unroll
            for (int g = 0; g < DF_GROUP; ++g) {
                v0h[g] = make_float4(0.f, 0.f, 0.f, 0.f);
                v1h[g] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (g < gv) {
                    const float4 *vj = reinterpret_cast<const float4 *>(V + (int64_t)(j0 + g) * n);
                    v0h[g] = vj[u];
                    if (two) v1h[g] = vj[u1];
                }
            }
#pragma unroll
            for (int g = 0; g < DF_GROUP; ++g) {
                if (g < gv) {
                    cdot_an(v0h[g].x, v0h[g].y, a0.x, a0.y, re[g], im[g]);
                    cdot_an(v0h[g].z, v0h[g].w, a0.z, a0.w, re[g], im[g]);
                    cdot_an(v1h[g].x, v1h[g].y, a1.x, a1.y, re[g], im[g]);
                    cdot_an(v1h[g].z, v1h[g].w, a1.z, a1.w, re[g], im[g]);
                }
            }
        }
#pragma unroll
        for (int g = 0; g < DF_GROUP; ++g) {
            if (g < gv) {
                DfAcc r_, i_;
                r_.hi = re[g].hi - sigma; r_.lo = re[g].lo;      // exact differences
                i_.hi = im[g].hi - sigma; i_.lo = im[g].lo;
                const double sr = dfwarp_sum(r_), si = dfwarp_sum(i_);
                if (lane == 0) { red[warp][2 * (j0 + g)] = sr; red[warp][2 * (j0 + g) + 1] = si; }
            }
        }
    }
    const double wsum = dfwarp_sum(wn);
    if (lane == 0) red[warp][2 * DST_MAX_VEC] = wsum;
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * nvec; q += DF_THREADS) {
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
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const double *pd = reinterpret_cast<const double *>(partials);
    for (int q = warp; q < 2 * nvec + 1; q += NW) {
        double s_ = 0.0;
        if (q < 2 * nvec) {
            for (unsigned k = lane; k < gridDim.x; k += 32) s_ += __ldcg(pd + (size_t)k * 2 * nvec + q);
        } else if (wnrm2) {
            for (unsigned k = lane; k < gridDim.x; k += 32) s_ += __ldcg(wnrm_partials + k);
        }
        s_ = dwarp_sum(s_);
        if (lane == 0) {
            if (q < 2 * nvec) reinterpret_cast<double *>(h)[q] = s_;
            else if (wnrm2) *wnrm2 = s_;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *ticket = 0u;
}

// ---- FP32-stored basis, fed by bulk asynchronous copies --------------------
//
// The same projection as project_f32_kernel, but the basis and w reach shared
// memory through a ring of TMA_SLOTS 16 KB bulk copies completed on mbarriers:
// a producer warp keeps up to 96 KB per CTA in flight (two CTAs per SM),
// independent of the arithmetic, in contiguous 16 KB transfers, refilling a
// slot once all eight consumer warps have released it.  Each CTA owns one group
// of TMA_GROUP basis vectors over a contiguous slice of entries, cut into
// 2048-entry chunks; the copy sequence is, per chunk, the chunk of w and then
// the chunks of the group's vectors.  The CTAs of the groups of one slice are
// consecutive in the grid and run at the same time, so each chunk of w comes
// from HBM once and from L2 for the other groups (reducing every vector's chunk
// contribution over the warp instead, to read w once in one CTA, made the
// consumers the bottleneck).  Each chunk's contribution is accumulated in the
// anchored scheme with a bound taken from that chunk of w, then folded into a
// df32 per-thread sum.
constexpr int TMA_CHUNK = 2048;                 // entries per copy (16 KB)
constexpr int TMA_SLOTS = 6;                    // ring: 6 x 16 KB (two CTAs per SM)
constexpr int TMA_SMEM = TMA_SLOTS * TMA_CHUNK * 8;
constexpr unsigned TMA_WAIT_LIMIT = 1u << 22;   // try_wait attempts before a wait is declared failed
constexpr int TMA_GROUP = 8;                    // basis vectors per projection CTA (at most)

constexpr int TMA_THREADS = DF_THREADS + 32;   // eight consumer warps and one producer warp

// Failure handling.  A consumer warp that meets a failed wait (or sees that
// another warp failed) stops consuming at once: it neither reads nor releases
// that slot or any later one, and records how many copies it waited for.  A
// copy is issued into a slot only after every consumer warp has released the
// copy before it in that slot, and a warp releases only copies it waited for,
// so at exit the copies that may still be in flight are exactly those from the
// smallest completed-wait count over the consumer warps up to the last one
// issued - at most one per slot, each the latest phase of its slot's full
// mbarrier.  Thread 0 waits for each of them with the standard limit
// (whatever limit the consumers used) before the CTA touches its results or
// exits.  `wait_limit` bounds the consumers' and the producer's waits.
__global__ void __launch_bounds__(TMA_THREADS, 2)
project_tma_kernel(int64_t n, int nvec, const float2 *__restrict__ V, const float2 *__restrict__ w,
                   double2 *__restrict__ partials, const double *gate, double2 *__restrict__ h,
                   double *__restrict__ wnrm2, unsigned *__restrict__ ticket, double *err, unsigned wait_limit) {
    if (gate != nullptr && !(gate[0] < 0.5 * gate[3])) {           // DGKS: no second pass needed
        if (blockIdx.x == 0)
            for (int j = threadIdx.x; j < nvec; j += TMA_THREADS) h[j] = make_double2(0.0, 0.0);
        return;
    }
    constexpr int NW = DF_THREADS / 32;              // consumer warps
    constexpr int U = TMA_CHUNK / 2;                 // float4 units (two entries) per chunk
    constexpr int UPT = U / DF_THREADS;              // units per consumer thread per chunk
    extern __shared__ __align__(128) float4 ring[];  // TMA_SLOTS x U
    __shared__ __align__(8) uint64_t full[TMA_SLOTS], empty[TMA_SLOTS];
    __shared__ double red[NW][2 * TMA_GROUP + 1];
    __shared__ int failed, s_issued, s_done[NW];
    volatile int *vfailed = &failed;                 // polled across warps
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // CTA = (slice, group): the ngr CTAs of a slice are consecutive, so they stream the
    // slice's chunks of w at the same time and all but one read them from L2
    const int ngr = (nvec + TMA_GROUP - 1) / TMA_GROUP;
    const int nsl = (int)gridDim.x / ngr;
    const int slice = (int)blockIdx.x / ngr, grp = (int)blockIdx.x % ngr;
    // groups as even as possible (sizes differ by one at most), so that the CTAs of a
    // slice move through its chunks at the same pace
    const int j0 = grp * nvec / ngr, gv = (grp + 1) * nvec / ngr - j0;
    int64_t b, e;
    {
        int64_t per = (n + nsl - 1) / nsl;
        per += per & 1;
        b = (int64_t)slice * per;
        e = b + per < n ? b + per : n;
    }
    const int64_t len = e > b ? e - b : 0;
    const int nch = (int)((len + TMA_CHUNK - 1) / TMA_CHUNK);
    const int K = nch * (1 + gv);                    // copies this CTA consumes
    if (tid == 0) {
        for (int q = 0; q < TMA_SLOTS; ++q) {
            mbar_init(&full[q], 1);                  // the producer's arrival + the copy's bytes
            mbar_init(&empty[q], NW);                // one arrival per consumer warp
        }
        failed = 0;
        s_issued = 0;
        for (int q = 0; q < NW; ++q) s_done[q] = 0;
        mbar_fence_init();
    }
    __syncthreads();
    DfAcc wn;
    wn.zero();
    if (warp == NW) {
        // producer warp: lane 0 issues the copies in consumption order, refilling a
        // slot once every consumer warp has released it
        if (lane == 0) {
            int pc = 0, pq = 0, k = 0;
            for (; k < K && !*vfailed; ++k) {
                const int slot = k % TMA_SLOTS;
                if (k >= TMA_SLOTS &&
                    !mbar_wait_bounded(&empty[slot], (unsigned)(((k / TMA_SLOTS) - 1) & 1), wait_limit)) {
                    *vfailed = 1;
                    break;
                }
                const int64_t c0 = b + (int64_t)pc * TMA_CHUNK;
                const int64_t cnt = e - c0 < TMA_CHUNK ? e - c0 : TMA_CHUNK;
                const float2 *src = pq == 0 ? w + c0 : V + (int64_t)(j0 + pq - 1) * n + c0;
                const unsigned bytes = (unsigned)(cnt * (int64_t)sizeof(float2));
                mbar_arrive_expect_tx(&full[slot], bytes);
                bulk_g2s(ring + (size_t)slot * U, src, bytes, &full[slot]);
                if (++pq > gv) { pq = 0; ++pc; }
            }
            s_issued = k;
        }
    } else {
        int k = 0;                                   // copies this warp waited for (and released)
        // warp-uniform: the slot of copy k, or nullptr once a wait failed here or elsewhere
        auto wait_item = [&]() -> const float4 * {
            const int slot = k % TMA_SLOTS;
            bool ok = __shfl_sync(0xffffffffu, *vfailed == 0 ? 1 : 0, 0) != 0;
            if (ok) ok = mbar_wait_bounded(&full[slot], (unsigned)((k / TMA_SLOTS) & 1), wait_limit);
            ok = __all_sync(0xffffffffu, ok) != 0;
            if (!ok) {
                if (lane == 0) *vfailed = 1;
                return nullptr;
            }
            return (const float4 *)(ring + (size_t)slot * U);
        };
        auto release_item = [&]() {
            __syncwarp();                            // the warp is done with slot k
            if (lane == 0) mbar_arrive(&empty[k % TMA_SLOTS]);
            ++k;
        };
        bool stop = false;
        {
            const int g = grp;
            DfAcc R[TMA_GROUP], I[TMA_GROUP];
#pragma unroll
            for (int q = 0; q < TMA_GROUP; ++q) { R[q].zero(); I[q].zero(); }
            for (int c = 0; c < nch && !stop; ++c) {
                const int64_t c0 = b + (int64_t)c * TMA_CHUNK;
                const int units = (int)(((e - c0 < TMA_CHUNK) ? e - c0 : TMA_CHUNK) >> 1);
                float4 a[UPT];
                float bound = 0.f;
                {
                    const float4 *sw4 = wait_item();
                    if (!sw4) { stop = true; break; }
#pragma unroll
                    for (int i = 0; i < UPT; ++i) {
                        const int u = tid + i * DF_THREADS;
                        a[i] = u < units ? sw4[u] : make_float4(0.f, 0.f, 0.f, 0.f);
                        bound += (fabsf(a[i].x) + fabsf(a[i].y)) + (fabsf(a[i].z) + fabsf(a[i].w));
                        if (g == 0) {                    // ||w||^2: the first group's CTA of the slice
                            float p, r;
                            p = a[i].x * a[i].x; r = fmaf(a[i].x, a[i].x, -p); wn.add(p, r);
                            p = a[i].y * a[i].y; r = fmaf(a[i].y, a[i].y, -p); wn.add(p, r);
                            p = a[i].z * a[i].z; r = fmaf(a[i].z, a[i].z, -p); wn.add(p, r);
                            p = a[i].w * a[i].w; r = fmaf(a[i].w, a[i].w, -p); wn.add(p, r);
                        }
                    }
                    release_item();
                }
                const float sigma = anchor_above(bound);
#pragma unroll
                for (int q = 0; q < TMA_GROUP; ++q) {
                    if (q >= gv) break;
                    const float4 *sv = wait_item();
                    if (!sv) { stop = true; break; }
                    AnAcc re, im;
                    re.init(sigma);
                    im.init(sigma);
#pragma unroll
                    for (int i = 0; i < UPT; ++i) {
                        const int u = tid + i * DF_THREADS;
                        if (u < units) {
                            const float4 v = sv[u];
                            cdot_an(v.x, v.y, a[i].x, a[i].y, re, im);
                            cdot_an(v.z, v.w, a[i].z, a[i].w, re, im);
                        }
                    }
                    df_add(R[q].hi, R[q].lo, re.hi - sigma, re.lo);
                    df_add(I[q].hi, I[q].lo, im.hi - sigma, im.lo);
                    release_item();
                }
            }
#pragma unroll
            for (int q = 0; q < TMA_GROUP; ++q) {
                if (q < gv && !stop) {
                    const double sr = dfwarp_sum(R[q]), si = dfwarp_sum(I[q]);
                    if (lane == 0) {
                        red[warp][2 * q] = sr;
                        red[warp][2 * q + 1] = si;
                    }
                }
            }
        }
        if (lane == 0) s_done[warp] = k;
    }
    __syncthreads();
    // after a failed wait: wait (standard limit) for every copy that may still be in flight
    if (tid == 0 && *vfailed) {
        int lo = s_done[0];
        for (int q = 1; q < NW; ++q) lo = s_done[q] < lo ? s_done[q] : lo;
        for (int q = lo; q < s_issued; ++q)
            mbar_wait_bounded(&full[q % TMA_SLOTS], (unsigned)((q / TMA_SLOTS) & 1), TMA_WAIT_LIMIT);
    }
    __syncthreads();
    // every issued copy was waited for by the consumers (or the producer stopped
    // issuing after a failed wait); the ring is idle here
    const double wsum = warp < NW ? dfwarp_sum(wn) : 0.0;
    if (lane == 0 && warp < NW) red[warp][2 * TMA_GROUP] = wsum;
    __syncthreads();
    if (*vfailed && tid == 0 && err) *err = 1.0;
    // partials [slice][nvec]: this CTA's group of coefficients of its slice
    for (int q = tid; q < 2 * gv; q += TMA_THREADS) {
        double s_ = 0.0;
#pragma unroll
        for (int kk = 0; kk < NW; ++kk) s_ += red[kk][q];
        reinterpret_cast<double *>(partials + (int64_t)slice * nvec + j0)[q] = s_;
    }
    // ||w||^2 partial of the slice goes after the coefficient partials of all slices
    double *wparts = reinterpret_cast<double *>(partials + (int64_t)nsl * nvec);
    if (tid == 0 && grp == 0) {
        double s_ = 0.0;
#pragma unroll
        for (int kk = 0; kk < NW; ++kk) s_ += red[kk][2 * TMA_GROUP];
        wparts[slice] = s_;
    }
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const double *pd = reinterpret_cast<const double *>(partials);
    for (int q = warp; q < 2 * nvec + 1; q += NW) {
        double s_ = 0.0;
        if (q < 2 * nvec) {
            for (int kk = lane; kk < nsl; kk += 32) s_ += __ldcg(pd + (size_t)kk * 2 * nvec + q);
        } else if (wnrm2) {
            for (int kk = lane; kk < nsl; kk += 32) s_ += __ldcg(wparts + kk);
        }
        s_ = dwarp_sum(s_);
        if (lane == 0) {
            if (q < 2 * nvec) reinterpret_cast<double *>(h)[q] = s_;
            else if (wnrm2) *wnrm2 = s_;
        }
    }
    __syncthreads();
    if (tid == 0) *ticket = 0u;
}

// The update w <- w - sum_j V_j h_j of update_f32_kernel (same per-entry
// arithmetic: anchor max |w component| + sum_j |h_j|_1, the vectors in order,
// rounded once), with the basis streamed through the bulk-copy ring of
// project_tma_kernel: per chunk of the CTA's slice the consumers read w from
// global memory into registers, take the chunks of all nvec vectors from the
// ring, and store the result with its norm.  w is read and written once, every
// basis vector read once.  Same failure handling as project_tma_kernel (a
// consumer that meets a failed wait stops; the copies in flight are waited
// for; *err = 1 and the chunks not reached keep their old w).
__global__ void __launch_bounds__(TMA_THREADS, 2)
update_tma_kernel(int64_t n, int nvec, const float2 *__restrict__ V, const double2 *__restrict__ h,
                  float2 *__restrict__ w, double *__restrict__ nrm_partials, const double *gate,
                  double *__restrict__ nrm2, double *__restrict__ counter, unsigned *__restrict__ ticket,
                  double *err, unsigned wait_limit) {
    if (gate != nullptr && !(gate[0] < 0.5 * gate[3])) return;     // DGKS: no second pass needed
    constexpr int NW = DF_THREADS / 32;
    constexpr int U = TMA_CHUNK / 2;
    constexpr int UPT = U / DF_THREADS;
    extern __shared__ __align__(128) float4 ring[];
    __shared__ __align__(8) uint64_t full[TMA_SLOTS], empty[TMA_SLOTS];
    __shared__ float4 hs[DST_MAX_VEC];
    __shared__ double red[NW];
    __shared__ float h1_sh;
    __shared__ int failed, s_issued, s_done[NW];
    volatile int *vfailed = &failed;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int64_t b, e;
    df_slice2(n, b, e);
    const int64_t len = e > b ? e - b : 0;
    const int nch = (int)((len + TMA_CHUNK - 1) / TMA_CHUNK);
    const int K = nch * nvec;
    for (int j = tid; j < nvec; j += TMA_THREADS) {
        const double2 c = h[j];
        const float rh = (float)c.x, ih = (float)c.y;
        hs[j] = make_float4(rh, (float)(c.x - (double)rh), ih, (float)(c.y - (double)ih));
    }
    if (warp == 0) {
        double t = 0.0;
        for (int j = lane; j < nvec; j += 32) t += fabs(h[j].x) + fabs(h[j].y);
        t = dwarp_sum(t);
        if (lane == 0) h1_sh = (float)t;
    }
    if (tid == 0) {
        for (int q = 0; q < TMA_SLOTS; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], NW);
        }
        failed = 0;
        s_issued = 0;
        for (int q = 0; q < NW; ++q) s_done[q] = 0;
        mbar_fence_init();
    }
    __syncthreads();
    DfAcc nr;
    nr.zero();
    if (warp == NW) {
        if (lane == 0) {
            int pc = 0, pq = 0, k = 0;
            for (; k < K && !*vfailed; ++k) {
                const int slot = k % TMA_SLOTS;
                if (k >= TMA_SLOTS &&
                    !mbar_wait_bounded(&empty[slot], (unsigned)(((k / TMA_SLOTS) - 1) & 1), wait_limit)) {
                    *vfailed = 1;
                    break;
                }
                const int64_t c0 = b + (int64_t)pc * TMA_CHUNK;
                const int64_t cnt = e - c0 < TMA_CHUNK ? e - c0 : TMA_CHUNK;
                const unsigned bytes = (unsigned)(cnt * (int64_t)sizeof(float2));
                mbar_arrive_expect_tx(&full[slot], bytes);
                bulk_g2s(ring + (size_t)slot * U, V + (int64_t)pq * n + c0, bytes, &full[slot]);
                if (++pq == nvec) { pq = 0; ++pc; }
            }
            s_issued = k;
        }
    } else {
        int k = 0;
        auto wait_item = [&]() -> const float4 * {
            const int slot = k % TMA_SLOTS;
            bool ok = __shfl_sync(0xffffffffu, *vfailed == 0 ? 1 : 0, 0) != 0;
            if (ok) ok = mbar_wait_bounded(&full[slot], (unsigned)((k / TMA_SLOTS) & 1), wait_limit);
            ok = __all_sync(0xffffffffu, ok) != 0;
            if (!ok) {
                if (lane == 0) *vfailed = 1;
                return nullptr;
            }
            return (const float4 *)(ring + (size_t)slot * U);
        };
        auto release_item = [&]() {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[k % TMA_SLOTS]);
            ++k;
        };
        const float h1 = h1_sh;
        float4 *w4 = reinterpret_cast<float4 *>(w);
        bool stop = false;
        for (int c = 0; c < nch && !stop; ++c) {
            const int64_t c0 = b + (int64_t)c * TMA_CHUNK;
            const int units = (int)(((e - c0 < TMA_CHUNK) ? e - c0 : TMA_CHUNK) >> 1);
            const int64_t g0 = c0 >> 1;                  // the chunk's first float4 of w
            float sg[UPT];
            AnAcc acc[UPT][4];
#pragma unroll
            for (int i = 0; i < UPT; ++i) {
                const int u = tid + i * DF_THREADS;
                const float4 a = u < units ? w4[g0 + u] : make_float4(0.f, 0.f, 0.f, 0.f);
                sg[i] = anchor_above(fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))) + h1);
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][q].init(sg[i]);
                acc[i][0].add(a.x); acc[i][1].add(a.y); acc[i][2].add(a.z); acc[i][3].add(a.w);
            }
            for (int j = 0; j < nvec; ++j) {
                const float4 *sv = wait_item();
                if (!sv) { stop = true; break; }
                const float4 cj = hs[j];
#pragma unroll
                for (int i = 0; i < UPT; ++i) {
                    const int u = tid + i * DF_THREADS;
                    if (u < units) {
                        const float4 v = sv[u];
                        caxpy_an(v.x, v.y, cj, acc[i][0], acc[i][1]);
                        caxpy_an(v.z, v.w, cj, acc[i][2], acc[i][3]);
                    }
                }
                release_item();
            }
            if (stop) break;
#pragma unroll
            for (int i = 0; i < UPT; ++i) {
                const int u = tid + i * DF_THREADS;
                if (u >= units) continue;
                const float4 o = make_float4((acc[i][0].hi - sg[i]) + acc[i][0].lo, (acc[i][1].hi - sg[i]) + acc[i][1].lo,
                                             (acc[i][2].hi - sg[i]) + acc[i][2].lo, (acc[i][3].hi - sg[i]) + acc[i][3].lo);
                w4[g0 + u] = o;
                float p, r;
                p = o.x * o.x; r = fmaf(o.x, o.x, -p); nr.add(p, r);
                p = o.y * o.y; r = fmaf(o.y, o.y, -p); nr.add(p, r);
                p = o.z * o.z; r = fmaf(o.z, o.z, -p); nr.add(p, r);
                p = o.w * o.w; r = fmaf(o.w, o.w, -p); nr.add(p, r);
            }
        }
        if (lane == 0) s_done[warp] = k;
    }
    __syncthreads();
    if (tid == 0 && *vfailed) {
        int lo = s_done[0];
        for (int q = 1; q < NW; ++q) lo = s_done[q] < lo ? s_done[q] : lo;
        for (int q = lo; q < s_issued; ++q)
            mbar_wait_bounded(&full[q % TMA_SLOTS], (unsigned)((q / TMA_SLOTS) & 1), TMA_WAIT_LIMIT);
    }
    __syncthreads();
    const double s_ = warp < NW ? dfwarp_sum(nr) : 0.0;
    if (lane == 0 && warp < NW) red[warp] = s_;
    __syncthreads();
    if (*vfailed && tid == 0 && err) *err = 1.0;
    if (!nrm_partials) return;
    if (tid == 0) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < NW; ++q) t += red[q];
        nrm_partials[blockIdx.x] = t;
    }
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last || tid >= 32) return;
    __threadfence();
    double t = 0.0;
    for (unsigned q = tid; q < gridDim.x; q += 32) t += __ldcg(nrm_partials + q);
    t = dwarp_sum(t);
    if (tid == 0) {
        *nrm2 = t;
        if (counter) *counter += 1.0;
        *ticket = 0u;
    }
}

// x (FP64) <- x + sum_j V_j y_j at the end of a cycle, with the FP32-stored
// basis streamed through the bulk-copy ring of project_tma_kernel: per chunk of
// the CTA's slice the consumers accumulate every vector's chunk as it lands, in
// the arithmetic of combine_df_kernel<false> per entry (df32 sum over the
// vectors in order, one conversion; bit for bit the same), then read, update
// and store the chunk of x.  Same failure handling as project_tma_kernel
// (*err = 1; the chunks not reached keep their old x).
__global__ void __launch_bounds__(TMA_THREADS, 2)
combine_tma_kernel(int64_t n, int k, const float2 *__restrict__ V, const double2 *__restrict__ y,
                   double2 *__restrict__ x, double *err, unsigned wait_limit) {
    constexpr int NW = DF_THREADS / 32;
    constexpr int U = TMA_CHUNK / 2;
    constexpr int UPT = U / DF_THREADS;
    extern __shared__ __align__(128) float4 ring[];
    __shared__ __align__(8) uint64_t full[TMA_SLOTS], empty[TMA_SLOTS];
    __shared__ float4 ys[DST_MAX_VEC];              // -y split: (re_hi, re_lo, im_hi, im_lo)
    __shared__ int failed, s_issued, s_done[NW];
    volatile int *vfailed = &failed;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int64_t b, e;
    df_slice2(n, b, e);
    const int64_t len = e > b ? e - b : 0;
    const int nch = (int)((len + TMA_CHUNK - 1) / TMA_CHUNK);
    const int K = nch * k;
    for (int j = tid; j < k; j += TMA_THREADS) {
        const double2 c = y[j];
        const float rh = (float)(-c.x), ih = (float)(-c.y);
        ys[j] = make_float4(rh, (float)(-c.x - (double)rh), ih, (float)(-c.y - (double)ih));
    }
    if (tid == 0) {
        for (int q = 0; q < TMA_SLOTS; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], NW);
        }
        failed = 0;
        s_issued = 0;
        for (int q = 0; q < NW; ++q) s_done[q] = 0;
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == NW) {
        if (lane == 0) {
            int pc = 0, pq = 0, kk = 0;
            for (; kk < K && !*vfailed; ++kk) {
                const int slot = kk % TMA_SLOTS;
                if (kk >= TMA_SLOTS &&
                    !mbar_wait_bounded(&empty[slot], (unsigned)(((kk / TMA_SLOTS) - 1) & 1), wait_limit)) {
                    *vfailed = 1;
                    break;
                }
                const int64_t c0 = b + (int64_t)pc * TMA_CHUNK;
                const int64_t cnt = e - c0 < TMA_CHUNK ? e - c0 : TMA_CHUNK;
                const unsigned bytes = (unsigned)(cnt * (int64_t)sizeof(float2));
                mbar_arrive_expect_tx(&full[slot], bytes);
                bulk_g2s(ring + (size_t)slot * U, V + (int64_t)pq * n + c0, bytes, &full[slot]);
                if (++pq == k) { pq = 0; ++pc; }
            }
            s_issued = kk;
        }
    } else {
        int q = 0;                                   // copies this warp waited for (and released)
        auto wait_item = [&]() -> const float4 * {
            const int slot = q % TMA_SLOTS;
            bool ok = __shfl_sync(0xffffffffu, *vfailed == 0 ? 1 : 0, 0) != 0;
            if (ok) ok = mbar_wait_bounded(&full[slot], (unsigned)((q / TMA_SLOTS) & 1), wait_limit);
            ok = __all_sync(0xffffffffu, ok) != 0;
            if (!ok) {
                if (lane == 0) *vfailed = 1;
                return nullptr;
            }
            return (const float4 *)(ring + (size_t)slot * U);
        };
        auto release_item = [&]() {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[q % TMA_SLOTS]);
            ++q;
        };
        bool stop = false;
        for (int c = 0; c < nch && !stop; ++c) {
            const int64_t c0 = b + (int64_t)c * TMA_CHUNK;
            const int units = (int)(((e - c0 < TMA_CHUNK) ? e - c0 : TMA_CHUNK) >> 1);
            DfAcc ar[UPT][2], ai[UPT][2];
#pragma unroll
            for (int i = 0; i < UPT; ++i)
#pragma unroll
                for (int t = 0; t < 2; ++t) { ar[i][t].zero(); ai[i][t].zero(); }
            for (int j = 0; j < k; ++j) {
                const float4 *sv = wait_item();
                if (!sv) { stop = true; break; }
                const float4 cj = ys[j];
#pragma unroll
                for (int i = 0; i < UPT; ++i) {
                    const int u = tid + i * DF_THREADS;
                    if (u < units) {
                        const float4 v = sv[u];
                        caxpy_sub<false>(v.x, v.y, 0.f, 0.f, cj, ar[i][0], ai[i][0]);
                        caxpy_sub<false>(v.z, v.w, 0.f, 0.f, cj, ar[i][1], ai[i][1]);
                    }
                }
                release_item();
            }
            if (stop) break;
#pragma unroll
            for (int i = 0; i < UPT; ++i) {
                const int u = tid + i * DF_THREADS;
                if (u >= units) continue;
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int64_t idx = c0 + 2 * (int64_t)u + t;
                    double2 acc = x[idx];
                    acc.x += ar[i][t].value();
                    acc.y += ai[i][t].value();
                    x[idx] = acc;
                }
            }
        }
        if (lane == 0) s_done[warp] = q;
    }
    __syncthreads();
    if (tid == 0 && *vfailed) {
        int lo = s_done[0];
        for (int w = 1; w < NW; ++w) lo = s_done[w] < lo ? s_done[w] : lo;
        for (int w = lo; w < s_issued; ++w)
            mbar_wait_bounded(&full[w % TMA_SLOTS], (unsigned)((w / TMA_SLOTS) & 1), TMA_WAIT_LIMIT);
        if (err) *err = 1.0;
    }
    __syncthreads();
}

// w <- w - sum_j V_j h_j for an FP32-stored unit-norm basis and FP32 w (h in
// FP64, split per CTA), rounded to FP32 once; partials of ||w||^2 of the
// stored result.  Per entry the bound is |w component| + sum_j |h_j|_1.
__global__ void __launch_bounds__(DF_THREADS)
update_f32_kernel(int64_t n, int nvec, const float2 *__restrict__ V, const double2 *__restrict__ h,
                  float2 *__restrict__ w, double *__restrict__ nrm_partials, const double *gate,
                  double *__restrict__ nrm2, double *__restrict__ counter, unsigned *__restrict__ ticket) {
    if (gate != nullptr && !(gate[0] < 0.5 * gate[3])) return;     // DGKS: no second pass needed
    constexpr int NW = DF_THREADS / 32;
    __shared__ float4 hs[DST_MAX_VEC];     // (re_hi, re_lo, im_hi, im_lo)
    __shared__ double red[NW];
    __shared__ float h1_sh;
    for (int j = threadIdx.x; j < nvec; j += DF_THREADS) {
        const double2 c = h[j];
        const float rh = (float)c.x, ih = (float)c.y;
        hs[j] = make_float4(rh, (float)(c.x - (double)rh), ih, (float)(c.y - (double)ih));
    }
    if (threadIdx.x < 32) {
        double t = 0.0;
        for (int j = threadIdx.x; j < nvec; j += 32) t += fabs(h[j].x) + fabs(h[j].y);
        t = dwarp_sum(t);
        if (threadIdx.x == 0) h1_sh = (float)t;
    }
    __syncthreads();
    const float h1 = h1_sh;
    int64_t b, e;
    df_slice2(n, b, e);
    float4 *wh = reinterpret_cast<float4 *>(w);
    const float4 *v0 = reinterpret_cast<const float4 *>(V);
    const int64_t vs = n >> 1;           // float4 per stored vector
    const int64_t ub = b >> 1, ue = (e + 1) >> 1;     // the slice in float4 units (two entries each)
    DfAcc nr;
    nr.zero();
    // two units per thread and step, DF_THREADS apart: two independent loads
    // of every basis vector in flight
    for (int64_t u = ub + threadIdx.x; u < ue; u += 2 * DF_THREADS) {
        const int64_t u1 = u + DF_THREADS;
        const bool two = u1 < ue;
        const float4 a0 = wh[u];
        const float4 a1 = two ? wh[u1] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float s0 =
            anchor_above(fmaxf(fmaxf(fabsf(a0.x), fabsf(a0.y)), fmaxf(fabsf(a0.z), fabsf(a0.w))) + h1);
        const float s1 =
            anchor_above(fmaxf(fmaxf(fabsf(a1.x), fabsf(a1.y)), fmaxf(fabsf(a1.z), fabsf(a1.w))) + h1);
        AnAcc acc[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) { acc[k].init(s0); acc[4 + k].init(s1); }
        acc[0].add(a0.x); acc[1].add(a0.y); acc[2].add(a0.z); acc[3].add(a0.w);
        acc[4].add(a1.x); acc[5].add(a1.y); acc[6].add(a1.z); acc[7].add(a1.w);
        float4 v0h = v0[u], v1h = two ? v0[u1] : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int j = 0; j < nvec; ++j) {
            float4 n0 = v0h, n1 = v1h;       // next vector in flight
            if (j + 1 < nvec) {
                const float4 *vn = v0 + (int64_t)(j + 1) * vs;
                n0 = vn[u];
                if (two) n1 = vn[u1];
            }
            const float4 c = hs[j];
            caxpy_an(v0h.x, v0h.y, c, acc[0], acc[1]);
            caxpy_an(v0h.z, v0h.w, c, acc[2], acc[3]);
            caxpy_an(v1h.x, v1h.y, c, acc[4], acc[5]);
            caxpy_an(v1h.z, v1h.w, c, acc[6], acc[7]);
            v0h = n0;
            v1h = n1;
        }
        const float4 o0 = make_float4((acc[0].hi - s0) + acc[0].lo, (acc[1].hi - s0) + acc[1].lo,
                                      (acc[2].hi - s0) + acc[2].lo, (acc[3].hi - s0) + acc[3].lo);
        const float4 o1 = make_float4((acc[4].hi - s1) + acc[4].lo, (acc[5].hi - s1) + acc[5].lo,
                                      (acc[6].hi - s1) + acc[6].lo, (acc[7].hi - s1) + acc[7].lo);
        wh[u] = o0;
        if (two) wh[u1] = o1;
        float p, r;
        p = o0.x * o0.x; r = fmaf(o0.x, o0.x, -p); nr.add(p, r);
        p = o0.y * o0.y; r = fmaf(o0.y, o0.y, -p); nr.add(p, r);
        p = o0.z * o0.z; r = fmaf(o0.z, o0.z, -p); nr.add(p, r);
        p = o0.w * o0.w; r = fmaf(o0.w, o0.w, -p); nr.add(p, r);
        if (two) {
            p = o1.x * o1.x; r = fmaf(o1.x, o1.x, -p); nr.add(p, r);
            p = o1.y * o1.y; r = fmaf(o1.y, o1.y, -p); nr.add(p, r);
            p = o1.z * o1.z; r = fmaf(o1.z, o1.z, -p); nr.add(p, r);
            p = o1.w * o1.w; r = fmaf(o1.w, o1.w, -p); nr.add(p, r);
        }
    }
    const double s_ = dfwarp_sum(nr);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s_;
    __syncthreads();
    if (!nrm_partials) return;
    if (threadIdx.x == 0) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < NW; ++k) t += red[k];
        nrm_partials[blockIdx.x] = t;
    }
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    double t = 0.0;
    for (unsigned k = threadIdx.x; k < gridDim.x; k += 32) t += __ldcg(nrm_partials + k);
    t = dwarp_sum(t);
    if (threadIdx.x == 0) {
        *nrm2 = t;
        if (counter) *counter += 1.0;
        *ticket = 0u;
    }
}

// v <- v / sqrt(*nrm2) in df32 (both planes; VL = false: the hi plane,
// rounded once to FP32).
template <bool VL>
__global__ void scale_df_kernel(int64_t n, float2 *__restrict__ v, const double *__restrict__ nrm2) {
    __shared__ float s_sh[2];     // split of 1/sqrt, once per CTA (FP64 division is slow here)
    if (threadIdx.x == 0) {
        const double sd = 1.0 / sqrt(*nrm2);
        s_sh[0] = (float)sd;
        s_sh[1] = (float)(sd - (double)s_sh[0]);
    }
    __syncthreads();
    const float sh = s_sh[0], sl = s_sh[1];
    float2 *vh = v, *vl = v + n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = vh[i], al = VL ? vl[i] : make_float2(0.f, 0.f);
        float p, e, s, t;
        df_prod(a.x, al.x, sh, sl, p, e);
        s = p + e; t = e - (s - p);
        float2 oh, ol;
        oh.x = s; ol.x = t;
        df_prod(a.y, al.y, sh, sl, p, e);
        s = p + e; t = e - (s - p);
        oh.y = s; ol.y = t;
        vh[i] = oh;
        if (VL) vl[i] = ol;
    }
}

// v <- v / sqrt(*nrm2) for an FP32-stored vector (the same compensated
// product as scale_df_kernel<false>, rounded once), two entries per 16-byte
// access, up to eight CTAs per SM, each computing the FP64 factor once.
__global__ void __launch_bounds__(256) scale_f32_kernel(int64_t n, float2 *__restrict__ v,
                                                        const double *__restrict__ nrm2) {
    __shared__ float s_sh[2];
    if (threadIdx.x == 0) {
        const double sd = 1.0 / sqrt(*nrm2);
        s_sh[0] = (float)sd;
        s_sh[1] = (float)(sd - (double)s_sh[0]);
    }
    __syncthreads();
    const float sh = s_sh[0], sl = s_sh[1];
    float4 *v4 = reinterpret_cast<float4 *>(v);
    const int64_t nu = n >> 1;
    auto sc = [&](float a) {
        float p, e;
        df_prod(a, 0.f, sh, sl, p, e);
        return p + e;
    };
    // four independent 16-byte loads in flight per thread
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; u + 3 * T < nu; u += 4 * T) {
        float4 a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = v4[u + k * T];
#pragma unroll
        for (int k = 0; k < 4; ++k) v4[u + k * T] = make_float4(sc(a[k].x), sc(a[k].y), sc(a[k].z), sc(a[k].w));
    }
    for (; u < nu; u += T) {
        const float4 a = v4[u];
        v4[u] = make_float4(sc(a.x), sc(a.y), sc(a.z), sc(a.w));
    }
}

// dst (df32) <- src (FP64) / sqrt(*nrm2): the restart vector of a cycle
// (VL = false: rounded to FP32).
template <bool VL>
__global__ void split_f64_df_kernel(int64_t n, const double2 *__restrict__ src, const double *__restrict__ nrm2,
                                    float2 *__restrict__ dst) {
    __shared__ double s_sh;
    if (threadIdx.x == 0) s_sh = 1.0 / sqrt(*nrm2);
    __syncthreads();
    const double sc = s_sh;
    float2 *dh = dst, *dl = dst + n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = src[i];
        const double xr = a.x * sc, xi = a.y * sc;
        const float hr = (float)xr, hi = (float)xi;
        dh[i] = make_float2(hr, hi);
        if (VL) dl[i] = make_float2((float)(xr - (double)hr), (float)(xi - (double)hi));
    }
}

// x (FP64) <- x + sum_j V_j y_j with V in df32 and y in FP64 (end of a
// cycle): the sum runs in df32 (y split once per CTA), one conversion per entry.
template <bool VL>
__global__ void __launch_bounds__(DF_THREADS)
combine_df_kernel(int64_t n, int k, const float2 *__restrict__ V, const double2 *__restrict__ y,
                  double2 *__restrict__ x) {
    __shared__ float4 ys[DST_MAX_VEC];    // -y split: (re_hi, re_lo, im_hi, im_lo)
    for (int j = threadIdx.x; j < k; j += DF_THREADS) {
        const double2 c = y[j];
        const float rh = (float)(-c.x), ih = (float)(-c.y);
        ys[j] = make_float4(rh, (float)(-c.x - (double)rh), ih, (float)(-c.y - (double)ih));
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        DfAcc ar, ai;
        ar.zero();
        ai.zero();
        for (int j = 0; j < k; ++j) {
            const float2 *vj = V + (int64_t)j * (VL ? 2 : 1) * n;
            const float2 vh = vj[i], vl = VL ? vj[n + i] : make_float2(0.f, 0.f);
            caxpy_sub<VL>(vh.x, vh.y, vl.x, vl.y, ys[j], ar, ai);     // acc -= v (-y) = acc + v y
        }
        double2 acc = x[i];
        acc.x += ar.value();
        acc.y += ai.value();
        x[i] = acc;
    }
}

}  // namespace dst

using namespace dst;

static unsigned df_stream_blocks(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

int dst_k_project_df(int64_t n, int nvec, const float2 *V, const float2 *w, bool w_hi_only, double2 *h,
                     double2 *partials, int nblk, cudaStream_t s, double *wnrm2, double *wnrm_partials,
                     const double *gate, unsigned *ticket, bool vlo) {
    if (n & 1) return DST_ERR_ARG;     // two entries per 16-byte load
    if (!vlo && !w_hi_only) return DST_ERR_ARG;     // an FP32-stored basis has no lo planes at all
    double *wp = wnrm2 ? wnrm_partials : nullptr;
    if (!vlo)
        project_f32_kernel<<<nblk, DF_THREADS, 0, s>>>(n, nvec, V, w, partials, wp, gate, h, wnrm2, ticket);
    else if (w_hi_only)
        project_df_kernel<true><<<nblk, DF_THREADS, 0, s>>>(n, nvec, V, w, partials, wp, gate, h, wnrm2, ticket);
    else
        project_df_kernel<false><<<nblk, DF_THREADS, 0, s>>>(n, nvec, V, w, partials, wp, gate, h, wnrm2, ticket);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_tma_projection_blocks(int64_t n) {
    int64_t b = (n + 2047) / 2048;
    if (b > 2 * 152) b = 2 * 152;
    return (int)(b < 1 ? 1 : b);
}

int dst_k_project_tma(int64_t n, int nvec, const float2 *V, const float2 *w, double2 *h, double2 *partials, int nblk,
                      cudaStream_t s, double *wnrm2, const double *gate, unsigned *ticket, double *err) {
    if (n & 1) return DST_ERR_ARG;
    static bool configured[64] = {};
    int dev = 0;
    DST_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        DST_CUDA_TRY(cudaFuncSetAttribute(project_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TMA_SMEM));
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    // nblk slices at most (the partials hold nblk x (nvec + 1)), one CTA per slice and group
    // of TMA_GROUP basis vectors, one wave of two CTAs per SM
    const int ngr = (nvec + TMA_GROUP - 1) / TMA_GROUP;
    int nsl = 2 * 152 / ngr;
    if (nsl > nblk) nsl = nblk;
    if (nsl < 1) nsl = 1;
    project_tma_kernel<<<nsl * ngr, TMA_THREADS, TMA_SMEM, s>>>(n, nvec, V, w, partials, gate, h, wnrm2, ticket, err,
                                                                dst_internal_wait_limit(TMA_WAIT_LIMIT));
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_update_tma(int64_t n, int nvec, const float2 *V, const double2 *h, float2 *w, double *nrm2,
                     double *partials, int nblk, cudaStream_t s, const double *gate, double *counter,
                     unsigned *ticket, double *err) {
    if (n & 1) return DST_ERR_ARG;
    static bool configured[64] = {};
    int dev = 0;
    DST_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        DST_CUDA_TRY(cudaFuncSetAttribute(update_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TMA_SMEM));
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    double *pp = nrm2 ? partials : nullptr;
    update_tma_kernel<<<nblk, TMA_THREADS, TMA_SMEM, s>>>(n, nvec, V, h, w, pp, gate, nrm2, counter, ticket, err,
                                                          dst_internal_wait_limit(TMA_WAIT_LIMIT));
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_combine_tma(int64_t n, int k, const float2 *V, const double2 *y, double2 *x, int nblk, cudaStream_t s,
                      double *err) {
    if (n & 1) return DST_ERR_ARG;
    if (k < 1) return DST_OK;
    static bool configured[64] = {};
    int dev = 0;
    DST_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        DST_CUDA_TRY(cudaFuncSetAttribute(combine_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TMA_SMEM));
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    combine_tma_kernel<<<nblk, TMA_THREADS, TMA_SMEM, s>>>(n, k, V, y, x, err,
                                                           dst_internal_wait_limit(TMA_WAIT_LIMIT));
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_update_df(int64_t n, int nvec, const float2 *V, const double2 *h, float2 *w, bool w_hi_only, double *nrm2,
                    double *partials, int nblk, cudaStream_t s, const double *gate, double *counter,
                    unsigned *ticket, bool vlo) {
    if (n & 1) return DST_ERR_ARG;
    if (!vlo && !w_hi_only) return DST_ERR_ARG;
    double *pp = nrm2 ? partials : nullptr;
    if (!vlo)
        update_f32_kernel<<<nblk, DF_THREADS, 0, s>>>(n, nvec, V, h, w, pp, gate, nrm2, counter, ticket);
    else if (w_hi_only)
        update_df_kernel<true><<<nblk, DF_THREADS, 0, s>>>(n, nvec, V, h, w, pp, gate, nrm2, counter, ticket);
    else
        update_df_kernel<false><<<nblk, DF_THREADS, 0, s>>>(n, nvec, V, h, w, pp, gate, nrm2, counter, ticket);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_scale_df(int64_t n, float2 *v, const double *nrm2, cudaStream_t s, bool vlo) {
    if (vlo) {
        scale_df_kernel<true><<<df_stream_blocks(n), 256, 0, s>>>(n, v, nrm2);
    } else {
        if (n & 1) return DST_ERR_ARG;          // two entries per 16-byte access
        int64_t b = (n / 2 + 1023) / 1024;
        if (b > 8 * 152) b = 8 * 152;
        scale_f32_kernel<<<(unsigned)(b < 1 ? 1 : b), 256, 0, s>>>(n, v, nrm2);
    }
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_split_f64_df(int64_t n, const double2 *src, const double *nrm2, float2 *dst, cudaStream_t s, bool vlo) {
    if (vlo) split_f64_df_kernel<true><<<df_stream_blocks(n), 256, 0, s>>>(n, src, nrm2, dst);
    else split_f64_df_kernel<false><<<df_stream_blocks(n), 256, 0, s>>>(n, src, nrm2, dst);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

int dst_k_combine_df(int64_t n, int k, const float2 *V, const double2 *y, double2 *x, cudaStream_t s, bool vlo) {
    if (vlo) combine_df_kernel<true><<<df_stream_blocks(n), DF_THREADS, 0, s>>>(n, k, V, y, x);
    else combine_df_kernel<false><<<df_stream_blocks(n), DF_THREADS, 0, s>>>(n, k, V, y, x);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

// ---- testing entry point: the Gram-Schmidt kernels of the mixed solve -----------

extern "C" int dst_testing_fp32_arnoldi(int mode, int64_t n, int nvec, const void *V, void *w, void *h, void *nrm2,
                                        void *stream) {
    if (mode < 0 || mode > 5 || n < 2 || (n & 1) || nvec < 1 || nvec > DST_MAX_VEC || !V || !w || !h ||
        ((mode == 2 || mode == 3) && !nrm2)) {
        dst_internal_set_error_detail("dst_testing_fp32_arnoldi: bad mode, size (n even >= 2, 1 <= nvec <= 64) "
                                      "or pointer");
        return DST_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nblk_reg = std::min(dst_reduction_blocks(n), 3 * 152);
    const int nblk = (mode == 1 || mode == 3 || mode == 5) ? dst_tma_projection_blocks(n)
                                                            : (mode == 2 ? dst_reduction_blocks(n) : nblk_reg);
    const size_t pbytes = sizeof(double2) * (size_t)nblk * (nvec + 1);
    char *scr = nullptr;
    if (cudaMallocAsync((void **)&scr, pbytes + 256 + 256, s) != cudaSuccess) {
        cudaGetLastError();
        return DST_ERR_OOM;
    }
    double2 *partials = (double2 *)scr;
    unsigned *ticket = (unsigned *)(scr + ((pbytes + 255) & ~(size_t)255));
    double *err = (double *)(ticket + 8);
    int rc = DST_OK;
    if (cudaMemsetAsync(ticket, 0, 64, s) != cudaSuccess) rc = DST_ERR_CUDA;
    if (rc == DST_OK) {
        if (mode == 0)
            rc = dst_k_project_df(n, nvec, (const float2 *)V, (const float2 *)w, true, (double2 *)h, partials, nblk, s,
                                  nullptr, nullptr, nullptr, ticket, false);
        else if (mode == 1)
            rc = dst_k_project_tma(n, nvec, (const float2 *)V, (const float2 *)w, (double2 *)h, partials, nblk, s,
                                   nullptr, nullptr, ticket, err);
        else if (mode == 2)
            rc = dst_k_update_df(n, nvec, (const float2 *)V, (const double2 *)h, (float2 *)w, true, (double *)nrm2,
                                 (double *)partials, nblk, s, nullptr, nullptr, ticket + 1, false);
        else if (mode == 3)
            rc = dst_k_update_tma(n, nvec, (const float2 *)V, (const double2 *)h, (float2 *)w, (double *)nrm2,
                                  (double *)partials, nblk, s, nullptr, nullptr, ticket + 1, err);
        else if (mode == 4)
            rc = dst_k_combine_df(n, nvec, (const float2 *)V, (const double2 *)h, (double2 *)w, s, false);
        else
            rc = dst_k_combine_tma(n, nvec, (const float2 *)V, (const double2 *)h, (double2 *)w, nblk, s, err);
    }
    double e = 0.0;
    if (rc == DST_OK && (mode == 1 || mode == 3 || mode == 5) &&
        (cudaMemcpyAsync(&e, err, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess))
        rc = DST_ERR_CUDA;
    cudaFreeAsync(scr, s);
    if (rc == DST_OK && e != 0.0) {
        dst_internal_set_error_detail("dst_testing_fp32_arnoldi: a bulk-copy wait timed out");
        rc = DST_ERR_CUDA;
    }
    return rc;
}
