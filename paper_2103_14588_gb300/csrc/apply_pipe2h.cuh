// 2+1 FP32 operator apply with two threads per output node, one spinor
// component each (meshes without an open axis; potential depending on x only,
// or none).
//
// Same operator, tiles and arithmetic per component as the pipelined kernel
// of apply_pipe.cuh (Appendix A's element matrices summed into [1,4,1] /
// [-1,0,1] tensor stencils; fields_std_rows; the two time stencils through
// running accumulators): a CTA owns a PipeTile<2, TV> output tile and its
// chunk of time layers, all staged in shared memory at once (the chunk's
// planes plus a halo plane on each side).  What changes is the work per
// thread.  The x and y stencils act on each component alone, and alpha =
// (sigma_x, sigma_y) couples the two components only through the convection
// fields, so thread h of a pair forms the fields of component h and takes its
// partner's two convection fields by lane shuffles.  Half the registers and
// twice the threads per CTA: the 2+1 plane of the bench workload (96^2 nodes)
// gives 432 CTAs, too few to hide shared-memory latency with one thread per
// node.
#pragma once

#include "apply_pipe.cuh"

namespace dst {

template <int TV>
struct Pipe2hShape {
    using Tile = PipeTile<2, TV>;
    static constexpr int TX = Tile::TX, TY = Tile::TY, TT = Tile::TT, RY = Tile::RY;
    static constexpr int BX = TX + 2, BY = TY + 2, BOX = BX * BY;
    static constexpr int NODE_BYTES = 16;                    // two FP32 complex components
    static constexpr int PLANES = TT + 2;                    // the whole chunk, resident at once
    static constexpr int NTHR = 2 * TX * (TY / RY);
    static constexpr int SMEM = PLANES * BOX * NODE_BYTES;
    static constexpr int PLAN = (BOX + NTHR - 1) / NTHR;     // box nodes copied per thread and plane
    static_assert(SMEM <= 56 * 1024, "the chunk must fit the shared-memory budget of four CTAs per SM");
};

template <int TV, bool NOV>
__global__ void __launch_bounds__(Pipe2hShape<TV>::NTHR, 3)
apply_pipe2h_kernel(OpParams p, const float2 *__restrict__ x, float2 *__restrict__ y, int64_t tiles_x) {
    using S = Pipe2hShape<TV>;
    constexpr int RY = S::RY;
    extern __shared__ __align__(16) char ring[];
    const int64_t tile = blockIdx.x, chunk = blockIdx.y;
    const int64_t x0 = (tile % tiles_x) * S::TX;
    const int64_t y0 = (tile / tiles_x) * S::TY;
    const int h = threadIdx.x & 1, col = threadIdx.x >> 1;
    const int tx = col % S::TX, ty = (col / S::TX) * RY;
    const int64_t ix = x0 + tx, iy = y0 + ty;
    const int64_t nx = p.ax[0].n, ny = p.ax[1].n;
    const int64_t N = p.nt;
    const int64_t t0 = 1 + chunk * S::TT;
    const int64_t t1 = min(t0 + (int64_t)S::TT, N + 1);
    const int nplanes = (int)(t1 - t0 + 2);
    const int64_t pfirst = t0 - 1;
    const int64_t plane_elems = nx * ny * 2;
    const size_t plane_bytes = (size_t)plane_elems * sizeof(float2);
    const int i_lo = (int)max((int64_t)0, 1 - pfirst);
    const int i_hi = (int)min((int64_t)(nplanes - 1), N - pfirst);
    const int i_last = (int)(N - pfirst);
    // every plane of the chunk in flight at once: box node b = threadIdx.x + j NTHR
    {
        int src[S::PLAN], dst[S::PLAN];
#pragma unroll
        for (int j = 0; j < S::PLAN; ++j) {
            const int b = threadIdx.x + j * S::NTHR;
            dst[j] = -1;
            src[j] = -1;
            if (b >= S::BOX) continue;
            const int64_t gx = axis_nbr(p.ax[0], x0 - 1 + b % S::BX);
            const int64_t gy = axis_nbr(p.ax[1], y0 - 1 + b / S::BX);
            dst[j] = b * S::NODE_BYTES;
            if (gx >= 0 && gy >= 0) src[j] = (int)((gy * nx + gx) * S::NODE_BYTES);
        }
        const char *layer = reinterpret_cast<const char *>(x) + (pfirst - 1) * (int64_t)plane_bytes;
        for (int i = 0; i < S::PLANES; ++i, layer += plane_bytes) {
            if (i < i_lo || i > i_hi) continue;
            char *slot = ring + (size_t)i * S::BOX * S::NODE_BYTES;
#pragma unroll
            for (int j = 0; j < S::PLAN; ++j)
                if (dst[j] >= 0) cp_async16(slot + dst[j], layer + (src[j] >= 0 ? src[j] : 0), src[j] >= 0);
        }
        cp_async_commit();
    }
    bool valid[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) valid[r] = ix < nx && iy + r < ny;
    const StdConst<float> sc = std_const<2, float>(p);
    // beta = +1 for component 0, -1 for component 1
    const float fm = h == 0 ? -(float)p.m * sc.km : (float)p.m * sc.km;
    float wa = 0.f, wb = 0.f;
    if (!NOV && valid[0]) {
        NodeCoef<2, float> k;
        node_coef<2, float>(p, ix, iy, 0, k);
        const float wl = h ? k.wl[1] : k.wl[0], wr = h ? k.wr[1] : k.wr[0];
        wa = -0.5f * sc.km * (wl + wr);
        wb = -0.5f * sc.km * (wr - wl);
    }
    const float ka1 = h == 0 ? sc.ka[1] : -sc.ka[1];
    char *ydst = reinterpret_cast<char *>(y + (t0 - 1) * plane_elems + (iy * nx + ix) * 2 + h);
    const size_t row_bytes = (size_t)nx * 2 * sizeof(float2);
    const int c0 = ty * S::BX + tx;                          // box node (x - 1, y - 1) of row 0
    float2 accP[RY], accC[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) { accP[r] = make_float2(0.f, 0.f); accC[r] = make_float2(0.f, 0.f); }
    // one wait and one barrier for the whole chunk (a barrier per plane, consuming
    // each plane as it lands, measured slower: 14.2 against 13.2 us at 96^2 x 96)
    cp_async_wait<0>();
    __syncthreads();
#pragma unroll
    for (int i = 0; i < S::PLANES; ++i) {
        if (i >= nplanes) break;
        const bool have = i >= i_lo && i <= i_hi;
        const char *slot = ring + (size_t)i * S::BOX * S::NODE_BYTES + 8 * h;
        float2 GC[RY], GM[RY];
        if (have) {
            float2 rM[RY + 2], rC[RY + 2];
#pragma unroll
            for (int q = 0; q < RY + 2; ++q) {
                const char *row = slot + (size_t)(c0 + q * S::BX) * S::NODE_BYTES;
                const float2 a0 = *reinterpret_cast<const float2 *>(row);
                const float2 a1 = *reinterpret_cast<const float2 *>(row + S::NODE_BYTES);
                const float2 a2 = *reinterpret_cast<const float2 *>(row + 2 * S::NODE_BYTES);
                rM[q].x = fmaf(4.f, a1.x, a0.x + a2.x); rM[q].y = fmaf(4.f, a1.y, a0.y + a2.y);
                rC[q].x = a2.x - a0.x; rC[q].y = a2.y - a0.y;
            }
            float2 PCx[RY], PCy[RY];
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                const float2 PM = cfma_r(4.f, rM[r + 1], cadd(rM[r], rM[r + 2]));
                PCx[r] = cfma_r(4.f, rC[r + 1], cadd(rC[r], rC[r + 2]));
                PCy[r] = csub(rM[r + 2], rM[r]);
                GC[r].x = -sc.kc * PM.y; GC[r].y = sc.kc * PM.x;
                GM[r] = NOV ? cmul_r(fm, PM) : cfma_r(wb, PCx[r], cmul_r(wa, PM));
            }
            // i alpha: component h takes the partner's convection fields,
            // sigma_x: + i ka0 Q_x; sigma_y: +- ka1 Q_y (+ for h = 0; see add_i_alpha)
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                float2 qx, qy;
                qx.x = __shfl_xor_sync(0xffffffffu, PCx[r].x, 1); qx.y = __shfl_xor_sync(0xffffffffu, PCx[r].y, 1);
                qy.x = __shfl_xor_sync(0xffffffffu, PCy[r].x, 1); qy.y = __shfl_xor_sync(0xffffffffu, PCy[r].y, 1);
                GM[r].x = fmaf(-sc.ka[0], qx.y, GM[r].x); GM[r].y = fmaf(sc.ka[0], qx.x, GM[r].y);
                GM[r].x = fmaf(ka1, qy.x, GM[r].x); GM[r].y = fmaf(ka1, qy.y, GM[r].y);
            }
        } else {
#pragma unroll
            for (int r = 0; r < RY; ++r) { GC[r] = make_float2(0.f, 0.f); GM[r] = make_float2(0.f, 0.f); }
        }
        // y(pl-1) += G_C' + G_M'; y(pl) += (pl < N ? 4 G_M' : G_C' + 2 G_M'); y(pl+1) = G_M' - G_C'
        const bool last = i >= i_last;
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            accP[r] = cadd(accP[r], cadd(GC[r], GM[r]));
            if (last) accC[r] = cadd(accC[r], cfma_r(2.f, GM[r], GC[r]));
            else accC[r] = cfma_r(4.f, GM[r], accC[r]);
            if (valid[r] && i >= 2) *reinterpret_cast<float2 *>(ydst + r * row_bytes) = accP[r];
            accP[r] = accC[r];
            accC[r] = csub(GM[r], GC[r]);
        }
        if (i >= 2) ydst += plane_bytes;
    }
}

template <int TV>
int launch_apply_pipe2h(const OpParams &p, const float2 *x, float2 *y, cudaStream_t s) {
    using S = Pipe2hShape<TV>;
    const int64_t tx = (p.ax[0].n + S::TX - 1) / S::TX;
    const int64_t ty = (p.ax[1].n + S::TY - 1) / S::TY;
    const int64_t chunks = (p.nt + S::TT - 1) / S::TT;
    const int64_t tiles = tx * ty;
    if (tiles <= 0 || tiles > 0x7fffffffLL || chunks > 65535) return DST_ERR_ARG;
    if (p.ax[0].n * p.ax[1].n * S::NODE_BYTES >= (1LL << 31)) return launch_apply<2, 2, float>(p, x, y, s);
    static bool configured[2][DST_MAX_DEVICES_APPLY] = {};
    int dev = 0;
    DST_CUDA_TRY(cudaGetDevice(&dev));
    const int nov = p.vmode == 2 ? 1 : 0;
    auto kern = nov ? apply_pipe2h_kernel<TV, true> : apply_pipe2h_kernel<TV, false>;
    if (dev < 0 || dev >= DST_MAX_DEVICES_APPLY || !configured[nov][dev]) {
        DST_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM));
        if (dev >= 0 && dev < DST_MAX_DEVICES_APPLY) configured[nov][dev] = true;
    }
    kern<<<dim3((unsigned)tiles, (unsigned)chunks), S::NTHR, S::SMEM, s>>>(p, x, y, tx);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

}  // namespace dst
