// 3+1 operator apply with z-columns per thread (meshes whose nodes all have the
// standard interior stencils: periodic or Dirichlet axes; potential depending on
// x only, or none).
//
// Same operator as apply_pipe.cuh (Appendix A's element matrices summed into
// [1,4,1] / [-1,0,1] tensor stencils, combined with the spin matrices, then the
// two time stencils through running accumulators).  What changes is the work
// per thread: a thread owns RZ consecutive z outputs at one (x, y).  For each
// staged time plane it walks the RZ + 2 z-slices of its column once: per slice
// the x and y stencils of the 3 x 3 (x, y) neighbourhood give three fields
// (M_x M_y, C_x M_y, M_x C_y; the x-only potential needs no fourth, see
// fields_std), kept for the last three slices; when a slice
// arrives, the z stencils of the output below it are completed from the
// window.  Each staged node and each x-y stencil then serves up to three
// outputs instead of one: about half the shared-memory loads and
// floating-point work of one output per thread.
//
// Planes are staged by cp.async into a ring of shared-memory slots; the copy
// sources of the CTA's box (byte offset in a layer, -1 outside a Dirichlet wall)
// are computed once into a shared table.
#pragma once

#include "apply_pipe.cuh"

namespace dst {

template <typename T, int RZ>
struct ZblkShape {
    static constexpr int TX = 16, TY = 8, TT = 8;
    static constexpr int BX = TX + 2, BY = TY + 2, BZ = RZ + 2;
    static constexpr int BOX = BX * BY * BZ;
    static constexpr int NODE_BYTES = 4 * 2 * (int)sizeof(T);
    static constexpr int CHUNKS = NODE_BYTES / 16;
    static constexpr int NTHR = TX * TY;
    static constexpr int SLOT = BOX * NODE_BYTES;
    static constexpr int STAGES = 3 * SLOT <= 110 * 1024 ? 3 : 2;
    static constexpr int SMEM = STAGES * SLOT + BOX * (int)sizeof(int);
};

// The x-y fields of one z-slice for the thread's (x, y): unscaled sums
//   FM = [1,4,1]_y [1,4,1]_x,  FCx = [1,4,1]_y [-1,0,1]_x,  FCy = [-1,0,1]_y [1,4,1]_x.
template <typename T>
struct ZFields {
    typename C2<T>::type M[4], Cx[4], Cy[4];
};

template <typename T, typename Get>
__device__ __forceinline__ void zslice_fields(Get get, ZFields<T> &F) {
    using V = typename C2<T>::type;
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
        const NodeV<4, T> n0 = get(dy, 0), n1 = get(dy, 1), n2 = get(dy, 2);
        const T wy = dy == 1 ? (T)4 : (T)1;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const V x0 = n0.c[c], x1 = n1.c[c], x2 = n2.c[c];
            V rM, rC;
            rM.x = fma((T)4, x1.x, x0.x + x2.x); rM.y = fma((T)4, x1.y, x0.y + x2.y);
            rC.x = x2.x - x0.x; rC.y = x2.y - x0.y;
            if (dy == 0) {
                F.M[c] = rM; F.Cx[c] = rC; F.Cy[c].x = -rM.x; F.Cy[c].y = -rM.y;
            } else {
                F.M[c] = cfma_r(wy, rM, F.M[c]);
                F.Cx[c] = cfma_r(wy, rC, F.Cx[c]);
                if (dy == 2) F.Cy[c] = cadd(F.Cy[c], rM);
            }
        }
    }
}

// G_C' and G_M' (scaled as in apply_pipe.cuh) of the output whose z-slices are A, B, C.
// WV: G_M' = a QM + b QCx with the x-only potential weights of fields_std.
template <typename T, bool WV>
__device__ __forceinline__ void zcombine(const ZFields<T> &A, const ZFields<T> &Bf, const ZFields<T> &Cf,
                                         const StdConst<T> &sc, T m, const T (&wa)[2], const T (&wb)[2],
                                         typename C2<T>::type *GC, typename C2<T>::type *GM) {
    using V = typename C2<T>::type;
    V QCx[4], QCy[4], QCz[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        // (A + 4 B) + C: the association of the one-output-per-thread kernel, so that
        // FP64 results agree bit for bit between the two tile variants
        const V QM = cadd(cfma_r((T)4, Bf.M[c], A.M[c]), Cf.M[c]);
        QCx[c] = cadd(cfma_r((T)4, Bf.Cx[c], A.Cx[c]), Cf.Cx[c]);
        QCy[c] = cadd(cfma_r((T)4, Bf.Cy[c], A.Cy[c]), Cf.Cy[c]);
        QCz[c] = csub(Cf.M[c], A.M[c]);
        GC[c].x = -sc.kc * QM.y; GC[c].y = sc.kc * QM.x;
        if (WV) {
            const int sb = Beta<3>::s(c) > 0 ? 0 : 1;
            GM[c] = cfma_r(wb[sb], QCx[c], cmul_r(wa[sb], QM));
        } else {
            const T f = Beta<3>::s(c) > 0 ? -m * sc.km : m * sc.km;
            GM[c] = cmul_r(f, QM);
        }
    }
    add_i_alpha<4>(0, sc.ka[0], QCx, GM);
    add_i_alpha<4>(1, sc.ka[1], QCy, GM);
    add_i_alpha<4>(2, sc.ka[2], QCz, GM);
}

// The plane loop of one CTA.
template <typename T, int RZ, bool WV>
__device__ __forceinline__ void zblk_planes(const OpParams &p, const typename C2<T>::type *__restrict__ x,
                                            typename C2<T>::type *__restrict__ y, char *ring, const int *src_tab,
                                            int64_t x0, int64_t y0, int64_t z0, int64_t t0, int64_t t1,
                                            const StdConst<T> &sc, const T (&wa)[2], const T (&wb)[2]) {
    using V = typename C2<T>::type;
    using S = ZblkShape<T, RZ>;
    const int tx = threadIdx.x % S::TX, ty = threadIdx.x / S::TX;
    const int64_t ix = x0 + tx, iy = y0 + ty;
    const int64_t nx = p.ax[0].n, ny = p.ax[1].n, nz = p.ax[2].n;
    const int64_t N = p.nt;
    const bool colv = ix < nx && iy < ny;
    const int nplanes = (int)(t1 - t0 + 2);
    const int64_t pfirst = t0 - 1;
    const int64_t plane_elems = nx * ny * nz * 4;
    const size_t plane_bytes = (size_t)plane_elems * sizeof(V);
    const int i_lo = (int)max((int64_t)0, 1 - pfirst);
    const int i_hi = (int)min((int64_t)(nplanes - 1), N - pfirst);
    const int i_last = (int)(N - pfirst);
    const char *xsrc = reinterpret_cast<const char *>(x) + (pfirst - 1) * (int64_t)plane_bytes;
    int issue_slot = 0;
    const char *issue_src = xsrc;
    auto issue_next = [&](int i) {
        if (i >= i_lo && i <= i_hi) {
            char *slot = ring + (size_t)issue_slot * S::SLOT;
            for (int j = threadIdx.x; j < S::BOX * S::CHUNKS; j += S::NTHR) {
                const int node = j / S::CHUNKS, part = j % S::CHUNKS;
                const int so = src_tab[node];
                cp_async16(slot + node * S::NODE_BYTES + part * 16, issue_src + (so >= 0 ? so : 0) + part * 16, so >= 0);
            }
        }
        cp_async_commit();
        issue_src += plane_bytes;
        issue_slot = issue_slot + 1 == S::STAGES ? 0 : issue_slot + 1;
    };
    V accP[RZ][4], accC[RZ][4];
#pragma unroll
    for (int r = 0; r < RZ; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) { accP[r][c] = cz<V>(); accC[r][c] = cz<V>(); }
    const int64_t self = (z0 * ny + iy) * nx + ix;              // node of output 0 in a layer
    char *ydst = reinterpret_cast<char *>(y + (t0 - 1) * plane_elems + self * 4);
    const size_t zstride = (size_t)nx * ny * 4 * sizeof(V);
    const int cbase = ty * S::BX + tx;                           // box (x - 1, y - 1) of the column at bz = 0
    for (int i = 0; i < S::STAGES - 1; ++i) issue_next(i);
    int si = 0;
    for (int i = 0; i < nplanes; ++i) {
        cp_async_wait_n(S::STAGES - 2);
        __syncthreads();
        issue_next(i + S::STAGES - 1);
        const bool have = i >= i_lo && i <= i_hi;
        const char *slot = ring + (size_t)si * S::SLOT;
        si = si + 1 == S::STAGES ? 0 : si + 1;
        const bool last = i >= i_last;
        ZFields<T> F0, F1, F2;
#pragma unroll
        for (int bz = 0; bz < RZ + 2; ++bz) {
            ZFields<T> &F = (bz % 3 == 0) ? F0 : ((bz % 3 == 1) ? F1 : F2);
            if (have) {
                auto get = [&](int dy, int dx) { return smem_node<4, T>(slot, (bz * S::BY + dy) * S::BX + cbase + dx); };
                zslice_fields<T>(get, F);
            }
            if (bz >= 2) {
                const int r = bz - 2;
                V GC[4], GM[4];
                if (have) {
                    const ZFields<T> &A = ((bz - 2) % 3 == 0) ? F0 : (((bz - 2) % 3 == 1) ? F1 : F2);
                    const ZFields<T> &Bm = ((bz - 1) % 3 == 0) ? F0 : (((bz - 1) % 3 == 1) ? F1 : F2);
                    zcombine<T, WV>(A, Bm, F, sc, (T)p.m, wa, wb, GC, GM);
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) { GC[c] = cz<V>(); GM[c] = cz<V>(); }
                }
                // y(pl-1) += G_C' + G_M'; y(pl) += (pl < N ? 4 G_M' : G_C' + 2 G_M'); y(pl+1) = G_M' - G_C'
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    accP[r][c] = cadd(accP[r][c], cadd(GC[c], GM[c]));
                    if (last) accC[r][c] = cadd(accC[r][c], cfma_r((T)2, GM[c], GC[c]));
                    else accC[r][c] = cfma_r((T)4, GM[c], accC[r][c]);
                }
                if (colv && z0 + r < nz && i >= 2)
                    store_node<4, T>(reinterpret_cast<V *>(ydst + r * zstride), 0, accP[r]);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    accP[r][c] = accC[r][c];
                    accC[r][c] = csub(GM[c], GC[c]);
                }
            }
        }
        if (i >= 2) ydst += plane_bytes;
    }
    cp_async_wait<0>();
}

template <typename T, int RZ, bool NOV>
__global__ void __launch_bounds__(ZblkShape<T, RZ>::NTHR, 2)
apply_zblk_kernel(OpParams p, const typename C2<T>::type *__restrict__ x, typename C2<T>::type *__restrict__ y,
                  int64_t tiles_x, int64_t tiles_y) {
    using S = ZblkShape<T, RZ>;
    extern __shared__ __align__(16) char smz[];
    char *ring = smz;
    int *src_tab = reinterpret_cast<int *>(smz + S::STAGES * S::SLOT);
    const int64_t tile = blockIdx.x, chunk = blockIdx.y;
    const int64_t x0 = (tile % tiles_x) * S::TX;
    const int64_t y0 = ((tile / tiles_x) % tiles_y) * S::TY;
    const int64_t z0 = (tile / (tiles_x * tiles_y)) * RZ;
    const int tx = threadIdx.x % S::TX, ty = threadIdx.x / S::TX;
    const int64_t ix = x0 + tx, iy = y0 + ty;
    const int64_t nx = p.ax[0].n, ny = p.ax[1].n, nz = p.ax[2].n;
    const int64_t t0 = 1 + chunk * S::TT;
    const int64_t t1 = min(t0 + (int64_t)S::TT, p.nt + 1);
    // copy sources of the box, once per CTA
    for (int b = threadIdx.x; b < S::BOX; b += S::NTHR) {
        const int bx = b % S::BX, by = (b / S::BX) % S::BY, bz = b / (S::BX * S::BY);
        const int64_t gx = axis_nbr(p.ax[0], x0 - 1 + bx);
        const int64_t gy = axis_nbr(p.ax[1], y0 - 1 + by);
        const int64_t gz = axis_nbr(p.ax[2], z0 - 1 + bz);
        src_tab[b] = (gx >= 0 && gy >= 0 && gz >= 0) ? (int)(((gz * ny + gy) * nx + gx) * S::NODE_BYTES) : -1;
    }
    __syncthreads();
    const bool colv = ix < nx && iy < ny;
    const StdConst<T> sc = std_const<3, T>(p);
    T wa[2] = {(T)0, (T)0}, wb[2] = {(T)0, (T)0};
    if (!NOV && colv) {
        NodeCoef<3, T> k;
        node_coef<3, T>(p, ix, iy, z0 < nz ? z0 : 0, k);
        for (int sb = 0; sb < 2; ++sb) {
            wa[sb] = (T)(-0.5) * sc.km * (k.wl[sb] + k.wr[sb]);
            wb[sb] = (T)(-0.5) * sc.km * (k.wr[sb] - k.wl[sb]);
        }
    }
    zblk_planes<T, RZ, !NOV>(p, x, y, ring, src_tab, x0, y0, z0, t0, t1, sc, wa, wb);
}

// ---- FP32: two threads per column, each with two of the four spinor components ----
//
// The x, y and z stencils act on each spinor component alone; only the alpha
// matrices couple components, and alpha_k = [[0, sigma_k], [sigma_k, 0]] couples
// component pairs (0, 1) and (2, 3).  So thread h of a column (h = 0, 1) computes
// the fields of components 2h, 2h + 1 and takes the partner's three convection
// fields by lane shuffles (12 floats per output).  Half the registers per thread,
// twice the threads per CTA: twice the resident warps of the four-component kernel
// for the same shared-memory ring.  Same arithmetic, in the same order, per component.

struct ZFieldsH {
    float2 M[2], Cx[2], Cy[2];
};

template <typename Get>
__device__ __forceinline__ void zslice_fields_h(Get get, ZFieldsH &F) {
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
        const float4 n0 = get(dy, 0), n1 = get(dy, 1), n2 = get(dy, 2);
        const float wy = dy == 1 ? 4.f : 1.f;
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const float2 x0 = l ? make_float2(n0.z, n0.w) : make_float2(n0.x, n0.y);
            const float2 x1 = l ? make_float2(n1.z, n1.w) : make_float2(n1.x, n1.y);
            const float2 x2 = l ? make_float2(n2.z, n2.w) : make_float2(n2.x, n2.y);
            float2 rM, rC;
            rM.x = fmaf(4.f, x1.x, x0.x + x2.x); rM.y = fmaf(4.f, x1.y, x0.y + x2.y);
            rC.x = x2.x - x0.x; rC.y = x2.y - x0.y;
            if (dy == 0) {
                F.M[l] = rM; F.Cx[l] = rC; F.Cy[l].x = -rM.x; F.Cy[l].y = -rM.y;
            } else {
                F.M[l] = cfma_r(wy, rM, F.M[l]);
                F.Cx[l] = cfma_r(wy, rC, F.Cx[l]);
                if (dy == 2) F.Cy[l] = cadd(F.Cy[l], rM);
            }
        }
    }
}

// G_C', G_M' of the thread's two components (global 2h, 2h + 1); wa, wb (WV) or
// fm (the -beta m km factor) already carry the components' beta sign.
template <bool WV>
__device__ __forceinline__ void zcombine_h(const ZFieldsH &A, const ZFieldsH &Bf, const ZFieldsH &Cf,
                                           const StdConst<float> &sc, float fm, float wa, float wb,
                                           float2 (&GC)[2], float2 (&GM)[2]) {
    float2 QCx[2], QCy[2], QCz[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const float2 QM = cadd(cfma_r(4.f, Bf.M[l], A.M[l]), Cf.M[l]);
        QCx[l] = cadd(cfma_r(4.f, Bf.Cx[l], A.Cx[l]), Cf.Cx[l]);
        QCy[l] = cadd(cfma_r(4.f, Bf.Cy[l], A.Cy[l]), Cf.Cy[l]);
        QCz[l] = csub(Cf.M[l], A.M[l]);
        GC[l].x = -sc.kc * QM.y; GC[l].y = sc.kc * QM.x;
        GM[l] = WV ? cfma_r(wb, QCx[l], cmul_r(wa, QM)) : cmul_r(fm, QM);
    }
    // the partner's fields (its local components 0, 1)
    float2 PCx[2], PCy[2], PCz[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        PCx[l].x = __shfl_xor_sync(0xffffffffu, QCx[l].x, 1); PCx[l].y = __shfl_xor_sync(0xffffffffu, QCx[l].y, 1);
        PCy[l].x = __shfl_xor_sync(0xffffffffu, QCy[l].x, 1); PCy[l].y = __shfl_xor_sync(0xffffffffu, QCy[l].y, 1);
        PCz[l].x = __shfl_xor_sync(0xffffffffu, QCz[l].x, 1); PCz[l].y = __shfl_xor_sync(0xffffffffu, QCz[l].y, 1);
    }
    // i alpha_k: component l of this half takes the partner's component 1 - l (x: i s, y: +-s)
    // or l (z: +-i s), the sign - for l = 1 (see add_i_alpha)
    auto addi = [](float2 &g, float2 a, float f) { g.x = fmaf(-f, a.y, g.x); g.y = fmaf(f, a.x, g.y); };
    addi(GM[0], PCx[1], sc.ka[0]); addi(GM[1], PCx[0], sc.ka[0]);
    GM[0].x = fmaf(sc.ka[1], PCy[1].x, GM[0].x); GM[0].y = fmaf(sc.ka[1], PCy[1].y, GM[0].y);
    GM[1].x = fmaf(-sc.ka[1], PCy[0].x, GM[1].x); GM[1].y = fmaf(-sc.ka[1], PCy[0].y, GM[1].y);
    addi(GM[0], PCz[0], sc.ka[2]); addi(GM[1], PCz[1], -sc.ka[2]);
}

template <int RZ, bool NOV>
__global__ void __launch_bounds__(2 * ZblkShape<float, RZ>::NTHR, 2)
apply_zblk_h_kernel(OpParams p, const float2 *__restrict__ x, float2 *__restrict__ y, int64_t tiles_x,
                    int64_t tiles_y) {
    using S = ZblkShape<float, RZ>;
    constexpr int NT = 2 * S::NTHR;
    extern __shared__ __align__(16) char smz[];
    char *ring = smz;
    int *src_tab = reinterpret_cast<int *>(smz + S::STAGES * S::SLOT);
    const int64_t tile = blockIdx.x, chunk = blockIdx.y;
    const int64_t x0 = (tile % tiles_x) * S::TX;
    const int64_t y0 = ((tile / tiles_x) % tiles_y) * S::TY;
    const int64_t z0 = (tile / (tiles_x * tiles_y)) * RZ;
    const int h = threadIdx.x & 1, col = threadIdx.x >> 1;
    const int tx = col % S::TX, ty = col / S::TX;
    const int64_t ix = x0 + tx, iy = y0 + ty;
    const int64_t nx = p.ax[0].n, ny = p.ax[1].n, nz = p.ax[2].n;
    const int64_t N = p.nt;
    const int64_t t0 = 1 + chunk * S::TT;
    const int64_t t1 = min(t0 + (int64_t)S::TT, N + 1);
    for (int b = threadIdx.x; b < S::BOX; b += NT) {
        const int bx = b % S::BX, by = (b / S::BX) % S::BY, bz = b / (S::BX * S::BY);
        const int64_t gx = axis_nbr(p.ax[0], x0 - 1 + bx);
        const int64_t gy = axis_nbr(p.ax[1], y0 - 1 + by);
        const int64_t gz = axis_nbr(p.ax[2], z0 - 1 + bz);
        src_tab[b] = (gx >= 0 && gy >= 0 && gz >= 0) ? (int)(((gz * ny + gy) * nx + gx) * S::NODE_BYTES) : -1;
    }
    __syncthreads();
    const bool colv = ix < nx && iy < ny;
    const StdConst<float> sc = std_const<3, float>(p);
    // beta = +1 for components 0, 1 (h = 0), -1 for 2, 3
    const float fm = h == 0 ? -(float)p.m * sc.km : (float)p.m * sc.km;
    float wa = 0.f, wb = 0.f;
    if (!NOV && colv) {
        NodeCoef<3, float> k;
        node_coef<3, float>(p, ix, iy, z0 < nz ? z0 : 0, k);
        const float wl = h ? k.wl[1] : k.wl[0], wr = h ? k.wr[1] : k.wr[0];
        wa = -0.5f * sc.km * (wl + wr);
        wb = -0.5f * sc.km * (wr - wl);
    }
    const int nplanes = (int)(t1 - t0 + 2);
    const int64_t pfirst = t0 - 1;
    const int64_t plane_elems = nx * ny * nz * 4;
    const size_t plane_bytes = (size_t)plane_elems * sizeof(float2);
    const int i_lo = (int)max((int64_t)0, 1 - pfirst);
    const int i_hi = (int)min((int64_t)(nplanes - 1), N - pfirst);
    const int i_last = (int)(N - pfirst);
    const char *issue_src = reinterpret_cast<const char *>(x) + (pfirst - 1) * (int64_t)plane_bytes;
    int issue_slot = 0;
    auto issue_next = [&](int i) {
        if (i >= i_lo && i <= i_hi) {
            char *slot = ring + (size_t)issue_slot * S::SLOT;
            for (int j = threadIdx.x; j < S::BOX * S::CHUNKS; j += NT) {
                const int node = j / S::CHUNKS, part = j % S::CHUNKS;
                const int so = src_tab[node];
                cp_async16(slot + node * S::NODE_BYTES + part * 16, issue_src + (so >= 0 ? so : 0) + part * 16, so >= 0);
            }
        }
        cp_async_commit();
        issue_src += plane_bytes;
        issue_slot = issue_slot + 1 == S::STAGES ? 0 : issue_slot + 1;
    };
    float2 accP[RZ][2], accC[RZ][2];
#pragma unroll
    for (int r = 0; r < RZ; ++r)
#pragma unroll
        for (int l = 0; l < 2; ++l) { accP[r][l] = make_float2(0.f, 0.f); accC[r][l] = make_float2(0.f, 0.f); }
    const int64_t self = (z0 * ny + iy) * nx + ix;
    char *ydst = reinterpret_cast<char *>(y + (t0 - 1) * plane_elems + self * 4 + 2 * h);
    const size_t zstride = (size_t)nx * ny * 4 * sizeof(float2);
    const int cbase = ty * S::BX + tx;
    for (int i = 0; i < S::STAGES - 1; ++i) issue_next(i);
    int si = 0;
    for (int i = 0; i < nplanes; ++i) {
        cp_async_wait_n(S::STAGES - 2);
        __syncthreads();
        issue_next(i + S::STAGES - 1);
        const bool have = i >= i_lo && i <= i_hi;
        const char *slot = ring + (size_t)si * S::SLOT + 16 * h;
        si = si + 1 == S::STAGES ? 0 : si + 1;
        const bool last = i >= i_last;
        ZFieldsH F0, F1, F2;
#pragma unroll
        for (int bz = 0; bz < RZ + 2; ++bz) {
            ZFieldsH &F = (bz % 3 == 0) ? F0 : ((bz % 3 == 1) ? F1 : F2);
            if (have) {
                auto get = [&](int dy, int dx) {
                    return *reinterpret_cast<const float4 *>(slot + ((bz * S::BY + dy) * S::BX + cbase + dx) * S::NODE_BYTES);
                };
                zslice_fields_h(get, F);
            }
            if (bz >= 2) {
                const int r = bz - 2;
                float2 GC[2], GM[2];
                if (have) {
                    const ZFieldsH &A = ((bz - 2) % 3 == 0) ? F0 : (((bz - 2) % 3 == 1) ? F1 : F2);
                    const ZFieldsH &Bm = ((bz - 1) % 3 == 0) ? F0 : (((bz - 1) % 3 == 1) ? F1 : F2);
                    zcombine_h<!NOV>(A, Bm, F, sc, fm, wa, wb, GC, GM);
                } else {
#pragma unroll
                    for (int l = 0; l < 2; ++l) { GC[l] = make_float2(0.f, 0.f); GM[l] = make_float2(0.f, 0.f); }
                }
#pragma unroll
                for (int l = 0; l < 2; ++l) {
                    accP[r][l] = cadd(accP[r][l], cadd(GC[l], GM[l]));
                    if (last) accC[r][l] = cadd(accC[r][l], cfma_r(2.f, GM[l], GC[l]));
                    else accC[r][l] = cfma_r(4.f, GM[l], accC[r][l]);
                }
                if (colv && z0 + r < nz && i >= 2)
                    *reinterpret_cast<float4 *>(ydst + r * zstride) =
                        make_float4(accP[r][0].x, accP[r][0].y, accP[r][1].x, accP[r][1].y);
#pragma unroll
                for (int l = 0; l < 2; ++l) {
                    accP[r][l] = accC[r][l];
                    accC[r][l] = csub(GM[l], GC[l]);
                }
            }
        }
        if (i >= 2) ydst += plane_bytes;
    }
    cp_async_wait<0>();
}

template <typename T, int RZ>
int launch_apply_zblk(const OpParams &p, const typename C2<T>::type *x, typename C2<T>::type *y, cudaStream_t s) {
    using S = ZblkShape<T, RZ>;
    const int64_t tx = (p.ax[0].n + S::TX - 1) / S::TX;
    const int64_t ty = (p.ax[1].n + S::TY - 1) / S::TY;
    const int64_t tz = (p.ax[2].n + RZ - 1) / RZ;
    const int64_t chunks = (p.nt + S::TT - 1) / S::TT;
    const int64_t tiles = tx * ty * tz;
    if (tiles <= 0 || tiles > 0x7fffffffLL || chunks > 65535) return DST_ERR_ARG;
    if (p.ax[0].n * p.ax[1].n * p.ax[2].n * S::NODE_BYTES >= (1LL << 31)) return launch_apply<3, 4, T>(p, x, y, s);
    static bool configured[2][DST_MAX_DEVICES_APPLY] = {};
    int dev = 0;
    DST_CUDA_TRY(cudaGetDevice(&dev));
    const int nov = p.vmode == 2 ? 1 : 0;
    if constexpr (sizeof(T) == 4) {
        // two threads per column (ZFieldsH)
        auto kern = nov ? apply_zblk_h_kernel<RZ, true> : apply_zblk_h_kernel<RZ, false>;
        if (dev < 0 || dev >= DST_MAX_DEVICES_APPLY || !configured[nov][dev]) {
            DST_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM));
            if (dev >= 0 && dev < DST_MAX_DEVICES_APPLY) configured[nov][dev] = true;
        }
        kern<<<dim3((unsigned)tiles, (unsigned)chunks), 2 * S::NTHR, S::SMEM, s>>>(p, x, y, tx, ty);
    } else {
        auto kern = nov ? apply_zblk_kernel<T, RZ, true> : apply_zblk_kernel<T, RZ, false>;
        if (dev < 0 || dev >= DST_MAX_DEVICES_APPLY || !configured[nov][dev]) {
            DST_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM));
            if (dev >= 0 && dev < DST_MAX_DEVICES_APPLY) configured[nov][dev] = true;
        }
        kern<<<dim3((unsigned)tiles, (unsigned)chunks), S::NTHR, S::SMEM, s>>>(p, x, y, tx, ty);
    }
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

}  // namespace dst
