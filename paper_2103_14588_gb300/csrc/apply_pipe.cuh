// Pipelined operator apply: time planes staged through a shared-memory ring
// by asynchronous copies (cp.async, L2 -> shared, zero-filled outside
// non-periodic boundaries), several planes in flight per CTA.
//
// Same operator and evaluation order as apply_impl.cuh: per time plane the
// spatial sum-factorised fields of Appendix A's element matrices
// (D^0 = (x)M, D^k = C on axis k, M elsewhere) combined with the spin matrices
// into G_C (partner of the time convection C_t) and G_M (partner of the time
// mass M_t), then the two time stencils through two running accumulators per
// output.  One CTA owns a spatial tile (one output node per thread) and a
// chunk of time layers; it walks the chunk's planes plus one halo plane on
// each side.  Each plane of the tile + spatial halo is copied once into the
// ring; every thread then reads its 3^d neighbourhood from shared memory.
// One barrier per plane: after it, the slot consumed one plane earlier is
// free and the copies of the next-but-(S-1) plane are issued into it.
#pragma once

#include "apply_fast.cuh"

#define DST_MAX_DEVICES_APPLY 64

namespace dst {

// Output tile TX x TY x TZ per CTA and TT time layers; each thread computes RY
// consecutive y outputs (2+1: the x stencils of the rows they share are
// computed once).
// TV selects one of the tile shapes the autotuner chooses from (variant 0 is
// the default): smaller tiles and time chunks give small meshes more CTAs.
template <int D, int TV = 0> struct PipeTile;
template <> struct PipeTile<1, 0> { static constexpr int TX = 256, TY = 1, TZ = 1, TT = 32, RY = 1; };
template <> struct PipeTile<1, 1> { static constexpr int TX = 128, TY = 1, TZ = 1, TT = 16, RY = 1; };
template <> struct PipeTile<1, 2> { static constexpr int TX = 64, TY = 1, TZ = 1, TT = 8, RY = 1; };
template <> struct PipeTile<2, 0> { static constexpr int TX = 32, TY = 8, TZ = 1, TT = 8, RY = 2; };
template <> struct PipeTile<2, 1> { static constexpr int TX = 32, TY = 8, TZ = 1, TT = 4, RY = 2; };
template <> struct PipeTile<2, 2> { static constexpr int TX = 16, TY = 8, TZ = 1, TT = 8, RY = 2; };
template <> struct PipeTile<3, 0> { static constexpr int TX = 16, TY = 4, TZ = 4, TT = 8, RY = 1; };

template <int D, int NC, typename T, int TV = 0>
struct PipeShape {
    using Tile = PipeTile<D, TV>;
    static constexpr int BX = Tile::TX + 2;
    static constexpr int BY = D >= 2 ? Tile::TY + 2 : 1;
    static constexpr int BZ = D >= 3 ? Tile::TZ + 2 : 1;
    static constexpr int BOX = BX * BY * BZ;                          // nodes per staged plane
    static constexpr int NODE_BYTES = NC * 2 * (int)sizeof(T);        // 16, 32 or 64
    static constexpr int CHUNKS = NODE_BYTES / 16;                    // 16-byte copies per node
    static constexpr int NTHR = Tile::TX * (Tile::TY / Tile::RY) * Tile::TZ;
    // two planes per step (twice the independent work per barrier) when one
    // output per thread and an eight-plane ring fits comfortably; otherwise one
    // plane per step, 4 or 3 stages
    static constexpr bool PAIR = Tile::RY == 1 && BOX * NODE_BYTES * 8 <= 72 * 1024;
    // the whole chunk (TT planes + two halo planes) resident at once when it is
    // small: every copy is issued before the first plane is consumed, so the
    // latency of the HBM reads is paid once per CTA instead of once per slot
    static constexpr bool FULL = !PAIR && (Tile::TT + 2) * BOX * NODE_BYTES <= 56 * 1024;
    static constexpr int STAGES =
        FULL ? Tile::TT + 2 : (PAIR ? 8 : ((BOX * NODE_BYTES * 4 <= 96 * 1024) ? 4 : 3));
    static constexpr int SMEM = STAGES * BOX * NODE_BYTES;
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool ok) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = ok ? 16 : 0;     // n = 0: nothing read, 16 zero bytes written
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
// wait_group with a count known only after unrolling (0 .. 15)
__device__ __forceinline__ void cp_async_wait_n(int n) {
    switch (n) {
    case 0: cp_async_wait<0>(); break;   case 1: cp_async_wait<1>(); break;
    case 2: cp_async_wait<2>(); break;   case 3: cp_async_wait<3>(); break;
    case 4: cp_async_wait<4>(); break;   case 5: cp_async_wait<5>(); break;
    case 6: cp_async_wait<6>(); break;   case 7: cp_async_wait<7>(); break;
    case 8: cp_async_wait<8>(); break;   case 9: cp_async_wait<9>(); break;
    case 10: cp_async_wait<10>(); break; case 11: cp_async_wait<11>(); break;
    case 12: cp_async_wait<12>(); break; case 13: cp_async_wait<13>(); break;
    case 14: cp_async_wait<14>(); break; default: cp_async_wait<15>(); break;
    }
}

// The 16-byte copies one thread issues for every plane: source byte offset
// within a time layer (-1: outside a non-periodic boundary, zero-filled) and
// destination byte offset within a ring slot.  Computed once per thread, so
// the plane loop does no index arithmetic (periodic wrap needs 64-bit modulo).
template <int D, int NC, typename T, int TV>
struct CopyPlan {
    static constexpr int PER_THREAD =
        (PipeShape<D, NC, T, TV>::BOX * PipeShape<D, NC, T, TV>::CHUNKS + PipeShape<D, NC, T, TV>::NTHR - 1) /
        PipeShape<D, NC, T, TV>::NTHR;
    int src[PER_THREAD];
    int dst[PER_THREAD];
};

template <int D, int NC, typename T, int TV>
__device__ __forceinline__ void make_copy_plan(const OpParams &p, int64_t x0, int64_t y0, int64_t z0,
                                               CopyPlan<D, NC, T, TV> &cp) {
    using S = PipeShape<D, NC, T, TV>;
    const int64_t nx = p.ax[0].n, ny = p.ax[1].n;
#pragma unroll
    for (int j = 0; j < CopyPlan<D, NC, T, TV>::PER_THREAD; ++j) {
        const int i = threadIdx.x + j * S::NTHR;
        cp.dst[j] = -1;
        cp.src[j] = -1;
        if (i >= S::BOX * S::CHUNKS) continue;
        const int node = i / S::CHUNKS, part = i % S::CHUNKS;
        const int bx = node % S::BX, by = (node / S::BX) % S::BY, bz = node / (S::BX * S::BY);
        const int64_t gx = axis_nbr(p.ax[0], x0 - 1 + bx);
        const int64_t gy = D >= 2 ? axis_nbr(p.ax[1], y0 - 1 + by) : 0;
        const int64_t gz = D >= 3 ? axis_nbr(p.ax[2], z0 - 1 + bz) : 0;
        cp.dst[j] = node * S::NODE_BYTES + part * 16;
        if (gx >= 0 && gy >= 0 && gz >= 0) cp.src[j] = (int)(((gz * ny + gy) * nx + gx) * S::NODE_BYTES + part * 16);
    }
}

// Issue the copies of one plane (tile box, one-node halo) into a ring slot.
template <int D, int NC, typename T, int TV>
__device__ __forceinline__ void issue_plane(const CopyPlan<D, NC, T, TV> &cp, const char *layer, char *slot) {
#pragma unroll
    for (int j = 0; j < CopyPlan<D, NC, T, TV>::PER_THREAD; ++j)
        if (cp.dst[j] >= 0) cp_async16(slot + cp.dst[j], layer + (cp.src[j] >= 0 ? cp.src[j] : 0), cp.src[j] >= 0);
}

template <int NC, typename T>
__device__ __forceinline__ NodeV<NC, T> smem_node(const char *slot, int node) {
    NodeV<NC, T> v;
    if (sizeof(T) == 4) {
        const float4 *q = reinterpret_cast<const float4 *>(slot + (size_t)node * NC * 8);
#pragma unroll
        for (int k = 0; k < NC / 2; ++k) {
            const float4 f = q[k];
            v.c[2 * k].x = f.x; v.c[2 * k].y = f.y; v.c[2 * k + 1].x = f.z; v.c[2 * k + 1].y = f.w;
        }
    } else {
        const double2 *q = reinterpret_cast<const double2 *>(slot + (size_t)node * NC * 16);
#pragma unroll
        for (int c = 0; c < NC; ++c) { const double2 f = q[c]; v.c[c].x = f.x; v.c[c].y = f.y; }
    }
    return v;
}

// Per-kernel constants of the standard interior stencils.  With
// M = h/6 [1,4,1] and C = 1/2 [-1,0,1] on every axis, the spatial fields are
// unscaled [1,4,1] / [-1,0,1] sums times fixed factors; those factors, the 1/2
// and h_t/6 of the time stencils and the mass m are folded into these
// constants, so G_C' = G_C / 2 and G_M' = (h_t/6) G_M come out directly.
template <typename T>
struct StdConst {
    T kc;        // G_C' = i kc PM                      (kc = 1/2 prod h_k/6)
    T km;        // mass part of G_M': -beta m km PM    (km = (h_t/6) prod h_k/6)
    T ka[3];     // alpha_k part of G_M': i ka[k] alpha_k PC_k  (ka = (h_t/6) 1/2 prod_{j!=k} h_j/6)
};

template <int D, typename T>
__host__ __device__ inline StdConst<T> std_const(const OpParams &p) {
    StdConst<T> c;
    double pm = 1.0;
    for (int k = 0; k < D; ++k) pm *= p.ax[k].h / 6.0;
    const double ht6 = p.ht / 6.0;
    c.kc = (T)(0.5 * pm);
    c.km = (T)(ht6 * pm);
    for (int k = 0; k < 3; ++k) {
        double q = 0.5 * ht6;
        for (int j = 0; j < D; ++j)
            if (j != k) q *= p.ax[j].h / 6.0;
        c.ka[k] = (T)q;
    }
    return c;
}

// i s (alpha_k P)[c] accumulated into G (NC = 2: alpha = (sigma_x, sigma_y);
// NC = 4: alpha_k = [[0, sigma_k], [sigma_k, 0]]).
template <int NC, typename V, typename T>
__device__ __forceinline__ void add_i_alpha(int k, T s, const V *P, V *G) {
    // i * (a.x + i a.y) * s = (-s a.y, s a.x)
    auto addi = [&](V &g, V a, T f) { g.x = fma(-f, a.y, g.x); g.y = fma(f, a.x, g.y); };
    if (NC == 2) {
        if (k == 0) { addi(G[0], P[1], s); addi(G[1], P[0], s); }
        else {      // sigma_y: (-i b, i a): i*(-i b) = b, i*(i a) = -a
            G[0].x = fma(s, P[1].x, G[0].x); G[0].y = fma(s, P[1].y, G[0].y);
            G[1].x = fma(-s, P[0].x, G[1].x); G[1].y = fma(-s, P[0].y, G[1].y);
        }
    } else {
        if (k == 0) { addi(G[0], P[3], s); addi(G[1], P[2], s); addi(G[2], P[1], s); addi(G[3], P[0], s); }
        else if (k == 1) {
            G[0].x = fma(s, P[3].x, G[0].x); G[0].y = fma(s, P[3].y, G[0].y);
            G[1].x = fma(-s, P[2].x, G[1].x); G[1].y = fma(-s, P[2].y, G[1].y);
            G[2].x = fma(s, P[1].x, G[2].x); G[2].y = fma(s, P[1].y, G[2].y);
            G[3].x = fma(-s, P[0].x, G[3].x); G[3].y = fma(-s, P[0].y, G[3].y);
        } else {    // sigma_z: (a, -b)
            addi(G[0], P[2], s); addi(G[1], P[3], -s); addi(G[2], P[0], s); addi(G[3], P[1], -s);
        }
    }
}

// G_C' and G_M' of a node whose stencils are the standard interior ones.
// WV: x-only potential.  The mass-plus-potential x stencil of a node between
// elements of weights w_l, w_r (w = m beta + V) is (w_l, 2 (w_l + w_r), w_r)
// = (w_l + w_r)/2 [1,4,1] + (w_r - w_l)/2 [-1,0,1], so G_M' = a QM + b QCx with
// a = -km (w_l + w_r) / 2 and b = -km (w_r - w_l) / 2: both fields are needed
// anyway, and b = 0 away from a jump of V.
template <int D, int NC, typename T, bool WV, typename Get>
__device__ __forceinline__ void fields_std(Get get, const StdConst<T> &sc, T m, const T (&wa)[2], const T (&wb)[2],
                                           typename C2<T>::type *GC, typename C2<T>::type *GM) {
    using V = typename C2<T>::type;
    const int NZ = D >= 3 ? 3 : 1, NY = D >= 2 ? 3 : 1;
    V QM[NC], QCx[NC], QCy[NC], QCz[NC];   // sums over z of [1,4,1] (and [-1,0,1] for z)
#pragma unroll
    for (int c = 0; c < NC; ++c) { QM[c] = cz<V>(); QCx[c] = cz<V>(); QCy[c] = cz<V>(); QCz[c] = cz<V>(); }
#pragma unroll
    for (int dz = 0; dz < NZ; ++dz) {
        V PM[NC], PCx[NC], PCy[NC];
#pragma unroll
        for (int dy = 0; dy < NY; ++dy) {
            const int r = (dz * NY + dy) * 3;
            const NodeV<NC, T> n0 = get(r), n1 = get(r + 1), n2 = get(r + 2);
            const T wy = (D >= 2 && dy == 1) ? (T)4 : (T)1;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const V x0 = n0.c[c], x1 = n1.c[c], x2 = n2.c[c];
                V rM, rC;
                rM.x = fma((T)4, x1.x, x0.x + x2.x); rM.y = fma((T)4, x1.y, x0.y + x2.y);
                rC.x = x2.x - x0.x; rC.y = x2.y - x0.y;
                if (dy == 0) {
                    PM[c] = rM; PCx[c] = rC;
                    if (D >= 2) { PCy[c].x = -rM.x; PCy[c].y = -rM.y; }
                } else {
                    PM[c] = cfma_r(wy, rM, PM[c]);
                    PCx[c] = cfma_r(wy, rC, PCx[c]);
                    if (D >= 2 && dy == 2) PCy[c] = cadd(PCy[c], rM);
                }
            }
        }
        const T wz = (D >= 3 && dz == 1) ? (T)4 : (T)1;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            QM[c] = cfma_r(wz, PM[c], QM[c]);
            QCx[c] = cfma_r(wz, PCx[c], QCx[c]);
            if (D >= 2) QCy[c] = cfma_r(wz, PCy[c], QCy[c]);
            if (D >= 3) {
                if (dz == 0) QCz[c] = cmul_r((T)(-1), PM[c]);
                else if (dz == 2) QCz[c] = cadd(QCz[c], PM[c]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        GC[c].x = -sc.kc * QM[c].y; GC[c].y = sc.kc * QM[c].x;             // i kc QM
        if (WV) {
            const int sb = Beta<D>::s(c) > 0 ? 0 : 1;
            GM[c] = cfma_r(wb[sb], QCx[c], cmul_r(wa[sb], QM[c]));          // weights carry m beta + V
        } else {
            const T f = Beta<D>::s(c) > 0 ? -m * sc.km : m * sc.km;          // -beta m km
            GM[c] = cmul_r(f, QM[c]);
        }
    }
    add_i_alpha<NC>(0, sc.ka[0], QCx, GM);
    if (D >= 2) add_i_alpha<NC>(1, sc.ka[1], QCy, GM);
    if (D >= 3) add_i_alpha<NC>(2, sc.ka[2], QCz, GM);
}

// 2+1, standard interior stencils, RY consecutive y outputs of one thread:
// the x stencils of the RY + 2 rows are computed once and shared.
// get(q, dx): node of row q (0 .. RY+1) and column dx (0 .. 2).
template <int NC, typename T, bool WV, int RY, typename Get>
__device__ __forceinline__ void fields_std_rows(Get get, const StdConst<T> &sc, T m, const T (&wa)[2], const T (&wb)[2],
                                                typename C2<T>::type (*GC)[NC], typename C2<T>::type (*GM)[NC]) {
    using V = typename C2<T>::type;
    V rM[RY + 2][NC], rC[RY + 2][NC];
#pragma unroll
    for (int q = 0; q < RY + 2; ++q) {
        const NodeV<NC, T> n0 = get(q, 0), n1 = get(q, 1), n2 = get(q, 2);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const V x0 = n0.c[c], x1 = n1.c[c], x2 = n2.c[c];
            rM[q][c].x = fma((T)4, x1.x, x0.x + x2.x); rM[q][c].y = fma((T)4, x1.y, x0.y + x2.y);
            rC[q][c].x = x2.x - x0.x; rC[q][c].y = x2.y - x0.y;
        }
    }
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        V PM[NC], PCx[NC], PCy[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            PM[c] = cfma_r((T)4, rM[r + 1][c], cadd(rM[r][c], rM[r + 2][c]));
            PCx[c] = cfma_r((T)4, rC[r + 1][c], cadd(rC[r][c], rC[r + 2][c]));
            PCy[c] = csub(rM[r + 2][c], rM[r][c]);
            GC[r][c].x = -sc.kc * PM[c].y; GC[r][c].y = sc.kc * PM[c].x;
            if (WV) {
                const int sb = Beta<2>::s(c) > 0 ? 0 : 1;
                GM[r][c] = cfma_r(wb[sb], PCx[c], cmul_r(wa[sb], PM[c]));
            } else {
                const T f = Beta<2>::s(c) > 0 ? -m * sc.km : m * sc.km;
                GM[r][c] = cmul_r(f, PM[c]);
            }
        }
        add_i_alpha<NC>(0, sc.ka[0], PCx, GM[r]);
        add_i_alpha<NC>(1, sc.ka[1], PCy, GM[r]);
    }
}

// STD: every node of the mesh has the standard interior stencils on every axis
// (no open axis), so the general-coefficient branch is not compiled in.
// One CTA's work: output tile `tile` over the time chunk `chunk`, staged through
// `ring` (PipeShape::SMEM bytes of shared memory), PipeShape::NTHR threads.
// Ends with every copy complete; a caller that reuses the ring for another
// tile synchronises the CTA first.
template <int D, int NC, typename T, bool NOV, bool STD, int TV = 0>
__device__ __forceinline__ void apply_pipe_tile(const OpParams &p, const typename C2<T>::type *__restrict__ x,
                                                typename C2<T>::type *__restrict__ y, int64_t tiles_x,
                                                int64_t tiles_y, int64_t tile, int64_t chunk, char *ring) {
    using V = typename C2<T>::type;
    using S = PipeShape<D, NC, T, TV>;
    using Tile = typename S::Tile;
    constexpr int RY = Tile::RY;
    constexpr int TYT = Tile::TY / RY;                  // threads along y

    const int64_t x0 = (tile % tiles_x) * Tile::TX;
    const int64_t y0 = ((tile / tiles_x) % tiles_y) * Tile::TY;
    const int64_t z0 = (tile / (tiles_x * tiles_y)) * Tile::TZ;
    const int tx = threadIdx.x % Tile::TX;
    const int ty = ((threadIdx.x / Tile::TX) % TYT) * RY;     // first of the thread's RY output rows
    const int tz = threadIdx.x / (Tile::TX * TYT);
    const int64_t ix = x0 + tx, iy = y0 + ty, iz = z0 + tz;
    const int64_t nx = p.ax[0].n, ny = p.ax[1].n, nz = p.ax[2].n;
    const int64_t N = p.nt;
    const int64_t t0 = 1 + chunk * Tile::TT;
    const int64_t t1 = min(t0 + (int64_t)Tile::TT, N + 1);
    const int64_t plane_elems = nx * ny * nz * NC;
    const int64_t self = (iz * ny + iy) * nx + ix;
    const int nplanes = (int)(t1 - t0 + 2);            // planes t0-1 .. t1
    const int64_t pfirst = t0 - 1;

    bool valid[RY];
    bool stdn[RY];
    bool any_valid = false, all_std = true;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        valid[r] = ix < nx && iy + r < ny && iz < nz;
        any_valid = any_valid || valid[r];
    }
    NodeCoef<D, T> k;      // coefficients of output row 0 (x and z are shared by all rows)
    if (valid[0]) node_coef<D, T>(p, ix, iy, iz, k);
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        // standard interior stencils on every axis (periodic / Dirichlet axes,
        // and open axes away from their two end nodes)
        bool sd = valid[r] && k.cx.eL && k.cx.eR;
        if (D >= 2 && valid[r]) {
            const Coef3<T> cy = r == 0 ? k.cy : axis_coef<T>(p.ax[1], iy + r);
            sd = sd && cy.eL && cy.eR;
        }
        if (D >= 3) sd = sd && k.cz.eL && k.cz.eR;
        stdn[r] = sd;
        all_std = all_std && (sd || !valid[r]);
    }
    all_std = all_std && valid[0];
    const StdConst<T> sc = std_const<D, T>(p);
    T wa[2], wb[2];  // mass-plus-potential weights of the standard path (fields_std), h_x / 6 in StdConst
    for (int sb = 0; sb < 2; ++sb) {
        const T wl = valid[0] ? k.wl[sb] : (T)0, wr = valid[0] ? k.wr[sb] : (T)0;
        wa[sb] = (T)(-0.5) * sc.km * (wl + wr); wb[sb] = (T)(-0.5) * sc.km * (wr - wl);
    }
    CopyPlan<D, NC, T, TV> cplan;
    make_copy_plan<D, NC, T, TV>(p, x0, y0, z0, cplan);
    const T h6 = (T)(p.ht / 6.0);
    const int NY = D >= 2 ? 3 : 1;
    const int c0 = (tz * S::BY + ty) * S::BX + tx;      // box index of the (-1,-1,-1) neighbour of row 0

    // Plane-loop bookkeeping in 32-bit, relative to the chunk: plane i is time
    // layer pfirst + i; it exists iff i_lo <= i <= i_hi; outputs are stored
    // for i >= 2; the final layer's diagonal applies for i >= i_last.
    const int i_lo = (int)max((int64_t)0, 1 - pfirst);
    const int i_hi = (int)min((int64_t)(nplanes - 1), N - pfirst);
    const int i_last = (int)(N - pfirst);
    const size_t plane_bytes = (size_t)plane_elems * sizeof(V);
    const size_t slot_bytes = (size_t)S::BOX * S::NODE_BYTES;
    const char *xsrc = reinterpret_cast<const char *>(x) + (pfirst - 1) * (int64_t)plane_bytes;   // plane i = xsrc + i*plane_bytes
    char *ydst = reinterpret_cast<char *>(y + (t0 - 1) * plane_elems + self * NC);               // layer t0, row 0
    const size_t row_bytes = (size_t)nx * NC * sizeof(V);
    int issue_slot = 0;
    const char *issue_src = xsrc;

    auto issue_next = [&](int i) {      // plane i into the next ring slot (i strictly increasing)
        if (i >= i_lo && i <= i_hi) issue_plane<D, NC, T, TV>(cplan, issue_src, ring + (size_t)issue_slot * slot_bytes);
        cp_async_commit();
        issue_src += plane_bytes;
        issue_slot = issue_slot + 1 == S::STAGES ? 0 : issue_slot + 1;
    };
    // G_C' = G_C / 2 and G_M' = (h_t / 6) G_M of plane i (ring slot si) for the thread's RY outputs
    auto plane_fields = [&](int i, int si, V (*GC)[NC], V (*GM)[NC]) {
        const bool have = i >= i_lo && i <= i_hi;
        const char *slot = ring + (size_t)si * slot_bytes;
        if (STD) {
            // rows / columns past the mesh end read initialised shared memory
            // (wrapped or zero-filled halo) and are not stored
            if (!have) {
#pragma unroll
                for (int r = 0; r < RY; ++r)
#pragma unroll
                    for (int c = 0; c < NC; ++c) { GC[r][c] = cz<V>(); GM[r][c] = cz<V>(); }
            } else if (RY > 1) {
                auto getq = [&](int q, int dx) { return smem_node<NC, T>(slot, c0 + q * S::BX + dx); };
                fields_std_rows<NC, T, !NOV, RY>(getq, sc, (T)p.m, wa, wb, GC, GM);
            } else {
                auto get = [&](int q) {
                    const int dz = q / (3 * NY), dy = (q / 3) % NY, dx = q % 3;
                    return smem_node<NC, T>(slot, c0 + (dz * S::BY + dy) * S::BX + dx);
                };
                fields_std<D, NC, T, !NOV>(get, sc, (T)p.m, wa, wb, GC[0], GM[0]);
            }
            return;
        }
        if (have && RY > 1 && all_std) {
            auto getq = [&](int q, int dx) { return smem_node<NC, T>(slot, c0 + q * S::BX + dx); };
            fields_std_rows<NC, T, !NOV, RY>(getq, sc, (T)p.m, wa, wb, GC, GM);
            return;
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            if (have && valid[r]) {
                const int cr = c0 + r * S::BX;
                auto get = [&](int q) {
                    const int dz = q / (3 * NY), dy = (q / 3) % NY, dx = q % 3;
                    return smem_node<NC, T>(slot, cr + (dz * S::BY + dy) * S::BX + dx);
                };
                if (stdn[r]) {
                    fields_std<D, NC, T, !NOV>(get, sc, (T)p.m, wa, wb, GC[r], GM[r]);
                } else {
                    NodeCoef<D, T> kr;
                    if (r == 0) kr = k;
                    else node_coef<D, T>(p, ix, iy + r, iz, kr);
                    if (NOV) fields_nov<D, NC, T>(get, kr, (T)p.m, GC[r], GM[r]);
                    else fields<D, NC, T>(get, kr, GC[r], GM[r]);
#pragma unroll
                    for (int c = 0; c < NC; ++c) { GC[r][c] = cmul_r((T)0.5, GC[r][c]); GM[r][c] = cmul_r(h6, GM[r][c]); }
                }
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c) { GC[r][c] = cz<V>(); GM[r][c] = cz<V>(); }
            }
        }
    };

    V accP[RY][NC], accC[RY][NC];
#pragma unroll
    for (int r = 0; r < RY; ++r)
#pragma unroll
        for (int c = 0; c < NC; ++c) { accP[r][c] = cz<V>(); accC[r][c] = cz<V>(); }
    // y(pl-1) += G_C' + G_M'; y(pl) += (pl < N ? 4 G_M' : G_C' + 2 G_M'); y(pl+1) = G_M' - G_C'
    auto accumulate = [&](int i, V (*GC)[NC], V (*GM)[NC]) {
        const bool last = i >= i_last;
#pragma unroll
        for (int r = 0; r < RY; ++r) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                accP[r][c] = cadd(accP[r][c], cadd(GC[r][c], GM[r][c]));
                if (last) accC[r][c] = cadd(accC[r][c], cfma_r((T)2, GM[r][c], GC[r][c]));
                else accC[r][c] = cfma_r((T)4, GM[r][c], accC[r][c]);
            }
            if (valid[r] && i >= 2) store_node<NC, T>(reinterpret_cast<V *>(ydst + r * row_bytes), 0, accP[r]);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                accP[r][c] = accC[r][c];
                accC[r][c] = csub(GM[r][c], GC[r][c]);
            }
        }
        if (i >= 2) ydst += plane_bytes;
    };

    if (S::FULL) {
        // every plane of the chunk in flight at once; one wait and one barrier,
        // then the planes' independent loads and arithmetic can interleave
#pragma unroll
        for (int i = 0; i < S::STAGES; ++i) issue_next(i);
        cp_async_wait<0>();
        __syncthreads();
#pragma unroll
        for (int i = 0; i < S::STAGES; ++i) {
            if (i < nplanes) {
                V GC[RY][NC], GM[RY][NC];
                plane_fields(i, i, GC, GM);
                accumulate(i, GC, GM);
            }
        }
    } else if (S::PAIR) {
        // ring of 8: planes i, i+1 computed while up to six more are in flight
#pragma unroll
        for (int i = 0; i < S::STAGES - 2; ++i) issue_next(i);
        int si = 0;
        for (int i = 0; i < nplanes; i += 2) {
            cp_async_wait<S::STAGES - 4>();
            __syncthreads();
            issue_next(i + S::STAGES - 2);
            issue_next(i + S::STAGES - 1);
            V GC0[RY][NC], GM0[RY][NC], GC1[RY][NC], GM1[RY][NC];
            plane_fields(i, si, GC0, GM0);
            plane_fields(i + 1, si + 1, GC1, GM1);
            si = (si + 2) & (S::STAGES - 1);
            accumulate(i, GC0, GM0);
            if (i + 1 < nplanes) accumulate(i + 1, GC1, GM1);
        }
    } else {
#pragma unroll
        for (int i = 0; i < S::STAGES - 1; ++i) issue_next(i);
        int si = 0;
        for (int i = 0; i < nplanes; ++i) {
            cp_async_wait<S::STAGES - 2>();
            __syncthreads();
            issue_next(i + S::STAGES - 1);
            V GC[RY][NC], GM[RY][NC];
            plane_fields(i, si, GC, GM);
            si = si + 1 == S::STAGES ? 0 : si + 1;
            accumulate(i, GC, GM);
        }
    }
    cp_async_wait<0>();
    (void)any_valid;
}

template <int D, int NC, typename T, bool NOV, bool STD, int TV>
__global__ void __launch_bounds__(PipeShape<D, NC, T, TV>::NTHR,
                                  sizeof(T) == 8 ? 1 : (D == 3 ? (STD ? 2 : 1) : 3))
apply_pipe_kernel(OpParams p, const typename C2<T>::type *__restrict__ x, typename C2<T>::type *__restrict__ y,
                  int64_t tiles_x, int64_t tiles_y) {
    extern __shared__ __align__(16) char ring[];
    apply_pipe_tile<D, NC, T, NOV, STD, TV>(p, x, y, tiles_x, tiles_y, blockIdx.x, blockIdx.y, ring);
}

template <int D, int NC, typename T, int TV>
int launch_apply_pipe_v(const OpParams &p, const typename C2<T>::type *x, typename C2<T>::type *y, cudaStream_t s) {
    using S = PipeShape<D, NC, T, TV>;
    using Tile = PipeTile<D, TV>;
    const int64_t tx = (p.ax[0].n + Tile::TX - 1) / Tile::TX;
    const int64_t ty = (p.ax[1].n + Tile::TY - 1) / Tile::TY;
    const int64_t tz = (p.ax[2].n + Tile::TZ - 1) / Tile::TZ;
    const int64_t chunks = (p.nt + Tile::TT - 1) / Tile::TT;
    const int64_t tiles = tx * ty * tz;
    if (tiles <= 0 || tiles > 0x7fffffffLL || chunks > 65535) return DST_ERR_ARG;
    // byte offsets within one time layer are kept in 32 bits
    if (p.ax[0].n * p.ax[1].n * p.ax[2].n * S::NODE_BYTES >= (1LL << 31)) return launch_apply<D, NC, T>(p, x, y, s);
    dim3 grid((unsigned)tiles, (unsigned)chunks);
    // the shared-memory opt-in is a per-device function attribute: set it once per device
    static bool configured[4][DST_MAX_DEVICES_APPLY] = {};
    int dev = 0;
    DST_CUDA_TRY(cudaGetDevice(&dev));
    const int nov = p.vmode == 2 ? 1 : 0;
    bool all_std = true;        // no open axis: every node has the standard stencils
    for (int k = 0; k < D; ++k) all_std = all_std && p.ax[k].bc != DST_BC_OPEN;
    const int var = nov + 2 * (all_std ? 1 : 0);
    auto kern = var == 0   ? apply_pipe_kernel<D, NC, T, false, false, TV>
                : var == 1 ? apply_pipe_kernel<D, NC, T, true, false, TV>
                : var == 2 ? apply_pipe_kernel<D, NC, T, false, true, TV>
                           : apply_pipe_kernel<D, NC, T, true, true, TV>;
    if (dev < 0 || dev >= DST_MAX_DEVICES_APPLY || !configured[var][dev]) {
        DST_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM));
        if (dev >= 0 && dev < DST_MAX_DEVICES_APPLY) configured[var][dev] = true;
    }
    kern<<<grid, S::NTHR, S::SMEM, s>>>(p, x, y, tx, ty);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

// Number of tile variants per spatial dimension (3+1: the one-output-per-thread
// tiles of this file, and the z-columns of apply_zblk.cuh).
constexpr int pipe_tile_variants(int d) { return d == 3 ? 2 : 3; }

template <typename T, int RZ>
int launch_apply_zblk(const OpParams &p, const typename C2<T>::type *x, typename C2<T>::type *y, cudaStream_t s);

// Launch with the tile variant the parameters carry for this precision.
template <int D, int NC, typename T>
int launch_apply_pipe(const OpParams &p, const typename C2<T>::type *x, typename C2<T>::type *y, cudaStream_t s) {
    const int tv = p.tile_variant[sizeof(T) == 4 ? DST_FP32 : DST_FP64];
    if constexpr (D == 3) {
        bool all_std = true;
        for (int k = 0; k < 3; ++k) all_std = all_std && p.ax[k].bc != DST_BC_OPEN;
        if (tv == 1 && all_std && p.vmode != 1) return launch_apply_zblk<T, sizeof(T) == 4 ? 4 : 2>(p, x, y, s);
    }
    if (D == 3 || tv <= 0) return launch_apply_pipe_v<D, NC, T, 0>(p, x, y, s);
    if constexpr (D < 3) {
        if (tv == 1) return launch_apply_pipe_v<D, NC, T, 1>(p, x, y, s);
        return launch_apply_pipe_v<D, NC, T, 2>(p, x, y, s);
    }
    return DST_ERR_ARG;
}

}  // namespace dst
