// Streaming operator apply for potentials that depend on x only (or vanish).
//
// Same operator and evaluation order as apply_impl.cuh (sum-factorised Q1
// stencils, spatial fields per time plane combined with the spin matrices,
// time stencils through two running accumulators), but organised for
// bandwidth: one thread owns one spatial node and marches through a chunk of
// time planes.  Its spatial
// neighbours come straight from global memory through L1 as 16-byte vector
// loads - every node of a plane is read by up to 3^d threads of the same CTA,
// so L1/L2 absorb the reuse and DRAM sees each x value about once - and
// nothing is staged in shared memory, so there are no barriers.  In FP32 the
// loads of plane p+1 are issued before plane p is combined (software
// pipelining).
#pragma once

#include "apply_impl.cuh"

namespace dst {

template <int D> struct FastTile;
template <> struct FastTile<1> { static constexpr int TX = 128, TY = 1, TZ = 1, TT = 16; };
template <> struct FastTile<2> { static constexpr int TX = 32, TY = 4, TZ = 1, TT = 8; };
template <> struct FastTile<3> { static constexpr int TX = 32, TY = 4, TZ = 1, TT = 8; };

template <int NC, typename T>
struct NodeV {
    typename C2<T>::type c[NC];
};

// Vector load of one node's NC complex values (zero when absent).
template <int NC, typename T>
__device__ __forceinline__ void load_node(const typename C2<T>::type *__restrict__ base, int64_t node, bool ok,
                                          NodeV<NC, T> &v) {
    using V = typename C2<T>::type;
    if (!ok) {
#pragma unroll
        for (int c = 0; c < NC; ++c) v.c[c] = cz<V>();
        return;
    }
    const V *p = base + node * NC;
    if (sizeof(T) == 4) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
        for (int k = 0; k < NC / 2; ++k) {
            float4 f = __ldg(q + k);
            v.c[2 * k].x = f.x; v.c[2 * k].y = f.y; v.c[2 * k + 1].x = f.z; v.c[2 * k + 1].y = f.w;
        }
    } else {
        const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double2 f = __ldg(q + c);
            v.c[c].x = f.x; v.c[c].y = f.y;
        }
    }
}

template <int NC, typename T>
__device__ __forceinline__ void store_node(typename C2<T>::type *__restrict__ base, int64_t node,
                                           const typename C2<T>::type *val) {
    using V = typename C2<T>::type;
    V *p = base + node * NC;
    if (sizeof(T) == 4) {
        float4 *q = reinterpret_cast<float4 *>(p);
#pragma unroll
        for (int k = 0; k < NC / 2; ++k)
            q[k] = make_float4(val[2 * k].x, val[2 * k].y, val[2 * k + 1].x, val[2 * k + 1].y);
    } else {
        double2 *q = reinterpret_cast<double2 *>(p);
#pragma unroll
        for (int c = 0; c < NC; ++c) q[c] = make_double2(val[c].x, val[c].y);
    }
}

// Neighbour offsets of one thread within one time plane, per axis: node index
// = xo[dx] + yo[dy] + zo[dz]; an absent neighbour (outside a non-periodic
// axis) carries a large negative offset so that any sum with it is < 0.
// Planes of up to 2^31 - 1 nodes (checked by the launcher).
struct Nbr {
    int xo[3], yo[3], zo[3];
    __device__ __forceinline__ int at(int dz, int dy, int dx) const { return xo[dx] + yo[dy] + zo[dz]; }
};

template <int D>
__device__ __forceinline__ void neighbours(const OpParams &p, int64_t ix, int64_t iy, int64_t iz, Nbr &nb) {
    const int nx = (int)p.ax[0].n, nxy = (int)(p.ax[0].n * p.ax[1].n);
    const int ABSENT = -(1 << 30);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int64_t xx = axis_nbr(p.ax[0], ix - 1 + k);
        nb.xo[k] = xx >= 0 ? (int)xx : ABSENT;
        if (D >= 2) {
            const int64_t yy = axis_nbr(p.ax[1], iy - 1 + k);
            nb.yo[k] = yy >= 0 ? (int)yy * nx : ABSENT;
        } else {
            nb.yo[k] = (int)iy * nx;
        }
        if (D >= 3) {
            const int64_t zz = axis_nbr(p.ax[2], iz - 1 + k);
            nb.zo[k] = zz >= 0 ? (int)zz * nxy : ABSENT;
        } else {
            nb.zo[k] = (int)iz * nxy;
        }
    }
}

template <int D, int NC, typename T>
struct Plane {
    NodeV<NC, T> v[D == 1 ? 3 : (D == 2 ? 9 : 27)];
};

template <int D, int NC, typename T>
__device__ __forceinline__ void load_plane(const typename C2<T>::type *__restrict__ layer, const Nbr &nb,
                                           bool have, Plane<D, NC, T> &pl) {
    const int NY = D >= 2 ? 3 : 1;
#pragma unroll
    for (int dy = 0; dy < NY; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
            const int id = nb.at(1, dy, dx);
            load_node<NC, T>(layer, id, have && id >= 0, pl.v[dy * 3 + dx]);
        }
}

// G_C, G_M of one output node from its 3^d neighbourhood; get(r) returns the
// node of neighbourhood row r (r = (dz*NY + dy)*3 + dx), from registers or memory.
template <int D, int NC, typename T, typename Get>
__device__ __forceinline__ void fields(Get get, const NodeCoef<D, T> &k, typename C2<T>::type *GC,
                                       typename C2<T>::type *GM) {
    using V = typename C2<T>::type;
    const int NZ = D >= 3 ? 3 : 1, NY = D >= 2 ? 3 : 1;
    V sM[NC], sW[NC], sCx[NC], sCy[NC], sCz[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) { sM[c] = cz<V>(); sW[c] = cz<V>(); sCx[c] = cz<V>(); sCy[c] = cz<V>(); sCz[c] = cz<V>(); }
    // x-direction weights of the mass + potential term for beta = +1 / -1
    T wx[2][3];
#pragma unroll
    for (int sb = 0; sb < 2; ++sb) {
        wx[sb][0] = k.wl[sb] * k.cx.ml[0];
        wx[sb][1] = k.wl[sb] * k.cx.ml[1] + k.wr[sb] * k.cx.mr[1];
        wx[sb][2] = k.wr[sb] * k.cx.mr[2];
    }
#pragma unroll
    for (int dz = 0; dz < NZ; ++dz) {
        V pM[NC], pCx[NC], pCy[NC], pW[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) { pM[c] = cz<V>(); pCx[c] = cz<V>(); pCy[c] = cz<V>(); pW[c] = cz<V>(); }
#pragma unroll
        for (int dy = 0; dy < NY; ++dy) {
            const int r = (dz * NY + dy) * 3;
            const NodeV<NC, T> n0 = get(r), n1 = get(r + 1), n2 = get(r + 2);
            const T my = D >= 2 ? k.cy.m[dy] : (T)1;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int sb = Beta<D>::s(c) > 0 ? 0 : 1;
                const V x0 = n0.c[c], x1 = n1.c[c], x2 = n2.c[c];
                const V rM = cfma_r(k.cx.m[0], x0, cfma_r(k.cx.m[1], x1, cmul_r(k.cx.m[2], x2)));
                const V rC = cfma_r(k.cx.c[0], x0, cfma_r(k.cx.c[1], x1, cmul_r(k.cx.c[2], x2)));
                const V rW = cfma_r(wx[sb][0], x0, cfma_r(wx[sb][1], x1, cmul_r(wx[sb][2], x2)));
                pM[c] = cfma_r(my, rM, pM[c]);
                pCx[c] = cfma_r(my, rC, pCx[c]);
                pW[c] = cfma_r(my, rW, pW[c]);
                if (D >= 2) pCy[c] = cfma_r(k.cy.c[dy], rM, pCy[c]);
            }
        }
        const T mz = D >= 3 ? k.cz.m[dz] : (T)1;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            sM[c] = cfma_r(mz, pM[c], sM[c]);
            sCx[c] = cfma_r(mz, pCx[c], sCx[c]);
            sW[c] = cfma_r(mz, pW[c], sW[c]);
            if (D >= 2) sCy[c] = cfma_r(mz, pCy[c], sCy[c]);
            if (D >= 3) sCz[c] = cfma_r(k.cz.c[dz], pM[c], sCz[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) { GC[c] = cmul_i(sM[c]); GM[c].x = -sW[c].x; GM[c].y = -sW[c].y; }
    V aS[NC];
    alpha_apply<NC>(0, sCx, aS);
#pragma unroll
    for (int c = 0; c < NC; ++c) GM[c] = cadd(GM[c], cmul_i(aS[c]));
    if (D >= 2) {
        alpha_apply<NC>(1, sCy, aS);
#pragma unroll
        for (int c = 0; c < NC; ++c) GM[c] = cadd(GM[c], cmul_i(aS[c]));
    }
    if (D >= 3) {
        alpha_apply<NC>(2, sCz, aS);
#pragma unroll
        for (int c = 0; c < NC; ++c) GM[c] = cadd(GM[c], cmul_i(aS[c]));
    }
}

// fields() for a vanishing potential: the mass term is m beta S_M, so the
// weighted x stencil and its y / z sums are skipped.
template <int D, int NC, typename T, typename Get>
__device__ __forceinline__ void fields_nov(Get get, const NodeCoef<D, T> &k, T m, typename C2<T>::type *GC,
                                           typename C2<T>::type *GM) {
    using V = typename C2<T>::type;
    const int NZ = D >= 3 ? 3 : 1, NY = D >= 2 ? 3 : 1;
    V sM[NC], sCx[NC], sCy[NC], sCz[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) { sM[c] = cz<V>(); sCx[c] = cz<V>(); sCy[c] = cz<V>(); sCz[c] = cz<V>(); }
#pragma unroll
    for (int dz = 0; dz < NZ; ++dz) {
        V pM[NC], pCx[NC], pCy[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) { pM[c] = cz<V>(); pCx[c] = cz<V>(); pCy[c] = cz<V>(); }
#pragma unroll
        for (int dy = 0; dy < NY; ++dy) {
            const int r = (dz * NY + dy) * 3;
            const NodeV<NC, T> n0 = get(r), n1 = get(r + 1), n2 = get(r + 2);
            const T my = D >= 2 ? k.cy.m[dy] : (T)1;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const V x0 = n0.c[c], x1 = n1.c[c], x2 = n2.c[c];
                const V rM = cfma_r(k.cx.m[0], x0, cfma_r(k.cx.m[1], x1, cmul_r(k.cx.m[2], x2)));
                const V rC = cfma_r(k.cx.c[0], x0, cfma_r(k.cx.c[1], x1, cmul_r(k.cx.c[2], x2)));
                pM[c] = cfma_r(my, rM, pM[c]);
                pCx[c] = cfma_r(my, rC, pCx[c]);
                if (D >= 2) pCy[c] = cfma_r(k.cy.c[dy], rM, pCy[c]);
            }
        }
        const T mz = D >= 3 ? k.cz.m[dz] : (T)1;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            sM[c] = cfma_r(mz, pM[c], sM[c]);
            sCx[c] = cfma_r(mz, pCx[c], sCx[c]);
            if (D >= 2) sCy[c] = cfma_r(mz, pCy[c], sCy[c]);
            if (D >= 3) sCz[c] = cfma_r(k.cz.c[dz], pM[c], sCz[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        GC[c] = cmul_i(sM[c]);
        const T mb = Beta<D>::s(c) > 0 ? -m : m;        // -(m beta)
        GM[c] = cmul_r(mb, sM[c]);
    }
    V aS[NC];
    alpha_apply<NC>(0, sCx, aS);
#pragma unroll
    for (int c = 0; c < NC; ++c) GM[c] = cadd(GM[c], cmul_i(aS[c]));
    if (D >= 2) {
        alpha_apply<NC>(1, sCy, aS);
#pragma unroll
        for (int c = 0; c < NC; ++c) GM[c] = cadd(GM[c], cmul_i(aS[c]));
    }
    if (D >= 3) {
        alpha_apply<NC>(2, sCz, aS);
#pragma unroll
        for (int c = 0; c < NC; ++c) GM[c] = cadd(GM[c], cmul_i(aS[c]));
    }
}

template <int D, int NC, typename T>
__global__ void __launch_bounds__(FastTile<D>::TX * FastTile<D>::TY * FastTile<D>::TZ)
apply_fast_kernel(OpParams p, const typename C2<T>::type *__restrict__ x, typename C2<T>::type *__restrict__ y,
                  int64_t tiles_x, int64_t tiles_y) {
    using V = typename C2<T>::type;
    using Tile = FastTile<D>;
    constexpr bool PREFETCH = sizeof(T) == 4 && D <= 2;
    const int64_t tile = blockIdx.x;
    const int64_t chunk = blockIdx.y;
    const int64_t x0 = (tile % tiles_x) * Tile::TX;
    const int64_t y0 = ((tile / tiles_x) % tiles_y) * Tile::TY;
    const int64_t z0 = (tile / (tiles_x * tiles_y)) * Tile::TZ;
    const int tx = threadIdx.x % Tile::TX;
    const int ty = (threadIdx.x / Tile::TX) % Tile::TY;
    const int tz = threadIdx.x / (Tile::TX * Tile::TY);
    const int64_t ix = x0 + tx, iy = y0 + ty, iz = z0 + tz;
    const int64_t nx = p.ax[0].n, ny = p.ax[1].n, nz = p.ax[2].n;
    if (ix >= nx || iy >= ny || iz >= nz) return;
    const int64_t N = p.nt;
    const int64_t t0 = 1 + chunk * Tile::TT;
    const int64_t t1 = min(t0 + (int64_t)Tile::TT, N + 1);
    const int64_t plane_nodes = nx * ny * nz;
    const int64_t self = (iz * ny + iy) * nx + ix;

    NodeCoef<D, T> k;
    node_coef<D, T>(p, ix, iy, iz, k);
    Nbr nb;
    neighbours<D>(p, ix, iy, iz, nb);
    const T h6 = (T)(p.ht / 6.0);

    V accP[NC], accC[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) { accP[c] = cz<V>(); accC[c] = cz<V>(); }

    constexpr int K = D == 1 ? 3 : (D == 2 ? 9 : 27);
    Plane<D, NC, T> cur, nxt;   // used only when prefetching (1+1, 2+1 in FP32)
    int64_t pl = t0 - 1;
    if (PREFETCH) load_plane<D, NC, T>(x + (pl - 1) * plane_nodes * NC, nb, pl >= 1 && pl <= N, cur);
    for (; pl <= t1; ++pl) {
        const bool have = pl >= 1 && pl <= N;
        if (PREFETCH && pl + 1 <= t1)
            load_plane<D, NC, T>(x + pl * plane_nodes * NC, nb, pl + 1 >= 1 && pl + 1 <= N, nxt);
        V GC[NC], GM[NC];
        if (have) {
            if (PREFETCH) {
                fields<D, NC, T>([&](int r) { return cur.v[r]; }, k, GC, GM);
            } else {
                const V *layer = x + (pl - 1) * plane_nodes * NC;
                fields<D, NC, T>([&](int r) {
                    NodeV<NC, T> v;
                    const int NY = D >= 2 ? 3 : 1;
                    const int id = nb.at(r / (3 * NY), (r / 3) % NY, r % 3);
                    load_node<NC, T>(layer, id, id >= 0, v);
                    return v;
                }, k, GC, GM);
            }
        } else {
#pragma unroll
            for (int c = 0; c < NC; ++c) { GC[c] = cz<V>(); GM[c] = cz<V>(); }
        }
        const T cdiag = pl < N ? (T)0 : (T)0.5;
        const T mdiag = pl < N ? 4 * h6 : 2 * h6;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            accP[c] = cfma_r((T)0.5, GC[c], cfma_r(h6, GM[c], accP[c]));
            accC[c] = cfma_r(cdiag, GC[c], cfma_r(mdiag, GM[c], accC[c]));
        }
        if (pl - 1 >= t0 && pl - 1 < t1) store_node<NC, T>(y + (pl - 2) * plane_nodes * NC, self, accP);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            accP[c] = accC[c];
            accC[c] = cfma_r((T)(-0.5), GC[c], cmul_r(h6, GM[c]));
        }
        if (PREFETCH) {
#pragma unroll
            for (int q = 0; q < K; ++q) cur.v[q] = nxt.v[q];
        }
    }
}

template <int D, int NC, typename T>
int launch_apply_fast(const OpParams &p, const typename C2<T>::type *x, typename C2<T>::type *y, cudaStream_t s) {
    using Tile = FastTile<D>;
    const int64_t tx = (p.ax[0].n + Tile::TX - 1) / Tile::TX;
    const int64_t ty = (p.ax[1].n + Tile::TY - 1) / Tile::TY;
    const int64_t tz = (p.ax[2].n + Tile::TZ - 1) / Tile::TZ;
    const int64_t chunks = (p.nt + Tile::TT - 1) / Tile::TT;
    const int64_t tiles = tx * ty * tz;
    if (tiles <= 0 || tiles > 0x7fffffffLL || chunks > 65535) return DST_ERR_ARG;
    if (p.ax[0].n * p.ax[1].n * p.ax[2].n >= (1LL << 30)) return launch_apply<D, NC, T>(p, x, y, s);
    dim3 grid((unsigned)tiles, (unsigned)chunks);
    apply_fast_kernel<D, NC, T><<<grid, Tile::TX * Tile::TY * Tile::TZ, 0, s>>>(p, x, y, tx, ty);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

}  // namespace dst
