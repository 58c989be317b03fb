// Matrix-free operator apply y = D_w22 x and right-hand side b = -D_w21 psi0.
//
// The weak form of Sec. 2.1 (Eqs. 6-12) summed element by element (Sec. 2.2)
// on a structured Q1 mesh is a tensor-product stencil (Sec. 2.2: on a grid
// the FEM relation between nodes is a finite-difference stencil).  With the
// rows premultiplied by gamma^0 the element operator of Appendix A becomes
//     A_e = i D^t (x) I + i sum_k D^k (x) alpha_k - D^0 (x) (m beta + V_e),
// and each D^mu is a Kronecker product of 1D Q1 matrices: the mass
// M = h/6 [[2,1],[1,2]] and the convection C = [[-1/2,1/2],[-1/2,1/2]]
// (row = test node, column = trial node).  Assembled along one axis they are
// 3-point stencils whose end coefficients drop the missing element.
//
// Evaluation order (sum factorisation, spatial first): for every time plane
// p of x the kernel forms, per spinor component, the spatial fields
//     S_M  = (M_z M_y M_x) x_p            (goes with C_t: the i d_t term)
//     S_Ck = (... C_k ...) x_p             (goes with M_t: the alpha_k terms)
//     S_w  = (M_z M_y M^w_x) x_p           (goes with M_t: the m beta + V term)
// and combines them with the spin matrices into G_C = i S_M and
// G_M = i sum_k alpha_k S_Ck - S_w.  The time stencils then read
//     y(t) = sum_{p in t-1..t+1} C_t[t][p] G_C(p) + M_t[t][p] G_M(p),
// so each thread keeps just two running output accumulators while it streams
// the planes of its time chunk (the t = 0 layer is known: its plane is zero
// in the apply and is the only input of the right-hand side).
//
// One CTA owns a spatial tile (TX x TY x TZ outputs) and a chunk of TT time
// layers; every plane of the tile plus a one-node halo is staged in shared
// memory (periodic halos wrap, halos outside a non-periodic axis are zero).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace dst {

template <typename T> struct C2;
template <> struct C2<double> { using type = double2; };
template <> struct C2<float> { using type = float2; };

template <int D> struct ApplyTile;
template <> struct ApplyTile<1> { static constexpr int TX = 128, TY = 1, TZ = 1, TT = 32; };
template <> struct ApplyTile<2> { static constexpr int TX = 32, TY = 8, TZ = 1, TT = 16; };
template <> struct ApplyTile<3> { static constexpr int TX = 16, TY = 4, TZ = 4, TT = 8; };

template <typename V> __device__ __forceinline__ V cz() { V r; r.x = 0; r.y = 0; return r; }
template <typename V, typename T> __device__ __forceinline__ V cmul_r(T a, V v) { V r; r.x = a * v.x; r.y = a * v.y; return r; }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { V r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { V r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename V, typename T> __device__ __forceinline__ V cfma_r(T a, V v, V acc) {
    V r; r.x = fma(a, v.x, acc.x); r.y = fma(a, v.y, acc.y); return r;
}
// multiply by i
template <typename V> __device__ __forceinline__ V cmul_i(V v) { V r; r.x = -v.y; r.y = v.x; return r; }

// 3-point coefficients of one axis at one unknown node.
template <typename T>
struct Coef3 {
    T m[3];       // mass stencil (left, centre, right)
    T c[3];       // convection stencil
    T ml[3];      // left-element part of the mass stencil: eL*h/6*(1,2,0)
    T mr[3];      // right-element part: eR*h/6*(0,2,1)
    int64_t eL_idx, eR_idx;   // element indices (meaningful when present)
    bool eL, eR;
};

template <typename T>
__device__ __forceinline__ Coef3<T> axis_coef(const AxisDesc &a, int64_t i) {
    Coef3<T> k;
    int64_t g = i + a.u0;
    if (a.bc == DST_BC_PERIODIC) {
        k.eL = true; k.eR = true;
        k.eL_idx = (g - 1 + a.nel) % a.nel; k.eR_idx = g % a.nel;
    } else if (a.bc == DST_BC_OPEN) {
        k.eL = g >= 1; k.eR = g <= a.nel - 1;
        k.eL_idx = g - 1; k.eR_idx = g;
    } else {
        k.eL = true; k.eR = true;
        k.eL_idx = g - 1; k.eR_idx = g;
    }
    T h6 = (T)(a.h / 6.0);
    T l = k.eL ? (T)1 : (T)0, r = k.eR ? (T)1 : (T)0;
    k.ml[0] = l * h6; k.ml[1] = 2 * l * h6; k.ml[2] = 0;
    k.mr[0] = 0; k.mr[1] = 2 * r * h6; k.mr[2] = r * h6;
    for (int j = 0; j < 3; ++j) k.m[j] = k.ml[j] + k.mr[j];
    k.c[0] = -l * (T)0.5; k.c[1] = (l - r) * (T)0.5; k.c[2] = r * (T)0.5;
    return k;
}

// Neighbour index along an axis (-1 if it is not an unknown node).
__device__ __forceinline__ int64_t axis_nbr(const AxisDesc &a, int64_t i) {
    if (a.bc == DST_BC_PERIODIC) return (i % a.n + a.n) % a.n;
    return (i >= 0 && i < a.n) ? i : -1;
}

template <int D> struct Beta;   // beta = gamma^0 signs per component
template <> struct Beta<1> { __device__ static constexpr int s(int c) { return c == 0 ? 1 : -1; } };
template <> struct Beta<2> { __device__ static constexpr int s(int c) { return c == 0 ? 1 : -1; } };
template <> struct Beta<3> { __device__ static constexpr int s(int c) { return c < 2 ? 1 : -1; } };

// alpha_k S for the representation used: NC = 2: alpha = (sigma_x, sigma_y);
// NC = 4: alpha_k = [[0, sigma_k], [sigma_k, 0]].
template <typename V>
__device__ __forceinline__ void sigma_apply(int k, V a, V b, V &ra, V &rb) {
    if (k == 0) { ra = b; rb = a; }                                         // sigma_x
    else if (k == 1) { V nb = cmul_i(b); ra.x = -nb.x; ra.y = -nb.y; rb = cmul_i(a); }  // sigma_y: (-i b, i a)
    else { ra = a; rb.x = -b.x; rb.y = -b.y; }                              // sigma_z
}

template <int NC, typename V>
__device__ __forceinline__ void alpha_apply(int k, const V *S, V *out) {
    if (NC == 2) {
        sigma_apply(k, S[0], S[1], out[0], out[1]);
    } else {
        sigma_apply(k, S[2], S[3], out[0], out[1]);
        sigma_apply(k, S[0], S[1], out[2], out[3]);
    }
}

// Per-thread constants for the spatial stencils of one output node.
template <int D, typename T>
struct NodeCoef {
    Coef3<T> cx, cy, cz;
    T wl[2], wr[2];     // separable: x-element weights (m*beta + V) for beta = +1 / -1
    T vc[8];            // general: V of the 2^D elements around the node (corner order x fastest)
};

template <int D, typename T>
__device__ __forceinline__ void node_coef(const OpParams &p, int64_t ix, int64_t iy, int64_t iz,
                                          NodeCoef<D, T> &nc) {
    nc.cx = axis_coef<T>(p.ax[0], ix);
    if (D >= 2) nc.cy = axis_coef<T>(p.ax[1], iy);
    if (D >= 3) nc.cz = axis_coef<T>(p.ax[2], iz);
    const int64_t nelx = p.ax[0].nel;
    if (p.vmode != 1) {
        for (int s = 0; s < 2; ++s) {
            nc.wl[s] = nc.cx.eL ? (T)p.wx[s * nelx + nc.cx.eL_idx] : (T)0;
            nc.wr[s] = nc.cx.eR ? (T)p.wx[s * nelx + nc.cx.eR_idx] : (T)0;
        }
    } else {
        nc.wl[0] = nc.wr[0] = (T)p.m; nc.wl[1] = nc.wr[1] = (T)(-p.m);
        const int64_t nely = p.ax[1].nel;
        for (int corner = 0; corner < (1 << D); ++corner) {
            int sx = corner & 1, sy = (corner >> 1) & 1, sz = (corner >> 2) & 1;
            bool ok = sx ? nc.cx.eR : nc.cx.eL;
            int64_t ex = sx ? nc.cx.eR_idx : nc.cx.eL_idx, ey = 0, ez = 0;
            if (D >= 2) { ok = ok && (sy ? nc.cy.eR : nc.cy.eL); ey = sy ? nc.cy.eR_idx : nc.cy.eL_idx; }
            if (D >= 3) { ok = ok && (sz ? nc.cz.eR : nc.cz.eL); ez = sz ? nc.cz.eR_idx : nc.cz.eL_idx; }
            nc.vc[corner] = ok ? (T)p.Vel[(ez * nely + ey) * nelx + ex] : (T)0;
        }
    }
}

// Spatial fields of one node from the staged box, combined with the spin
// matrices into G_C (C_t partner) and G_M (M_t partner).
// box: shared array [(bz*BY + by)*BX + bx][NC]; (bx, by, bz) = centre.
template <int D, int NC, typename T, int BX, int BY>
__device__ __forceinline__ void spatial_G(const typename C2<T>::type *box, int bx, int by, int bz,
                                          const NodeCoef<D, T> &k, bool vgen,
                                          typename C2<T>::type *GC, typename C2<T>::type *GM) {
    using V = typename C2<T>::type;
    V SM[NC], SW[NC], SC[3][NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int sb = Beta<D>::s(c) > 0 ? 0 : 1;
        const T wl = k.wl[sb], wr = k.wr[sb];
        V sM = cz<V>(), sW = cz<V>(), sCx = cz<V>(), sCy = cz<V>(), sCz = cz<V>(), sV = cz<V>();
        const int NZ = D >= 3 ? 3 : 1, NY = D >= 2 ? 3 : 1;
#pragma unroll
        for (int dz = 0; dz < NZ; ++dz) {
            V pM = cz<V>(), pCx = cz<V>(), pCy = cz<V>(), pW = cz<V>();
            V pL[2] = {cz<V>(), cz<V>()}, pR[2] = {cz<V>(), cz<V>()};   // general V: per (sy) row sums
#pragma unroll
            for (int dy = 0; dy < NY; ++dy) {
                const int zz = D >= 3 ? bz - 1 + dz : bz, yy = D >= 2 ? by - 1 + dy : by;
                const V *row = box + ((zz * BY + yy) * BX + (bx - 1)) * NC + c;
                V x0 = row[0], x1 = row[NC], x2 = row[2 * NC];
                V rM = cfma_r(k.cx.m[0], x0, cfma_r(k.cx.m[1], x1, cmul_r(k.cx.m[2], x2)));
                V rC = cfma_r(k.cx.c[0], x0, cfma_r(k.cx.c[1], x1, cmul_r(k.cx.c[2], x2)));
                V rL = cfma_r(k.cx.ml[0], x0, cmul_r(k.cx.ml[1], x1));
                V rR = cfma_r(k.cx.mr[1], x1, cmul_r(k.cx.mr[2], x2));
                V rW = cadd(cmul_r(wl, rL), cmul_r(wr, rR));
                T my = D >= 2 ? k.cy.m[dy] : (T)1;
                pM = cfma_r(my, rM, pM);
                pCx = cfma_r(my, rC, pCx);
                pW = cfma_r(my, rW, pW);
                if (D >= 2) {
                    pCy = cfma_r(k.cy.c[dy], rM, pCy);
                    if (vgen) {
                        pL[0] = cfma_r(k.cy.ml[dy], rL, pL[0]); pL[1] = cfma_r(k.cy.mr[dy], rL, pL[1]);
                        pR[0] = cfma_r(k.cy.ml[dy], rR, pR[0]); pR[1] = cfma_r(k.cy.mr[dy], rR, pR[1]);
                    }
                } else if (vgen) {
                    pL[0] = rL; pR[0] = rR;
                }
            }
            T mz = D >= 3 ? k.cz.m[dz] : (T)1;
            sM = cfma_r(mz, pM, sM);
            sCx = cfma_r(mz, pCx, sCx);
            sW = cfma_r(mz, pW, sW);
            if (D >= 2) sCy = cfma_r(mz, pCy, sCy);
            if (D >= 3) sCz = cfma_r(k.cz.c[dz], pM, sCz);
            if (vgen) {
                // corners: x side (L/R) x y side (L/R) x z side (L/R)
                if (D == 1) {
                    sV = cadd(cmul_r(k.vc[0], pL[0]), cmul_r(k.vc[1], pR[0]));
                } else if (D == 2) {
                    sV = cadd(sV, cadd(cadd(cmul_r(k.vc[0], pL[0]), cmul_r(k.vc[1], pR[0])),
                                       cadd(cmul_r(k.vc[2], pL[1]), cmul_r(k.vc[3], pR[1]))));
                } else {
                    T zl = k.cz.ml[dz], zr = k.cz.mr[dz];
                    V lo = cadd(cadd(cmul_r(k.vc[0], pL[0]), cmul_r(k.vc[1], pR[0])),
                                cadd(cmul_r(k.vc[2], pL[1]), cmul_r(k.vc[3], pR[1])));
                    V hi = cadd(cadd(cmul_r(k.vc[4], pL[0]), cmul_r(k.vc[5], pR[0])),
                                cadd(cmul_r(k.vc[6], pL[1]), cmul_r(k.vc[7], pR[1])));
                    sV = cfma_r(zl, lo, cfma_r(zr, hi, sV));
                }
            }
        }
        SM[c] = sM;
        SW[c] = vgen ? cadd(cmul_r((T)(Beta<D>::s(c)) * k.wl[0] , sM), sV) : sW;
        SC[0][c] = sCx;
        if (D >= 2) SC[1][c] = sCy;
        if (D >= 3) SC[2][c] = sCz;
    }
    // spin combination
#pragma unroll
    for (int c = 0; c < NC; ++c) { GC[c] = cmul_i(SM[c]); GM[c].x = -SW[c].x; GM[c].y = -SW[c].y; }
#pragma unroll
    for (int kk = 0; kk < D; ++kk) {
        V aS[NC];
        alpha_apply<NC>(kk, SC[kk], aS);
#pragma unroll
        for (int c = 0; c < NC; ++c) GM[c] = cadd(GM[c], cmul_i(aS[c]));
    }
}

template <int D, int NC, typename T>
struct ApplyShape {
    using Tile = ApplyTile<D>;
    static constexpr int BX = Tile::TX + 2;
    static constexpr int BY = D >= 2 ? Tile::TY + 2 : 1;
    static constexpr int BZ = D >= 3 ? Tile::TZ + 2 : 1;
    static constexpr int BOX = BX * BY * BZ;
    static constexpr int NTHR = Tile::TX * Tile::TY * Tile::TZ;
};

// Stage plane `layer_ptr` (one time layer, n_spatial*NC complex) of the tile
// box into shared memory; zero outside non-periodic axes.
template <int D, int NC, typename T>
__device__ __forceinline__ void stage_plane(const OpParams &p, const typename C2<T>::type *layer_ptr,
                                            typename C2<T>::type *box, int64_t x0, int64_t y0, int64_t z0) {
    using V = typename C2<T>::type;
    using S = ApplyShape<D, NC, T>;
    const int64_t nx = p.ax[0].n, ny = p.ax[1].n;
    for (int i = threadIdx.x; i < S::BOX; i += S::NTHR) {
        int bx = i % S::BX, by = (i / S::BX) % S::BY, bz = i / (S::BX * S::BY);
        int64_t gx = axis_nbr(p.ax[0], x0 - 1 + bx);
        int64_t gy = D >= 2 ? axis_nbr(p.ax[1], y0 - 1 + by) : 0;
        int64_t gz = D >= 3 ? axis_nbr(p.ax[2], z0 - 1 + bz) : 0;
        V *dst = box + (int64_t)i * NC;
        if (gx >= 0 && gy >= 0 && gz >= 0) {
            const V *src = layer_ptr + ((gz * ny + gy) * nx + gx) * NC;
#pragma unroll
            for (int c = 0; c < NC; ++c) dst[c] = src[c];
        } else {
#pragma unroll
            for (int c = 0; c < NC; ++c) dst[c] = cz<V>();
        }
    }
}

// y = A x over one (tile, time chunk) per CTA.
template <int D, int NC, typename T>
__global__ void __launch_bounds__(ApplyShape<D, NC, T>::NTHR)
apply_kernel(OpParams p, const typename C2<T>::type *__restrict__ x, typename C2<T>::type *__restrict__ y,
             int64_t tiles_x, int64_t tiles_y, int64_t tiles_z) {
    using V = typename C2<T>::type;
    using S = ApplyShape<D, NC, T>;
    using Tile = typename S::Tile;
    __shared__ V box[S::BOX * NC];

    const int64_t ntiles = tiles_x * tiles_y * tiles_z;
    const int64_t tile = blockIdx.x % ntiles;
    const int64_t chunk = blockIdx.x / ntiles;
    const int64_t x0 = (tile % tiles_x) * Tile::TX;
    const int64_t y0 = ((tile / tiles_x) % tiles_y) * Tile::TY;
    const int64_t z0 = (tile / (tiles_x * tiles_y)) * Tile::TZ;
    const int tx = threadIdx.x % Tile::TX;
    const int ty = (threadIdx.x / Tile::TX) % Tile::TY;
    const int tz = threadIdx.x / (Tile::TX * Tile::TY);
    const int64_t ix = x0 + tx, iy = y0 + ty, iz = z0 + tz;
    const int64_t nx = p.ax[0].n, ny = p.ax[1].n, nz = p.ax[2].n;
    const bool valid = ix < nx && iy < ny && iz < nz;
    const int64_t N = p.nt;
    const int64_t t0 = 1 + chunk * Tile::TT;                 // first output layer (1-based)
    const int64_t t1 = min(t0 + (int64_t)Tile::TT, N + 1);   // one past the last
    const int64_t plane = nx * ny * nz * NC;
    const int64_t node_off = ((iz * ny + iy) * nx + ix) * NC;

    NodeCoef<D, T> k;
    if (valid) node_coef<D, T>(p, ix, iy, iz, k);
    const bool vgen = p.vmode == 1;
    const T h6 = (T)(p.ht / 6.0);

    V accP[NC], accC[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) { accP[c] = cz<V>(); accC[c] = cz<V>(); }

    for (int64_t pl = t0 - 1; pl <= t1; ++pl) {
        const bool have = pl >= 1 && pl <= N;
        V GC[NC], GM[NC];
        if (have) {
            __syncthreads();
            stage_plane<D, NC, T>(p, x + (pl - 1) * plane, box, x0, y0, z0);
            __syncthreads();
        }
        if (have && valid) {
            spatial_G<D, NC, T, S::BX, S::BY>(box, tx + 1, D >= 2 ? ty + 1 : 0, D >= 3 ? tz + 1 : 0, k, vgen, GC, GM);
        } else {
#pragma unroll
            for (int c = 0; c < NC; ++c) { GC[c] = cz<V>(); GM[c] = cz<V>(); }
        }
        // y(pl-1) += C_t[pl-1][pl] G_C + M_t[pl-1][pl] G_M = G_C/2 + h/6 G_M; then complete
        const T cdiag = pl < N ? (T)0 : (T)0.5;
        const T mdiag = pl < N ? 4 * h6 : 2 * h6;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            accP[c] = cfma_r((T)0.5, GC[c], cfma_r(h6, GM[c], accP[c]));
            accC[c] = cfma_r(cdiag, GC[c], cfma_r(mdiag, GM[c], accC[c]));
        }
        if (valid && pl - 1 >= t0 && pl - 1 < t1) {
            V *dst = y + (pl - 2) * plane + node_off;
#pragma unroll
            for (int c = 0; c < NC; ++c) dst[c] = accP[c];
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            accP[c] = accC[c];
            accC[c] = cfma_r((T)(-0.5), GC[c], cmul_r(h6, GM[c]));
        }
    }
}

// b(layer 1) = -( C_t[1][0] G_C(psi0) + M_t[1][0] G_M(psi0) ) = G_C/2 - h/6 G_M.
template <int D, int NC>
__global__ void __launch_bounds__(ApplyShape<D, NC, double>::NTHR)
rhs_kernel(OpParams p, const double2 *__restrict__ psi0, double2 *__restrict__ b,
           int64_t tiles_x, int64_t tiles_y, int64_t tiles_z) {
    using V = double2;
    using S = ApplyShape<D, NC, double>;
    using Tile = typename S::Tile;
    __shared__ V box[S::BOX * NC];
    const int64_t tile = blockIdx.x;
    const int64_t x0 = (tile % tiles_x) * Tile::TX;
    const int64_t y0 = ((tile / tiles_x) % tiles_y) * Tile::TY;
    const int64_t z0 = (tile / (tiles_x * tiles_y)) * Tile::TZ;
    const int tx = threadIdx.x % Tile::TX;
    const int ty = (threadIdx.x / Tile::TX) % Tile::TY;
    const int tz = threadIdx.x / (Tile::TX * Tile::TY);
    const int64_t ix = x0 + tx, iy = y0 + ty, iz = z0 + tz;
    const int64_t nx = p.ax[0].n, ny = p.ax[1].n, nz = p.ax[2].n;
    const bool valid = ix < nx && iy < ny && iz < nz;
    stage_plane<D, NC, double>(p, psi0, box, x0, y0, z0);
    __syncthreads();
    if (!valid) return;
    NodeCoef<D, double> k;
    node_coef<D, double>(p, ix, iy, iz, k);
    V GC[NC], GM[NC];
    spatial_G<D, NC, double, S::BX, S::BY>(box, tx + 1, D >= 2 ? ty + 1 : 0, D >= 3 ? tz + 1 : 0, k, p.vmode == 1, GC, GM);
    const double h6 = p.ht / 6.0;
    V *dst = b + ((iz * ny + iy) * nx + ix) * NC;
#pragma unroll
    for (int c = 0; c < NC; ++c) dst[c] = cfma_r(-h6, GM[c], cmul_r(0.5, GC[c]));
}

template <int D, int NC, typename T>
int launch_apply(const OpParams &p, const typename C2<T>::type *x, typename C2<T>::type *y, cudaStream_t s) {
    using Tile = ApplyTile<D>;
    using S = ApplyShape<D, NC, T>;
    const int64_t tx = (p.ax[0].n + Tile::TX - 1) / Tile::TX;
    const int64_t ty = (p.ax[1].n + Tile::TY - 1) / Tile::TY;
    const int64_t tz = (p.ax[2].n + Tile::TZ - 1) / Tile::TZ;
    const int64_t chunks = (p.nt + Tile::TT - 1) / Tile::TT;
    const int64_t blocks = tx * ty * tz * chunks;
    if (blocks <= 0 || blocks > 0x7fffffffLL) return DST_ERR_ARG;
    apply_kernel<D, NC, T><<<(unsigned)blocks, S::NTHR, 0, s>>>(p, x, y, tx, ty, tz);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

template <int D, int NC>
int launch_rhs(const OpParams &p, const double2 *psi0, double2 *b, cudaStream_t s) {
    using Tile = ApplyTile<D>;
    using S = ApplyShape<D, NC, double>;
    const int64_t plane = p.ax[0].n * p.ax[1].n * p.ax[2].n * NC;
    DST_CUDA_TRY(cudaMemsetAsync(b, 0, sizeof(double2) * plane * p.nt, s));
    const int64_t tx = (p.ax[0].n + Tile::TX - 1) / Tile::TX;
    const int64_t ty = (p.ax[1].n + Tile::TY - 1) / Tile::TY;
    const int64_t tz = (p.ax[2].n + Tile::TZ - 1) / Tile::TZ;
    const int64_t blocks = tx * ty * tz;
    if (blocks <= 0 || blocks > 0x7fffffffLL) return DST_ERR_ARG;
    rhs_kernel<D, NC><<<(unsigned)blocks, S::NTHR, 0, s>>>(p, psi0, b, tx, ty, tz);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

}  // namespace dst
