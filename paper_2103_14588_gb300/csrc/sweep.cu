// Crank-Nicolson sweep: a time-marching right preconditioner for flexible GMRES.
//
// The paper's conclusion (Sec. 5) asks for a preconditioner and points at
// decomposing the time direction.  Row t of D_w22 (Eq. 11) tests against the
// hat function of time node t, the sum of its halves on the elements (t-1, t)
// and (t, t+1).  Testing each time element against a constant instead gives
// Crank-Nicolson, the block lower-bidiagonal
//     B[t, t] = Bd = i M_s + (h_t/2) K_s,   B[t, t-1] = Bl = -i M_s + (h_t/2) K_s,
// with M_s the spatial mass matrix and K_s the spatial part of the operator
// (the sum of i alpha_k D^k - (m beta + V) D^0 over the spatial element
// matrices of Appendix A).  Averaging adjacent element rows, S = (I + U) / 2
// (U the shift to the next layer, the last layer keeping 1/2), reproduces the
// time derivative of D_w22 exactly and its spatial part up to a second
// difference in time.  The preconditioner is M = B^-1 S^-1:
//   s = S^-1 v:  s_{N-1} = 2 v_{N-1},  s_t = 2 v_t - s_{t+1}          (time scan)
//   x = B^-1 s:  x_0 = Bd^-1 s_0,      x_t = Bd^-1 (s_t - Bl x_{t-1}) (forward march)
// one spatial solve with Bd per layer.
//
// GPU layout of the work (FP32 vectors, the precision of the inner solve):
//   1. time scan, one thread per spatial entry, backward over the layers;
//   2. FFT over the periodic spatial axes of every (layer, x-node) plane, in
//      shared memory (mixed-radix Stockham, one warp per line);
//   3. the march per frequency of those axes:
//      spectral mode (every axis periodic, constant potential): M_s and K_s are
//        diagonal in frequency with NC x NC blocks, so the march is one scan over
//        t per frequency with a fixed 2 x 2 / 4 x 4 recurrence;
//      banded mode (x Dirichlet, y / z periodic, potential depending on x only):
//        per frequency of (y, z) each layer solve is block tridiagonal along x,
//        solved by a block Thomas elimination whose factors (computed once per
//        mesh in FP64) are stored; NC lanes of a warp march one frequency;
//   4. inverse FFT back to the node layout.
// The result is the same linear map as the assembled sweep (up to FP32
// rounding); meshes of other kinds (open axes, two or more non-periodic axes,
// a potential varying along a periodic axis) get DST_ERR_ARG.
#include <cmath>
#include <cstring>
#include <vector>

#include "blas.h"
#include "internal.h"
#include "sweep.h"
#include "fft.cuh"

namespace {

constexpr double PI = 3.14159265358979323846;

// ---- small complex helpers -------------------------------------------------
struct cd {
    double x, y;
};
__host__ __device__ inline cd mkcd(double a, double b) { return cd{a, b}; }
__host__ __device__ inline cd operator+(cd a, cd b) { return cd{a.x + b.x, a.y + b.y}; }
__host__ __device__ inline cd operator-(cd a, cd b) { return cd{a.x - b.x, a.y - b.y}; }
__host__ __device__ inline cd operator*(cd a, cd b) { return cd{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__host__ __device__ inline cd cdiv(cd a, cd b) {
    const double d = b.x * b.x + b.y * b.y;
    return cd{(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 csubf(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// acc + a * b
__device__ __forceinline__ float2 cfmaf(float2 a, float2 b, float2 acc) {
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}

// ---- spin structure: each row of alpha_k has one non-zero entry -------------
// (alpha_k v)_c = phi_k(c) v_{pi_k(c)}; beta = diag(s_c).
// NC = 2 (1+1, 2+1): alpha_x = sigma_x, alpha_y = sigma_y, beta = sigma_z.
// NC = 4 (3+1, Dirac representation): alpha_k = [[0, sigma_k], [sigma_k, 0]], beta = diag(1, 1, -1, -1).
__host__ __device__ inline int spin_pi(int nc, int k, int c) {
    if (nc == 2) return 1 - c;
    return k == 2 ? (c + 2) & 3 : 3 - c;
}
__host__ __device__ inline cd spin_phi(int nc, int k, int c) {
    if (k == 0) return mkcd(1.0, 0.0);
    if (k == 1) return (c & 1) ? mkcd(0.0, 1.0) : mkcd(0.0, -1.0);     // sigma_y rows: (-i, i)
    return (c & 1) ? mkcd(-1.0, 0.0) : mkcd(1.0, 0.0);                  // sigma_z in the off-diagonal blocks
}
__host__ __device__ inline double beta_s(int nc, int c) { return nc == 2 ? (c == 0 ? 1.0 : -1.0) : (c < 2 ? 1.0 : -1.0); }

// A layer-operator block a I + sum_k b_k alpha_k + diag(dc), dense NC x NC.
struct Blk {
    cd a, b[3];
    double dc[4];
};
__host__ __device__ inline void blk_dense(const Blk &B, int nc, int nk, cd (*out)[4]) {
    for (int c = 0; c < nc; ++c)
        for (int d = 0; d < nc; ++d) out[c][d] = mkcd(0.0, 0.0);
    for (int c = 0; c < nc; ++c) {
        out[c][c] = out[c][c] + B.a + mkcd(B.dc[c], 0.0);
        for (int k = 0; k < nk; ++k) out[c][spin_pi(nc, k, c)] = out[c][spin_pi(nc, k, c)] + B.b[k] * spin_phi(nc, k, c);
    }
}

// In-place inverse of an NC x NC complex matrix (Gauss-Jordan, partial pivoting).
__host__ __device__ inline void inv_small(cd (*A)[4], int n, cd (*R)[4]) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) R[i][j] = mkcd(i == j ? 1.0 : 0.0, 0.0);
    for (int col = 0; col < n; ++col) {
        int p = col;
        double best = A[col][col].x * A[col][col].x + A[col][col].y * A[col][col].y;
        for (int r = col + 1; r < n; ++r) {
            const double v = A[r][col].x * A[r][col].x + A[r][col].y * A[r][col].y;
            if (v > best) { best = v; p = r; }
        }
        if (p != col)
            for (int j = 0; j < n; ++j) {
                cd t = A[col][j]; A[col][j] = A[p][j]; A[p][j] = t;
                t = R[col][j]; R[col][j] = R[p][j]; R[p][j] = t;
            }
        const cd piv = A[col][col];
        for (int j = 0; j < n; ++j) { A[col][j] = cdiv(A[col][j], piv); R[col][j] = cdiv(R[col][j], piv); }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const cd f = A[r][col];
            for (int j = 0; j < n; ++j) { A[r][j] = A[r][j] - f * A[col][j]; R[r][j] = R[r][j] - f * R[col][j]; }
        }
    }
}

// Symbols of the 1D Q1 stencils at frequency theta: mass h (2 + cos th) / 3, convection i sin th.
__host__ __device__ inline double mass_sym(double h, double th) { return h * (2.0 + cos(th)) / 3.0; }

// ---- 1. time scan: s = S^-1 v -----------------------------------------------
// The loads of the next PD layers are issued before a layer is combined.
__global__ void time_scan_kernel(int64_t per, int64_t nt, const float2 *__restrict__ v, float2 *__restrict__ s) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= per) return;
    constexpr int PD = 8;
    float2 ring[PD];
#pragma unroll
    for (int q = 0; q < PD; ++q) ring[q] = nt - 1 - q >= 0 ? v[(nt - 1 - q) * per + e] : make_float2(0.f, 0.f);
    float2 acc = make_float2(0.f, 0.f);
    for (int64_t k0 = 0; k0 < nt; k0 += PD) {
#pragma unroll
        for (int q = 0; q < PD; ++q) {
            const int64_t t = nt - 1 - (k0 + q);
            if (t >= 0) {
                const float2 a = ring[q];
                if (t - PD >= 0) ring[q] = v[(t - PD) * per + e];
                acc = make_float2(2.f * a.x - acc.x, 2.f * a.y - acc.y);
                s[t * per + e] = acc;
            }
        }
    }
}

// ---- 3a. spectral march: one thread per frequency ---------------------------
// Blocks of frequency f:  Bd = i M^ + (h_t/2) K^,  Bl = -i M^ + (h_t/2) K^ with
// K^ = sum_k alpha_k (i sin th_k) i prod_{j != k} m_j - (m beta + V0) prod_j m_j.
template <int NC>
__global__ void march_spectral_kernel(SweepGeom g, float2 *__restrict__ x) {
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nf = (int64_t)g.n1 * g.n2;
    if (f >= nf) return;
    // frequencies of the axes: FFT dims (outer n1, inner n2) map to physical axes ax1, ax2
    double th[3] = {0.0, 0.0, 0.0};
    const int i1 = (int)(f / g.n2), i2 = (int)(f % g.n2);
    if (g.ax1 >= 0) th[g.ax1] = 2.0 * PI * i1 / g.n1;
    if (g.ax2 >= 0) th[g.ax2] = 2.0 * PI * i2 / g.n2;
    double mk[3], pm = 1.0;
    for (int k = 0; k < 3; ++k) {
        mk[k] = k < g.d ? mass_sym(g.h[k], th[k]) : 1.0;
        pm *= mk[k];
    }
    Blk kb;                       // K^ as a block
    kb.a = mkcd(0.0, 0.0);
    for (int k = 0; k < 3; ++k) {
        double o = k < g.d ? -sin(th[k]) : 0.0;                   // i alpha_k (i sin) = -sin alpha_k
        for (int j = 0; j < g.d; ++j)
            if (j != k) o *= mk[j];
        kb.b[k] = mkcd(0.5 * g.ht * o, 0.0);
    }
    for (int c = 0; c < 4; ++c) kb.dc[c] = c < NC ? -0.5 * g.ht * (g.m * beta_s(NC, c) + g.V0) * pm : 0.0;
    Blk bd = kb, bl = kb;
    bd.a = mkcd(0.0, pm);
    bl.a = mkcd(0.0, -pm);
    cd D[4][4], L[4][4], P[4][4];
    blk_dense(bd, NC, g.d, D);
    blk_dense(bl, NC, g.d, L);
    inv_small(D, NC, P);
    // Q = P Bl; x_t = P s_t - Q x_{t-1}
    float2 Pf[NC][NC], Qf[NC][NC];
    for (int c = 0; c < NC; ++c)
        for (int e = 0; e < NC; ++e) {
            cd q = mkcd(0.0, 0.0);
            for (int d = 0; d < NC; ++d) q = q + P[c][d] * L[d][e];
            Pf[c][e] = make_float2((float)P[c][e].x, (float)P[c][e].y);
            Qf[c][e] = make_float2((float)q.x, (float)q.y);
        }
    float2 xp[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) xp[c] = make_float2(0.f, 0.f);
    // the loads of the next PD layers are in flight while a layer is combined
    constexpr int PD = 4;
    float2 ring[PD][NC];
#pragma unroll
    for (int q = 0; q < PD; ++q)
#pragma unroll
        for (int c = 0; c < NC; ++c)
            ring[q][c] = q < g.nt ? x[((int64_t)q * nf + f) * NC + c] : make_float2(0.f, 0.f);
    for (int64_t t0 = 0; t0 < g.nt; t0 += PD) {
#pragma unroll
        for (int q = 0; q < PD; ++q) {
            const int64_t t = t0 + q;
            if (t < g.nt) {
                float2 sv[NC], xn[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) sv[c] = ring[q][c];
                if (t + PD < g.nt) {
#pragma unroll
                    for (int c = 0; c < NC; ++c) ring[q][c] = x[((t + PD) * nf + f) * NC + c];
                }
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                    for (int d = 0; d < NC; ++d) {
                        acc = cfmaf(Pf[c][d], sv[d], acc);
                        acc = csubf(acc, cmulf(Qf[c][d], xp[d]));
                    }
                    xn[c] = acc;
                }
                float2 *pt = x + (t * nf + f) * NC;
#pragma unroll
                for (int c = 0; c < NC; ++c) { xp[c] = xn[c]; pt[c] = xn[c]; }
            }
        }
    }
}

// ---- 3b. banded mode: block Thomas along x per frequency of (y, z) -----------
// Unknown x node i (geometric node i + 1 of a Dirichlet axis), offset o in {-1, 0, 1}.
struct XRow {
    double M, C;      // 1D mass (h/6 [1,4,1]) and convection (1/2 [-1,0,1]) entries
    double W[2];      // element-weighted mass with w_e = s m + V_e, for beta sign s = +1 / -1
};
__host__ __device__ inline XRow xrow(const SweepGeom &g, const double *Vx, int i, int o) {
    XRow r;
    const double h6 = g.h[0] / 6.0;
    const int gi = i + 1;                       // geometric node
    const double vl = Vx ? Vx[gi - 1] : 0.0;    // element left of the node
    const double vr = Vx ? Vx[gi] : 0.0;        // element right of the node
    if (o == 0) {
        r.M = 4.0 * h6;
        r.C = 0.0;
        r.W[0] = 2.0 * h6 * ((g.m + vl) + (g.m + vr));
        r.W[1] = 2.0 * h6 * ((-g.m + vl) + (-g.m + vr));
    } else if (o < 0) {
        r.M = h6;
        r.C = -0.5;
        r.W[0] = h6 * (g.m + vl);
        r.W[1] = h6 * (-g.m + vl);
    } else {
        r.M = h6;
        r.C = 0.5;
        r.W[0] = h6 * (g.m + vr);
        r.W[1] = h6 * (-g.m + vr);
    }
    return r;
}

// Block (i, o) of Bd (sgn = +1) or Bl (sgn = -1) at (y, z) frequency symbols my, mz, sy, sz.
__host__ __device__ inline Blk xblock(const SweepGeom &g, const XRow &r, int nc, double my, double mz, double sy,
                                      double sz, double sgn) {
    Blk B;
    const double myz = my * mz, ht2 = 0.5 * g.ht;
    B.a = mkcd(0.0, sgn * r.M * myz);
    B.b[0] = mkcd(0.0, ht2 * r.C * myz);                   // i alpha_x C_x
    B.b[1] = mkcd(-ht2 * r.M * sy * mz, 0.0);               // i alpha_y M_x (i sin th_y)
    B.b[2] = mkcd(-ht2 * r.M * my * sz, 0.0);               // i alpha_z M_x (i sin th_z)
    for (int c = 0; c < 4; ++c) B.dc[c] = c < nc ? -ht2 * r.W[beta_s(nc, c) > 0 ? 0 : 1] * myz : 0.0;
    return B;
}

__device__ inline void yz_symbols(const SweepGeom &g, int64_t f, double &my, double &mz, double &sy, double &sz) {
    double th[3] = {0.0, 0.0, 0.0};
    const int i1 = (int)(f / g.n2), i2 = (int)(f % g.n2);
    if (g.ax1 >= 0) th[g.ax1] = 2.0 * PI * i1 / g.n1;
    if (g.ax2 >= 0) th[g.ax2] = 2.0 * PI * i2 / g.n2;
    my = g.d >= 2 ? mass_sym(g.h[1], th[1]) : 1.0;
    mz = g.d >= 3 ? mass_sym(g.h[2], th[2]) : 1.0;
    sy = g.d >= 2 ? sin(th[1]) : 0.0;
    sz = g.d >= 3 ? sin(th[2]) : 0.0;
}

// Factors of the block-tridiagonal Bd per frequency, in FP64, stored in FP32:
// table[(f * n + i) * 2 + 0] = L_i = Bd(i, -1) D_{i-1}^-1, [.. + 1] = D_i^-1 with
// D_i = Bd(i, 0) - L_i Bd(i-1, +1); each an NC x NC row-major block.
template <int NC>
__global__ void banded_factor_kernel(SweepGeom g, const double *__restrict__ Vx, float2 *__restrict__ table) {
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nf = (int64_t)g.n1 * g.n2;
    if (f >= nf) return;
    double my, mz, sy, sz;
    yz_symbols(g, f, my, mz, sy, sz);
    const int n = g.nx;
    cd Dinv[4][4], T[4][4], Lm[4][4], U[4][4], Dp[4][4], tmp[4][4];
    for (int i = 0; i < n; ++i) {
        blk_dense(xblock(g, xrow(g, Vx, i, 0), NC, my, mz, sy, sz, 1.0), NC, g.d, Dp);
        if (i > 0) {
            blk_dense(xblock(g, xrow(g, Vx, i, -1), NC, my, mz, sy, sz, 1.0), NC, g.d, T);
            blk_dense(xblock(g, xrow(g, Vx, i - 1, 1), NC, my, mz, sy, sz, 1.0), NC, g.d, U);
            for (int c = 0; c < NC; ++c)
                for (int e = 0; e < NC; ++e) {
                    cd acc = mkcd(0.0, 0.0);
                    for (int d = 0; d < NC; ++d) acc = acc + T[c][d] * Dinv[d][e];
                    Lm[c][e] = acc;
                }
            for (int c = 0; c < NC; ++c)
                for (int e = 0; e < NC; ++e) {
                    cd acc = mkcd(0.0, 0.0);
                    for (int d = 0; d < NC; ++d) acc = acc + Lm[c][d] * U[d][e];
                    Dp[c][e] = Dp[c][e] - acc;
                }
        } else {
            for (int c = 0; c < NC; ++c)
                for (int e = 0; e < NC; ++e) Lm[c][e] = mkcd(0.0, 0.0);
        }
        inv_small(Dp, NC, tmp);
        float2 *o = table + ((size_t)f * n + i) * 2 * NC * NC;
        for (int c = 0; c < NC; ++c)
            for (int e = 0; e < NC; ++e) {
                Dinv[c][e] = tmp[c][e];
                o[c * NC + e] = make_float2((float)Lm[c][e].x, (float)Lm[c][e].y);
                o[NC * NC + c * NC + e] = make_float2((float)tmp[c][e].x, (float)tmp[c][e].y);
            }
    }
}

// FP32 coefficients of row c of the blocks (i, o) of Bd / Bl at one (y, z)
// frequency, from the x-row entries xr = (M, C, W+, W-) and the frequency scalars
// myz = my mz, sy mz, my sz:  a = i sgn M myz,  b_x = i (h_t/2) C myz,
// b_y = -(h_t/2) M sy mz,  b_z = -(h_t/2) M my sz,  dc = -(h_t/2) W_beta(c) myz.
struct FreqF {
    float myz, symz, mysz, ht2;
};
template <int NC>
__device__ __forceinline__ float2 row_apply(const float4 xr, const FreqF &q, float sgn, int c, int nk,
                                            const float2 *p) {
    const float M = xr.x, C = xr.y, Wc = (NC == 2 ? (c == 0) : (c < 2)) ? xr.z : xr.w;
    // diagonal: (i sgn M myz - ht2 W myz) v_c
    const float2 v = p[c];
    const float ar = -q.ht2 * Wc * q.myz, ai = sgn * M * q.myz;
    float2 acc = make_float2(ar * v.x - ai * v.y, ar * v.y + ai * v.x);
    // alpha_x: i ht2 C myz phi_x(c) v_pi  (phi_x = 1)
    {
        const float2 u = p[NC == 2 ? 1 - c : 3 - c];
        const float bi = q.ht2 * C * q.myz;
        acc.x -= bi * u.y;
        acc.y += bi * u.x;
    }
    if (nk >= 2) {                       // alpha_y: -(ht2 M sy mz) phi_y(c) v_pi, phi_y = -i (even c), +i (odd c)
        const float2 u = p[NC == 2 ? 1 - c : 3 - c];
        const float br = -q.ht2 * M * q.symz;
        if (c & 1) { acc.x -= br * u.y; acc.y += br * u.x; }
        else { acc.x += br * u.y; acc.y -= br * u.x; }
    }
    if (nk >= 3) {                       // alpha_z: -(ht2 M my sz) phi_z(c) v_pi, phi_z = +1 (even c), -1 (odd c)
        const float2 u = p[(c + 2) & 3];
        const float br = -q.ht2 * M * q.mysz * ((c & 1) ? -1.f : 1.f);
        acc.x += br * u.x;
        acc.y += br * u.y;
    }
    return acc;
}

// NC lanes march one frequency.  Per team in shared memory: the x-line buffer
// (the previous layer's solution, overwritten by the forward elimination's y and
// then by this layer's solution) and the layer's right-hand side line; per CTA
// the x-row entries of every node and offset.  Work layout [t][x][f][c].
template <int NC>
__global__ void march_banded_kernel(SweepGeom g, const double *__restrict__ Vx, const float2 *__restrict__ table,
                                    float2 *__restrict__ x) {
    extern __shared__ __align__(16) float4 msm[];
    const int n = g.nx;
    const int64_t nf = (int64_t)g.n1 * g.n2;
    const int teams = blockDim.x / NC;
    const int team = threadIdx.x / NC, c = threadIdx.x % NC;
    const int64_t f = blockIdx.x * (int64_t)teams + team;
    const bool live = f < nf;
    const int64_t fl = live ? f : 0;
    float4 *xr = msm;                                                    // [n][3]
    float2 *buf = reinterpret_cast<float2 *>(xr + 3 * n) + (size_t)team * 2 * n * NC;
    float2 *sln = buf + n * NC;
    for (int k = threadIdx.x; k < 3 * n; k += blockDim.x) {
        const XRow r = xrow(g, Vx, k / 3, k % 3 - 1);
        xr[k] = make_float4((float)r.M, (float)r.C, (float)r.W[0], (float)r.W[1]);
    }
    const unsigned lanebase = (threadIdx.x & 31) - c;
    double my, mz, sy, sz;
    yz_symbols(g, fl, my, mz, sy, sz);
    FreqF q;
    q.myz = (float)(my * mz);
    q.symz = (float)(sy * mz);
    q.mysz = (float)(my * sz);
    q.ht2 = (float)(0.5 * g.ht);
    for (int i = c; i < n * NC; i += NC) buf[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const float2 *tab = table + (size_t)fl * n * 2 * NC * NC + c * NC;   // row c of L_i at tab + i * 2 NC^2
    for (int64_t t = 0; t < g.nt; ++t) {
        float2 *xt = x + ((t * n) * nf + fl) * NC + c;                  // node i at xt + i * nf * NC
        for (int i = 0; i < n; ++i) sln[i * NC + c] = live ? xt[(int64_t)i * nf * NC] : make_float2(0.f, 0.f);
        __syncwarp();
        // forward elimination, the factor rows of the next node loaded one node ahead
        float2 Ln[NC];
#pragma unroll
        for (int d = 0; d < NC; ++d) Ln[d] = tab[d];
        float2 yprev = make_float2(0.f, 0.f);
        for (int i = 0; i < n; ++i) {
            float2 Lc[NC];
#pragma unroll
            for (int d = 0; d < NC; ++d) Lc[d] = Ln[d];
            if (i + 1 < n) {
#pragma unroll
                for (int d = 0; d < NC; ++d) Ln[d] = tab[(size_t)(i + 1) * 2 * NC * NC + d];
            }
            float2 r = sln[i * NC + c];
            if (t > 0) {
                for (int o = -1; o <= 1; ++o) {
                    if (i + o < 0 || i + o >= n) continue;
                    r = csubf(r, row_apply<NC>(xr[3 * i + o + 1], q, -1.f, c, g.d, buf + (i + o) * NC));
                }
            }
            float2 y = r;
#pragma unroll
            for (int d = 0; d < NC; ++d) {
                float2 yd;
                yd.x = __shfl_sync(0xffffffffu, yprev.x, lanebase + d);
                yd.y = __shfl_sync(0xffffffffu, yprev.y, lanebase + d);
                y = csubf(y, cmulf(Lc[d], yd));
            }
            __syncwarp();                            // every lane has read x_{t-1}[i - 1]
            if (i > 0) buf[(i - 1) * NC + c] = yprev;
            yprev = y;
        }
        buf[(n - 1) * NC + c] = yprev;
        __syncwarp();
        // back substitution x_i = D_i^-1 (y_i - Bd(i, +1) x_{i+1}), factor rows one node ahead
        float2 Dn[NC];
#pragma unroll
        for (int d = 0; d < NC; ++d) Dn[d] = tab[(size_t)(n - 1) * 2 * NC * NC + NC * NC + d];
        for (int i = n - 1; i >= 0; --i) {
            float2 Dc[NC];
#pragma unroll
            for (int d = 0; d < NC; ++d) Dc[d] = Dn[d];
            if (i > 0) {
#pragma unroll
                for (int d = 0; d < NC; ++d) Dn[d] = tab[(size_t)(i - 1) * 2 * NC * NC + NC * NC + d];
            }
            float2 u = buf[i * NC + c];
            if (i + 1 < n) u = csubf(u, row_apply<NC>(xr[3 * i + 2], q, 1.f, c, g.d, buf + (i + 1) * NC));
            float2 xi = make_float2(0.f, 0.f);
#pragma unroll
            for (int d = 0; d < NC; ++d) {
                float2 ud;
                ud.x = __shfl_sync(0xffffffffu, u.x, lanebase + d);
                ud.y = __shfl_sync(0xffffffffu, u.y, lanebase + d);
                xi = cfmaf(Dc[d], ud, xi);
            }
            __syncwarp();                            // every lane has read y_i and x_{i+1}
            buf[i * NC + c] = xi;
            sln[i * NC + c] = xi;
            __syncwarp();
        }
        if (live)
            for (int i = 0; i < n; ++i) xt[(int64_t)i * nf * NC] = sln[i * NC + c];
        __syncwarp();
    }
}

}  // namespace

int dst_sweep_plan(const dst_mesh *mesh, SweepPlan &p) {
    std::memset(&p, 0, sizeof(p));
    const int d = mesh->d;
    int nonper = 0;
    for (int k = 0; k < d; ++k) {
        if (mesh->bc[k] == DST_BC_OPEN) {
            dst_internal_set_error_detail("Crank-Nicolson sweep: open axes are not supported");
            return DST_ERR_ARG;
        }
        if (mesh->bc[k] != DST_BC_PERIODIC) ++nonper;
    }
    if (nonper > 1 || (nonper == 1 && mesh->bc[0] != DST_BC_DIRICHLET)) {
        dst_internal_set_error_detail("Crank-Nicolson sweep: at most one non-periodic axis, and it must be x");
        return DST_ERR_ARG;
    }
    if (mesh->nt < 1) return DST_ERR_ARG;
    const bool banded = nonper == 1;
    // potential: constant on a spectral mesh, x-only on a banded one
    double V0 = 0.0;
    if (!mesh->V.empty()) {
        if (mesh->v_general) {
            dst_internal_set_error_detail("Crank-Nicolson sweep: the potential must depend on x only");
            return DST_ERR_ARG;
        }
        if (!banded) {
            V0 = mesh->V[0];
            for (int64_t e = 1; e < mesh->nel[0]; ++e)
                if (mesh->V[e] != V0) {
                    dst_internal_set_error_detail("Crank-Nicolson sweep: a potential varying along a periodic axis");
                    return DST_ERR_ARG;
                }
        }
    }
    SweepGeom &g = p.g;
    g.d = d;
    g.nc = mesh->nc;
    g.nt = mesh->nt;
    g.ht = mesh->ht;
    g.m = mesh->m;
    g.V0 = V0;
    for (int k = 0; k < 3; ++k) g.h[k] = mesh->h[k];
    g.nx = (int)mesh->nu[0];
    // FFT dims: the periodic axes, outer (n1) the slower one
    int per_axes[3], np = 0;
    for (int k = banded ? 1 : 0; k < d; ++k) per_axes[np++] = k;
    g.ax1 = g.ax2 = -1;
    g.n1 = g.n2 = 1;
    SweepFft &a = p.fft;
    a.nc = mesh->nc;
    a.nbx = banded ? (int)mesh->nu[0] : 1;
    a.sbx = 1;
    a.ns_nodes = mesh->n_spatial;
    int64_t stride[3] = {1, mesh->nu[0], mesh->nu[0] * mesh->nu[1]};
    if (np == 1) {
        g.ax2 = per_axes[0];
        g.n2 = (int)mesh->nu[per_axes[0]];
        a.s2 = stride[per_axes[0]];
        a.s1 = 0;
    } else if (np == 2) {
        g.ax2 = per_axes[0];
        g.ax1 = per_axes[1];
        g.n2 = (int)mesh->nu[per_axes[0]];
        g.n1 = (int)mesh->nu[per_axes[1]];
        a.s2 = stride[per_axes[0]];
        a.s1 = stride[per_axes[1]];
    } else if (np == 3) {
        dst_internal_set_error_detail("Crank-Nicolson sweep: a 3+1 mesh needs a Dirichlet x axis");
        return DST_ERR_ARG;
    }
    a.n1 = g.n1;
    a.n2 = g.n2;
    dst_fft::radices(a.n1, a.rad1, a.nrad1);
    dst_fft::radices(a.n2, a.rad2, a.nrad2);
    p.banded = banded;
    p.has_fft = np > 0;
    p.nb = banded ? mesh->nt * mesh->nu[0] : mesh->nt;
    const int64_t nf = (int64_t)g.n1 * g.n2;
    const int nmax = g.n1 > g.n2 ? g.n1 : g.n2;
    if (nmax > 4096) {
        dst_internal_set_error_detail("Crank-Nicolson sweep: a periodic axis longer than 4096 nodes");
        return DST_ERR_ARG;
    }
    const size_t limit = 200 * 1024;
    if (p.has_fft && !dst_fft::choose_layout<float2>(a, p.nb, limit)) {
        dst_internal_set_error_detail("Crank-Nicolson sweep: a periodic plane too large for shared memory");
        return DST_ERR_ARG;
    }
    p.fft_smem = dst_fft::fft_smem_bytes<float2>(a);
    p.table_bytes = banded ? sizeof(float2) * (size_t)nf * g.nx * 2 * g.nc * g.nc : 0;
    // banded march: teams of NC lanes, shared memory of one x-line per team
    if (banded) {
        const size_t line = 2 * sizeof(float2) * (size_t)g.nx * g.nc;      // the x-line and the right-hand side line
        int teams = (int)((96 * 1024) / line);
        const int per_warp = 32 / g.nc;
        if (teams > 128 / g.nc) teams = 128 / g.nc;
        if (teams < per_warp) teams = per_warp;        // one warp at least (idle lanes if the line is long)
        teams = teams / per_warp * per_warp;
        p.march_threads = teams * g.nc;
        p.march_smem = line * teams + sizeof(float4) * 3 * (size_t)g.nx;
        if (p.march_smem > 200 * 1024) {
            dst_internal_set_error_detail("Crank-Nicolson sweep: x axis too long for the banded march");
            return DST_ERR_ARG;
        }
    }
    p.vx = banded && !mesh->V.empty();
    return DST_OK;
}

size_t dst_sweep_scratch_bytes(const SweepPlan &p, int64_t n_unknowns) {
    size_t b = (sizeof(float2) * (size_t)n_unknowns + 255) & ~(size_t)255;
    b += (p.table_bytes + 255) & ~(size_t)255;
    b += ((size_t)(p.g.nx + 2) * sizeof(double) + 255) & ~(size_t)255;
    return b;
}

int dst_sweep_setup(const dst_mesh *mesh, SweepPlan &p, void *scratch, cudaStream_t s) {
    char *base = (char *)scratch;
    size_t off = 0;
    p.work = (float2 *)(base + off);
    off += (sizeof(float2) * (size_t)mesh->n_unknowns + 255) & ~(size_t)255;
    p.table = p.banded ? (float2 *)(base + off) : nullptr;
    off += (p.table_bytes + 255) & ~(size_t)255;
    p.dvx = p.vx ? (double *)(base + off) : nullptr;
    if (p.vx)
        DST_CUDA_TRY(cudaMemcpyAsync(p.dvx, mesh->V.data(), sizeof(double) * mesh->nel[0], cudaMemcpyHostToDevice, s));
    if (p.banded) {
        const int64_t nf = (int64_t)p.g.n1 * p.g.n2;
        const unsigned blocks = (unsigned)((nf + 63) / 64);
        if (p.g.nc == 2) banded_factor_kernel<2><<<blocks, 64, 0, s>>>(p.g, p.dvx, p.table);
        else banded_factor_kernel<4><<<blocks, 64, 0, s>>>(p.g, p.dvx, p.table);
        DST_CUDA_TRY(cudaGetLastError());
    }
    return DST_OK;
}

// z = M v on FP32 vectors; `work` (n_unknowns float2) is the plan's scratch; v and z
// may not overlap work; z may equal v only if there is no FFT (it is written last).
int dst_sweep_apply(const SweepPlan &p, int64_t n_unknowns, const float2 *v, float2 *z, cudaStream_t s) {
    const int64_t per = n_unknowns / p.g.nt;
    const int64_t nf = (int64_t)p.g.n1 * p.g.n2;
    float2 *work = p.work;
    // 1. s = S^-1 v (into z if an FFT follows, else into work)
    float2 *sdst = p.has_fft ? z : work;
    time_scan_kernel<<<(unsigned)((per + 255) / 256), 256, 0, s>>>(per, p.g.nt, v, sdst);
    DST_CUDA_TRY(cudaGetLastError());
    // 2. forward FFT of every plane: z -> work (frequency layout)
    static bool configured[64] = {};
    int dev = 0;
    DST_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        DST_CUDA_TRY(cudaFuncSetAttribute(dst_fft::fft_planes_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          200 * 1024));
        DST_CUDA_TRY(cudaFuncSetAttribute(march_banded_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          200 * 1024));
        DST_CUDA_TRY(cudaFuncSetAttribute(march_banded_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          200 * 1024));
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    const dim3 fgrid((unsigned)p.nb, (unsigned)(p.g.nc / p.fft.ncb));
    if (p.has_fft) {
        dst_fft::fft_planes_kernel<float2><<<fgrid, dst_fft::FFT_THREADS, p.fft_smem, s>>>(p.fft, 0, z, work);
        DST_CUDA_TRY(cudaGetLastError());
    }
    // 3. the march, in place on work
    if (!p.banded) {
        const unsigned blocks = (unsigned)((nf + 127) / 128);
        if (p.g.nc == 2) march_spectral_kernel<2><<<blocks, 128, 0, s>>>(p.g, work);
        else march_spectral_kernel<4><<<blocks, 128, 0, s>>>(p.g, work);
    } else {
        const int teams = p.march_threads / p.g.nc;
        const unsigned blocks = (unsigned)((nf + teams - 1) / teams);
        if (p.g.nc == 2) march_banded_kernel<2><<<blocks, p.march_threads, p.march_smem, s>>>(p.g, p.dvx, p.table, work);
        else march_banded_kernel<4><<<blocks, p.march_threads, p.march_smem, s>>>(p.g, p.dvx, p.table, work);
    }
    DST_CUDA_TRY(cudaGetLastError());
    // 4. inverse FFT: work -> z (without an FFT the march ran on the node layout)
    if (p.has_fft) {
        dst_fft::fft_planes_kernel<float2><<<fgrid, dst_fft::FFT_THREADS, p.fft_smem, s>>>(p.fft, 1, work, z);
        DST_CUDA_TRY(cudaGetLastError());
    } else {
        DST_CUDA_TRY(cudaMemcpyAsync(z, work, sizeof(float2) * n_unknowns, cudaMemcpyDeviceToDevice, s));
    }
    return DST_OK;
}

extern "C" int dst_precond_apply(const dst_mesh *mesh, int kind, const void *v, void *z, void *stream) {
    if (!mesh || !v || !z || v == z) return DST_ERR_ARG;
    if (kind == DST_PRECOND_BLOCK_JACOBI) {
        cudaStream_t s = (cudaStream_t)stream;
        int rc = dst_internal_jacobi_setup(const_cast<dst_mesh *>(mesh), s);
        return rc ? rc : dst_internal_jacobi_apply(mesh, (const float2 *)v, (float2 *)z, s);
    }
    if (kind != DST_PRECOND_CN_SWEEP && kind != DST_PRECOND_CN_LEARNED) {
        dst_internal_set_error_detail("dst_precond_apply: unknown preconditioner kind");
        return DST_ERR_ARG;
    }
    if (kind == DST_PRECOND_CN_LEARNED && !dst_internal_unet_fits(mesh->unet, mesh)) {
        dst_internal_set_error_detail("dst_precond_apply: no network for this mesh (dst_set_learned_precond)");
        return DST_ERR_ARG;
    }
    SweepPlan p;
    int rc = dst_sweep_plan(mesh, p);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    void *scratch = nullptr;
    const int64_t n = mesh->n_unknowns;
    const size_t sweep_bytes = (dst_sweep_scratch_bytes(p, n) + 255) & ~(size_t)255;
    const size_t vec_bytes = ((size_t)n * sizeof(float2) + 255) & ~(size_t)255;
    const size_t bytes = sweep_bytes + (kind == DST_PRECOND_CN_LEARNED ? 2 * vec_bytes : 0);
    if (cudaMallocAsync(&scratch, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return DST_ERR_OOM;
    }
    rc = dst_sweep_setup(mesh, p, scratch, s);
    if (rc == DST_OK) rc = dst_sweep_apply(p, n, (const float2 *)v, (float2 *)z, s);
    if (rc == DST_OK && kind == DST_PRECOND_CN_LEARNED) {
        float2 *tmp = reinterpret_cast<float2 *>((char *)scratch + sweep_bytes);
        float2 *rho = reinterpret_cast<float2 *>((char *)scratch + sweep_bytes + vec_bytes);
        int nk = 0;
        rc = dst_internal_apply(mesh, DST_FP32, z, tmp, s);                 // rho = v - A M_CN(v)
        if (rc == DST_OK) rc = dst_k_sub_f32(n, (const float2 *)v, tmp, rho, s);
        if (rc == DST_OK) rc = dst_internal_unet_correct(mesh->unet, mesh, rho, (float2 *)z, tmp, s, &nk);
    }
    cudaFreeAsync(scratch, s);
    return rc;
}
