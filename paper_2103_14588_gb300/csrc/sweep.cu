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

#include "internal.h"
#include "sweep.h"

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
__device__ __forceinline__ float2 caddf(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
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
__global__ void time_scan_kernel(int64_t per, int64_t nt, const float2 *__restrict__ v, float2 *__restrict__ s) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= per) return;
    float2 acc = make_float2(0.f, 0.f);
    for (int64_t t = nt - 1; t >= 0; --t) {
        const float2 a = v[t * per + e];
        acc = make_float2(2.f * a.x - acc.x, 2.f * a.y - acc.y);
        s[t * per + e] = acc;
    }
}

// ---- 2 / 4. FFT of planes over the periodic axes ------------------------------
constexpr int FFT_THREADS = 256;
constexpr int FFT_WARPS = FFT_THREADS / 32;

// One line of length n (stride st in the plane) through the Stockham stages
// `rad`, by one warp, with twiddles w[j] = exp(sign 2 pi i j / n) from the
// table and two scratch lines a, b of n entries.
__device__ void warp_fft_line(float2 *line, int st, int n, const int *rad, int nrad, const float2 *w, float2 *a,
                              float2 *b) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < n; i += 32) a[i] = line[i * st];
    __syncwarp();
    float2 *d0 = a, *d1 = b;
    int Ns = 1;
    for (int s = 0; s < nrad; ++s) {
        const int R = rad[s];
        const int q = n / R;               // butterflies of this stage
        const int step = n / (Ns * R);     // twiddle index unit: exp(sign 2 pi i k / (Ns R)) = w[k * step]
        for (int j = lane; j < q; j += 32) {
            const int k = j % Ns;
            const int dst = (j / Ns) * Ns * R + k;
            if (R == 2) {
                const float2 v0 = d0[j], v1 = cmulf(d0[j + q], w[k * step]);
                d1[dst] = caddf(v0, v1);
                d1[dst + Ns] = csubf(v0, v1);
            } else if (R == 4) {
                const float2 v0 = d0[j];
                const float2 v1 = cmulf(d0[j + q], w[k * step]);
                const float2 v2 = cmulf(d0[j + 2 * q], w[(2 * k * step) % n]);
                const float2 v3 = cmulf(d0[j + 3 * q], w[(3 * k * step) % n]);
                // omega = w[n/4] = exp(sign i pi/2) = sign * i
                const float2 om = w[n / 4];
                const float2 t0 = caddf(v0, v2), t1 = csubf(v0, v2);
                const float2 t2 = caddf(v1, v3), t3 = cmulf(om, csubf(v1, v3));
                d1[dst] = caddf(t0, t2);
                d1[dst + Ns] = caddf(t1, t3);
                d1[dst + 2 * Ns] = csubf(t0, t2);
                d1[dst + 3 * Ns] = csubf(t1, t3);
            } else {
                // general radix: V_o = sum_r v_r exp(sign 2 pi i r o / R), v_r twiddled
                for (int o = 0; o < R; ++o) {
                    float2 acc = make_float2(0.f, 0.f);
                    for (int r = 0; r < R; ++r) {
                        const float2 vr = cmulf(d0[j + r * q], w[(int)(((long long)r * k * step) % n)]);
                        acc = cfmaf(w[(int)(((long long)r * o * q) % n)], vr, acc);
                    }
                    d1[dst + o * Ns] = acc;
                }
            }
        }
        __syncwarp();
        float2 *t = d0; d0 = d1; d1 = t;
        Ns *= R;
    }
    for (int i = lane; i < n; i += 32) line[i * st] = d0[i];
    __syncwarp();
}

// One CTA per plane (batch b = layer, or layer x x-node in banded mode) and
// component group: load into shared memory, FFT along the inner then the outer
// axis, store.  Forward: node layout in, frequency layout [b][f][c] out;
// inverse (sign +1): frequency layout in, node layout out, scaled by 1/(n1 n2).
__global__ void __launch_bounds__(FFT_THREADS)
fft_planes_kernel(SweepFft a, int inverse, const float2 *__restrict__ in, float2 *__restrict__ out) {
    extern __shared__ __align__(16) float2 sm[];
    const int n1 = a.n1, n2 = a.n2, nc = a.nc, ncb = a.ncb;
    const int nf = n1 * n2;
    float2 *plane = sm;                                   // [ncb][n1][n2]
    float2 *w1 = plane + (size_t)ncb * nf;                // twiddles of the outer axis (n1)
    float2 *w2 = w1 + n1;                                 // twiddles of the inner axis (n2)
    float2 *scr = w2 + n2;                                // per warp two lines of nmax
    const int nmax = n1 > n2 ? n1 : n2;
    const int64_t b = blockIdx.x;
    const int c0 = blockIdx.y * ncb;
    const int64_t base = (b / a.nbx) * a.ns_nodes + (b % a.nbx);       // node index of (i1, i2) = (0, 0)
    const float sign = inverse ? 1.f : -1.f;
    for (int j = threadIdx.x; j < n1; j += FFT_THREADS) {
        float sn, cs;
        sincospif(2.f * (float)j / (float)n1, &sn, &cs);
        w1[j] = make_float2(cs, sign * sn);
    }
    for (int j = threadIdx.x; j < n2; j += FFT_THREADS) {
        float sn, cs;
        sincospif(2.f * (float)j / (float)n2, &sn, &cs);
        w2[j] = make_float2(cs, sign * sn);
    }
    // load
    for (int idx = threadIdx.x; idx < nf * ncb; idx += FFT_THREADS) {
        const int cc = idx % ncb, f = idx / ncb;
        const int i1 = f / n2, i2 = f % n2;
        float2 v;
        if (inverse) v = in[(b * nf + f) * nc + c0 + cc];
        else v = in[(base + (int64_t)i1 * a.s1 + (int64_t)i2 * a.s2) * nc + c0 + cc];
        plane[(size_t)cc * nf + f] = v;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    float2 *sa = scr + (size_t)warp * 2 * nmax, *sb = sa + nmax;
    if (n2 > 1)
        for (int line = warp; line < ncb * n1; line += FFT_WARPS)
            warp_fft_line(plane + (size_t)line * n2, 1, n2, a.rad2, a.nrad2, w2, sa, sb);
    __syncthreads();
    if (n1 > 1)
        for (int line = warp; line < ncb * n2; line += FFT_WARPS) {
            const int cc = line / n2, i2 = line % n2;
            warp_fft_line(plane + (size_t)cc * nf + i2, n2, n1, a.rad1, a.nrad1, w1, sa, sb);
        }
    __syncthreads();
    const float scale = inverse ? 1.f / (float)nf : 1.f;
    for (int idx = threadIdx.x; idx < nf * ncb; idx += FFT_THREADS) {
        const int cc = idx % ncb, f = idx / ncb;
        const int i1 = f / n2, i2 = f % n2;
        float2 v = plane[(size_t)cc * nf + f];
        v.x *= scale;
        v.y *= scale;
        if (inverse) out[(base + (int64_t)i1 * a.s1 + (int64_t)i2 * a.s2) * nc + c0 + cc] = v;
        else out[(b * nf + f) * nc + c0 + cc] = v;
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
    for (int64_t t = 0; t < g.nt; ++t) {
        float2 *p = x + (t * nf + f) * NC;
        float2 s[NC], xn[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) s[c] = p[c];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int d = 0; d < NC; ++d) {
                acc = cfmaf(Pf[c][d], s[d], acc);
                const float2 q = cmulf(Qf[c][d], xp[d]);
                acc = csubf(acc, q);
            }
            xn[c] = acc;
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) { xp[c] = xn[c]; p[c] = xn[c]; }
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

// Row c of a structured block applied to the vector at node slot p of a team's
// buffer (NC complex per node): a v_c + sum_k b_k phi_k(c) v_{pi_k(c)} + dc_c v_c.
template <int NC>
__device__ __forceinline__ float2 blk_row(const float2 (&bk)[5], int c, const float2 *p, int nk) {
    float2 acc = cmulf(bk[0], p[c]);
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (k < nk) acc = cfmaf(bk[1 + k], p[spin_pi(NC, k, c)], acc);
    return cfmaf(bk[4], p[c], acc);
}
// The coefficients of row c of a block in FP32: a, b_k phi_k(c), dc_c.
template <int NC>
__device__ __forceinline__ void blk_coefs(const Blk &B, int c, float2 (&bk)[5]) {
    bk[0] = make_float2((float)B.a.x, (float)B.a.y);
    for (int k = 0; k < 3; ++k) {
        const cd v = B.b[k] * spin_phi(NC, k, c);
        bk[1 + k] = make_float2((float)v.x, (float)v.y);
    }
    bk[4] = make_float2((float)B.dc[c], 0.f);
}

// NC lanes march one frequency; each team keeps its x-line (n nodes x NC) in
// shared memory: the previous layer's solution, overwritten by the forward
// elimination's y and then by this layer's solution.  Work layout [t][x][f][c].
template <int NC>
__global__ void march_banded_kernel(SweepGeom g, const double *__restrict__ Vx, const float2 *__restrict__ table,
                                    float2 *__restrict__ x) {
    extern __shared__ __align__(16) float2 bufs[];
    const int n = g.nx;
    const int64_t nf = (int64_t)g.n1 * g.n2;
    const int team = threadIdx.x / NC, c = threadIdx.x % NC;
    const int64_t f = blockIdx.x * (int64_t)(blockDim.x / NC) + team;
    const bool live = f < nf;
    const int64_t fl = live ? f : 0;
    float2 *buf = bufs + (size_t)team * n * NC;
    const unsigned lanebase = (threadIdx.x & 31) - c;
    double my, mz, sy, sz;
    yz_symbols(g, fl, my, mz, sy, sz);
    for (int i = c; i < n * NC; i += NC) buf[i] = make_float2(0.f, 0.f);
    __syncwarp();
    const float2 *tab = table + (size_t)fl * n * 2 * NC * NC;
    for (int64_t t = 0; t < g.nt; ++t) {
        float2 *xt = x + ((t * n) * nf + fl) * NC;         // node i at xt + i * nf * NC
        float2 yprev = make_float2(0.f, 0.f);
        for (int i = 0; i < n; ++i) {
            // r_i = s_t[i] - sum_o Bl(i, o) x_{t-1}[i + o]
            float2 r = live ? xt[(int64_t)i * nf * NC + c] : make_float2(0.f, 0.f);
            if (t > 0) {
                for (int o = -1; o <= 1; ++o) {
                    if (i + o < 0 || i + o >= n) continue;
                    float2 bk[5];
                    blk_coefs<NC>(xblock(g, xrow(g, Vx, i, o), NC, my, mz, sy, sz, -1.0), c, bk);
                    r = csubf(r, blk_row<NC>(bk, c, buf + (i + o) * NC, g.d));
                }
            }
            // y_i = r_i - L_i y_{i-1}
            const float2 *Li = tab + (size_t)i * 2 * NC * NC + c * NC;
            float2 y = r;
#pragma unroll
            for (int d = 0; d < NC; ++d) {
                float2 yd;
                yd.x = __shfl_sync(0xffffffffu, yprev.x, lanebase + d);
                yd.y = __shfl_sync(0xffffffffu, yprev.y, lanebase + d);
                y = csubf(y, cmulf(Li[d], yd));
            }
            __syncwarp();                            // every lane has read x_{t-1}[i - 1]
            if (i > 0) buf[(i - 1) * NC + c] = yprev;
            yprev = y;
        }
        buf[(n - 1) * NC + c] = yprev;
        __syncwarp();
        // x_i = D_i^-1 (y_i - Bd(i, +1) x_{i+1})
        for (int i = n - 1; i >= 0; --i) {
            float2 u = buf[i * NC + c];
            if (i + 1 < n) {
                float2 bk[5];
                blk_coefs<NC>(xblock(g, xrow(g, Vx, i, 1), NC, my, mz, sy, sz, 1.0), c, bk);
                u = csubf(u, blk_row<NC>(bk, c, buf + (i + 1) * NC, g.d));
            }
            const float2 *Di = tab + (size_t)i * 2 * NC * NC + NC * NC + c * NC;
            float2 xi = make_float2(0.f, 0.f);
#pragma unroll
            for (int d = 0; d < NC; ++d) {
                float2 ud;
                ud.x = __shfl_sync(0xffffffffu, u.x, lanebase + d);
                ud.y = __shfl_sync(0xffffffffu, u.y, lanebase + d);
                xi = cfmaf(Di[d], ud, xi);
            }
            __syncwarp();                            // every lane has read y_i and x_{i+1}
            buf[i * NC + c] = xi;
            if (live) xt[(int64_t)i * nf * NC + c] = xi;
            __syncwarp();
        }
    }
}

void radices(int n, int *r, int &nr) {
    nr = 0;
    while (n % 4 == 0) { r[nr++] = 4; n /= 4; }
    while (n % 2 == 0) { r[nr++] = 2; n /= 2; }
    for (int p = 3; n > 1; p += 2)
        while (n % p == 0) { r[nr++] = p; n /= p; }
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
    radices(a.n1, a.rad1, a.nrad1);
    radices(a.n2, a.rad2, a.nrad2);
    p.banded = banded;
    p.has_fft = np > 0;
    p.nb = banded ? mesh->nt * mesh->nu[0] : mesh->nt;
    const int64_t nf = (int64_t)g.n1 * g.n2;
    const int nmax = g.n1 > g.n2 ? g.n1 : g.n2;
    if (nmax > 4096) {
        dst_internal_set_error_detail("Crank-Nicolson sweep: a periodic axis longer than 4096 nodes");
        return DST_ERR_ARG;
    }
    const size_t fixed = sizeof(float2) * ((size_t)g.n1 + g.n2 + (size_t)FFT_WARPS * 2 * nmax);
    const size_t limit = 200 * 1024;
    // components per FFT CTA: all of them when the plane fits and the planes alone fill the GPU
    a.ncb = mesh->nc;
    while (a.ncb > 1 && (fixed + sizeof(float2) * (size_t)a.ncb * nf > limit || p.nb * (mesh->nc / a.ncb) < 304))
        a.ncb /= 2;
    p.fft_smem = fixed + sizeof(float2) * (size_t)a.ncb * nf;
    if (p.has_fft && p.fft_smem > limit) {
        dst_internal_set_error_detail("Crank-Nicolson sweep: a periodic plane too large for shared memory");
        return DST_ERR_ARG;
    }
    p.table_bytes = banded ? sizeof(float2) * (size_t)nf * g.nx * 2 * g.nc * g.nc : 0;
    // banded march: teams of NC lanes, shared memory of one x-line per team
    if (banded) {
        const size_t line = sizeof(float2) * (size_t)g.nx * g.nc;
        int teams = (int)((96 * 1024) / line);
        const int per_warp = 32 / g.nc;
        if (teams > 128 / g.nc) teams = 128 / g.nc;
        if (teams < per_warp) teams = per_warp;        // one warp at least (idle lanes if the line is long)
        teams = teams / per_warp * per_warp;
        p.march_threads = teams * g.nc;
        p.march_smem = line * teams;
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
        DST_CUDA_TRY(cudaFuncSetAttribute(fft_planes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        DST_CUDA_TRY(cudaFuncSetAttribute(march_banded_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          200 * 1024));
        DST_CUDA_TRY(cudaFuncSetAttribute(march_banded_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          200 * 1024));
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    const dim3 fgrid((unsigned)p.nb, (unsigned)(p.g.nc / p.fft.ncb));
    if (p.has_fft) {
        fft_planes_kernel<<<fgrid, FFT_THREADS, p.fft_smem, s>>>(p.fft, 0, z, work);
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
        fft_planes_kernel<<<fgrid, FFT_THREADS, p.fft_smem, s>>>(p.fft, 1, work, z);
        DST_CUDA_TRY(cudaGetLastError());
    } else {
        DST_CUDA_TRY(cudaMemcpyAsync(z, work, sizeof(float2) * n_unknowns, cudaMemcpyDeviceToDevice, s));
    }
    return DST_OK;
}

extern "C" int dst_precond_apply(const dst_mesh *mesh, int kind, const void *v, void *z, void *stream) {
    if (!mesh || !v || !z || v == z) return DST_ERR_ARG;
    if (kind != DST_PRECOND_CN_SWEEP) {
        dst_internal_set_error_detail("dst_precond_apply: unknown preconditioner kind");
        return DST_ERR_ARG;
    }
    SweepPlan p;
    int rc = dst_sweep_plan(mesh, p);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    void *scratch = nullptr;
    const size_t bytes = dst_sweep_scratch_bytes(p, mesh->n_unknowns);
    if (cudaMallocAsync(&scratch, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return DST_ERR_OOM;
    }
    rc = dst_sweep_setup(mesh, p, scratch, s);
    if (rc == DST_OK) rc = dst_sweep_apply(p, mesh->n_unknowns, (const float2 *)v, (float2 *)z, s);
    cudaFreeAsync(scratch, s);
    return rc;
}
