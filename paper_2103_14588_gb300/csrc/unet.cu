// Learned right preconditioner: a convolutional U-Net trained on the GPU.
//
// The paper names no preconditioner; its conclusion (Sec. 5) asks for one.  The
// network corrects the Crank-Nicolson sweep M_CN (sweep.cu):
//     M(v) = M_CN(v) + s U(rho / s),   rho = v - A M_CN(v),  s = ||rho||,
// so U is trained to map the sweep's residual to the sweep's error.  Training
// pairs come from the method itself: e random, r = A e (FP32 operator apply),
// z = M_CN(r), input rho = r - A z, target e - z (the exact solution of
// A d = rho), both divided by ||rho||; loss ||U(rho^) - t^||^2 / ||t^||^2; Adam.
//
// Network (three levels, 16 / 32 / 64 channels, C = 2 NC field channels, channel
// 2c = Re psi_c and 2c + 1 = Im psi_c, which is the complex unknown vector read as
// [node][channel] floats):
//   e1a conv3 C->16 ReLU, e1b conv3 16->16 ReLU = s1; pool;
//   e2a conv3 16->32 ReLU, e2b conv3 32->32 ReLU = s2; pool;
//   e3a conv3 32->64 ReLU, e3b conv3 64->64 ReLU; upsample;
//   u2p conv1 64->32, + s2, u2c conv3 32->32 ReLU; upsample;
//   u1p conv1 32->16, + s1, u1c conv3 16->16 ReLU; out conv1 16->C.
// pool = mean over 2^D blocks (cells past an odd end count as zero), upsample =
// nearest.  Convolutions run on BF16 tensor cores with FP32 accumulation
// (unet_kernels.cuh); parameters are kept in FP32 (Adam) and rounded to BF16.
// Parameter order and layout of the flat vector: per layer in the order above
// its weight (co, ci, kernel offsets row-major over the grid axes) then its bias.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "blas.h"
#include "internal.h"
#include "sweep.h"
#include "unet_kernels.cuh"

using namespace dst_nn;

namespace {

constexpr int NLAYER = 11;
enum { E1A, E1B, E2A, E2B, E3A, E3B, U2P, U2C, U1P, U1C, OUT };

struct Layer {
    int ci, co, taps, level;
    int kpad, co8;          // K padded to 16, output rows padded to 8
    int64_t woff, boff;     // offsets of weight and bias in the flat parameter vector
};

__global__ void pool_fwd_kernel(UGrid f, UGrid c, int ch, const float *__restrict__ in, float *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= c.N * ch) return;
    const int k = (int)(i % ch);
    int64_t q = i / ch;
    int cc[4];
    coords(c, q, cc);
    float s = 0.f;
    const int nb = 1 << f.D;
    for (int m = 0; m < nb; ++m) {
        int64_t r = 0;
        bool ok = true;
        for (int a = 0; a < f.D; ++a) {
            const int x = 2 * cc[a] + ((m >> (f.D - 1 - a)) & 1);
            if (x >= f.n[a]) { ok = false; break; }
            r = r * f.n[a] + x;
        }
        if (ok) s += in[r * ch + k];
    }
    out[i] = s / (float)nb;
}

// d_fine[p] += d_coarse[p / 2] / 2^D
__global__ void pool_bwd_kernel(UGrid f, UGrid c, int ch, const float *__restrict__ dc, float *__restrict__ df) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= f.N * ch) return;
    const int k = (int)(i % ch);
    int cf[4];
    coords(f, i / ch, cf);
    int64_t q = 0;
    for (int a = 0; a < f.D; ++a) q = q * c.n[a] + cf[a] / 2;
    df[i] += dc[q * ch + k] / (float)(1 << f.D);
}

// fine[p] = coarse[p / 2]
__global__ void up_fwd_kernel(UGrid f, UGrid c, int ch, const float *__restrict__ in, float *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= f.N * ch) return;
    const int k = (int)(i % ch);
    int cf[4];
    coords(f, i / ch, cf);
    int64_t q = 0;
    for (int a = 0; a < f.D; ++a) q = q * c.n[a] + cf[a] / 2;
    out[i] = in[q * ch + k];
}

// d_coarse[q] = sum of d_fine over the cells p with p / 2 = q
__global__ void up_bwd_kernel(UGrid f, UGrid c, int ch, const float *__restrict__ df, float *__restrict__ dc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= c.N * ch) return;
    const int k = (int)(i % ch);
    int cc[4];
    coords(c, i / ch, cc);
    float s = 0.f;
    for (int m = 0; m < (1 << f.D); ++m) {
        int64_t r = 0;
        bool ok = true;
        for (int a = 0; a < f.D; ++a) {
            const int x = 2 * cc[a] + ((m >> (f.D - 1 - a)) & 1);
            if (x >= f.n[a]) { ok = false; break; }
            r = r * f.n[a] + x;
        }
        if (ok) s += df[r * ch + k];
    }
    dc[i] = s;
}

// dz = d * (y > 0)
__global__ void relu_mask_kernel(int64_t n, const float *__restrict__ d, const float *__restrict__ y,
                                 float *__restrict__ dz) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dz[i] = y[i] > 0.f ? d[i] : 0.f;
}

// db[co] += sum_n dz[n][co] (one CTA per channel, fixed order)
__global__ void bias_grad_kernel(int64_t N, int co, const float *__restrict__ dz, float *__restrict__ db) {
    __shared__ float red[256];
    const int c = blockIdx.x;
    float s = 0.f;
    for (int64_t n = threadIdx.x; n < N; n += blockDim.x) s += dz[n * co + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[c] += red[0];
}

// internal weights: wf[co8][kpad] bf16 (k = tap * ci + c) and the mirrored transpose
// wt[ci8][kpadT] (k' = tap' * co + o, tap' = taps - 1 - tap) for the input gradient
__global__ void pack_weights_kernel(Layer L, const float *__restrict__ p, __nv_bfloat16 *__restrict__ wf,
                                    __nv_bfloat16 *__restrict__ wt, int kpadT) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nf = (int64_t)L.co8 * L.kpad;
    if (i < nf) {
        const int o = (int)(i / L.kpad), k = (int)(i % L.kpad);
        float v = 0.f;
        if (o < L.co && k < L.taps * L.ci) {
            const int tap = k / L.ci, c = k % L.ci;
            v = p[L.woff + ((int64_t)o * L.ci + c) * L.taps + tap];
        }
        wf[i] = __float2bfloat16_rn(v);
    }
    if (wt) {
        const int ci8 = (L.ci + 7) / 8 * 8;
        if (i < (int64_t)ci8 * kpadT) {
            const int c = (int)(i / kpadT), k = (int)(i % kpadT);
            float v = 0.f;
            if (c < L.ci && k < L.taps * L.co) {
                const int tapT = k / L.co, o = k % L.co;
                v = p[L.woff + ((int64_t)o * L.ci + c) * L.taps + (L.taps - 1 - tapT)];
            }
            wt[i] = __float2bfloat16_rn(v);
        }
    }
}

// flat gradient (parameter layout) from the internal dW[co][kpad]
__global__ void unpack_wgrad_kernel(Layer L, const float *__restrict__ dw, float *__restrict__ g) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)L.co * L.ci * L.taps;
    if (i >= n) return;
    const int tap = (int)(i % L.taps);
    const int c = (int)((i / L.taps) % L.ci);
    const int o = (int)(i / ((int64_t)L.taps * L.ci));
    g[L.woff + i] = dw[(size_t)o * L.kpad + tap * L.ci + c];
}

__global__ void adam_kernel(int64_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// sum of squares of a float array into *out (FP64 accumulation, one CTA)
__global__ void sumsq_kernel(int64_t n, const float *__restrict__ a, double *__restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)a[i] * a[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// the norm s = sqrt(sum of squares) as a float scalar (the input scale of the network)
__global__ void sqrt_scalar_kernel(const double *__restrict__ ss, float *__restrict__ s) {
    if (threadIdx.x == 0) *s = (float)sqrt(*ss);
}

// loss = ||y - t / s||^2 / ||t / s||^2 into *loss, dy = 2 (y - t / s) / ||t / s||^2
__global__ void loss_kernel(int64_t n, const float *__restrict__ y, const float *__restrict__ t,
                            const float *__restrict__ s, const double *__restrict__ tt, float *__restrict__ dy,
                            double *__restrict__ loss) {
    __shared__ double red[256];
    const float inv = 1.0f / *s;
    const double tn = *tt * (double)inv * inv;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const float r = y[i] - t[i] * inv;
        acc += (double)r * r;
        dy[i] = (float)(2.0 * r / tn);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] / tn;
}

// z += g s y (the network's output scaled back; y [N][C] is the same floats as a complex vector)
__global__ void axpy_scaled_kernel(int64_t n, const float *__restrict__ s, const float *__restrict__ g,
                                   const float *__restrict__ y, float *__restrict__ z) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) z[i] += *g * *s * y[i];
}

// <y, t / s> and ||y||^2 accumulated into acc[0], acc[1] (one CTA, FP64)
__global__ void dot_kernel(int64_t n, const float *__restrict__ y, const float *__restrict__ t,
                           const float *__restrict__ s, double *__restrict__ acc) {
    __shared__ double r1[256], r2[256];
    const float inv = 1.0f / *s;
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        a += (double)y[i] * (double)(t[i] * inv);
        b += (double)y[i] * (double)y[i];
    }
    r1[threadIdx.x] = a;
    r2[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) { r1[threadIdx.x] += r1[threadIdx.x + w]; r2[threadIdx.x] += r2[threadIdx.x + w]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { acc[0] += r1[0]; acc[1] += r2[0]; }
}

// Partial sums of <a, r> = sum conj(a_i) r_i (re, im) and ||a||^2 over complex
// vectors, one triple per CTA (FP64), for the least-squares scale of the correction.
constexpr int LS_PARTS = 304;
constexpr int WGRAD_SPLITS = 64;                 // node ranges of the weight-gradient GEMM
__global__ void __launch_bounds__(256) ls_partials_kernel(int64_t n, const float2 *__restrict__ a,
                                                          const float2 *__restrict__ r, double *__restrict__ part) {
    __shared__ double red[3][256];
    double re = 0.0, im = 0.0, aa = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 ai = a[i], ri = r[i];
        re += (double)ai.x * ri.x + (double)ai.y * ri.y;
        im += (double)ai.x * ri.y - (double)ai.y * ri.x;
        aa += (double)ai.x * ai.x + (double)ai.y * ai.y;
    }
    red[0][threadIdx.x] = re; red[1][threadIdx.x] = im; red[2][threadIdx.x] = aa;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) part[3 * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

// z += alpha y with alpha = <a, r> / ||a||^2 from the partials (0 when a = 0);
// every CTA sums the partials in the same order, so all use the same alpha.
__global__ void __launch_bounds__(256) ls_axpy_kernel(int64_t n, int nparts, const double *__restrict__ part,
                                                      const float2 *__restrict__ y, float2 *__restrict__ z) {
    __shared__ float2 alpha;
    if (threadIdx.x == 0) {
        double re = 0.0, im = 0.0, aa = 0.0;
        for (int b = 0; b < nparts; ++b) { re += part[3 * b]; im += part[3 * b + 1]; aa += part[3 * b + 2]; }
        alpha = aa > 0.0 ? make_float2((float)(re / aa), (float)(im / aa)) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const float2 yi = y[i];
        float2 zi = z[i];
        zi.x += alpha.x * yi.x - alpha.y * yi.y;
        zi.y += alpha.x * yi.y + alpha.y * yi.x;
        z[i] = zi;
    }
}

// standard normal pairs from splitmix64 of (seed, index) by Box-Muller
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__global__ void randn_kernel(int64_t n, uint64_t seed, float2 *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t a = mix64(seed ^ mix64((uint64_t)i));
    const double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    const double u2 = (mix64(a) >> 11) * (1.0 / 9007199254740992.0);
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    out[i] = make_float2((float)(r * cs), (float)(r * sn));
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

struct dst_unet {
    int device;
    int d, nc, C;
    UGrid grid[3];
    Layer L[NLAYER];
    int64_t nparams;
    float *params, *grads, *adam_m, *adam_v;     // FP32 [nparams]
    __nv_bfloat16 *wf[NLAYER], *wt[NLAYER];
    int kpadT[NLAYER];
    float *dw;                                   // largest co x kpad
    float *dw_part;                              // WGRAD_SPLITS partials of dw
    // activations [N][ch] and their gradients
    float *x0, *a1, *s1, *p1, *a2, *s2, *p2, *a3, *h3, *u2, *q2, *r2, *u1, *q1, *r1, *y;
    float *g_big1, *g_big2, *g_big3, *gs1, *gs2, *g_mid;   // gradient scratch
    float *scale;                                          // device scalar s
    float *gamma;                                          // device scalar: output scale of the correction
    double gamma_host;
    double *dscr;                                          // device doubles: [0] sum sq, [1] loss, [2] target sumsq
    double *part;                                          // LS_PARTS x 3 partial sums of the correction's scale
    int64_t act_floats;
    void *mem;
    size_t mem_bytes;
    bool packed;
};

static UGrid coarse(const UGrid &f) {
    UGrid c;
    c.D = f.D;
    c.N = 1;
    for (int a = 0; a < f.D; ++a) {
        c.n[a] = (f.n[a] + 1) / 2;
        c.N *= c.n[a];
    }
    for (int a = f.D; a < 4; ++a) c.n[a] = 1;
    return c;
}

static int unet_create(const dst_mesh *mesh, dst_unet **out) {
    dst_unet *u = new (std::nothrow) dst_unet();
    if (!u) return DST_ERR_OOM;
    std::memset(u, 0, sizeof(*u));
    DST_CUDA_TRY(cudaGetDevice(&u->device));
    u->d = mesh->d;
    u->nc = mesh->nc;
    u->C = 2 * mesh->nc;
    UGrid &g1 = u->grid[0];
    g1.D = mesh->d + 1;
    g1.n[0] = (int)mesh->nt;
    for (int a = 1; a < g1.D; ++a) g1.n[a] = (int)mesh->nu[mesh->d - a];     // t, [z], [y], x
    for (int a = g1.D; a < 4; ++a) g1.n[a] = 1;
    g1.N = mesh->nt * mesh->n_spatial;
    u->grid[1] = coarse(g1);
    u->grid[2] = coarse(u->grid[1]);
    int taps3 = 1;
    for (int a = 0; a < g1.D; ++a) taps3 *= 3;
    const int spec[NLAYER][4] = {{-1, 16, 3, 0}, {16, 16, 3, 0}, {16, 32, 3, 1}, {32, 32, 3, 1}, {32, 64, 3, 2},
                                 {64, 64, 3, 2}, {64, 32, 1, 1}, {32, 32, 3, 1}, {32, 16, 1, 0}, {16, 16, 3, 0},
                                 {16, -1, 1, 0}};
    int64_t off = 0;
    for (int l = 0; l < NLAYER; ++l) {
        Layer &L = u->L[l];
        L.ci = spec[l][0] < 0 ? u->C : spec[l][0];
        L.co = spec[l][1] < 0 ? u->C : spec[l][1];
        L.taps = spec[l][2] == 3 ? taps3 : 1;
        L.level = spec[l][3];
        L.kpad = (L.taps * L.ci + 15) / 16 * 16;
        L.co8 = (L.co + 7) / 8 * 8;
        L.woff = off;
        off += (int64_t)L.co * L.ci * L.taps;
        L.boff = off;
        off += L.co;
        u->kpadT[l] = (L.taps * L.co + 15) / 16 * 16;
    }
    u->nparams = off;
    // one device allocation for everything
    const int64_t N1 = g1.N, N2 = u->grid[1].N, N3 = u->grid[2].N;
    std::vector<size_t> sizes;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t total = 0;
    auto take = [&](size_t b) { size_t o = total; total += al(b); return o; };
    const size_t o_par = take(4 * sizeof(float) * u->nparams);
    size_t o_wf[NLAYER], o_wt[NLAYER];
    size_t maxdw = 0;
    for (int l = 0; l < NLAYER; ++l) {
        const Layer &L = u->L[l];
        o_wf[l] = take(sizeof(__nv_bfloat16) * (size_t)L.co8 * L.kpad);
        o_wt[l] = take(sizeof(__nv_bfloat16) * (size_t)((L.ci + 7) / 8 * 8) * u->kpadT[l]);
        maxdw = std::max(maxdw, (size_t)L.co * L.kpad);
    }
    const size_t o_dw = take(sizeof(float) * maxdw);
    const size_t o_dwp = take(sizeof(float) * maxdw * WGRAD_SPLITS);
    const int64_t acts[] = {N1 * u->C, N1 * 16, N1 * 16, N2 * 16, N2 * 32, N2 * 32, N3 * 32, N3 * 64, N3 * 64,
                            N2 * 64, N2 * 32, N2 * 32, N1 * 32, N1 * 16, N1 * 16, N1 * u->C};
    size_t o_act[16];
    for (int k = 0; k < 16; ++k) o_act[k] = take(sizeof(float) * acts[k]);
    const int64_t big = std::max(std::max(N1 * 32, N2 * 64), N3 * 64);
    const size_t o_g1 = take(sizeof(float) * big), o_g2 = take(sizeof(float) * big), o_g3 = take(sizeof(float) * big);
    const size_t o_gs1 = take(sizeof(float) * N1 * 16), o_gs2 = take(sizeof(float) * N2 * 32);
    const size_t o_gm = take(sizeof(float) * big);
    const size_t o_sc = take(sizeof(float) * 4), o_ds = take(sizeof(double) * 4);
    const size_t o_pt = take(sizeof(double) * 3 * LS_PARTS);
    if (cudaMalloc(&u->mem, total) != cudaSuccess) {
        cudaGetLastError();
        delete u;
        return DST_ERR_OOM;
    }
    u->mem_bytes = total;
    char *b = (char *)u->mem;
    u->params = (float *)(b + o_par);
    u->grads = u->params + u->nparams;
    u->adam_m = u->grads + u->nparams;
    u->adam_v = u->adam_m + u->nparams;
    for (int l = 0; l < NLAYER; ++l) {
        u->wf[l] = (__nv_bfloat16 *)(b + o_wf[l]);
        u->wt[l] = (__nv_bfloat16 *)(b + o_wt[l]);
    }
    u->dw = (float *)(b + o_dw);
    u->dw_part = (float *)(b + o_dwp);
    float **acts_p[16] = {&u->x0, &u->a1, &u->s1, &u->p1, &u->a2, &u->s2, &u->p2, &u->a3, &u->h3,
                          &u->u2, &u->q2, &u->r2, &u->u1, &u->q1, &u->r1, &u->y};
    for (int k = 0; k < 16; ++k) *acts_p[k] = (float *)(b + o_act[k]);
    u->g_big1 = (float *)(b + o_g1);
    u->g_big2 = (float *)(b + o_g2);
    u->g_big3 = (float *)(b + o_g3);
    u->gs1 = (float *)(b + o_gs1);
    u->gs2 = (float *)(b + o_gs2);
    u->g_mid = (float *)(b + o_gm);
    u->scale = (float *)(b + o_sc);
    u->gamma = u->scale + 1;
    u->dscr = (double *)(b + o_ds);
    u->part = (double *)(b + o_pt);
    cudaError_t e = cudaMemset(u->mem, 0, total);
    const float one = 1.0f;
    if (e == cudaSuccess) e = cudaMemcpy(u->gamma, &one, sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(u->mem);
        delete u;
        DST_CUDA_TRY(e);
    }
    u->gamma_host = 1.0;
    *out = u;
    return DST_OK;
}

static int pack(dst_unet *u, cudaStream_t s) {
    for (int l = 0; l < NLAYER; ++l) {
        const Layer &L = u->L[l];
        const int64_t n = std::max((int64_t)L.co8 * L.kpad, (int64_t)((L.ci + 7) / 8 * 8) * u->kpadT[l]);
        pack_weights_kernel<<<nblk(n), 256, 0, s>>>(L, u->params, u->wf[l], l == E1A ? nullptr : u->wt[l], u->kpadT[l]);
    }
    DST_CUDA_TRY(cudaGetLastError());
    u->packed = true;
    return DST_OK;
}

template <int NT>
static void launch_conv(const ConvArgs &a, cudaStream_t s) {
    const int64_t tiles = (a.g.N + 15) / 16;
    conv_fwd_kernel<NT><<<(unsigned)((tiles + 3) / 4), 128, 0, s>>>(a);
}

static int conv(dst_unet *u, int l, const float *in, float *out, const float *res, bool relu, const float *in_scale,
                cudaStream_t s) {
    const Layer &L = u->L[l];
    ConvArgs a;
    a.g = u->grid[L.level];
    a.ci = L.ci; a.taps = L.taps; a.kpad = L.kpad; a.co = L.co;
    a.in = in; a.w = u->wf[l]; a.bias = u->params + L.boff; a.res = res; a.in_scale = in_scale;
    a.relu = relu ? 1 : 0; a.out = out; a.flip = 0;
    switch (L.co8 / 8) {
        case 1: launch_conv<1>(a, s); break;
        case 2: launch_conv<2>(a, s); break;
        case 4: launch_conv<4>(a, s); break;
        case 8: launch_conv<8>(a, s); break;
        default: return DST_ERR_ARG;
    }
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

// input gradient of layer l: dx[n][ci] = sum dz[n - off][co] W[co][ci][tap]
static int conv_dgrad(dst_unet *u, int l, const float *dz, float *dx, cudaStream_t s) {
    const Layer &L = u->L[l];
    ConvArgs a;
    a.g = u->grid[L.level];
    a.ci = L.co; a.taps = L.taps; a.kpad = u->kpadT[l]; a.co = L.ci;
    a.in = dz; a.w = u->wt[l]; a.bias = nullptr; a.res = nullptr; a.in_scale = nullptr;
    a.relu = 0; a.out = dx; a.flip = 0;
    // wt holds the mirrored taps already
    switch ((L.ci + 7) / 8) {
        case 2: launch_conv<2>(a, s); break;
        case 4: launch_conv<4>(a, s); break;
        case 8: launch_conv<8>(a, s); break;
        default: return DST_ERR_ARG;
    }
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

static int conv_wgrad(dst_unet *u, int l, const float *in, const float *dz, const float *in_scale, cudaStream_t s) {
    const Layer &L = u->L[l];
    const UGrid &g = u->grid[L.level];
    WgradArgs a;
    a.g = g; a.ci = L.ci; a.taps = L.taps; a.kpad = L.kpad; a.co = L.co;
    a.in = in; a.dz = dz; a.in_scale = in_scale; a.dw = u->dw_part;
    const int64_t splits = std::min<int64_t>(WGRAD_SPLITS, (g.N + 1023) / 1024);
    a.nodes_per_cta = ((g.N + splits - 1) / splits + 15) / 16 * 16;
    const int ktiles = L.kpad / 8;
    dim3 grid((unsigned)splits, (unsigned)((ktiles + 3) / 4), (unsigned)((L.co + 15) / 16));
    // every (co < L.co, k < kpad) entry of every split's partial is written by exactly one warp
    conv_wgrad_kernel<<<grid, 128, 0, s>>>(a);
    const int64_t ndw = (int64_t)L.co * L.kpad;
    sum_partials_kernel<<<nblk(ndw), 256, 0, s>>>(ndw, (int)splits, u->dw_part, u->dw);
    const int64_t nw = (int64_t)L.co * L.ci * L.taps;
    unpack_wgrad_kernel<<<nblk(nw), 256, 0, s>>>(L, u->dw, u->grads);
    bias_grad_kernel<<<L.co, 256, 0, s>>>(g.N, L.co, dz, u->grads + L.boff);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

// y = U(x / s) on the node grid (x: the complex unknown vector as [N][C] floats)
static int forward(dst_unet *u, const float *x, const float *in_scale, cudaStream_t s) {
    int rc;
    if (!u->packed && (rc = pack(u, s))) return rc;
    const UGrid &g1 = u->grid[0], &g2 = u->grid[1], &g3 = u->grid[2];
    if ((rc = conv(u, E1A, x, u->a1, nullptr, true, in_scale, s))) return rc;
    if ((rc = conv(u, E1B, u->a1, u->s1, nullptr, true, nullptr, s))) return rc;
    pool_fwd_kernel<<<nblk(g2.N * 16), 256, 0, s>>>(g1, g2, 16, u->s1, u->p1);
    if ((rc = conv(u, E2A, u->p1, u->a2, nullptr, true, nullptr, s))) return rc;
    if ((rc = conv(u, E2B, u->a2, u->s2, nullptr, true, nullptr, s))) return rc;
    pool_fwd_kernel<<<nblk(g3.N * 32), 256, 0, s>>>(g2, g3, 32, u->s2, u->p2);
    if ((rc = conv(u, E3A, u->p2, u->a3, nullptr, true, nullptr, s))) return rc;
    if ((rc = conv(u, E3B, u->a3, u->h3, nullptr, true, nullptr, s))) return rc;
    up_fwd_kernel<<<nblk(g2.N * 64), 256, 0, s>>>(g2, g3, 64, u->h3, u->u2);
    if ((rc = conv(u, U2P, u->u2, u->q2, u->s2, false, nullptr, s))) return rc;
    if ((rc = conv(u, U2C, u->q2, u->r2, nullptr, true, nullptr, s))) return rc;
    up_fwd_kernel<<<nblk(g1.N * 32), 256, 0, s>>>(g1, g2, 32, u->r2, u->u1);
    if ((rc = conv(u, U1P, u->u1, u->q1, u->s1, false, nullptr, s))) return rc;
    if ((rc = conv(u, U1C, u->q1, u->r1, nullptr, true, nullptr, s))) return rc;
    if ((rc = conv(u, OUT, u->r1, u->y, nullptr, false, nullptr, s))) return rc;
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

// gradients of every parameter (into u->grads, overwritten) for dy = dL/dy
static int backward(dst_unet *u, const float *x, const float *in_scale, const float *dy, cudaStream_t s) {
    const UGrid &g1 = u->grid[0], &g2 = u->grid[1], &g3 = u->grid[2];
    float *dA = u->g_big1, *dB = u->g_big2, *dZ = u->g_big3;
    int rc;
    DST_CUDA_TRY(cudaMemsetAsync(u->grads, 0, sizeof(float) * u->nparams, s));
    // out (conv1 16 -> C): input r1
    if ((rc = conv_wgrad(u, OUT, u->r1, dy, nullptr, s))) return rc;
    if ((rc = conv_dgrad(u, OUT, dy, dA, s))) return rc;                      // d r1
    relu_mask_kernel<<<nblk(g1.N * 16), 256, 0, s>>>(g1.N * 16, dA, u->r1, dZ);
    if ((rc = conv_wgrad(u, U1C, u->q1, dZ, nullptr, s))) return rc;
    if ((rc = conv_dgrad(u, U1C, dZ, dA, s))) return rc;                      // d q1
    DST_CUDA_TRY(cudaMemcpyAsync(u->gs1, dA, sizeof(float) * g1.N * 16, cudaMemcpyDeviceToDevice, s));   // d s1
    if ((rc = conv_wgrad(u, U1P, u->u1, dA, nullptr, s))) return rc;
    if ((rc = conv_dgrad(u, U1P, dA, dB, s))) return rc;                      // d u1 (g1, 32)
    up_bwd_kernel<<<nblk(g2.N * 32), 256, 0, s>>>(g1, g2, 32, dB, dA);       // d r2 (g2, 32)
    relu_mask_kernel<<<nblk(g2.N * 32), 256, 0, s>>>(g2.N * 32, dA, u->r2, dZ);
    if ((rc = conv_wgrad(u, U2C, u->q2, dZ, nullptr, s))) return rc;
    if ((rc = conv_dgrad(u, U2C, dZ, dA, s))) return rc;                      // d q2
    DST_CUDA_TRY(cudaMemcpyAsync(u->gs2, dA, sizeof(float) * g2.N * 32, cudaMemcpyDeviceToDevice, s));   // d s2
    if ((rc = conv_wgrad(u, U2P, u->u2, dA, nullptr, s))) return rc;
    if ((rc = conv_dgrad(u, U2P, dA, dB, s))) return rc;                      // d u2 (g2, 64)
    up_bwd_kernel<<<nblk(g3.N * 64), 256, 0, s>>>(g2, g3, 64, dB, dA);       // d h3 (g3, 64)
    relu_mask_kernel<<<nblk(g3.N * 64), 256, 0, s>>>(g3.N * 64, dA, u->h3, dZ);
    if ((rc = conv_wgrad(u, E3B, u->a3, dZ, nullptr, s))) return rc;
    if ((rc = conv_dgrad(u, E3B, dZ, dA, s))) return rc;                      // d a3
    relu_mask_kernel<<<nblk(g3.N * 64), 256, 0, s>>>(g3.N * 64, dA, u->a3, dZ);
    if ((rc = conv_wgrad(u, E3A, u->p2, dZ, nullptr, s))) return rc;
    if ((rc = conv_dgrad(u, E3A, dZ, dA, s))) return rc;                      // d p2 (g3, 32)
    pool_bwd_kernel<<<nblk(g2.N * 32), 256, 0, s>>>(g2, g3, 32, dA, u->gs2);  // d s2 += pool^T d p2
    relu_mask_kernel<<<nblk(g2.N * 32), 256, 0, s>>>(g2.N * 32, u->gs2, u->s2, dZ);
    if ((rc = conv_wgrad(u, E2B, u->a2, dZ, nullptr, s))) return rc;
    if ((rc = conv_dgrad(u, E2B, dZ, dA, s))) return rc;                      // d a2
    relu_mask_kernel<<<nblk(g2.N * 32), 256, 0, s>>>(g2.N * 32, dA, u->a2, dZ);
    if ((rc = conv_wgrad(u, E2A, u->p1, dZ, nullptr, s))) return rc;
    if ((rc = conv_dgrad(u, E2A, dZ, dA, s))) return rc;                      // d p1 (g2, 16)
    pool_bwd_kernel<<<nblk(g1.N * 16), 256, 0, s>>>(g1, g2, 16, dA, u->gs1);  // d s1 += pool^T d p1
    relu_mask_kernel<<<nblk(g1.N * 16), 256, 0, s>>>(g1.N * 16, u->gs1, u->s1, dZ);
    if ((rc = conv_wgrad(u, E1B, u->a1, dZ, nullptr, s))) return rc;
    if ((rc = conv_dgrad(u, E1B, dZ, dA, s))) return rc;                      // d a1
    relu_mask_kernel<<<nblk(g1.N * 16), 256, 0, s>>>(g1.N * 16, dA, u->a1, dZ);
    if ((rc = conv_wgrad(u, E1A, x, dZ, in_scale, s))) return rc;
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

// s = ||v|| of a float array into u->scale
static int norm_into_scale(dst_unet *u, const float *v, int64_t n, cudaStream_t s) {
    sumsq_kernel<<<1, 256, 0, s>>>(n, v, u->dscr);
    sqrt_scalar_kernel<<<1, 32, 0, s>>>(u->dscr, u->scale);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

// loss and gradients for input x (scaled by its norm) and target t (same scale)
static int loss_grad(dst_unet *u, const float *x, const float *t, cudaStream_t s) {
    const int64_t n = u->grid[0].N * u->C;
    int rc;
    if ((rc = norm_into_scale(u, x, n, s))) return rc;
    if ((rc = forward(u, x, u->scale, s))) return rc;
    sumsq_kernel<<<1, 256, 0, s>>>(n, t, u->dscr + 2);
    loss_kernel<<<1, 256, 0, s>>>(n, u->y, t, u->scale, u->dscr + 2, u->g_mid, u->dscr + 1);
    return backward(u, x, u->scale, u->g_mid, s);
}

// ---- preconditioner hook used by the solver --------------------------------------

int dst_internal_unet_correct(dst_unet *u, const dst_mesh *mesh, const float2 *rho, float2 *z, float2 *tmp,
                              cudaStream_t s, int *launches) {
    const int64_t n = u->grid[0].N * u->C, nc = n / 2;
    const float *x = reinterpret_cast<const float *>(rho);
    const float2 *y = reinterpret_cast<const float2 *>(u->y);
    *launches = (u->packed ? 0 : NLAYER) + 2 + 15 + 1 + 2;
    int rc;
    if ((rc = norm_into_scale(u, x, n, s))) return rc;
    if ((rc = forward(u, x, u->scale, s))) return rc;
    // the correction's scale for this input: alpha minimising ||rho - alpha A y||, so the
    // corrected direction never leaves a larger residual than the sweep alone
    if ((rc = dst_internal_apply(mesh, DST_FP32, y, tmp, s))) return rc;
    const int parts = (int)std::min<int64_t>(LS_PARTS, (nc + 2047) / 2048);
    ls_partials_kernel<<<parts, 256, 0, s>>>(nc, tmp, rho, u->part);
    ls_axpy_kernel<<<nblk(nc), 256, 0, s>>>(nc, parts, u->part, y, z);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

bool dst_internal_unet_fits(const dst_unet *u, const dst_mesh *mesh) {
    return u && u->d == mesh->d && u->grid[0].N == mesh->nt * mesh->n_spatial && u->device == mesh->device;
}

// ---- C ABI ----------------------------------------------------------------------------

extern "C" int dst_unet_create(const dst_mesh *mesh, dst_unet **out) {
    if (!mesh || !out) return DST_ERR_ARG;
    *out = nullptr;
    if (mesh->nt > 0x7fffffff || mesh->n_spatial * mesh->nt > (1LL << 40)) return DST_ERR_ARG;
    return dst_internal_guard("dst_unet_create", [&] { return unet_create(mesh, out); });
}

extern "C" int dst_unet_destroy(dst_unet *u) {
    if (!u) return DST_OK;
    cudaFree(u->mem);
    delete u;
    return DST_OK;
}

extern "C" int dst_unet_num_params(const dst_unet *u, int64_t *n) {
    if (!u || !n) return DST_ERR_ARG;
    *n = u->nparams;
    return DST_OK;
}

extern "C" int dst_unet_set_params(dst_unet *u, const float *host) {
    if (!u || !host) return DST_ERR_ARG;
    DST_CUDA_TRY(cudaMemcpy(u->params, host, sizeof(float) * u->nparams, cudaMemcpyHostToDevice));
    DST_CUDA_TRY(cudaMemset(u->adam_m, 0, 2 * sizeof(float) * u->nparams));
    const float one = 1.0f;
    DST_CUDA_TRY(cudaMemcpy(u->gamma, &one, sizeof(float), cudaMemcpyHostToDevice));
    u->gamma_host = 1.0;
    u->packed = false;
    return DST_OK;
}

extern "C" int dst_unet_get_params(const dst_unet *u, float *host) {
    if (!u || !host) return DST_ERR_ARG;
    DST_CUDA_TRY(cudaMemcpy(host, u->params, sizeof(float) * u->nparams, cudaMemcpyDeviceToHost));
    return DST_OK;
}

extern "C" int dst_unet_forward(dst_unet *u, const void *x, void *y, void *stream) {
    if (!u || !x || !y) return DST_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = u->grid[0].N * u->C;
    int rc = norm_into_scale(u, (const float *)x, n, s);
    if (rc == DST_OK) rc = forward(u, (const float *)x, u->scale, s);
    if (rc) return rc;
    DST_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(float) * n, s));
    axpy_scaled_kernel<<<nblk(n), 256, 0, s>>>(n, u->scale, u->gamma, u->y, (float *)y);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}

extern "C" int dst_unet_loss_grad(dst_unet *u, const void *x, const void *target, double *loss, float *grad_host,
                                  void *stream) {
    if (!u || !x || !target) return DST_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = loss_grad(u, (const float *)x, (const float *)target, s);
    if (rc) return rc;
    if (loss) DST_CUDA_TRY(cudaMemcpyAsync(loss, u->dscr + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (grad_host)
        DST_CUDA_TRY(cudaMemcpyAsync(grad_host, u->grads, sizeof(float) * u->nparams, cudaMemcpyDeviceToHost, s));
    DST_CUDA_TRY(cudaStreamSynchronize(s));
    return DST_OK;
}

static int train(dst_unet *u, dst_mesh *mesh, int steps, float lr, uint64_t seed, float *loss_host, cudaStream_t s) {
    if (!dst_internal_unet_fits(u, mesh)) {
        dst_internal_set_error_detail("dst_unet_train: the network was created for another mesh");
        return DST_ERR_ARG;
    }
    SweepPlan plan;
    int rc = dst_sweep_plan(mesh, plan);
    if (rc) return rc;
    const int64_t n = mesh->n_unknowns;
    const size_t vb = (sizeof(float2) * (size_t)n + 255) & ~(size_t)255;
    const size_t sweep_bytes = dst_sweep_scratch_bytes(plan, n);
    char *scr = nullptr;
    if (cudaMallocAsync((void **)&scr, 5 * vb + sweep_bytes + 256, s) != cudaSuccess) {
        cudaGetLastError();
        return DST_ERR_OOM;
    }
    float2 *e = (float2 *)scr, *r = (float2 *)(scr + vb), *z = (float2 *)(scr + 2 * vb), *az = (float2 *)(scr + 3 * vb),
           *tg = (float2 *)(scr + 4 * vb);
    double *lossd = nullptr;
    rc = dst_sweep_setup(mesh, plan, scr + 5 * vb, s);
    std::vector<double> losses(steps > 0 ? steps : 1);
    if (rc == DST_OK && cudaMallocAsync((void **)&lossd, sizeof(double) * (steps > 0 ? steps : 1), s) != cudaSuccess) {
        cudaGetLastError();
        rc = DST_ERR_OOM;
    }
    const float b1 = 0.9f, b2 = 0.999f;
    for (int it = 0; it < steps && rc == DST_OK; ++it) {
        // a training pair from the method: e random, r = A e, z = M_CN r, rho = r - A z, target e - z
        randn_kernel<<<nblk(n), 256, 0, s>>>(n, seed + (uint64_t)it * 0x9E3779B97F4A7C15ull, e);
        if ((rc = dst_internal_apply(mesh, DST_FP32, e, r, s))) break;
        if ((rc = dst_sweep_apply(plan, n, r, z, s))) break;
        if ((rc = dst_internal_apply(mesh, DST_FP32, z, az, s))) break;
        if ((rc = dst_k_sub_f32(n, r, az, r, s))) break;                  // r <- rho
        if ((rc = dst_k_sub_f32(n, e, z, tg, s))) break;                  // target
        if ((rc = loss_grad(u, (const float *)r, (const float *)tg, s))) break;
        if (cudaMemcpyAsync(lossd + it, u->dscr + 1, sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            rc = DST_ERR_CUDA;
            break;
        }
        const float c1 = 1.f - std::pow(b1, (float)(it + 1)), c2 = 1.f - std::pow(b2, (float)(it + 1));
        adam_kernel<<<nblk(u->nparams), 256, 0, s>>>(u->nparams, u->params, u->grads, u->adam_m, u->adam_v, lr, b1, b2,
                                                      c1, c2, 1e-8f);
        if ((rc = pack(u, s))) break;
    }
    // output scale: the least-squares factor gamma = <U, t> / ||U||^2 over fresh pairs, so
    // that the scaled correction's error on them is never above the sweep's own
    if (rc == DST_OK && steps > 0) {
        const int nval = 8;
        double *acc = u->dscr + 2;                      // [2], [3]; dscr[2] is reused by loss_grad only
        if (cudaMemsetAsync(acc, 0, 2 * sizeof(double), s) != cudaSuccess) rc = DST_ERR_CUDA;
        for (int it = 0; it < nval && rc == DST_OK; ++it) {
            randn_kernel<<<nblk(n), 256, 0, s>>>(n, ~seed + (uint64_t)it * 0xD1B54A32D192ED03ull, e);
            if ((rc = dst_internal_apply(mesh, DST_FP32, e, r, s))) break;
            if ((rc = dst_sweep_apply(plan, n, r, z, s))) break;
            if ((rc = dst_internal_apply(mesh, DST_FP32, z, az, s))) break;
            if ((rc = dst_k_sub_f32(n, r, az, r, s))) break;
            if ((rc = dst_k_sub_f32(n, e, z, tg, s))) break;
            const float *x = (const float *)r;
            if ((rc = norm_into_scale(u, x, 2 * n, s))) break;
            if ((rc = forward(u, x, u->scale, s))) break;
            dot_kernel<<<1, 256, 0, s>>>(2 * n, u->y, (const float *)tg, u->scale, acc);
        }
        double hacc[2] = {0.0, 0.0};
        if (rc == DST_OK && (cudaMemcpyAsync(hacc, acc, sizeof(hacc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                             cudaStreamSynchronize(s) != cudaSuccess))
            rc = DST_ERR_CUDA;
        if (rc == DST_OK) {
            double gmm = hacc[1] > 0.0 ? hacc[0] / hacc[1] : 0.0;
            if (!(gmm > 0.0)) gmm = 0.0;
            const float gf = (float)gmm;
            u->gamma_host = gmm;
            if (cudaMemcpyAsync(u->gamma, &gf, sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                rc = DST_ERR_CUDA;
        }
    }
    if (rc == DST_OK && steps > 0 && loss_host) {
        if (cudaMemcpyAsync(losses.data(), lossd, sizeof(double) * steps, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = DST_ERR_CUDA;
        for (int i = 0; i < steps; ++i) loss_host[i] = (float)losses[i];
    }
    if (lossd) cudaFreeAsync(lossd, s);
    cudaFreeAsync(scr, s);
    if (rc == DST_OK) DST_CUDA_TRY(cudaStreamSynchronize(s));
    return rc;
}

extern "C" int dst_unet_train(dst_unet *u, dst_mesh *mesh, int steps, float lr, uint64_t seed, float *loss_host,
                              void *stream) {
    if (!u || !mesh || steps < 0 || !(lr > 0)) return DST_ERR_ARG;
    return dst_internal_guard("dst_unet_train", [&] { return train(u, mesh, steps, lr, seed, loss_host, (cudaStream_t)stream); });
}

extern "C" int dst_unet_output_scale(const dst_unet *u, double *gamma) {
    if (!u || !gamma) return DST_ERR_ARG;
    *gamma = u->gamma_host;
    return DST_OK;
}

extern "C" int dst_set_learned_precond(dst_mesh *mesh, dst_unet *u) {
    if (!mesh) return DST_ERR_ARG;
    if (u && !dst_internal_unet_fits(u, mesh)) {
        dst_internal_set_error_detail("dst_set_learned_precond: the network was created for another mesh");
        return DST_ERR_ARG;
    }
    mesh->unet = u;
    return DST_OK;
}
