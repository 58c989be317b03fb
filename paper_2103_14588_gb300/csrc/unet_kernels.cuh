// Kernels of the convolutional U-Net preconditioner: implicit-GEMM convolutions
// on BF16 tensor cores with FP32 accumulation (mma.sync m16n8k16), and the
// element-wise pieces (pooling, upsampling, ReLU masks, bias gradients, Adam).
//
// Activations are FP32 arrays [node][channel] over a D-dimensional node grid
// (t slowest, then z, y, x; only the axes the mesh has); they are rounded to
// BF16 as they enter a convolution.  A convolution with kernel 3 in every axis
// (taps = 3^D, zero padding that keeps the size) or kernel 1 (one tap) is the
// cross-correlation out[n][co] = b[co] + sum_tap sum_ci in[n + off(tap)][ci] W[co][ci][tap],
// evaluated as a GEMM with M = nodes, N = output channels and K = taps x input
// channels; K index k = tap * Ci + ci, tap in row-major order of the kernel
// offsets (-1, 0, 1) per axis.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace dst_nn {

struct UGrid {
    int D;            // axes (2, 3 or 4)
    int n[4];         // nodes per axis, slowest first
    int64_t N;        // nodes
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// coordinates of node r (slowest axis first)
__device__ __forceinline__ void coords(const UGrid &g, int64_t r, int (&c)[4]) {
    for (int a = g.D - 1; a >= 0; --a) {
        c[a] = (int)(r % g.n[a]);
        r /= g.n[a];
    }
}

// node index of the neighbour of (c) at kernel tap `tap` (taps = 3^D), or -1 outside
__device__ __forceinline__ int64_t tap_node(const UGrid &g, const int (&c)[4], int tap, int taps) {
    if (taps == 1) {
        int64_t r = 0;
        for (int a = 0; a < g.D; ++a) r = r * g.n[a] + c[a];
        return r;
    }
    int64_t r = 0;
    int pw = taps / 3;
    for (int a = 0; a < g.D; ++a) {
        const int o = (tap / pw) % 3 - 1;
        pw /= 3;
        const int x = c[a] + o;
        if (x < 0 || x >= g.n[a]) return -1;
        r = r * g.n[a] + x;
    }
    return r;
}

struct ConvArgs {
    UGrid g;
    int ci, taps, kpad;             // input channels, kernel taps, K padded to 16
    int co;                         // output channels (stored); the weight rows are padded to 8 NT
    const float *in;                // [N][ci]
    const __nv_bfloat16 *w;         // [8 NT][kpad], k = tap * ci + c
    const float *bias;              // [co] or null
    const float *res;               // [N][co] added before the activation, or null
    const float *in_scale;          // device scalar s: the input is read as in / s (null: 1)
    int relu;
    float *out;                     // [N][co]
    int flip;                       // 1: taps mirrored (the input-gradient convolution)
};

// Two consecutive K entries (k even) of row node r as a bf16 pair.
__device__ __forceinline__ uint32_t a_pair(const ConvArgs &a, const int (&c)[4], bool valid, int k, float inv) {
    if (!valid || k >= a.taps * a.ci) return 0u;
    const int tap = k / a.ci, ch = k % a.ci;
    const int t = a.flip ? a.taps - 1 - tap : tap;
    const int64_t nb = tap_node(a.g, c, t, a.taps);
    if (nb < 0) return 0u;
    const float2 v = *reinterpret_cast<const float2 *>(a.in + nb * a.ci + ch);
    return pack_bf16(v.x * inv, v.y * inv);
}

// One warp: 16 consecutive nodes x 8 NT output channels.
template <int NT>
__global__ void __launch_bounds__(128) conv_fwd_kernel(ConvArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tg = lane & 3;
    const int64_t m0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * 16;
    if (m0 >= a.g.N) return;
    const int64_t r0 = m0 + g, r1 = m0 + g + 8;
    const bool v0 = r0 < a.g.N, v1 = r1 < a.g.N;
    int c0[4] = {0, 0, 0, 0}, c1[4] = {0, 0, 0, 0};
    if (v0) coords(a.g, r0, c0);
    if (v1) coords(a.g, r1, c1);
    const float inv = a.in_scale ? 1.0f / *a.in_scale : 1.0f;
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const uint32_t *w32 = reinterpret_cast<const uint32_t *>(a.w);
    const int kw = a.kpad / 2;                      // 32-bit words per weight row
    for (int kc = 0; kc < a.kpad; kc += 16) {
        uint32_t af[4];
        af[0] = a_pair(a, c0, v0, kc + 2 * tg, inv);
        af[1] = a_pair(a, c1, v1, kc + 2 * tg, inv);
        af[2] = a_pair(a, c0, v0, kc + 8 + 2 * tg, inv);
        af[3] = a_pair(a, c1, v1, kc + 8 + 2 * tg, inv);
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const uint32_t *wr = w32 + (size_t)(j * 8 + g) * kw + kc / 2;
            mma_16816(acc[j], af, __ldg(wr + tg), __ldg(wr + 4 + tg));
        }
    }
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int co = j * 8 + 2 * tg;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t r = h ? r1 : r0;
            if (r >= a.g.N) continue;
            for (int e = 0; e < 2; ++e) {
                const int cc = co + e;
                if (cc >= a.co) continue;
                float v = acc[j][2 * h + e];
                if (a.bias) v += a.bias[cc];
                if (a.res) v += a.res[r * a.co + cc];
                if (a.relu) v = fmaxf(v, 0.f);
                a.out[r * a.co + cc] = v;
            }
        }
    }
}

struct WgradArgs {
    UGrid g;
    int ci, taps, kpad, co;
    const float *in;        // layer input [N][ci]
    const float *dz;        // gradient of the layer's output before its activation [N][co]
    const float *in_scale;  // as in ConvArgs
    float *dw;              // [splits][co][kpad] FP32: one partial per node range (blockIdx.x)
    int64_t nodes_per_cta;  // node range of one CTA
};

// dW[co][k] = sum_n dz[n][co] in[n + off(tap(k))][ci(k)]: GEMM with M = co, N = k,
// K = nodes; one warp per (16 co x 8 k) tile over the CTA's node range, whose
// partial goes to its own slice of dw (summed afterwards in a fixed order, so
// that training is reproducible).
__global__ void __launch_bounds__(128) conv_wgrad_kernel(WgradArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tg = lane & 3;
    const int ktile = blockIdx.y * (blockDim.x >> 5) + warp;     // 8 k-columns each
    const int cot = blockIdx.z;                                  // 16 co each
    if (ktile * 8 >= a.kpad) return;
    const int kcol = ktile * 8 + g;                              // this lane's B column
    const bool kvalid = kcol < a.taps * a.ci;
    const int tap = kvalid ? kcol / a.ci : 0, ch = kvalid ? kcol % a.ci : 0;
    const int coA = cot * 16 + g, coB = coA + 8;
    const float inv = a.in_scale ? 1.0f / *a.in_scale : 1.0f;
    const int64_t n_begin = (int64_t)blockIdx.x * a.nodes_per_cta;
    int64_t n_end = n_begin + a.nodes_per_cta;
    if (n_end > a.g.N) n_end = a.g.N;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    auto dzv = [&](int64_t n, int co) -> float { return (n < n_end && co < a.co) ? a.dz[n * a.co + co] : 0.f; };
    auto inv_b = [&](int64_t n) -> float {
        if (n >= n_end || !kvalid) return 0.f;
        int c[4];
        coords(a.g, n, c);
        const int64_t nb = tap_node(a.g, c, tap, a.taps);
        return nb < 0 ? 0.f : a.in[nb * a.ci + ch] * inv;
    };
    for (int64_t n0 = n_begin; n0 < n_end; n0 += 16) {
        uint32_t af[4];
        const int64_t na = n0 + 2 * tg, nb8 = n0 + 8 + 2 * tg;
        af[0] = pack_bf16(dzv(na, coA), dzv(na + 1, coA));
        af[1] = pack_bf16(dzv(na, coB), dzv(na + 1, coB));
        af[2] = pack_bf16(dzv(nb8, coA), dzv(nb8 + 1, coA));
        af[3] = pack_bf16(dzv(nb8, coB), dzv(nb8 + 1, coB));
        const uint32_t b0 = pack_bf16(inv_b(na), inv_b(na + 1));
        const uint32_t b1 = pack_bf16(inv_b(nb8), inv_b(nb8 + 1));
        mma_16816(acc, af, b0, b1);
    }
    // D: (row co = cot*16 + g (+8), col k = ktile*8 + 2 tg + {0, 1})
    const int k0 = ktile * 8 + 2 * tg;
    const int rows[2] = {coA, coB};
    float *part = a.dw + (size_t)blockIdx.x * a.co * a.kpad;
    for (int h = 0; h < 2; ++h)
        for (int e = 0; e < 2; ++e)
            if (rows[h] < a.co && k0 + e < a.kpad) part[(size_t)rows[h] * a.kpad + k0 + e] = acc[2 * h + e];
}

// dw[i] = sum over the node-range partials, in order
__global__ void sum_partials_kernel(int64_t n, int splits, const float *__restrict__ part, float *__restrict__ dw) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float t = 0.f;
    for (int b = 0; b < splits; ++b) t += part[(size_t)b * n + i];
    dw[i] = t;
}

}  // namespace dst_nn
