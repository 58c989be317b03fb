// FFT of the planes of periodic axes in shared memory (used by the
// Crank-Nicolson sweep in FP32 and by the energy observable in FP64).
//
// Each CTA loads one plane (n1 x n2 nodes of one layer, or of one x node of a
// layer) of its component group into shared memory, transforms every line of
// the inner axis and then every line of the outer axis, and stores the result.
// The mixed-radix Stockham self-sorting scheme (stages of radix 4, 2, then odd
// primes; twiddles from a per-axis table w[j] = exp(sign 2 pi i j / n)) runs
// either over all lines of an axis at once, the CTA's threads sharing every
// stage's butterflies (when a second plane buffer fits in shared memory), or one
// line per warp with two scratch lines.
// Forward (sign -1): node layout in, frequency layout [b][f][c] out with
// f = i1 n2 + i2.  Inverse (sign +1): frequency layout in, node layout out,
// scaled by 1 / (n1 n2).
#pragma once

#include "sweep.h"

namespace dst_fft {

constexpr int FFT_THREADS = 256;
constexpr int FFT_WARPS = FFT_THREADS / 32;

template <typename V> struct Real;
template <> struct Real<float2> { using type = float; };
template <> struct Real<double2> { using type = double; };

template <typename V> __device__ __forceinline__ V mk(typename Real<V>::type a, typename Real<V>::type b) {
    V r; r.x = a; r.y = b; return r;
}
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    return mk<V>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cfma(V a, V b, V acc) {
    return mk<V>(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}

__device__ __forceinline__ void sincos_pi(float x, float *s, float *c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincos_pi(double x, double *s, double *c) { sincospi(x, s, c); }

template <typename V>
__device__ void warp_fft_line(V *line, int st, int n, const int *rad, int nrad, const V *w, V *a, V *b) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < n; i += 32) a[i] = line[i * st];
    __syncwarp();
    V *d0 = a, *d1 = b;
    int Ns = 1;
    for (int s = 0; s < nrad; ++s) {
        const int R = rad[s];
        const int q = n / R;               // butterflies of this stage
        const int step = n / (Ns * R);     // exp(sign 2 pi i k / (Ns R)) = w[k * step]
        for (int j = lane; j < q; j += 32) {
            const int k = j % Ns;
            const int dst = (j / Ns) * Ns * R + k;
            if (R == 2) {
                const V v0 = d0[j], v1 = cmul(d0[j + q], w[k * step]);
                d1[dst] = cadd(v0, v1);
                d1[dst + Ns] = csub(v0, v1);
            } else if (R == 4) {
                const V v0 = d0[j];
                const V v1 = cmul(d0[j + q], w[k * step]);
                const V v2 = cmul(d0[j + 2 * q], w[(2 * k * step) % n]);
                const V v3 = cmul(d0[j + 3 * q], w[(3 * k * step) % n]);
                const V om = w[n / 4];                       // exp(sign i pi / 2)
                const V t0 = cadd(v0, v2), t1 = csub(v0, v2);
                const V t2 = cadd(v1, v3), t3 = cmul(om, csub(v1, v3));
                d1[dst] = cadd(t0, t2);
                d1[dst + Ns] = cadd(t1, t3);
                d1[dst + 2 * Ns] = csub(t0, t2);
                d1[dst + 3 * Ns] = csub(t1, t3);
            } else {
                // general radix: V_o = sum_r v_r exp(sign 2 pi i r o / R), v_r twiddled
                for (int o = 0; o < R; ++o) {
                    V acc = mk<V>(0, 0);
                    for (int r = 0; r < R; ++r) {
                        const V vr = cmul(d0[j + r * q], w[(int)(((long long)r * k * step) % n)]);
                        acc = cfma(w[(int)(((long long)r * o * q) % n)], vr, acc);
                    }
                    d1[dst + o * Ns] = acc;
                }
            }
        }
        __syncwarp();
        V *t = d0; d0 = d1; d1 = t;
        Ns *= R;
    }
    for (int i = lane; i < n; i += 32) line[i * st] = d0[i];
    __syncwarp();
}

// All lines of one axis of the plane through the Stockham stages at once: each
// stage's butterflies of every line are spread over the CTA's threads, with a
// barrier between stages (ping-pong between the plane and a second buffer).
// Line l of the axis starts at l_base(l) and has element stride st; `nl` lines.
// Returns the buffer holding the result (the plane or the second buffer).
template <typename V>
__device__ V *cta_fft_axis(V *d0, V *d1, int n, int st, int nl, int lstride_in, int lsplit, int lstride_out,
                           const int *rad, int nrad, const V *w) {
    // line l = (la, lb) with la = l / lsplit, lb = l % lsplit; element i of line l at
    // la * lstride_out + lb * lstride_in + i * st (the same map in both buffers)
    int Ns = 1;
    for (int s = 0; s < nrad; ++s) {
        const int R = rad[s];
        const int q = n / R;
        const int step = n / (Ns * R);
        for (int idx = threadIdx.x; idx < nl * q; idx += blockDim.x) {
            const int l = idx / q, j = idx % q;
            const int base = (l / lsplit) * lstride_out + (l % lsplit) * lstride_in;
            const V *src = d0 + base;
            V *dst_ = d1 + base;
            const int k = j % Ns;
            const int dst = (j / Ns) * Ns * R + k;
            if (R == 2) {
                const V v0 = src[j * st], v1 = cmul(src[(j + q) * st], w[k * step]);
                dst_[dst * st] = cadd(v0, v1);
                dst_[(dst + Ns) * st] = csub(v0, v1);
            } else if (R == 4) {
                const V v0 = src[j * st];
                const V v1 = cmul(src[(j + q) * st], w[k * step]);
                const V v2 = cmul(src[(j + 2 * q) * st], w[(2 * k * step) % n]);
                const V v3 = cmul(src[(j + 3 * q) * st], w[(3 * k * step) % n]);
                const V om = w[n / 4];
                const V t0 = cadd(v0, v2), t1 = csub(v0, v2);
                const V t2 = cadd(v1, v3), t3 = cmul(om, csub(v1, v3));
                dst_[dst * st] = cadd(t0, t2);
                dst_[(dst + Ns) * st] = cadd(t1, t3);
                dst_[(dst + 2 * Ns) * st] = csub(t0, t2);
                dst_[(dst + 3 * Ns) * st] = csub(t1, t3);
            } else {
                for (int o = 0; o < R; ++o) {
                    V acc = mk<V>(0, 0);
                    for (int r = 0; r < R; ++r) {
                        const V vr = cmul(src[(j + r * q) * st], w[(int)(((long long)r * k * step) % n)]);
                        acc = cfma(w[(int)(((long long)r * o * q) % n)], vr, acc);
                    }
                    dst_[(dst + o * Ns) * st] = acc;
                }
            }
        }
        __syncthreads();
        V *t = d0; d0 = d1; d1 = t;
        Ns *= R;
    }
    return d0;
}

// Shared memory of one CTA: the plane, two twiddle tables, two scratch lines per warp.
template <typename V>
inline size_t fft_smem_bytes(const SweepFft &a) {
    const int nmax = a.n1 > a.n2 ? a.n1 : a.n2;
    const size_t scratch = a.pingpong ? (size_t)a.ncb * a.n1 * a.n2 : (size_t)FFT_WARPS * 2 * nmax;
    return sizeof(V) * ((size_t)a.ncb * a.n1 * a.n2 + a.n1 + a.n2 + scratch);
}

template <typename V>
__global__ void __launch_bounds__(FFT_THREADS)
fft_planes_kernel(SweepFft a, int inverse, const V *__restrict__ in, V *__restrict__ out) {
    using R = typename Real<V>::type;
    extern __shared__ __align__(16) unsigned char fft_sm_raw[];
    V *sm = reinterpret_cast<V *>(fft_sm_raw);
    const int n1 = a.n1, n2 = a.n2, nc = a.nc, ncb = a.ncb;
    const int nf = n1 * n2;
    V *plane = sm;                                        // [ncb][n1][n2]
    V *w1 = plane + (size_t)ncb * nf;                     // twiddles of the outer axis (n1)
    V *w2 = w1 + n1;                                      // twiddles of the inner axis (n2)
    V *scr = w2 + n2;                                     // second plane, or per warp two lines of nmax
    const int nmax = n1 > n2 ? n1 : n2;
    const int64_t b = blockIdx.x;
    const int c0 = blockIdx.y * ncb;
    const int64_t base = (b / a.nbx) * a.ns_nodes + (b % a.nbx) * a.sbx;   // node index of (i1, i2) = (0, 0)
    const R sign = inverse ? (R)1 : (R)-1;
    for (int j = threadIdx.x; j < n1; j += FFT_THREADS) {
        R sn, cs;
        sincos_pi((R)2 * (R)j / (R)n1, &sn, &cs);
        w1[j] = mk<V>(cs, sign * sn);
    }
    for (int j = threadIdx.x; j < n2; j += FFT_THREADS) {
        R sn, cs;
        sincos_pi((R)2 * (R)j / (R)n2, &sn, &cs);
        w2[j] = mk<V>(cs, sign * sn);
    }
    for (int idx = threadIdx.x; idx < nf * ncb; idx += FFT_THREADS) {
        const int cc = idx % ncb, f = idx / ncb;
        const int i1 = f / n2, i2 = f % n2;
        V v;
        if (inverse) v = in[(b * nf + f) * nc + c0 + cc];
        else v = in[(base + (int64_t)i1 * a.s1 + (int64_t)i2 * a.s2) * nc + c0 + cc];
        plane[(size_t)cc * nf + f] = v;
    }
    __syncthreads();
    if (a.pingpong) {
        // CTA-wide stages; scr is a second plane
        V *cur = plane;
        if (n2 > 1) cur = cta_fft_axis(cur, cur == plane ? scr : plane, n2, 1, ncb * n1, 0, 1, n2, a.rad2, a.nrad2, w2);
        if (n1 > 1)
            cur = cta_fft_axis(cur, cur == plane ? scr : plane, n1, n2, ncb * n2, 1, n2, nf, a.rad1, a.nrad1, w1);
        if (cur != plane) {
            for (int idx = threadIdx.x; idx < nf * ncb; idx += FFT_THREADS) plane[idx] = cur[idx];
            __syncthreads();
        }
    } else {
        const int warp = threadIdx.x >> 5;
        V *sa = scr + (size_t)warp * 2 * nmax, *sb = sa + nmax;
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
    }
    const R scale = inverse ? (R)1 / (R)nf : (R)1;
    for (int idx = threadIdx.x; idx < nf * ncb; idx += FFT_THREADS) {
        const int cc = idx % ncb, f = idx / ncb;
        const int i1 = f / n2, i2 = f % n2;
        V v = plane[(size_t)cc * nf + f];
        v.x *= scale;
        v.y *= scale;
        if (inverse) out[(base + (int64_t)i1 * a.s1 + (int64_t)i2 * a.s2) * nc + c0 + cc] = v;
        else out[(b * nf + f) * nc + c0 + cc] = v;
    }
}

// Pick the components per CTA and the stage layout for planes of a.n1 x a.n2:
// CTA-wide stages (second plane buffer) when they fit, else one line per warp;
// fewer components per CTA when the CTAs would not fill the GPU (nb planes per
// component group).  Returns false if nothing fits in `limit` bytes.
template <typename V>
inline bool choose_layout(SweepFft &a, int64_t nb, size_t limit) {
    for (int pp = 1; pp >= 0; --pp) {
        a.pingpong = pp;
        for (int ncb = a.nc; ncb >= 1; ncb /= 2) {
            a.ncb = ncb;
            if (fft_smem_bytes<V>(a) > limit) continue;
            if (ncb > 1 && nb * (a.nc / ncb) < 304) continue;
            return true;
        }
        a.ncb = 1;
        if (fft_smem_bytes<V>(a) <= limit) return true;
    }
    return false;
}

// Stockham radices of n: fours, a two, then odd primes.
inline void radices(int n, int *r, int &nr) {
    nr = 0;
    while (n % 4 == 0) { r[nr++] = 4; n /= 4; }
    while (n % 2 == 0) { r[nr++] = 2; n /= 2; }
    for (int p = 3; n > 1; p += 2)
        while (n % p == 0) { r[nr++] = p; n /= p; }
}

}  // namespace dst_fft
