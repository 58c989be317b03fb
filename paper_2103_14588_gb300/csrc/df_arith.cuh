// Error-free and compensated FP32 arithmetic shared by the Gram-Schmidt
// kernels of blas_df.cu and the batched persistent solver (batch.cu).
//
//   TwoProd(a, b): p = a*b, e = fma(a, b, -p)            (exact product, Dekker/FMA)
//   TwoSum(a, b):  s = a+b, e = (a-(s-bb)) + (b-bb)       (exact sum, Knuth)
// "df32" values are (hi, lo) pairs of floats (Dekker 1971; the compensated dot
// product of Ogita, Rump & Oishi 2005).
#pragma once

#include <cuda_runtime.h>

namespace dst {

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (p, e) with p + e = (ah + al)(bh + bl) up to the al*bl term (2^-48 relative)
__device__ __forceinline__ void df_prod(float ah, float al, float bh, float bl, float &p, float &e) {
    p = ah * bh;
    e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
}

struct DfAcc {
    float hi, lo;
    __device__ __forceinline__ void zero() { hi = 0.f; lo = 0.f; }
    // += p + e
    __device__ __forceinline__ void add(float p, float e) {
        float s, t;
        two_sum(hi, p, s, t);
        hi = s;
        lo += t + e;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// (ah, al) += (bh, bl) in df32, renormalised
__device__ __forceinline__ void df_add(float &ah, float &al, float bh, float bl) {
    float s, e;
    two_sum(ah, bh, s, e);
    e += al + bl;
    ah = s + e;
    al = e - (ah - s);
}

// Warp sum of a df32 value, in df32 (no FP64 work per lane); FP64 result
// valid in lane 0.
__device__ __forceinline__ double dfwarp_sum(DfAcc a) {
    float h = a.hi, l = a.lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float bh = __shfl_down_sync(0xffffffffu, h, o);
        const float bl = __shfl_down_sync(0xffffffffu, l, o);
        df_add(h, l, bh, bl);
    }
    return (double)h + (double)l;
}

__device__ __forceinline__ double dwarp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// (p, e): p + e = a b exactly, plus the lo cross terms that are present
template <bool AL, bool BL>
__device__ __forceinline__ void df_prod_t(float ah, float al, float bh, float bl, float &p, float &e) {
    p = ah * bh;
    e = fmaf(ah, bh, -p);
    if (BL) e = fmaf(ah, bl, e);
    if (AL) e = fmaf(al, bh, e);
}

// acc -= v c for one complex entry (v df32, c = (re_hi, re_lo, im_hi, im_lo))
template <bool VL = true>
__device__ __forceinline__ void caxpy_sub(float vhr, float vhi, float vlr, float vli, const float4 &c, DfAcc &ar,
                                          DfAcc &ai) {
    float p1, e1, p2, e2;
    df_prod_t<VL, true>(vhr, vlr, c.x, c.y, p1, e1);     // vr hr
    df_prod_t<VL, true>(vhi, vli, c.z, c.w, p2, e2);     // vi hi
    ar.add(-p1, -e1);
    ar.add(p2, e2);
    df_prod_t<VL, true>(vhr, vlr, c.z, c.w, p1, e1);     // vr hi
    df_prod_t<VL, true>(vhi, vli, c.x, c.y, p2, e2);     // vi hr
    ai.add(-p1, -e1);
    ai.add(-p2, -e2);
}

__device__ __forceinline__ void renorm(DfAcc &a) {
    const float s = a.hi + a.lo;
    a.lo = a.lo - (s - a.hi);
    a.hi = s;
}

// ---- FP32-stored basis: anchored error-free accumulation ------------------
//
// With the basis stored as single FP32 planes, the compensated sums of the
// hi/lo kernels spend most of their instructions in TwoSum (6 additions per
// term).  Here every thread first bounds the magnitude B of every partial sum
// it will form (the basis vectors have unit 2-norm, so each of their
// components is at most 1 in magnitude), picks a power of two sigma with
// 4B < sigma <= 8B, and accumulates into hi = sigma + (partial sum), so hi
// stays within [3/4, 5/4] sigma.  A product term a*b is added with one FMA,
// s = fl(hi + a b); since s and hi are within a factor 2 of each other,
// z = s - hi is exact (Sterbenz), so a b - z is exactly the rounding error
// of that FMA, and fma(a, b, -z) delivers it rounded once to FP32 into a
// plain lo.  Four instructions per term (two FMA, two additions) instead of
// TwoProd + TwoSum; hi - sigma is exact at the end.  Anchoring to a fixed
// power of two is the extraction idea of Rump, Ogita & Oishi's AccSum
// (SIAM J. Sci. Comput. 31, 2008); the result has the accuracy of a
// compensated dot product, about eps32^2 sigma per term.

// power of two sigma with 4 b < sigma <= 8 b (b >= 0); +inf when b is not
// finite or above 2^123, so that the results become NaN instead of wrong
__device__ __forceinline__ float anchor_above(float b) {
    const unsigned u = __float_as_uint(b * 1.001f) & 0x7f800000u;   // 2^floor(log2), 0 if subnormal
    if (u >= (123u + 127u) << 23) return __int_as_float(0x7f800000);
    return __uint_as_float(u + (3u << 23));
}

struct AnAcc {
    float hi, lo;
    __device__ __forceinline__ void init(float sigma) { hi = sigma; lo = 0.f; }
    // += a b (|a b| <= sigma / 4)
    __device__ __forceinline__ void madd(float a, float b) {
        const float s_ = fmaf(a, b, hi);
        const float z = s_ - hi;          // exact
        lo += fmaf(a, b, -z);             // the FMA's rounding error
        hi = s_;
    }
    // += x (|x| <= sigma / 4), FastTwoSum
    __device__ __forceinline__ void add(float x) {
        const float s_ = hi + x;
        const float z = s_ - hi;
        lo += x - z;
        hi = s_;
    }
};

// acc += conj(v) w for one complex entry, v and w FP32
__device__ __forceinline__ void cdot_an(float vr, float vi, float ar, float ai, AnAcc &re, AnAcc &im) {
    re.madd(vr, ar);
    re.madd(vi, ai);
    im.madd(vr, ai);
    im.madd(-vi, ar);
}

// acc -= v c for one complex entry (v FP32, c = (re_hi, re_lo, im_hi, im_lo))
// (the lo halves of c are 2^-24 of the hi halves: their products go straight to lo)
__device__ __forceinline__ void caxpy_an(float vr, float vi, const float4 &c, AnAcc &ar, AnAcc &ai) {
    ar.madd(-vr, c.x); ar.lo = fmaf(-vr, c.y, ar.lo);     // - vr hr
    ar.madd(vi, c.z);  ar.lo = fmaf(vi, c.w, ar.lo);      // + vi hi
    ai.madd(-vr, c.z); ai.lo = fmaf(-vr, c.w, ai.lo);     // - vr hi
    ai.madd(-vi, c.x); ai.lo = fmaf(-vi, c.y, ai.lo);     // - vi hr
}

}  // namespace dst
