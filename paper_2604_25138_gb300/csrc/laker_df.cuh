// Double-float ("df") arithmetic on the float32 pipes: a value is the unevaluated
// sum hi + lo of two floats (~48 significant bits).  GB300 executes float32 at
// ~74x its float64 rate, so float64-accurate work on the hot path is done here.
//
// Building blocks are the classical error-free transformations:
//   two_sum   (Knuth, TAOCP vol. 2):  a + b = s + e exactly;
//   two_prod  (Dekker 1971, with a fused multiply-add):  a * b = p + e exactly;
// dot products follow Ogita, Rump and Oishi, "Accurate sum and dot product"
// (SIAM J. Sci. Comput. 2005, algorithm Dot2), extended with the cross terms of
// double-float inputs; exp follows Tang's table-driven method (ACM TOMS 1989):
// x = (64 k + j) ln2/64 + r, |r| <= ln2/128, e^x = 2^k 2^(j/64) e^r with a
// Taylor polynomial for e^r and a double-float table of 2^(j/64).
#pragma once

#include <cuda_runtime.h>

#include <cmath>

namespace lk {

struct df2 {
    float hi, lo;
};

__device__ __forceinline__ df2 df_from(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to(df2 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {   // |a| >= |b|
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
__device__ __forceinline__ df2 df_add(df2 a, df2 b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    df2 r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ df2 df_mul(df2 a, df2 b) {
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    df2 r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ df2 df_mul_f(df2 a, float b) {
    float p, e;
    two_prod(a.hi, b, p, e);
    e = __fmaf_rn(a.lo, b, e);
    df2 r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

// Dot2 accumulator: running (p, s) with the final value p + s.
struct Dot2 {
    float p = 0.f, s = 0.f;
    __device__ __forceinline__ void add(df2 a, df2 b) {
        float h, r, q;
        two_prod(a.hi, b.hi, h, r);
        float np;
        two_sum(p, h, np, q);
        p = np;
        s = __fadd_rn(s, __fadd_rn(q, r));
        s = __fmaf_rn(a.hi, b.lo, s);
        s = __fmaf_rn(a.lo, b.hi, s);
    }
    __device__ __forceinline__ df2 value() const {
        df2 r;
        fast_two_sum(p, s, r.hi, r.lo);
        return r;
    }
};

// Dot product with the compensation itself accumulated error-free (the K = 3
// case of Ogita, Rump and Oishi's DotK): value = p + s + c.  Needed when the
// terms are orders of magnitude larger than the result -- e.g. (lambda I + G)
// alpha near convergence, |G_ij alpha_j| ~ 1e4 against an O(1) sum -- where
// Dot2's float32 compensation term would leave ~1e-7 absolute noise.
struct Dot3 {
    float p = 0.f, s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(df2 a, df2 b) {
        float h, r, q, np, ns, e;
        two_prod(a.hi, b.hi, h, r);
        two_sum(p, h, np, q);
        p = np;
        float t = __fadd_rn(q, r);
        t = __fmaf_rn(a.hi, b.lo, t);
        t = __fmaf_rn(a.lo, b.hi, t);
        two_sum(s, t, ns, e);
        s = ns;
        c = __fadd_rn(c, e);
    }
    __device__ __forceinline__ df2 value() const {
        df2 r;
        two_sum(p, s, r.hi, r.lo);
        r.lo = __fadd_rn(r.lo, c);
        df2 o;
        fast_two_sum(r.hi, r.lo, o.hi, o.lo);
        return o;
    }
};

// 2^(j/64), j = 0..63, as double-float pairs (hi at 2j, lo at 2j + 1), built
// by each thread block in its own shared memory from the float64 exp2 of the
// math library: no host upload, so no ordering against other streams and no
// set-up call.  The block must __syncthreads() before the first df_exp.
__device__ __forceinline__ void df_exp_table_init(float* tab) {
    for (int j = threadIdx.x; j < 64; j += blockDim.x) {
        const double v = exp2((double)j / 64.0);
        const float h = (float)v;
        tab[2 * j] = h;
        tab[2 * j + 1] = (float)(v - (double)h);
    }
}

// e^x for a double-float x with |x| < 80; relative error ~1e-14.
__device__ __forceinline__ df2 df_exp(df2 x, const float* tab) {
    // ln2/64 = HI + MID + LO (residual < 2e-22); HI has 12 significant bits so
    // k * HI is exact for |k| < 2^12.  Values computed to 60 digits with sympy.
    constexpr float INV_LN2_64 = 92.33248138427734f;       // 64 / ln 2
    constexpr float LN2_64_HI = 0.010829925537109375f;
    constexpr float LN2_64_MID = 4.991591140424134e-07f;
    constexpr float LN2_64_LO = 2.572804640231345e-14f;
    const float kf = rintf(x.hi * INV_LN2_64);
    const int k = (int)kf;
    // r = x - k ln2/64 in double-float
    df2 r = df_add(x, df2{-kf * LN2_64_HI, 0.f});
    r = df_add(r, df_mul_f(df2{LN2_64_MID, LN2_64_LO}, -kf));
    // e^r = 1 + r + r^2/2 + r^3 (1/6 + r/24 + r^2/120) ; the cubic tail in float
    const float t = r.hi;
    const float tail = t * t * t * __fmaf_rn(t, __fmaf_rn(t, 1.f / 120.f, 1.f / 24.f), 1.f / 6.f);
    df2 r2 = df_mul(r, r);
    r2.hi *= 0.5f;
    r2.lo *= 0.5f;
    df2 e = df_add(r, r2);
    e = df_add(e, df2{tail, 0.f});
    e = df_add(df2{1.f, 0.f}, e);
    const int j = k & 63;
    const int m = (k - j) / 64;
    e = df_mul(e, df2{tab[2 * j], tab[2 * j + 1]});
    return {ldexpf(e.hi, m), ldexpf(e.lo, m)};
}

}  // namespace lk
