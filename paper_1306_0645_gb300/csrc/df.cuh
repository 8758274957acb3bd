// df.cuh -- double-float ("df") arithmetic on the FP32 pipe for the
// FP64-accurate parts of the mixed-precision step.
//
// GB300 issues FP64 at 1/64 of its FP32 rate, so the assembly of the system
// (Sec. 2 limiter, Sec. 3.2 right-hand side), the refinement residual and
// the finalisation sums of the mixed solver are computed with unevaluated
// sums h + l of two floats.  The building blocks are the error-free
// transformations two-sum (Knuth) and two-product (by fused multiply-add),
// and the compensated dot product of Ogita, Rump and Oishi (2005, "Dot2").
// A df number carries 47 or more significant bits.
//
// FP64 operands are split into df with integer instructions only (no FP64
// conversion), relative to a power-of-two scale 2^K that brings a step's
// values into the FP32 exponent range.
// A difference of two FP64 values, where cancellation would expose the
// split's truncation, is formed in FP64 (one subtraction) and split after.
//
// Every FP32 operation here is an explicit _rn intrinsic so that the
// compiler cannot contract a product and a sum into one FMA, which would
// break the error-free transformations.
#pragma once
#include <cuda_runtime.h>

namespace fld {

struct df {
    float h, l;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }

// a + b with a relative error of a few units of 2^-48 in the result, also
// under cancellation (both parts summed error-free).
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.h, b.h);
    const df t = two_sum(a.l, b.l);
    s.l = __fadd_rn(s.l, t.h);
    s = fast_two_sum(s.h, s.l);
    s.l = __fadd_rn(s.l, t.l);
    return fast_two_sum(s.h, s.l);
}

// a - b accurate to a few units of 2^-48 of the difference itself (both
// parts subtracted error-free), also where a and b nearly cancel.
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a * b as an unnormalised pair (p, e) with p = fl(a.h b.h): for summing into
// an accumulator, which adds p error-free and e to its compensation.
__device__ __forceinline__ df df_mul_raw(df a, df b) {
    const df p = two_prod(a.h, b.h);
    return {p.h, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l))};
}

__device__ __forceinline__ df df_mul(df a, df b) {
    df p = two_prod(a.h, b.h);
    p.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
    return fast_two_sum(p.h, p.l);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
    df p = two_prod(a.h, b);
    p.l = __fmaf_rn(a.l, b, p.l);
    return fast_two_sum(p.h, p.l);
}

// a < b, for normalised df numbers
__device__ __forceinline__ bool df_lt(df a, df b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }

// 1 / sqrt(x) for x > 0 in the FP32 normal range: the hardware estimate
// y0 refined by one Newton step taken in df, y = y0 (1 + e/2 + 3 e^2/8)
// with e = 1 - x y0^2 kept as the unevaluated pair (1 - q.h) - q.l (q.h
// lies within a few units of 2^-22 of 1, so 1 - q.h is exact); relative
// error about 2^-47.
__device__ __forceinline__ df df_rsqrt(df x) {
    const float y0 = rsqrtf(x.h);
    const df q = df_mul(x, two_prod(y0, y0));
    const float eh = __fsub_rn(1.0f, q.h), el = -q.l;
    const df p = two_prod(y0, eh);
    const float e = __fadd_rn(eh, el);
    const float cl = __fmaf_rn(0.375f * p.h, e, 0.5f * __fmaf_rn(y0, el, p.l));
    df y = fast_two_sum(y0, 0.5f * p.h);
    y.l = __fadd_rn(y.l, cl);
    return fast_two_sum(y.h, y.l);
}

// Compensated accumulator of sums of df terms and df products (Dot2 in
// FP32): the value is s + c; the error of the result is of order
// 2^-48 sum |terms| (plus 2^-24 |result| if rounded to one float).
struct Acc2 {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float p) {
        const float t = __fadd_rn(s, p);
        const float z = __fsub_rn(t, s);
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z)));
        s = t;
    }
    __device__ __forceinline__ void add(df a) {
        add(a.h);
        c = __fadd_rn(c, a.l);
    }
    __device__ __forceinline__ void sub(df a) {
        add(-a.h);
        c = __fsub_rn(c, a.l);
    }
    // += a * b
    __device__ __forceinline__ void addmul(df a, df b) {
        const df p = two_prod(a.h, b.h);
        add(p.h);
        c = __fadd_rn(c, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l)));
    }
    // -= a * b
    __device__ __forceinline__ void submul(df a, df b) { addmul(df_neg(a), b); }
    __device__ __forceinline__ df value() const { return two_sum(s, c); }
};

// The FP32 number with biased exponent fe (>= 24) and fraction bits m23
// (23 bits), minus its leading bit: m23 * 2^(fe - 150), exact.
__device__ __forceinline__ float frac_value(unsigned sg, int fe, unsigned m23) {
    const unsigned eb = sg | ((unsigned)fe << 23);
    return __fsub_rn(__uint_as_float(eb | m23), __uint_as_float(eb));
}

// v * 2^-K as df, v finite: the high part holds the leading 24 significant
// bits (truncated), the low part the next 23, the rest is dropped (relative
// error below 2^-46).  Values below 2^(K-102) keep only their high part,
// values below 2^(K-126) flush to 0; above 2^(K+128) the result is
// infinite.  Integer instructions and one FP32 subtraction.
__device__ __forceinline__ df split64(double v, int K) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
    const int fe = (int)((hi >> 20) & 0x7FFu) - 896 - K;
    const unsigned sg = hi & 0x80000000u;
    const unsigned m23 = __funnelshift_l(lo, hi, 3) & 0x7FFFFFu;
    df r;
    if (fe >= 1) {
        r.h = fe <= 254 ? __uint_as_float(sg | ((unsigned)fe << 23) | m23) : __uint_as_float(sg | 0x7F800000u);
        r.l = fe >= 24 && fe <= 254 ? frac_value(sg, fe - 23, (lo >> 6) & 0x7FFFFFu) : 0.0f;
    } else {
        r.h = 0.0f;
        r.l = 0.0f;
    }
    return r;
}

// v * 2^-K rounded to the nearest float (ties away from zero), integer
// instructions only; below 2^(K-126) it flushes to 0.
__device__ __forceinline__ float round64(double v, int K) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
    const int fe = (int)((hi >> 20) & 0x7FFu) - 896 - K;
    const unsigned sg = hi & 0x80000000u;
    if (fe < 1) return 0.0f;
    if (fe > 254) return __uint_as_float(sg | 0x7F800000u);
    // a carry out of the fraction moves the exponent up, as rounding should
    const unsigned mag = (((unsigned)fe << 23) | (__funnelshift_l(lo, hi, 3) & 0x7FFFFFu)) + ((lo >> 28) & 1u);
    return __uint_as_float(sg | mag);
}

// f * 2^K as a double, exactly; FP32 subnormals flush to 0.
__device__ __forceinline__ double f2d(float f, int K) {
    const unsigned b = __float_as_uint(f);
    const int fe = (int)((b >> 23) & 0xFFu);
    if (fe == 0) return 0.0;
    const int de = fe + 896 + K;
    if (de <= 0) return 0.0;
    if (de > 2046) return __hiloint2double((int)((b & 0x80000000u) | 0x7FF00000u), 0);
    const unsigned hi = (b & 0x80000000u) | ((unsigned)de << 20) | ((b >> 3) & 0xFFFFFu);
    return __hiloint2double((int)hi, (int)(b << 29));
}

// (h + l) * 2^K as a double: two exact conversions and one FP64 addition.
__device__ __forceinline__ double df2d(df a, int K) { return f2d(a.h, K) + f2d(a.l, K); }

// Unbiased binary exponent of a finite double v > 0 plus one (2^(e-1) <=
// v < 2^e), from its bits; 0 gives -1100.
__device__ __host__ __forceinline__ int exp_above(double v) {
#ifdef __CUDA_ARCH__
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
#else
    unsigned long long u;
    __builtin_memcpy(&u, &v, sizeof u);
#endif
    const int e = (int)((u >> 52) & 0x7FFu);
    return e == 0 ? -1100 : e - 1022;
}

}  // namespace fld
