// limiter.cuh -- the flux limiter of Sec. 2 in FP64 and the exact FP32
// screen that settles capped faces, shared by the FP64 assembly
// (k_assemble.cu) and the mixed-precision assembly (k_mixed.cu).
//
// Flux limiter (Sec. 2): D = min{ c (9 kappa_f^2 + R^2)^(-1/2), D_max },
// R = max{ |E_2 - E_1| / (h E_f), R_min }, E_f arithmetic and kappa_f
// harmonic face means; Levermore-Pomraning alternative (Sec. 1 citation)
// with lambda(x) = (coth x - 1/x)/x, x = R/kappa_f.
#pragma once
#include "kernels.h"

namespace fld {

// Square-root-sum limiter without divisions in the common case.  With
// s = h E_f, a = max(|E_2 - E_1|, R_min s) (so R = a / s),
// P = 2 k1 k2 and K = k1 + k2 (so kappa_f = P / K):
//     D = c s K / sqrt(9 P^2 s^2 + a^2 K^2),
// and D >= D_max exactly when (c s K)^2 >= D_max^2 (9 P^2 s^2 + a^2 K^2),
// which settles the cap without a square root.  Degenerate or out-of-range
// arguments take the textbook form.
__device__ __forceinline__ double limiter_paper(double E1, double E2, double k1, double k2,
                                                double h, const PhysDev& p) {
    const double esum = E1 + E2;
    const bool thin = !(k1 > 0.0 && k2 > 0.0);
    if (esum > 0.0) {
        const double s = 0.5 * h * esum;
        double a = fabs(E2 - E1);
        const double amin = p.Rmin * s;
        if (a < amin) a = amin;
        const double P = thin ? 0.0 : 2.0 * k1 * k2;
        const double K = thin ? 1.0 : k1 + k2;
        const double Ps = P * s, aK = a * K;
        const double q = fma(9.0 * Ps, Ps, aK * aK);
        const double num = p.c * s * K;
        const double num2 = num * num, cap2 = p.Dmax * p.Dmax * q;
        if (q > 1e-290 && q < 1e290 && num2 > 1e-290 && num2 < 1e290 && cap2 < 1e290 &&
            cap2 > 1e-290) {
            if (num2 >= cap2) return p.Dmax;
            return num * rsqrt(q);
        }
        double R = a / s;
        double kf = thin ? 0.0 : P / K;
        double D = p.c / sqrt(9.0 * kf * kf + R * R);
        return D < p.Dmax ? D : p.Dmax;
    }
    // both face energies zero: R = R_min
    double kf = thin ? 0.0 : 2.0 * k1 * k2 / (k1 + k2);
    double D = p.c / sqrt(9.0 * kf * kf + p.Rmin * p.Rmin);
    return D < p.Dmax ? D : p.Dmax;
}

__device__ __forceinline__ double lp_lambda(double x) {
    if (x < 1e-2) {
        const double x2 = x * x;
        return 1.0 / 3.0 - x2 / 45.0 + 2.0 * x2 * x2 / 945.0;
    }
    return (1.0 / tanh(x) - 1.0 / x) / x;
}

__device__ __forceinline__ double limiter_lp(double E1, double E2, double k1, double k2, double h,
                                             const PhysDev& p) {
    const double Ef = 0.5 * (E1 + E2);
    const double kf = (k1 > 0.0 && k2 > 0.0) ? 2.0 * k1 * k2 / (k1 + k2) : 0.0;
    double R;
    if (Ef > 0.0) {
        R = fabs(E2 - E1) / (h * Ef);
        if (R < p.Rmin) R = p.Rmin;
    } else {
        R = p.Rmin;   // E >= 0 is validated, so E_f = 0 means E_1 = E_2 = 0
    }
    double D;
    if (kf == 0.0) {
        D = p.c / R;
    } else {
        const double x = R / kf;
        D = (x > 1e8) ? p.c / R : p.c * lp_lambda(x) / kf;
    }
    return D < p.Dmax ? D : p.Dmax;
}

__device__ __forceinline__ double face_D(double E1, double E2, double k1, double k2, double h,
                                         const PhysDev& p) {
    return p.limiter == 1 ? limiter_lp(E1, E2, k1, k2, h, p) : limiter_paper(E1, E2, k1, k2, h, p);
}

// Finite and >= 0 (or -0), tested on the bits with integer instructions
// (on the two 32-bit words: tests on the 64-bit pattern can be compiled as
// FP64 comparisons, instructions of the FP64 pipe).
__device__ __forceinline__ bool valid_bits(double v) {
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    return (hi >> 20) < 0x7FFu || (hi == 0x80000000u && lo == 0u);
}

// FP32 value of a finite non-negative double by exponent rebias and
// mantissa truncation, with integer instructions only (no FP64 pipe);
// ok becomes false outside the FP32 normal range.
__device__ __forceinline__ float f32_trunc(double x, bool& ok) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7FFu);
    if (((hi << 1) | lo) == 0u) return 0.0f;
    ok = ok && e >= 1023 - 126 && e <= 1023 + 127;
    const unsigned int fb = (hi & 0x80000000u) | ((unsigned int)(e - 896) << 23) | (__funnelshift_l(lo, hi, 3) & 0x7FFFFFu);
    return __int_as_float((int)fb);
}

// The two face energies as FP32 numbers sharing one power-of-two scale (the
// larger one's FP64 exponent maps to 2^0), by integer instructions only.
// The screen needs only their ratio, so E far below the FP32 range (a
// radiation field decaying over many steps) is screened all the same; a
// value 2^-126 or more below the other flushes to 0, which leaves the
// ratio |E2 - E1| / (E1 + E2) within FP32 rounding.  ok is false for
// negative or non-finite input.
__device__ __forceinline__ void pair32(double a, double b, float& fa, float& fb, bool& ok) {
    const unsigned long long ba = (unsigned long long)__double_as_longlong(a);
    const unsigned long long bb = (unsigned long long)__double_as_longlong(b);
    ok = ok && (ba >> 52) < 0x7FFull && (bb >> 52) < 0x7FFull;   // >= +0 and finite
    const int ea = (int)(ba >> 52), eb = (int)(bb >> 52);
    const int emax = ea > eb ? ea : eb;
    auto conv = [&](unsigned long long bits, int e) {
        const int ne = e - emax + 127;
        if (e == 0 || ne <= 0) return 0.0f;
        return __int_as_float((int)(((unsigned int)ne << 23) | (unsigned int)((bits >> 29) & 0x7FFFFFu)));
    };
    fa = conv(ba, ea);
    fb = conv(bb, eb);
}

// FP32 screen of the square-root-sum limiter: true only if the face is
// certainly capped, D = D_max, i.e. 9 (kappa_f L)^2 + (R L)^2 lies below
// the threshold with a margin far above the FP32 error of the estimate.
__device__ __forceinline__ bool capped32(float e1, float e2, float kL1, float kL2, float twoL_h,
                                         float thr) {
    const float esum = e1 + e2;
    if (!(esum > 0.0f)) return false;
    const float kf = (kL1 > 0.0f && kL2 > 0.0f) ? __fdividef(2.0f * kL1 * kL2, kL1 + kL2) : 0.0f;
    const float RL = __fdividef(fabsf(e2 - e1) * twoL_h, esum);
    const float X = 9.0f * kf * kf + RL * RL;
    return X < thr;
}

}  // namespace fld
