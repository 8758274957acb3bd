// k_assemble.cu -- per-cell opacity and per-face flux-limited diffusion
// coefficients of the backward-Euler correction system (FP64).
//
// Flux limiter (Sec. 2): D = min{ c (9 kappa_f^2 + R^2)^(-1/2), D_max },
// R = max{ |E_2 - E_1| / (h E_f), R_min }, E_f arithmetic and kappa_f
// harmonic face means; Levermore-Pomraning alternative (Sec. 1 citation)
// with lambda(x) = (coth x - 1/x)/x, x = R/kappa_f.
// System (Sec. 3.2, residual-correction form of backward Euler with the
// limiter lagged at E^n): w_f = dt D_f / h^2, m = 1 + dt (c kappa + adot/a),
// b = dt eta - dt (c kappa + adot/a) E + sum_f w_f (E_nbr - E).
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

__device__ __forceinline__ bool bad_value(double v) { return !(v >= 0.0) || !isfinite(v); }

__global__ void __launch_bounds__(256) k_assemble_faces(Dims d, PhysDev p, const double* __restrict__ E,
                                                       const double* __restrict__ nHI,
                                                       const double* __restrict__ eta, Op<double> op,
                                                       Op<float> op32, double* sc) {
    const long long sx = 1, sy = d.nx, sz = (long long)d.nx * d.ny;
    bool bad = false;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n;
         c += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(c, d, i, j, k);
        const double Ec = E[c], nc = nHI[c];
        bad |= bad_value(Ec) || bad_value(nc) || bad_value(eta[c]);
        const double kc = nc * p.sigma;
        const double m = 1.0 + p.dt * (p.c * kc + p.adot);
        double w[3];
        const int ijk[3] = {i, j, k};
        const int nn[3] = {d.nx, d.ny, d.nz};
        const int per[3] = {d.px, d.py, d.pz};
        const long long st[3] = {sx, sy, sz};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            long long lo;
            if (ijk[a] > 0) lo = c - st[a];
            else if (per[a]) lo = c + (long long)(nn[a] - 1) * st[a];
            else { w[a] = 0.0; continue; }
            const double D = face_D(E[lo], Ec, nHI[lo] * p.sigma, kc, p.h[a], p);
            w[a] = p.dt_h2[a] * D;
        }
        op.m[c] = m;
        op.wx[c] = w[0];
        op.wy[c] = w[1];
        op.wz[c] = w[2];
        if (op32.m) {
            op32.m[c] = (float)m;
            op32.wx[c] = (float)w[0];
            op32.wy[c] = (float)w[1];
            op32.wz[c] = (float)w[2];
        }
    }
    if (bad) sc[S_BAD] = 1.0;
}

__global__ void __launch_bounds__(RED_THREADS) k_assemble_rhs(Dims d, PhysDev p, const double* __restrict__ E,
                                                             const double* __restrict__ nHI,
                                                             const double* __restrict__ eta, Op<double> op,
                                                             Op<float> op32, double* __restrict__ b,
                                                             RedArgs ra) {
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    double acc[1] = {0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n;
         c += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(c, d, i, j, k);
        const double Ec = E[c];
        double flux = 0.0, wsum = 0.0;
        // x faces
        {
            const double wl = op.wx[c];
            if (i > 0) flux += wl * (E[c - 1] - Ec);
            else if (d.px) flux += wl * (E[c + d.nx - 1] - Ec);
            const long long up = (i < d.nx - 1) ? c + 1 : (d.px ? c - (d.nx - 1) : -1);
            const double wu = up >= 0 ? op.wx[up] : 0.0;
            if (up >= 0) flux += wu * (E[up] - Ec);
            wsum += wl + wu;
        }
        {
            const double wl = op.wy[c];
            if (j > 0) flux += wl * (E[c - sy] - Ec);
            else if (d.py) flux += wl * (E[c + (long long)(d.ny - 1) * sy] - Ec);
            const long long up = (j < d.ny - 1) ? c + sy : (d.py ? c - (long long)(d.ny - 1) * sy : -1);
            const double wu = up >= 0 ? op.wy[up] : 0.0;
            if (up >= 0) flux += wu * (E[up] - Ec);
            wsum += wl + wu;
        }
        {
            const double wl = op.wz[c];
            if (k > 0) flux += wl * (E[c - sz] - Ec);
            else if (d.pz) flux += wl * (E[c + (long long)(d.nz - 1) * sz] - Ec);
            const long long up = (k < d.nz - 1) ? c + sz : (d.pz ? c - (long long)(d.nz - 1) * sz : -1);
            const double wu = up >= 0 ? op.wz[up] : 0.0;
            if (up >= 0) flux += wu * (E[up] - Ec);
            wsum += wl + wu;
        }
        const double sink = p.dt * (p.c * nHI[c] * p.sigma + p.adot);
        const double bc = p.dt * eta[c] - sink * Ec + flux;
        b[c] = bc;
        acc[0] += bc * bc;
        const double diag = op.m[c] + wsum;
        if (op.invd) op.invd[c] = 1.0 / diag;
        if (op32.invd) op32.invd[c] = 1.0f / (float)diag;
    }
    const bool ismax[1] = {false};
    grid_reduce<1>(acc, ismax, ra);
}

void launch_assemble_faces(const Dims& d, const PhysDev& p, const double* E, const double* nHI,
                           const double* eta, Op<double> op, Op<float> op32, double* sc,
                           cudaStream_t s) {
    k_assemble_faces<<<grid_blocks(d.n, 256), 256, 0, s>>>(d, p, E, nHI, eta, op, op32, sc);
}

void launch_assemble_rhs(const Dims& d, const PhysDev& p, const double* E, const double* nHI,
                         const double* eta, Op<double> op, Op<float> op32, double* b,
                         const RedArgs& ra, cudaStream_t s) {
    k_assemble_rhs<<<red_blocks(d.n), RED_THREADS, 0, s>>>(d, p, E, nHI, eta, op, op32, b, ra);
}

__global__ void k_opacity_update(long long n, const double* __restrict__ E, const double* __restrict__ nH,
                                 const double* nHI, double* out, double dt, double c, double sigma,
                                 double hnu, double alpha_B) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double h = nH[i];
        const double x = h > 0.0 ? nHI[i] / h : 0.0;
        const double gam = c * sigma * E[i] / hnu;
        const double ion = 1.0 - x;
        double xn = (x + dt * alpha_B * h * ion * ion) / (1.0 + dt * gam);
        xn = fmin(fmax(xn, 1e-12), 1.0);
        out[i] = xn * h;
    }
}

void launch_opacity_update(long long n, const double* E, const double* nH, const double* nHI,
                           double* out, double dt, double c, double sigma, double hnu,
                           double alpha_B, cudaStream_t s) {
    k_opacity_update<<<grid_blocks(n, 256), 256, 0, s>>>(n, E, nH, nHI, out, dt, c, sigma, hnu,
                                                         alpha_B);
}

}  // namespace fld
