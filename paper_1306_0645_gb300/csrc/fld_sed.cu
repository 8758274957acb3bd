// fld_sed.cu -- grey and multigroup spectral integrals (Sec. 2, Eqs.
// "opacity", "photoionization", "photoheating") and the per-cell fields
// built from them: group opacities and emissivities, photoionisation and
// photoheating rates.
//
// For frequency groups [nu_g, nu_{g+1}] (a grey field is the single group
// [nu_1, nu_max]) and species i = HI, HeI, HeII with thresholds nu_i:
//   K_gi = int sigma_i chi dnu              / N_g
//   P_gi = int sigma_i chi / nu dnu         / N_g
//   H_gi = int sigma_i chi (1 - nu_i/nu) dnu / N_g
//   F_g  = N_g / N,   N_g = int_g chi dnu,  N = int_{nu_1}^{nu_max} chi dnu,
// the species integrals running from max(nu_g, nu_i).  Then
//   kappa_g = sum_i n_i K_gi,  eta_g = F_g eta,
//   Gamma_i = sum_g (c E_g / h) P_gi,  G = sum_g (c E_g / rho_b) sum_i n_i H_gi.
// The normalisation N_g starts at the group's lower edge for all three
// integrals: photons below nu_i belong to E but species i cannot absorb
// them.
//
// Quadrature: composite Simpson's rule in u = ln nu, 2^14 intervals per
// integral, one thread block per integral, summed in a fixed order.
#include <cmath>
#include <string>

#include "fld.h"
#include "kernels.h"

namespace {

using namespace fld;

constexpr double H_PLANCK = 6.62607015e-27;   // erg s
constexpr double K_BOLTZ = 1.380649e-16;      // erg / K
constexpr int SIMPSON_N = 1 << 14;            // intervals (even)
constexpr int NCOEF = FLD_SED_NCOEF;

struct SedDev {
    int kind;
    double nu_mono, hkT, alpha;
    double nut[3], s0[3], beta[3], sx[3];
};

struct Edges {
    int groups;
    double e[FLD_MAX_GROUPS + 1];
};

__device__ double xsec(const SedDev& S, int sp, double nu) {
    if (nu < S.nut[sp]) return 0.0;
    const double r = nu / S.nut[sp];
    return S.s0[sp] * (S.beta[sp] * pow(r, -S.sx[sp]) + (1.0 - S.beta[sp]) * pow(r, -S.sx[sp] - 1.0));
}

__device__ double chi(const SedDev& S, double nu) {
    if (S.kind == FLD_SED_BLACKBODY) {
        const double x = S.hkT * nu;
        if (x > 700.0) return 0.0;
        return nu * nu * nu / expm1(x);
    }
    return pow(nu, -S.alpha);
}

// Integrand q of integral job: 0 chi; 1 sigma chi; 2 sigma chi / nu;
// 3 sigma chi (1 - nu_i / nu); times nu for the measure du = dnu / nu.
__device__ double integrand(const SedDev& S, int q, int sp, double u) {
    const double nu = exp(u);
    const double c = chi(S, nu) * nu;
    if (q == 0) return c;
    // a species' range starts at its threshold; exp(log(nu_i)) may round
    // just below it, where the cross section would read 0
    const double sg = xsec(S, sp, fmax(nu, S.nut[sp]));
    if (q == 1) return sg * c;
    if (q == 2) return sg * c / nu;
    return sg * c * (1.0 - S.nut[sp] / nu);
}

// Block b < 10 G: group g = b / 10, job k = b % 10 (0: N_g; 1..9: species
// (k-1) % 3, integrand 1 + (k-1) / 3); block 10 G: N.
__global__ void __launch_bounds__(256) k_sed_quad(SedDev S, Edges E, double* __restrict__ raw) {
    const int b = blockIdx.x;
    const int G = E.groups;
    double lo, hi;
    int q = 0, sp = 0;
    if (b < 10 * G) {
        const int g = b / 10, k = b % 10;
        lo = E.e[g];
        hi = E.e[g + 1];
        if (k > 0) {
            sp = (k - 1) % 3;
            q = 1 + (k - 1) / 3;
            lo = fmax(lo, S.nut[sp]);
        }
    } else {
        lo = E.e[0];
        hi = E.e[G];
    }
    double acc = 0.0;
    if (hi > lo) {
        const double ul = log(lo), uh = log(hi);
        const double hu = (uh - ul) / SIMPSON_N;
        for (int j = threadIdx.x; j <= SIMPSON_N; j += blockDim.x) {
            const double w = (j == 0 || j == SIMPSON_N) ? 1.0 : ((j & 1) ? 4.0 : 2.0);
            acc = fma(w, integrand(S, q, sp, ul + hu * j), acc);
        }
        acc *= hu / 3.0;
    }
    // fixed-order block reduction
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) raw[b] = v;
    }
}

// Coefficients from the raw integrals (or, for a line, from the cross
// sections at the line).  Row g: K_0..2, P_0..2, H_0..2, F.
__global__ void k_sed_finish(SedDev S, Edges E, const double* __restrict__ raw, double* __restrict__ coef) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= E.groups) return;
    double* row = coef + (long long)g * NCOEF;
    if (S.kind == FLD_SED_MONO) {
        const double nu0 = S.nu_mono;
        const bool in = E.e[g] <= nu0 && nu0 < E.e[g + 1];
        for (int i = 0; i < 3; i++) {
            const double sg = in ? xsec(S, i, nu0) : 0.0;
            row[i] = sg;
            row[3 + i] = sg / nu0;
            row[6 + i] = sg > 0.0 ? sg * (1.0 - S.nut[i] / nu0) : 0.0;
        }
        row[9] = in ? 1.0 : 0.0;
        return;
    }
    const double Ng = raw[10 * g], N = raw[10 * E.groups];
    for (int k = 1; k < 10; k++) {
        const int sp = (k - 1) % 3, q = (k - 1) / 3;   // q: 0 K, 1 P, 2 H
        row[3 * q + sp] = Ng > 0.0 ? raw[10 * g + k] / Ng : 0.0;
    }
    row[9] = N > 0.0 ? Ng / N : 0.0;
}

struct GroupArgs {
    int groups;
    double K[FLD_MAX_GROUPS][3];
    double F[FLD_MAX_GROUPS];
    double* kap[FLD_MAX_GROUPS];
    double* eta[FLD_MAX_GROUPS];
};

// kappa_g = sum_i n_i K_gi and eta_g = F_g eta, all groups in one pass
// over the densities.
__global__ void __launch_bounds__(256) k_group_fields(long long n, const double* __restrict__ nHI,
                                                    const double* __restrict__ nHeI,
                                                    const double* __restrict__ nHeII,
                                                    const double* __restrict__ eta, GroupArgs A) {
    GRID_LOOP(c, n) {
        const double a = nHI[c];
        const double b = nHeI ? nHeI[c] : 0.0;
        const double d = nHeII ? nHeII[c] : 0.0;
        const double e = eta ? eta[c] : 0.0;
        for (int g = 0; g < A.groups; g++) {
            A.kap[g][c] = fma(A.K[g][2], d, fma(A.K[g][1], b, A.K[g][0] * a));
            if (A.eta[g]) A.eta[g][c] = A.F[g] * e;
        }
    }
}

struct RateArgs {
    int groups;
    double P[FLD_MAX_GROUPS][3];   // times c / h
    double H[FLD_MAX_GROUPS][3];   // times c
    const double* E[FLD_MAX_GROUPS];
};

// Gamma_i = sum_g (c / h) P_gi E_g, G = (1 / rho_b) sum_g c E_g sum_i n_i H_gi.
__global__ void __launch_bounds__(256) k_photo_rates(long long n, RateArgs A, const double* __restrict__ nHI,
                                                    const double* __restrict__ nHeI,
                                                    const double* __restrict__ nHeII,
                                                    const double* __restrict__ rho, double* gHI, double* gHeI,
                                                    double* gHeII, double* heat) {
    GRID_LOOP(c, n) {
        const double dn[3] = {nHI ? nHI[c] : 0.0, nHeI ? nHeI[c] : 0.0, nHeII ? nHeII[c] : 0.0};
        double gam[3] = {0.0, 0.0, 0.0}, h = 0.0;
        for (int g = 0; g < A.groups; g++) {
            const double Eg = A.E[g][c];
#pragma unroll
            for (int i = 0; i < 3; i++) gam[i] = fma(A.P[g][i], Eg, gam[i]);
            h = fma(Eg, fma(A.H[g][2], dn[2], fma(A.H[g][1], dn[1], A.H[g][0] * dn[0])), h);
        }
        if (gHI) gHI[c] = gam[0];
        if (gHeI) gHeI[c] = gam[1];
        if (gHeII) gHeII[c] = gam[2];
        if (heat && rho) heat[c] = h / rho[c];
    }
}

fld_status fail(fld_status st, const std::string& msg) {
    fld::record_error(msg.c_str());
    return st;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

fld_status check_sed(const fld_sed* sed) {
    if (!sed) return fail(FLD_EINVAL, "null SED");
    if (sed->kind != FLD_SED_MONO && sed->kind != FLD_SED_BLACKBODY && sed->kind != FLD_SED_POWERLAW)
        return fail(FLD_EINVAL, "unknown SED kind " + std::to_string(sed->kind));
    if (sed->kind == FLD_SED_MONO && !finite_pos(sed->nu_mono)) return fail(FLD_EINVAL, "nu_mono must be > 0");
    if (sed->kind == FLD_SED_BLACKBODY && !finite_pos(sed->T)) return fail(FLD_EINVAL, "T must be > 0");
    if (sed->kind == FLD_SED_POWERLAW && !std::isfinite(sed->alpha)) return fail(FLD_EINVAL, "alpha must be finite");
    for (int i = 0; i < 3; i++) {
        const fld_xsec& x = sed->species[i];
        if (!finite_pos(x.nu_threshold) || !(std::isfinite(x.sigma0) && x.sigma0 >= 0.0) ||
            !std::isfinite(x.beta) || !std::isfinite(x.s))
            return fail(FLD_EINVAL, "invalid cross-section fit of species " + std::to_string(i));
    }
    return FLD_OK;
}

SedDev to_dev(const fld_sed* sed) {
    SedDev S;
    S.kind = sed->kind;
    S.nu_mono = sed->nu_mono;
    S.hkT = sed->kind == FLD_SED_BLACKBODY ? H_PLANCK / (K_BOLTZ * sed->T) : 0.0;
    S.alpha = sed->alpha;
    for (int i = 0; i < 3; i++) {
        S.nut[i] = sed->species[i].nu_threshold;
        S.s0[i] = sed->species[i].sigma0;
        S.beta[i] = sed->species[i].beta;
        S.sx[i] = sed->species[i].s;
    }
    return S;
}

fld_status check_groups(int groups, const double* coef) {
    if (groups < 1 || groups > FLD_MAX_GROUPS)
        return fail(FLD_EINVAL, "groups must lie in [1, " + std::to_string(FLD_MAX_GROUPS) + "]");
    if (!coef) return fail(FLD_EINVAL, "null coefficient table");
    for (int k = 0; k < groups * NCOEF; k++)
        if (!std::isfinite(coef[k])) return fail(FLD_EINVAL, "non-finite coefficient");
    return FLD_OK;
}

int blocks_for(long long n) {
    long long b = (n + 255) / 256;
    const long long cap = 152LL * 16;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

extern "C" {

fld_status fld_sed_default(fld_sed* sed) {
    if (!sed) return fail(FLD_EINVAL, "null SED");
    const double ev = 1.602176634e-12;
    sed->kind = FLD_SED_BLACKBODY;
    sed->T = 1e5;
    sed->alpha = 1.5;
    sed->nu_mono = 13.6 * ev / H_PLANCK;
    const double thr[3] = {13.6, 24.6, 54.4};
    const double s0[3] = {6.30e-18, 7.83e-18, 1.58e-18};
    const double beta[3] = {1.34, 1.66, 1.34};
    const double sx[3] = {2.99, 2.05, 2.99};
    for (int i = 0; i < 3; i++) {
        sed->species[i].nu_threshold = thr[i] * ev / H_PLANCK;
        sed->species[i].sigma0 = s0[i];
        sed->species[i].beta = beta[i];
        sed->species[i].s = sx[i];
    }
    return FLD_OK;
}

fld_status fld_sed_integrals(const fld_sed* sed, const double* edges, int groups, double* coef,
                             void* cuda_stream) {
    fld_status st = check_sed(sed);
    if (st) return st;
    if (groups < 1 || groups > FLD_MAX_GROUPS)
        return fail(FLD_EINVAL, "groups must lie in [1, " + std::to_string(FLD_MAX_GROUPS) + "]");
    if (!edges || !coef) return fail(FLD_EINVAL, "null edges or coefficient table");
    Edges E;
    E.groups = groups;
    for (int g = 0; g <= groups; g++) {
        if (!finite_pos(edges[g])) return fail(FLD_EINVAL, "group edges must be finite and > 0");
        if (g > 0 && !(edges[g] > edges[g - 1])) return fail(FLD_EINVAL, "group edges must increase");
        E.e[g] = edges[g];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double* d = nullptr;
    const int jobs = 10 * groups + 1;
    cudaError_t e = cudaMallocAsync(&d, (size_t)(jobs + groups * NCOEF) * sizeof(double), s);
    if (e != cudaSuccess) return fail(FLD_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    const SedDev S = to_dev(sed);
    if (sed->kind != FLD_SED_MONO) k_sed_quad<<<jobs, 256, 0, s>>>(S, E, d);
    k_sed_finish<<<1, 32, 0, s>>>(S, E, d, d + jobs);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(coef, d + jobs, (size_t)groups * NCOEF * sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(FLD_ECUDA, std::string("fld_sed_integrals: ") + cudaGetErrorString(e));
    return FLD_OK;
}

fld_status fld_group_fields(size_t n, int groups, const double* coef, const double* n_HI, const double* n_HeI,
                            const double* n_HeII, const double* eta, double* const* kappa, double* const* eta_out,
                            void* cuda_stream) {
    fld_status st = check_groups(groups, coef);
    if (st) return st;
    if (!n_HI || !kappa) return fail(FLD_EINVAL, "null n_HI or kappa list");
    GroupArgs A;
    A.groups = groups;
    for (int g = 0; g < groups; g++) {
        for (int i = 0; i < 3; i++) A.K[g][i] = coef[g * NCOEF + i];
        A.F[g] = coef[g * NCOEF + 9];
        if (!kappa[g]) return fail(FLD_EINVAL, "null kappa output of group " + std::to_string(g));
        A.kap[g] = kappa[g];
        A.eta[g] = eta_out ? eta_out[g] : nullptr;
        if (A.eta[g] && !eta) return fail(FLD_EINVAL, "group emissivities need eta");
    }
    if (n == 0) return FLD_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    k_group_fields<<<blocks_for((long long)n), 256, 0, s>>>((long long)n, n_HI, n_HeI, n_HeII, eta, A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FLD_ECUDA, std::string("fld_group_fields: ") + cudaGetErrorString(e));
    return FLD_OK;
}

fld_status fld_photo_rates(size_t n, int groups, const double* coef, const double* const* E, const double* n_HI,
                           const double* n_HeI, const double* n_HeII, const double* rho_b, double c,
                           double* gamma_HI, double* gamma_HeI, double* gamma_HeII, double* heating,
                           void* cuda_stream) {
    fld_status st = check_groups(groups, coef);
    if (st) return st;
    if (!E) return fail(FLD_EINVAL, "null E list");
    if (!finite_pos(c)) return fail(FLD_EINVAL, "c must be finite and > 0");
    if (heating && !rho_b) return fail(FLD_EINVAL, "the heating rate needs rho_b");
    RateArgs A;
    A.groups = groups;
    for (int g = 0; g < groups; g++) {
        if (!E[g]) return fail(FLD_EINVAL, "null E of group " + std::to_string(g));
        A.E[g] = E[g];
        for (int i = 0; i < 3; i++) {
            A.P[g][i] = c / H_PLANCK * coef[g * NCOEF + 3 + i];
            A.H[g][i] = c * coef[g * NCOEF + 6 + i];
        }
    }
    if (n == 0) return FLD_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    k_photo_rates<<<blocks_for((long long)n), 256, 0, s>>>((long long)n, A, n_HI, n_HeI, n_HeII, rho_b, gamma_HI,
                                                          gamma_HeI, gamma_HeII, heating);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FLD_ECUDA, std::string("fld_photo_rates: ") + cudaGetErrorString(e));
    return FLD_OK;
}

}  // extern "C"
