// k_cg.cu -- conjugate-gradient vector kernels (Table 1 outer solver),
// FP64 iterative-refinement kernels of the mixed-precision solve, and the
// step finaliser with the photon balance.
//
// Every dot product and norm goes through the deterministic two-level FP64
// reduction of common.cuh, so a given launch shape always adds in the same
// order.
#include "kernels.h"

namespace fld {


template <class T>
__global__ void __launch_bounds__(RED_THREADS) k_dot(long long n, const T* __restrict__ a,
                                                     const T* __restrict__ b, RedArgs ra) {
    DotAcc<T> da;
    GRID_LOOP(c, n) da.add(a[c], b[c]);
    double acc[1] = {da.value()};
    const bool mx[1] = {false};
    grid_reduce<1>(acc, mx, ra);
}

// p_out = z + beta p_in;  q = A p_out;  <p_out, q>  ->  alpha = rho / <p, q>.
// p is double-buffered because neighbours of p_out are formed from p_in.
template <class T>
__global__ void __launch_bounds__(RED_THREADS) k_cg_p_matvec(Dims d, Op<T> A, const T* __restrict__ z,
                                                             const T* __restrict__ p_in,
                                                             T* __restrict__ p_out, T* __restrict__ q,
                                                             RedArgs ra) {
    const T beta = (T)ra.sc[S_BETA];
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    DotAcc<T> da;
    COL_BEGIN(d)
        const T pc = z[c] + beta * p_in[c];
        T a = T(0), s = T(0);
#define NB(widx, nb)                                      \
    {                                                     \
        const T w_ = A.widx;                              \
        a += w_ * (z[nb] + beta * p_in[nb]);              \
        s += w_;                                          \
    }
        if (i > 0) NB(wx[c], c - 1) else if (d.px) NB(wx[c], c + d.nx - 1)
        if (i < d.nx - 1) NB(wx[c + 1], c + 1) else if (d.px) NB(wx[c - (d.nx - 1)], c - (d.nx - 1))
        if (j > 0) NB(wy[c], c - sy) else if (d.py) NB(wy[c], c + (long long)(d.ny - 1) * sy)
        if (j < d.ny - 1) NB(wy[c + sy], c + sy) else if (d.py) NB(wy[c - (long long)(d.ny - 1) * sy], c - (long long)(d.ny - 1) * sy)
        if (k > 0) NB(wz[c], c - sz) else if (d.pz) NB(wz[c], c + (long long)(d.nz - 1) * sz)
        if (k < d.nz - 1) NB(wz[c + sz], c + sz) else if (d.pz) NB(wz[c - (long long)(d.nz - 1) * sz], c - (long long)(d.nz - 1) * sz)
#undef NB
        const T qc = A.m[c] * pc + s * pc - a;
        p_out[c] = pc;
        q[c] = qc;
        da.add(pc, qc);
    }
    double acc[1] = {da.value()};
    const bool mx[1] = {false};
    grid_reduce<1>(acc, mx, ra);
}

// x += alpha p;  r -= alpha q;  ||r||^2.
template <class T>
__global__ void __launch_bounds__(RED_THREADS) k_cg_update(long long n, T* __restrict__ x, T* __restrict__ r,
                                                           const T* __restrict__ p, const T* __restrict__ q,
                                                           RedArgs ra) {
    const T alpha = (T)ra.sc[S_ALPHA];
    DotAcc<T> da;
    GRID_LOOP(c, n) {
        x[c] += alpha * p[c];
        const T rc = r[c] - alpha * q[c];
        r[c] = rc;
        da.add(rc, rc);
    }
    double acc[1] = {da.value()};
    const bool mx[1] = {false};
    grid_reduce<1>(acc, mx, ra);
}

template <class T>
__global__ void k_apply(Dims d, Op<T> A, const T* __restrict__ x, T* __restrict__ y) {
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    COL_BEGIN(d)
        const T xc = x[c];
        T acc = A.m[c] * xc;
        if (i > 0) acc += A.wx[c] * (xc - x[c - 1]); else if (d.px) acc += A.wx[c] * (xc - x[c + d.nx - 1]);
        if (i < d.nx - 1) acc += A.wx[c + 1] * (xc - x[c + 1]); else if (d.px) acc += A.wx[c - (d.nx - 1)] * (xc - x[c - (d.nx - 1)]);
        if (j > 0) acc += A.wy[c] * (xc - x[c - sy]); else if (d.py) acc += A.wy[c] * (xc - x[c + (long long)(d.ny - 1) * sy]);
        if (j < d.ny - 1) acc += A.wy[c + sy] * (xc - x[c + sy]); else if (d.py) acc += A.wy[c - (long long)(d.ny - 1) * sy] * (xc - x[c - (long long)(d.ny - 1) * sy]);
        if (k > 0) acc += A.wz[c] * (xc - x[c - sz]); else if (d.pz) acc += A.wz[c] * (xc - x[c + (long long)(d.nz - 1) * sz]);
        if (k < d.nz - 1) acc += A.wz[c + sz] * (xc - x[c + sz]); else if (d.pz) acc += A.wz[c - (long long)(d.nz - 1) * sz] * (xc - x[c - (long long)(d.nz - 1) * sz]);
        y[c] = acc;
    }
}

// FP64 residual r = b - A x with ||r||^2 and max |r|.  With diag (the
// stored diagonal m + sum_f w_f) the product is diag x - sum_f w_f x_nbr,
// seven FP64 operations per cell instead of thirteen; its rounding error,
// u diag |x| per cell, stays far below the 1e-8 relative residual the
// refinement targets because diag <= 1 + 12 max(w) and ||x|| <= ||b||.
__global__ void __launch_bounds__(RED_THREADS) k_residual64(Dims d, Op<double> A, const double* __restrict__ diag,
                                                            const double* __restrict__ b,
                                                            const double* __restrict__ x, double* __restrict__ r,
                                                            RedArgs ra) {
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    double acc[2] = {0.0, 0.0};
    COL_BEGIN(d)
        const double xc = x[c];
        double Ax;
        if (diag) {
            // b + sum_f w_f x_nbr, then r = b - (diag x - sum) in one FMA
            double s = b[c];
            if (i > 0) s = fma(A.wx[c], x[c - 1], s); else if (d.px) s = fma(A.wx[c], x[c + d.nx - 1], s);
            if (i < d.nx - 1) s = fma(A.wx[c + 1], x[c + 1], s); else if (d.px) s = fma(A.wx[c - (d.nx - 1)], x[c - (d.nx - 1)], s);
            if (j > 0) s = fma(A.wy[c], x[c - sy], s); else if (d.py) s = fma(A.wy[c], x[c + (long long)(d.ny - 1) * sy], s);
            if (j < d.ny - 1) s = fma(A.wy[c + sy], x[c + sy], s); else if (d.py) s = fma(A.wy[c - (long long)(d.ny - 1) * sy], x[c - (long long)(d.ny - 1) * sy], s);
            if (k > 0) s = fma(A.wz[c], x[c - sz], s); else if (d.pz) s = fma(A.wz[c], x[c + (long long)(d.nz - 1) * sz], s);
            if (k < d.nz - 1) s = fma(A.wz[c + sz], x[c + sz], s); else if (d.pz) s = fma(A.wz[c - (long long)(d.nz - 1) * sz], x[c - (long long)(d.nz - 1) * sz], s);
            Ax = 0.0;
            const double rd = fma(-diag[c], xc, s);
            if (r) r[c] = rd;
            acc[0] = fma(rd, rd, acc[0]);
            acc[1] = fmax(acc[1], fabs(rd));
            continue;
        } else {
            Ax = A.m[c] * xc;
            if (i > 0) Ax += A.wx[c] * (xc - x[c - 1]); else if (d.px) Ax += A.wx[c] * (xc - x[c + d.nx - 1]);
            if (i < d.nx - 1) Ax += A.wx[c + 1] * (xc - x[c + 1]); else if (d.px) Ax += A.wx[c - (d.nx - 1)] * (xc - x[c - (d.nx - 1)]);
            if (j > 0) Ax += A.wy[c] * (xc - x[c - sy]); else if (d.py) Ax += A.wy[c] * (xc - x[c + (long long)(d.ny - 1) * sy]);
            if (j < d.ny - 1) Ax += A.wy[c + sy] * (xc - x[c + sy]); else if (d.py) Ax += A.wy[c - (long long)(d.ny - 1) * sy] * (xc - x[c - (long long)(d.ny - 1) * sy]);
            if (k > 0) Ax += A.wz[c] * (xc - x[c - sz]); else if (d.pz) Ax += A.wz[c] * (xc - x[c + (long long)(d.nz - 1) * sz]);
            if (k < d.nz - 1) Ax += A.wz[c + sz] * (xc - x[c + sz]); else if (d.pz) Ax += A.wz[c - (long long)(d.nz - 1) * sz] * (xc - x[c - (long long)(d.nz - 1) * sz]);
        }
        const double rc = b[c] - Ax;
        if (r) r[c] = rc;
        acc[0] = fma(rc, rc, acc[0]);
        acc[1] = fmax(acc[1], fabs(rc));
    }
    const bool mx[2] = {false, true};
    grid_reduce<2>(acc, mx, ra);
}

// E_out = max(E + dE, 0) and the sums of the photon balance of the
// unfloored update (energy density units; the host applies dt, dt c sigma,
// dt adot/a and V / h nu): sum dE, sum eta, sum n_HI E^theta, sum E^theta
// with E^theta = E^n + theta dE (E^{n+1} for backward Euler), the energy the
// floor adds, and sum dE^2, sum E_out^2 for the relative change of the step.
// Seven FP64 operations per cell (the FP64 pipe bounds this kernel); the
// sign test and the floor run on the integer pipe.  BE: theta = 1.
template <bool BE>
__global__ void __launch_bounds__(RED_THREADS) k_finalize(long long n, PhysDev p, const double* __restrict__ E,
                                                          const double* __restrict__ dE,
                                                          const double* __restrict__ nHI,
                                                          const double* __restrict__ eta, double* E_out,
                                                          RedArgs ra) {
    double acc[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    GRID_LOOP(c, n) {
        const double d = dE[c];
        const double Ec = E[c];
        const double En = Ec + d;
        const double Et = BE ? En : fma(p.theta, d, Ec);
        acc[0] += d;
        acc[1] += eta[c];
        acc[2] = fma(nHI[c], Et, acc[2]);
        acc[6] += Et;
        const bool neg = __double_as_longlong(En) < 0;   // sign bit (also -0)
        if (neg) acc[3] -= En;
        const double Eo = neg ? 0.0 : En;
        acc[4] = fma(d, d, acc[4]);
        acc[5] = fma(Eo, Eo, acc[5]);
        E_out[c] = Eo;
    }
    const bool mx[7] = {false, false, false, false, false, false, false};
    grid_reduce<7>(acc, mx, ra);
}

__global__ void k_f64_to_f32(long long n, const double* __restrict__ a, float* __restrict__ b) {
    GRID_LOOP(c, n) b[c] = (float)a[c];
}
__global__ void k_f32_to_f64(long long n, const float* __restrict__ a, double* __restrict__ b) {
    GRID_LOOP(c, n) b[c] = (double)a[c];
}

// Convergence test of a CG loop run on the device as the body of a
// conditional (while) graph node: count the iteration and continue while
// ||r||^2 > threshold, fewer than the allowed iterations are done and no
// reduction produced a non-finite value.
__global__ void k_cg_check(cudaGraphConditionalHandle h, cudaGraphConditionalHandle h2, int both, double* sc) {
    const double k = sc[S_KITER] + 1.0;
    sc[S_KITER] = k;
    const bool cont = !(sc[S_RR] <= sc[S_THRESH]) && k < sc[S_MAXIT] && sc[S_NONFINITE] == 0.0;
    cudaGraphSetConditional(h, cont ? 1u : 0u);
    if (both) cudaGraphSetConditional(h2, cont ? 1u : 0u);
}

// Reductions done in chunks (slots of nch consecutive NUM_SLOTS blocks):
// slot s_sum summed and s_max maximised in chunk order, a non-finite flag
// of any chunk kept.
__global__ void k_combine_chunks(const double* __restrict__ csc, int nch, double* sc, int s_sum, int s_max) {
    double sum = 0.0, mx = 0.0, nf = 0.0;
    for (int q = 0; q < nch; q++) {
        const double* v = csc + (long long)q * NUM_SLOTS;
        sum += v[s_sum];
        mx = fmax(mx, v[s_max]);
        nf = fmax(nf, v[S_NONFINITE]);
    }
    sc[s_sum] = sum;
    sc[s_max] = mx;
    if (nf != 0.0) sc[S_NONFINITE] = nf;
}

// Reductions done in chunks: each listed slot summed over the chunks in
// chunk order, a non-finite flag of any chunk kept.
__global__ void k_combine_sums(const double* __restrict__ csc, int nch, double* sc, SlotList sl) {
    double nf = 0.0;
    for (int t = 0; t < sl.n; t++) {
        double sum = 0.0;
        for (int q = 0; q < nch; q++) sum += csc[(long long)q * NUM_SLOTS + sl.s[t]];
        sc[sl.s[t]] = sum;
    }
    for (int q = 0; q < nch; q++) nf = fmax(nf, csc[(long long)q * NUM_SLOTS + S_NONFINITE]);
    if (nf != 0.0) sc[S_NONFINITE] = nf;
}

// ---------------------------------------------------------------- launchers

void launch_combine_sums(const double* chunk_sc, int nch, double* sc, const SlotList& sl, cudaStream_t s) {
    k_combine_sums<<<1, 1, 0, s>>>(chunk_sc, nch, sc, sl);
}
void launch_combine_chunks(const double* chunk_sc, int nch, double* sc, int s_sum, int s_max, cudaStream_t s) {
    k_combine_chunks<<<1, 1, 0, s>>>(chunk_sc, nch, sc, s_sum, s_max);
}

void launch_f64_to_f32(long long n, const double* a, float* b, cudaStream_t s) {
    k_f64_to_f32<<<grid_blocks(n, 256), 256, 0, s>>>(n, a, b);
}
void launch_f32_to_f64(long long n, const float* a, double* b, cudaStream_t s) {
    k_f32_to_f64<<<grid_blocks(n, 256), 256, 0, s>>>(n, a, b);
}

void launch_cg_check(cudaGraphConditionalHandle h, double* sc, cudaStream_t s,
                     const cudaGraphConditionalHandle* h2) {
    k_cg_check<<<1, 1, 0, s>>>(h, h2 ? *h2 : h, h2 ? 1 : 0, sc);
}


template <class T>
void launch_dot(long long n, const T* a, const T* b, const RedArgs& ra, cudaStream_t s) {
    k_dot<T><<<red_blocks(n), RED_THREADS, 0, s>>>(n, a, b, ra);
}
template <class T>
void launch_cg_p_matvec(const Dims& d, Op<T> A, const T* z, const T* p_in, T* p_out, T* q,
                        const RedArgs& ra, cudaStream_t s) {
    ColShape sh = col_shape(d);
    k_cg_p_matvec<T><<<sh.grid, sh.block, 0, s>>>(d, A, z, p_in, p_out, q, ra);
}
template <class T>
void launch_cg_update(long long n, T* x, T* r, const T* p, const T* q, const RedArgs& ra,
                      cudaStream_t s) {
    k_cg_update<T><<<red_blocks(n), RED_THREADS, 0, s>>>(n, x, r, p, q, ra);
}
template <class T>
void launch_apply(const Dims& d, Op<T> A, const T* x, T* y, cudaStream_t s) {
    ColShape sh = col_shape(d);
    k_apply<T><<<sh.grid, sh.block, 0, s>>>(d, A, x, y);
}
ColShape residual64_shape(const Dims& d) { return col_shape(d); }

void launch_residual64(const Dims& d, Op<double> A, const double* diag, const double* b, const double* x,
                       double* r, const RedArgs& ra, cudaStream_t s) {
    const ColShape sh = residual64_shape(d);
    k_residual64<<<sh.grid, sh.block, 0, s>>>(d, A, diag, b, x, r, ra);
}
void launch_finalize(long long n, const PhysDev& p, const double* E, const double* dE,
                     const double* nHI, const double* eta, double* E_out, const RedArgs& ra,
                     cudaStream_t s) {
    if (p.theta == 1.0)
        k_finalize<true><<<red_blocks(n), RED_THREADS, 0, s>>>(n, p, E, dE, nHI, eta, E_out, ra);
    else
        k_finalize<false><<<red_blocks(n), RED_THREADS, 0, s>>>(n, p, E, dE, nHI, eta, E_out, ra);
}

#define INST(T)                                                                                     \
    template void launch_dot<T>(long long, const T*, const T*, const RedArgs&, cudaStream_t);        \
    template void launch_cg_p_matvec<T>(const Dims&, Op<T>, const T*, const T*, T*, T*,              \
                                        const RedArgs&, cudaStream_t);                              \
    template void launch_cg_update<T>(long long, T*, T*, const T*, const T*, const RedArgs&,         \
                                      cudaStream_t);                                                \
    template void launch_apply<T>(const Dims&, Op<T>, const T*, T*, cudaStream_t);
INST(float)
INST(double)

}  // namespace fld
