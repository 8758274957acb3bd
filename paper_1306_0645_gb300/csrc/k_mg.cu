// k_mg.cu -- geometric multigrid V-cycle pieces for the 7-point FLD system
// (the preconditioner of Table 1): coarse operators, red/black Gauss-Seidel
// and weighted Jacobi smoothing, residual, full-weighting restriction,
// trilinear prolongation, and the dense coarsest-grid solve.
//
// Cell-centred full coarsening; operators by rediscretisation (coarse face
// weight = sum of the 4 fine face weights across the coarse face / 16,
// coarse mass term = mean of the 8 children); prolongation trilinear with
// 1-D weights 3/4 (nearer coarse cell) and 1/4 (farther one), ghost cells
// equal to the boundary cell on zero-gradient axes and wrapped on periodic
// ones; restriction is the transpose of prolongation divided by 8.
#include "kernels.h"

namespace fld {

// Sum over the faces of cell c of w_f * u_nbr, and of w_f.
template <class T>
__device__ __forceinline__ void nbr_sums(const Dims& d, const Op<T>& A, long long c, int i, int j,
                                         int k, const T* __restrict__ u, T& swu, T& sw) {
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    T a = T(0), s = T(0);
    {
        const T wl = A.wx[c];
        if (i > 0) { a += wl * u[c - 1]; s += wl; }
        else if (d.px) { a += wl * u[c + d.nx - 1]; s += wl; }
        if (i < d.nx - 1) { const T wu = A.wx[c + 1]; a += wu * u[c + 1]; s += wu; }
        else if (d.px) { const long long up = c - (d.nx - 1); const T wu = A.wx[up]; a += wu * u[up]; s += wu; }
    }
    {
        const T wl = A.wy[c];
        if (j > 0) { a += wl * u[c - sy]; s += wl; }
        else if (d.py) { a += wl * u[c + (long long)(d.ny - 1) * sy]; s += wl; }
        if (j < d.ny - 1) { const T wu = A.wy[c + sy]; a += wu * u[c + sy]; s += wu; }
        else if (d.py) { const long long up = c - (long long)(d.ny - 1) * sy; const T wu = A.wy[up]; a += wu * u[up]; s += wu; }
    }
    {
        const T wl = A.wz[c];
        if (k > 0) { a += wl * u[c - sz]; s += wl; }
        else if (d.pz) { a += wl * u[c + (long long)(d.nz - 1) * sz]; s += wl; }
        if (k < d.nz - 1) { const T wu = A.wz[c + sz]; a += wu * u[c + sz]; s += wu; }
        else if (d.pz) { const long long up = c - (long long)(d.nz - 1) * sz; const T wu = A.wz[up]; a += wu * u[up]; s += wu; }
    }
    swu = a;
    sw = s;
}

// Sum over the faces of cell c of w_f * u_nbr * v_nbr (smoothing from a
// zero guess needs the red neighbours' values r * invd on the fly).
template <class T>
__device__ __forceinline__ T nbr_sum_prod(const Dims& d, const Op<T>& A, long long c, int i, int j,
                                          int k, const T* __restrict__ u, const T* __restrict__ v) {
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    T a = T(0);
    if (i > 0) a += A.wx[c] * u[c - 1] * v[c - 1];
    else if (d.px) a += A.wx[c] * u[c + d.nx - 1] * v[c + d.nx - 1];
    if (i < d.nx - 1) a += A.wx[c + 1] * u[c + 1] * v[c + 1];
    else if (d.px) { const long long up = c - (d.nx - 1); a += A.wx[up] * u[up] * v[up]; }
    if (j > 0) a += A.wy[c] * u[c - sy] * v[c - sy];
    else if (d.py) { const long long lo = c + (long long)(d.ny - 1) * sy; a += A.wy[c] * u[lo] * v[lo]; }
    if (j < d.ny - 1) a += A.wy[c + sy] * u[c + sy] * v[c + sy];
    else if (d.py) { const long long up = c - (long long)(d.ny - 1) * sy; a += A.wy[up] * u[up] * v[up]; }
    if (k > 0) a += A.wz[c] * u[c - sz] * v[c - sz];
    else if (d.pz) { const long long lo = c + (long long)(d.nz - 1) * sz; a += A.wz[c] * u[lo] * v[lo]; }
    if (k < d.nz - 1) a += A.wz[c + sz] * u[c + sz] * v[c + sz];
    else if (d.pz) { const long long up = c - (long long)(d.nz - 1) * sz; a += A.wz[up] * u[up] * v[up]; }
    return a;
}


// ------------------------------------------------------------ operators

// Rediscretised coarse operator in precision T (FP64 for the FP64 cycle;
// FP32 from the FP32 operator for the mixed solver's cycle, which alone
// reads the coarse levels there).
template <class T>
__global__ void k_coarsen(Dims f, Dims cd, Op<T> F, Op<T> C) {
    COL_BEGIN(cd)
        const int I = i, J = j, K = k;
        const long long fx = f.nx, fxy = (long long)f.nx * f.ny;
        const long long base = 2LL * I + fx * 2LL * J + fxy * 2LL * K;
        T ms = 0;
#pragma unroll
        for (int dk = 0; dk < 2; dk++)
#pragma unroll
            for (int dj = 0; dj < 2; dj++)
#pragma unroll
                for (int di = 0; di < 2; di++) ms += F.m[base + di + fx * dj + fxy * dk];
        T sx = 0, sy = 0, sz = 0;
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int b = 0; b < 2; b++) {
                sx += F.wx[base + fx * a + fxy * b];
                sy += F.wy[base + a + fxy * b];
                sz += F.wz[base + a + fx * b];
            }
        C.m[c] = ms * (T)0.125;
        C.wx[c] = sx * (T)0.0625;
        C.wy[c] = sy * (T)0.0625;
        C.wz[c] = sz * (T)0.0625;
    }
}

// Coarse Dirichlet face weights of side sd: the sum of the 4 fine weights
// across each coarse face / 16, as for interior faces.  k_coarsen set the
// coarse mass term to the mean of the 8 children's m, which holds their
// boundary weights / 8 = 2 w_c; the rediscretised mass term has w_c, so
// w_c is taken back off.
template <class T>
__global__ void k_coarsen_bnd(Dims f, Dims cd, int sd, Bnd F, Bnd C, Op<T> CA) {
    const int a = sd >> 1, hi = sd & 1;
    const long long nfc = bnd_side_size(cd, sd);
    const long long offc = bnd_offset(cd, sd), offf = bnd_offset(f, sd);
    const long long nuc = a == 0 ? cd.ny : cd.nx;
    const long long nuf = 2 * nuc;
    GRID_LOOP(fc, nfc) {
        const long long u = fc % nuc, v = fc / nuc;
        const long long f00 = offf + 2 * u + nuf * 2 * v;
        const double wc = ((F.w[f00] + F.w[f00 + 1]) + (F.w[f00 + nuf] + F.w[f00 + nuf + 1])) * 0.0625;
        C.w[offc + fc] = wc;
        long long i, j, k;
        if (a == 0) { i = hi ? cd.nx - 1 : 0; j = u; k = v; }
        else if (a == 1) { i = u; j = hi ? cd.ny - 1 : 0; k = v; }
        else { i = u; j = v; k = hi ? cd.nz - 1 : 0; }
        T& mc = CA.m[i + (long long)cd.nx * (j + (long long)cd.ny * k)];
        mc = (T)(mc - wc);
    }
}

// Inverse diagonal of A in precision T, the diagonal summed in the
// precision S of the operator src it is formed from.
template <class T, class S>
__global__ void k_invd(Dims d, Op<T> A, Op<S> src) {
    COL_BEGIN(d)
        S swu, sw;
        // u unused: pass m as a harmless array for the weight sum only
        nbr_sums<S>(d, src, c, i, j, k, src.m, swu, sw);
        const S diag = src.m[c] + sw;
        A.invd[c] = (T)((S)1 / diag);
    }
}

// ------------------------------------------------------------- smoothers

// First red/black Gauss-Seidel sweep from z = 0: red cells get r / diag,
// black cells (r + sum_f w_f z_red_nbr) / diag with the red values formed
// on the fly.
template <class T>
__global__ void k_smooth_zero(Dims d, Op<T> A, const T* __restrict__ r, T* __restrict__ z) {
    COL_BEGIN(d)
        if (((i + j + k) & 1) == 0) {
            z[c] = r[c] * A.invd[c];
        } else {
            z[c] = A.invd[c] * (r[c] + nbr_sum_prod<T>(d, A, c, i, j, k, r, A.invd));
        }
    }
}

// One colour of a red/black Gauss-Seidel sweep; every dimension is even on
// a smoothed level, so cell (2s + ((j + k + colour) & 1), j, k) enumerates
// the colour.
template <class T>
__global__ void k_rb_colour(Dims d, Op<T> A, const T* __restrict__ r, T* z, int colour) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int kch = (d.nz + (int)gridDim.z - 1) / (int)gridDim.z;
    const int k0 = (int)blockIdx.z * kch, k1 = min(d.nz, k0 + kch);
    if (s >= (d.nx >> 1) || j >= d.ny) return;
    const long long nxy = (long long)d.nx * d.ny;
    for (int k = k0; k < k1; k++) {
        const int i = 2 * s + ((j + k + colour) & 1);
        const long long c = (long long)k * nxy + (long long)j * d.nx + i;
        T swu, sw;
        nbr_sums<T>(d, A, c, i, j, k, z, swu, sw);
        z[c] = A.invd[c] * (r[c] + swu);
    }
}

// Weighted Jacobi: out = z + omega (r - A z) / diag, or omega r / diag from
// a zero guess.
template <class T>
__global__ void k_jacobi(Dims d, Op<T> A, const T* __restrict__ r, const T* __restrict__ z,
                         T* __restrict__ out, T omega, int zero_guess) {
    COL_BEGIN(d)
        if (zero_guess) {
            out[c] = omega * A.invd[c] * r[c];
        } else {
            T swu, sw;
            nbr_sums<T>(d, A, c, i, j, k, z, swu, sw);
            const T Az = A.m[c] * z[c] + sw * z[c] - swu;
            out[c] = z[c] + omega * A.invd[c] * (r[c] - Az);
        }
    }
}

template <class T>
__global__ void k_residual(Dims d, Op<T> A, const T* __restrict__ r, const T* __restrict__ z,
                           T* __restrict__ res) {
    COL_BEGIN(d)
        T swu, sw;
        nbr_sums<T>(d, A, c, i, j, k, z, swu, sw);
        res[c] = r[c] - (A.m[c] * z[c] + sw * z[c] - swu);
    }
}

// ------------------------------------------------------------- transfers

// Fine index of tap t (0..3 = offsets -1, 0, +1, +2 from 2I) along an axis,
// with the ghost rule; weights 1/4, 3/4, 3/4, 1/4.
__device__ __forceinline__ int fine_tap(int I, int t, int nf, int periodic) {
    int f = 2 * I - 1 + t;
    if (f < 0) f = periodic ? f + nf : 0;
    if (f >= nf) f = periodic ? f - nf : nf - 1;
    return f;
}

template <class T>
__global__ void k_restrict(Dims f, Dims cd, const T* __restrict__ rf, T* __restrict__ rc) {
    const T wt[4] = {T(0.25), T(0.75), T(0.75), T(0.25)};
    COL_BEGIN(cd)
        const int I = i, J = j, K = k;
        int fi[4], fj[4], fk[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
            fi[t] = fine_tap(I, t, f.nx, f.px);
            fj[t] = fine_tap(J, t, f.ny, f.py);
            fk[t] = fine_tap(K, t, f.nz, f.pz);
        }
        T acc = T(0);
#pragma unroll
        for (int tk = 0; tk < 4; tk++) {
            T acc_j = T(0);
#pragma unroll
            for (int tj = 0; tj < 4; tj++) {
                const long long row = (long long)f.nx * (fj[tj] + (long long)f.ny * fk[tk]);
                T acc_i = T(0);
#pragma unroll
                for (int ti = 0; ti < 4; ti++) acc_i += wt[ti] * rf[row + fi[ti]];
                acc_j += wt[tj] * acc_i;
            }
            acc += wt[tk] * acc_j;
        }
        rc[c] = acc * T(0.125);
    }
}

// Coarse neighbours of fine index i: nearer (weight 3/4) and farther (1/4).
__device__ __forceinline__ void coarse_pair(int i, int nc, int periodic, int& I0, int& I1) {
    I0 = i >> 1;
    int J = (i & 1) ? I0 + 1 : I0 - 1;
    if (J < 0) J = periodic ? nc - 1 : I0;
    if (J >= nc) J = periodic ? 0 : I0;
    I1 = J;
}

template <class T>
__global__ void k_prolong_add(Dims f, Dims cd, const T* __restrict__ ec, T* __restrict__ zf) {
    COL_BEGIN(f)
        int Ix[2], Iy[2], Iz[2];
        coarse_pair(i, cd.nx, cd.px, Ix[0], Ix[1]);
        coarse_pair(j, cd.ny, cd.py, Iy[0], Iy[1]);
        coarse_pair(k, cd.nz, cd.pz, Iz[0], Iz[1]);
        const T w[2] = {T(0.75), T(0.25)};
        T acc = T(0);
#pragma unroll
        for (int b = 0; b < 2; b++) {
            T acc_j = T(0);
#pragma unroll
            for (int a = 0; a < 2; a++) {
                const long long row = (long long)cd.nx * (Iy[a] + (long long)cd.ny * Iz[b]);
                acc_j += w[a] * (w[0] * ec[row + Ix[0]] + w[1] * ec[row + Ix[1]]);
            }
            acc += w[b] * acc_j;
        }
        zf[c] += acc;
    }
}

// ---------------------------------------------------------- coarsest grid

template <class T>
__global__ void k_dense_build(Dims d, Op<T> A, double* __restrict__ M) {
    const long long n = d.n;
    GRID_LOOP(c, n) {
        double* row = M + c * n;
        for (long long q = 0; q < n; q++) row[q] = 0.0;
    }
    // rows are owned by one thread each, so the adds below do not race
    GRID_LOOP(c, n) {
        int i, j, k;
        cell_ijk(c, d, i, j, k);
        double* row = M + c * n;
        const long long sy = d.nx, sz = (long long)d.nx * d.ny;
        double diag = (double)A.m[c];
        auto add = [&](T wt, long long nb) {
            const double w = (double)wt;
            diag += w;
            row[nb] -= w;
        };
        if (i > 0) add(A.wx[c], c - 1); else if (d.px) add(A.wx[c], c + d.nx - 1);
        if (i < d.nx - 1) add(A.wx[c + 1], c + 1); else if (d.px) add(A.wx[c - (d.nx - 1)], c - (d.nx - 1));
        if (j > 0) add(A.wy[c], c - sy); else if (d.py) add(A.wy[c], c + (long long)(d.ny - 1) * sy);
        if (j < d.ny - 1) add(A.wy[c + sy], c + sy); else if (d.py) add(A.wy[c - (long long)(d.ny - 1) * sy], c - (long long)(d.ny - 1) * sy);
        if (k > 0) add(A.wz[c], c - sz); else if (d.pz) add(A.wz[c], c + (long long)(d.nz - 1) * sz);
        if (k < d.nz - 1) add(A.wz[c + sz], c + sz); else if (d.pz) add(A.wz[c - (long long)(d.nz - 1) * sz], c - (long long)(d.nz - 1) * sz);
        row[c] += diag;
    }
}

// One CTA: in-place Cholesky of the dense SPD matrix M (row-major, lower
// triangle becomes L), then the explicit inverse Ainv = L^-T L^-1, one
// column per thread.  A non-positive pivot sets sc[S_BAD] = 2.
__global__ void k_chol_inverse(int n, double* M, double* Ainv, double* sc) {
    __shared__ int fail;
    if (threadIdx.x == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < n; j++) {
        if (threadIdx.x == 0) {
            const double piv = M[(long long)j * n + j];
            if (!(piv > 0.0)) { fail = 1; M[(long long)j * n + j] = 1.0; }
            else M[(long long)j * n + j] = sqrt(piv);
        }
        __syncthreads();
        const double ljj = M[(long long)j * n + j];
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) M[(long long)i * n + j] /= ljj;
        __syncthreads();
        // trailing update of the lower triangle: M[i][k] -= L[i][j] L[k][j], j < k <= i
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
            const double lij = M[(long long)i * n + j];
            for (int k = j + 1; k <= i; k++) M[(long long)i * n + k] -= lij * M[(long long)k * n + j];
        }
        __syncthreads();
    }
    if (fail && threadIdx.x == 0) sc[S_BAD] = 2.0;
    // inverse, column t: L y = e_t, then L^T x = y, written in Ainv[:, t]
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        for (int i = 0; i < t; i++) Ainv[(long long)i * n + t] = 0.0;
        for (int i = t; i < n; i++) {
            double s = (i == t) ? 1.0 : 0.0;
            for (int k = t; k < i; k++) s -= M[(long long)i * n + k] * Ainv[(long long)k * n + t];
            Ainv[(long long)i * n + t] = s / M[(long long)i * n + i];
        }
        for (int i = n - 1; i >= 0; i--) {
            double s = Ainv[(long long)i * n + t];
            for (int k = i + 1; k < n; k++) s -= M[(long long)k * n + i] * Ainv[(long long)k * n + t];
            Ainv[(long long)i * n + t] = s / M[(long long)i * n + i];
        }
    }
}

// Coarsest-grid setup for small grids, one CTA with the matrix in shared
// memory: Cholesky M = L L^T in precision T (the trailing update spread over
// all threads), X = L^-1 by forward substitution (one column per thread),
// and the inverse Ainv = X^T X, written as FP64 (exactly symmetric).  The
// mixed-precision solver takes T = float: its whole V-cycle is FP32.  A
// non-positive pivot sets sc[S_BAD] = 2.
template <class T>
__global__ void __launch_bounds__(1024) k_chol_inverse_smem(int n, const double* __restrict__ M,
                                                            double* __restrict__ Ainv, double* sc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* L = reinterpret_cast<T*>(smem_raw);   // n x n, row-major
    T* X = L + (long long)n * n;             // n x n, row-major, lower triangle
    __shared__ int fail;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) fail = 0;
    for (int q = tid; q < n * n; q += nt) {
        L[q] = (T)M[q];
        X[q] = T(0);
    }
    __syncthreads();
    for (int j = 0; j < n; j++) {
        if (tid == 0) {
            const T piv = L[j * n + j];
            if (!(piv > T(0))) { fail = 1; L[j * n + j] = T(1); }
            else L[j * n + j] = sqrt(piv);
        }
        __syncthreads();
        const T ljj = L[j * n + j];
        for (int i = j + 1 + tid; i < n; i += nt) L[i * n + j] /= ljj;
        __syncthreads();
        // trailing update of the lower triangle: (i, k) with j < k <= i
        const int m = n - j - 1;
        for (int q = tid; q < m * m; q += nt) {
            const int i = j + 1 + q / m, k = j + 1 + q % m;
            if (k <= i) L[i * n + k] -= L[i * n + j] * L[k * n + j];
        }
        __syncthreads();
    }
    for (int t = tid; t < n; t += nt)
        for (int i = t; i < n; i++) {
            T v = (i == t) ? T(1) : T(0);
            for (int k = t; k < i; k++) v -= L[i * n + k] * X[k * n + t];
            X[i * n + t] = v / L[i * n + i];
        }
    __syncthreads();
    for (int q = tid; q < n * n; q += nt) {
        const int a = q / n, b = q - a * n;
        T v = T(0);
        for (int i = a > b ? a : b; i < n; i++) v += X[i * n + a] * X[i * n + b];
        Ainv[q] = (double)v;
    }
    if (fail && tid == 0) sc[S_BAD] = 2.0;
}

// Coarsest-grid inverse for n <= 128, one CTA of 32 x 32 threads with the
// matrix in shared memory: in-place Gauss-Jordan elimination without
// pivoting (stable for the symmetric positive definite operator).  Step k
// replaces the matrix M by
//   M'[k][k] = 1/p,  M'[k][j] = M[k][j]/p,  M'[i][k] = -M[i][k]/p,
//   M'[i][j] = M[i][j] - M[i][k] M[k][j]/p      (p = M[k][k] > 0),
// every entry at once (read phase, barrier, write phase); after n steps M
// holds the inverse.  Each thread owns the entries (ty + 32 a, tx + 32 b).
// The result is written as FP64.  A non-positive pivot sets sc[S_BAD] = 2.
constexpr int GJ_MAX = 128;
template <class T, int PT>   // PT = entries per thread and axis, n <= 32 PT
__global__ void __launch_bounds__(1024) k_gj_inverse_smem(int n, const double* __restrict__ M,
                                                          double* __restrict__ Ainv, double* sc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* A = reinterpret_cast<T*>(smem_raw);
    __shared__ int fail;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if (threadIdx.x == 0) fail = 0;
    for (int q = threadIdx.x; q < n * n; q += 1024) A[q] = (T)M[q];
    __syncthreads();
    for (int k = 0; k < n; k++) {
        T p = A[k * n + k];
        if (!(p > T(0))) {
            if (threadIdx.x == 0) fail = 1;
            p = T(1);
        }
        const T ip = T(1) / p;
        T nv[PT][PT];
#pragma unroll
        for (int a = 0; a < PT; a++) {
            const int i = ty + 32 * a;
#pragma unroll
            for (int b = 0; b < PT; b++) {
                const int j = tx + 32 * b;
                if (i < n && j < n) {
                    if (i == k && j == k) nv[a][b] = ip;
                    else if (i == k) nv[a][b] = A[k * n + j] * ip;
                    else if (j == k) nv[a][b] = -A[i * n + k] * ip;
                    else nv[a][b] = A[i * n + j] - A[i * n + k] * (A[k * n + j] * ip);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int a = 0; a < PT; a++) {
            const int i = ty + 32 * a;
#pragma unroll
            for (int b = 0; b < PT; b++) {
                const int j = tx + 32 * b;
                if (i < n && j < n) A[i * n + j] = nv[a][b];
            }
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < n * n; q += 1024) Ainv[q] = (double)A[q];
    if (fail && threadIdx.x == 0) sc[S_BAD] = 2.0;
}

template <class T>
__global__ void k_coarse_apply(int n, const double* __restrict__ Ainv, const T* __restrict__ r,
                               T* __restrict__ z) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < n; j++) s += Ainv[(long long)j * n + i] * (double)r[j];
        z[i] = (T)s;
    }
}

// ---------------------------------------------------------------- launchers

static const int TPB = 256;

template <class T>
void launch_coarsen(const Dims& f, const Dims& c, Op<T> F, Op<T> C, cudaStream_t s) {
    ColShape sh = col_shape(c);
    k_coarsen<T><<<sh.grid, sh.block, 0, s>>>(f, c, F, C);
}
template <class T>
void launch_coarsen_bnd(const Dims& f, const Dims& c, int sd, Bnd F, Bnd C, Op<T> CA, cudaStream_t st) {
    k_coarsen_bnd<T><<<grid_blocks(bnd_side_size(c, sd), 256), 256, 0, st>>>(f, c, sd, F, C, CA);
}
template <class T>
void launch_invd(const Dims& d, Op<T> A, const Op<T>& src, cudaStream_t s) {
    ColShape sh = col_shape(d);
    k_invd<T, T><<<sh.grid, sh.block, 0, s>>>(d, A, src);
}
template <class T>
void launch_smooth_zero(const Dims& d, Op<T> A, const T* r, T* z, cudaStream_t s) {
    ColShape sh = col_shape(d);
    k_smooth_zero<T><<<sh.grid, sh.block, 0, s>>>(d, A, r, z);
}
template <class T>
void launch_rb_colour(const Dims& d, Op<T> A, const T* r, T* z, int colour, cudaStream_t s) {
    Dims h = d;
    h.nx = d.nx / 2;
    ColShape sh = col_shape(h);
    k_rb_colour<T><<<sh.grid, sh.block, 0, s>>>(d, A, r, z, colour);
}
template <class T>
void launch_jacobi(const Dims& d, Op<T> A, const T* r, const T* z, T* out, double omega,
                   bool zero_guess, cudaStream_t s) {
    ColShape sh = col_shape(d);
    k_jacobi<T><<<sh.grid, sh.block, 0, s>>>(d, A, r, z, out, (T)omega, zero_guess ? 1 : 0);
}
template <class T>
void launch_residual(const Dims& d, Op<T> A, const T* r, const T* z, T* res, cudaStream_t s) {
    ColShape sh = col_shape(d);
    k_residual<T><<<sh.grid, sh.block, 0, s>>>(d, A, r, z, res);
}
template <class T>
void launch_restrict(const Dims& f, const Dims& c, const T* rf, T* rc, cudaStream_t s) {
    ColShape sh = col_shape(c);
    k_restrict<T><<<sh.grid, sh.block, 0, s>>>(f, c, rf, rc);
}
template <class T>
void launch_prolong_add(const Dims& f, const Dims& c, const T* ec, T* zf, cudaStream_t s) {
    ColShape sh = col_shape(f);
    k_prolong_add<T><<<sh.grid, sh.block, 0, s>>>(f, c, ec, zf);
}
// shared memory of the in-CTA setup for an n x n matrix in precision T
// (factor and inverse), and whether it fits
static size_t chol_smem_bytes(long long n, size_t ts) { return 2 * (size_t)n * (size_t)n * ts; }
static const size_t CHOL_SMEM_MAX = 200 * 1024;

template <class T>
void launch_coarse_setup(const Dims& d, Op<T> A, double* dense, double* ainv, double* sc, bool fp32,
                         cudaStream_t s) {
    k_dense_build<T><<<1, TPB, 0, s>>>(d, A, dense);
    const size_t ts = fp32 ? sizeof(float) : sizeof(double);
    if (d.n <= GJ_MAX) {
        const size_t gb = (size_t)d.n * (size_t)d.n * ts;
        const int n = (int)d.n;
        auto go = [&](auto kern) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gb);
            kern<<<1, 1024, gb, s>>>(n, dense, ainv, sc);
        };
        if (fp32) {
            if (n <= 32) go(k_gj_inverse_smem<float, 1>);
            else if (n <= 64) go(k_gj_inverse_smem<float, 2>);
            else go(k_gj_inverse_smem<float, 4>);
        } else {
            if (n <= 32) go(k_gj_inverse_smem<double, 1>);
            else if (n <= 64) go(k_gj_inverse_smem<double, 2>);
            else go(k_gj_inverse_smem<double, 4>);
        }
        return;
    }
    const size_t bytes = chol_smem_bytes(d.n, ts);
    if (bytes <= CHOL_SMEM_MAX) {
        if (fp32) {
            cudaFuncSetAttribute(k_chol_inverse_smem<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
            k_chol_inverse_smem<float><<<1, 1024, bytes, s>>>((int)d.n, dense, ainv, sc);
        } else {
            cudaFuncSetAttribute(k_chol_inverse_smem<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
            k_chol_inverse_smem<double><<<1, 1024, bytes, s>>>((int)d.n, dense, ainv, sc);
        }
        return;
    }
    const int threads = d.n < 1024 ? (int)((d.n + 31) / 32 * 32) : 1024;
    k_chol_inverse<<<1, threads, 0, s>>>((int)d.n, dense, ainv, sc);
}
template <class T>
void launch_coarse_apply(int n, const double* ainv, const T* r, T* z, cudaStream_t s) {
    k_coarse_apply<T><<<(n + 127) / 128, 128, 0, s>>>(n, ainv, r, z);
}

#define INST(T)                                                                                    \
    template void launch_invd<T>(const Dims&, Op<T>, const Op<T>&, cudaStream_t);                   \
    template void launch_coarsen<T>(const Dims&, const Dims&, Op<T>, Op<T>, cudaStream_t);           \
    template void launch_coarsen_bnd<T>(const Dims&, const Dims&, int, Bnd, Bnd, Op<T>, cudaStream_t); \
    template void launch_coarse_setup<T>(const Dims&, Op<T>, double*, double*, double*, bool, cudaStream_t); \
    template void launch_smooth_zero<T>(const Dims&, Op<T>, const T*, T*, cudaStream_t);            \
    template void launch_rb_colour<T>(const Dims&, Op<T>, const T*, T*, int, cudaStream_t);         \
    template void launch_jacobi<T>(const Dims&, Op<T>, const T*, const T*, T*, double, bool,        \
                                   cudaStream_t);                                                  \
    template void launch_residual<T>(const Dims&, Op<T>, const T*, const T*, T*, cudaStream_t);     \
    template void launch_restrict<T>(const Dims&, const Dims&, const T*, T*, cudaStream_t);         \
    template void launch_prolong_add<T>(const Dims&, const Dims&, const T*, T*, cudaStream_t);      \
    template void launch_coarse_apply<T>(int, const double*, const T*, T*, cudaStream_t);
INST(float)
INST(double)

}  // namespace fld
