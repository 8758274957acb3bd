/*
 * fld_oracle.c -- plain FP64 CPU oracle for one implicit grey flux-limited
 * diffusion (FLD) radiation step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the package's smoke check and the
 * CPU-baseline leg of the benchmark use it.  It shares no source with the
 * CUDA path.
 *
 * What it computes (Norman et al. 2015, "Fully-Coupled Simulation of Cosmic
 * Reionization I", arXiv:1306.0645):
 *   - the grey FLD equation split off from the other physics (Sec. 3.2,
 *     Eq. "fld"):  dE/dt = div(D grad E) - (adot/a) E - c kappa E + eta;
 *   - the flux limiter D = min{c (9 kappa^2 + R^2)^(-1/2), D_max} with
 *     R = max{|dE|/E, R_min}, D_max = 0.006 c L_unit, R_min = 1e-20/L_unit,
 *     face E by arithmetic mean and face kappa by harmonic mean (Sec. 2,
 *     limiter definition after Eq. "cons_radiation");
 *   - the Levermore-Pomraning limiter the paper cites as an alternative
 *     (Sec. 1, LevermorePomraning1981);
 *   - opacity kappa = n_HI sigma for a monochromatic grey source
 *     (Eq. "opacity" with a single species and a delta-function SED);
 *   - comoving coordinates for cosmological runs (Sec. 3.2, Eq. "fld"
 *     with the adot/a term): cell widths are comoving, the gradients of the
 *     equation proper, so the limiter and the face weights see the proper
 *     widths a h, a the scale factor; E and eta are per comoving volume,
 *     kappa proper;
 *   - the implicit theta-method of Sec. 3.2 (theta = 1 backward Euler,
 *     theta = 1/2 the trapezoidal rule) with D lagged at E^n, so the step is
 *     one linear system, posed for the correction dE = E^{n+1} - E^n:
 *     with F(E) = div(D grad E) - (c kappa + adot/a) E + eta (eta and kappa
 *     held at t^n), dE - theta dt L dE = dt F(E^n), L the linear part of F;
 *   - the solver of Table 1: PCG, at most 50 iterations, tolerance 1e-8,
 *     preconditioned by a geometric multigrid cycle with red/black
 *     Gauss-Seidel relaxation, 1 pre- and 1 post-sweep.
 *
 * Where the paper is silent the oracle takes these readings (they are the
 * algorithm definition the CUDA path implements as well):
 *   - CGS units, L_unit = box length unless given; R uses the one-sided
 *     normal difference across the face only;
 *   - face kappa = 0 when either side is 0; R = R_min when both face E are 0;
 *   - LP limiter: with x = R/kappa_f, D = c lambda(x)/kappa_f,
 *     lambda(x) = (coth x - 1/x)/x, series 1/3 - x^2/45 + 2x^4/945 for
 *     x < 1e-2, and D = c/R when kappa_f = 0 or x > 1e8;
 *   - boundaries per face of the box: reflecting (zero gradient, no flux,
 *     face weight 0), periodic (wrap; both faces of the axis), Dirichlet
 *     (E fixed to E_b on the face, half a cell from the cell centre: the
 *     face takes D from the limiter with face E = (E + E_b)/2, normal
 *     difference |E - E_b| over h/2 and kappa_f = kappa of the cell, and
 *     weight theta dt D / (h h/2) on the diagonal), and outflow read as
 *     Dirichlet with E_b = 0, through which the limiter lets radiation
 *     stream out at |F| = c E_face when the cell is optically thin;
 *   - multigrid: full 2x coarsening of cell-centred grids while every
 *     dimension is even and the smallest one exceeds 4; trilinear
 *     prolongation P (ghost cells per boundary condition), restriction
 *     R = P^T / 8; coarse operator by rediscretisation (coarse face weight =
 *     sum of the 4 fine face weights across the coarse face / 16, also for
 *     Dirichlet boundary faces; coarse mass term = mean of the 8 children's
 *     mass terms, the boundary weights apart); dense Cholesky on the coarsest
 *     grid; one V(pre,post) cycle per PCG iteration, red = (i+j+k) even,
 *     pre-sweeps red then black, post-sweeps black then red (symmetric;
 *     or red then black, the order of Table 1's "nonsymmetric" relaxation,
 *     with paper_order);
 *     weighted Jacobi as the alternative smoother;
 *   - PCG from x0 = 0, stop when ||r||_2 / ||b||_2 <= rtol on the
 *     recursively updated residual; b = 0 gives dE = 0 in 0 iterations;
 *   - E^{n+1} = max(E^n + dE, 0): for backward Euler the exact solution is
 *     non-negative (A is an M-matrix and A E^{n+1} = E^n + dt eta >= 0), so
 *     negative values are solver-tolerance artefacts; the trapezoidal rule
 *     can undershoot for large dt, which the floor also catches.  The photon
 *     balance is taken on E^n + dE before the floor, and the floor's
 *     addition is reported.
 *
 * Layout: every field is a contiguous FP64 array, x fastest,
 * idx = i + nx (j + ny k).  The operator of a level is stored as the mass
 * term m_i = 1 + theta dt (c kappa_i + adot/a) + (the theta-scaled weights of
 * the cell's Dirichlet boundary faces) and three lower-face weights
 * theta dt D / h^2:
 * wx[idx] couples cell (i,j,k) with (i-1,j,k) (and with (nx-1,j,k) for i = 0
 * on a periodic axis; 0 on any other boundary), likewise wy, wz.
 * Row i of A:  (A u)_i = m_i u_i + sum_faces w_f (u_i - u_nbr).
 * The weights of Dirichlet faces are also kept per face, in one packed
 * boundary array (see side_offset), for the coarsening.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_ENOCONV = 3 };
enum { OR_LIMITER_PAPER = 0, OR_LIMITER_LP = 1 };
enum { OR_SMOOTH_RBGS = 0, OR_SMOOTH_JACOBI = 1 };

/* Faces of the box, side s = 2 axis + (0 lower, 1 upper). */
typedef struct {
    int n[3];          /* cells per axis */
    double h[3];       /* cell widths, cm */
    int periodic[3];   /* 1 = periodic axis (both faces) */
    int dirichlet[6];  /* per side: 1 = E fixed to ebc[side]; 0 = reflecting */
    double ebc[6];     /* Dirichlet value of each side (outflow: 0) */
} or_grid;

typedef struct {
    double dt;         /* s */
    double c;          /* cm/s */
    double L_unit;     /* cm */
    double dmax_coef;  /* 0.006 */
    double rmin_coef;  /* 1e-20 */
    double sigma;      /* cm^2 */
    double adot;       /* adot/a, 1/s */
    double hnu;        /* erg per photon, for photon counts */
    int limiter;
    double theta;      /* 1 backward Euler, 1/2 trapezoidal */
    double a;          /* cosmological scale factor (1: proper units) */
} or_phys;

typedef struct {
    int smoother;
    double omega;
    int pre, post;
    double rtol;
    int max_iter;
    int coarse_cap;    /* largest coarsest-grid size accepted */
    int paper_order;   /* RB-GS post-sweeps red then black (Table 1's
                          "nonsymmetric" relaxation); 0: black then red */
} or_solver;

typedef struct {
    int n[3];
    int periodic[3];
    double *m, *wx, *wy, *wz;
    int owned;
    int dirichlet[6];
    double* bnd;       /* packed Dirichlet face weights (NULL: none) */
} or_level;

#define OR_MAX_LEVELS 32

static size_t ncell(const int n[3]) { return (size_t)n[0] * n[1] * n[2]; }

/* Packed per-face boundary arrays: sides in the order x lo, x hi, y lo,
 * y hi, z lo, z hi; the face of cell (i,j,k) on an x side has index
 * j + ny k, on a y side i + nx k, on a z side i + nx j. */
static size_t side_size(const int n[3], int s) {
    int d = s / 2;
    if (d == 0) return (size_t)n[1] * n[2];
    if (d == 1) return (size_t)n[0] * n[2];
    return (size_t)n[0] * n[1];
}

static size_t side_offset(const int n[3], int s) {
    size_t o = 0;
    for (int q = 0; q < s; q++) o += side_size(n, q);
    return o;
}

size_t or_bnd_size(const int n[3]) { return side_offset(n, 6); }

/* Index of cell (i,j,k)'s face on side s in the packed array, or -1 when
 * the cell does not touch that side. */
static long side_face(const int n[3], int s, int i, int j, int k) {
    int d = s / 2, hi = s % 2;
    int ijk[3] = {i, j, k};
    if (ijk[d] != (hi ? n[d] - 1 : 0)) return -1;
    size_t f;
    if (d == 0) f = j + (size_t)n[1] * k;
    else if (d == 1) f = i + (size_t)n[0] * k;
    else f = i + (size_t)n[0] * j;
    return (long)(side_offset(n, s) + f);
}

static int any_dirichlet(const int dir[6]) {
    for (int s = 0; s < 6; s++)
        if (dir[s]) return 1;
    return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- limiter */

/* Levermore-Pomraning lambda(x) = (coth x - 1/x) / x. */
double or_lp_lambda(double x) {
    if (x < 1e-2) {
        double x2 = x * x;
        return 1.0 / 3.0 - x2 / 45.0 + 2.0 * x2 * x2 / 945.0;
    }
    return (1.0 / tanh(x) - 1.0 / x) / x;
}

/* Diffusion coefficient D on the face between two cells (Sec. 2):
 * E1, E2 the cell energies, k1, k2 the cell opacities, h the spacing
 * normal to the face. */
double or_face_D(double E1, double E2, double k1, double k2, double h,
                 const or_phys* p) {
    double Dmax = p->dmax_coef * p->c * p->L_unit;
    double Rmin = p->rmin_coef / p->L_unit;
    double Ef = 0.5 * (E1 + E2);                       /* arithmetic mean */
    double kf = (k1 > 0.0 && k2 > 0.0) ? 2.0 * k1 * k2 / (k1 + k2) : 0.0;
    double R;
    if (Ef > 0.0) {
        R = fabs(E2 - E1) / (h * Ef);
        if (R < Rmin) R = Rmin;
    } else {
        R = (E2 == E1) ? Rmin : 1e300;
    }
    double D;
    if (p->limiter == OR_LIMITER_LP) {
        if (kf == 0.0) {
            D = p->c / R;
        } else {
            double x = R / kf;
            if (x > 1e8) D = p->c / R;
            else D = p->c * or_lp_lambda(x) / kf;
        }
    } else {
        D = p->c / sqrt(9.0 * kf * kf + R * R);
    }
    return D < Dmax ? D : Dmax;
}

/* --------------------------------------------------------------- assembly */

static int valid_grid(const or_grid* g) {
    for (int d = 0; d < 3; d++) {
        if (g->n[d] < 1 || !(g->h[d] > 0.0)) return 0;
        if (g->periodic[d] && (g->dirichlet[2 * d] || g->dirichlet[2 * d + 1])) return 0;
    }
    for (int s = 0; s < 6; s++)
        if (g->dirichlet[s] && !(isfinite(g->ebc[s]) && g->ebc[s] >= 0.0)) return 0;
    return 1;
}

/* Build m, wx, wy, wz, the packed Dirichlet face weights bnd (may be NULL
 * when the grid has no Dirichlet side) and the right-hand side b of the
 * theta-method correction system A dE = b (Sec. 3.2), with the proper cell
 * widths h_d = a * (comoving width):
 *   w_f  = theta dt D_f / h_d^2                      (interior faces)
 *   w_b  = theta dt D_b / (h_d h_d / 2)              (Dirichlet faces)
 *   m_i  = 1 + theta dt (c kappa_i + adot/a) + sum of the cell's w_b
 *   b_i  = dt eta_i - dt (c kappa_i + adot/a) E_i
 *          + sum_f (w_f / theta) (E_nbr - E_i) + sum_b (w_b / theta) (E_b - E_i),
 * i.e. b = dt F(E^n) with the unscaled weights and A = I - theta dt L. */
int or_assemble(const or_grid* g, const or_phys* p, const double* E,
                const double* nHI, const double* eta, double* m, double* wx,
                double* wy, double* wz, double* b, double* bnd) {
    if (!valid_grid(g) || !(p->dt > 0.0) || p->sigma < 0.0) return OR_EINVAL;
    if (!(p->theta > 0.0 && p->theta <= 1.0)) return OR_EINVAL;
    if (!(p->a > 0.0 && isfinite(p->a))) return OR_EINVAL;
    if (any_dirichlet(g->dirichlet) && !bnd) return OR_EINVAL;
    const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
    const double th = p->theta;
    const double hp[3] = {p->a * g->h[0], p->a * g->h[1], p->a * g->h[2]};
    size_t N = ncell(g->n);
    for (size_t i = 0; i < N; i++)
        if (!(E[i] >= 0.0) || !(nHI[i] >= 0.0) || !(eta[i] >= 0.0) ||
            !isfinite(E[i]) || !isfinite(nHI[i]) || !isfinite(eta[i]))
            return OR_EINVAL;
    if (bnd) memset(bnd, 0, or_bnd_size(g->n) * sizeof(double));
    double* w[3] = {wx, wy, wz};
    const size_t stride[3] = {1, (size_t)nx, (size_t)nx * ny};
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int ijk[3] = {i, j, k};
                size_t c = i + (size_t)nx * (j + (size_t)ny * k);
                double kap = nHI[c] * p->sigma;
                double mass = 1.0 + th * p->dt * (p->c * kap + p->adot);
                for (int d = 0; d < 3; d++) {
                    size_t lo;
                    int has = 1;
                    if (ijk[d] > 0) lo = c - stride[d];
                    else if (g->periodic[d]) lo = c + (size_t)(g->n[d] - 1) * stride[d];
                    else { has = 0; lo = c; }
                    if (!has) { w[d][c] = 0.0; continue; }
                    double D = or_face_D(E[lo], E[c], nHI[lo] * p->sigma, kap,
                                         hp[d], p);
                    w[d][c] = th * p->dt * D / (hp[d] * hp[d]);
                }
                for (int sd = 0; sd < 6; sd++) {
                    if (!g->dirichlet[sd]) continue;
                    long f = side_face(g->n, sd, i, j, k);
                    if (f < 0) continue;
                    double h = hp[sd / 2];
                    double D = or_face_D(g->ebc[sd], E[c], kap, kap, 0.5 * h, p);
                    double wb = th * p->dt * D / (h * 0.5 * h);
                    bnd[f] = wb;
                    mass += wb;
                }
                m[c] = mass;
            }
    /* b needs every face weight, so it is a second pass. */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int ijk[3] = {i, j, k};
                size_t c = i + (size_t)nx * (j + (size_t)ny * k);
                double kap = nHI[c] * p->sigma;
                double flux = 0.0;
                for (int d = 0; d < 3; d++) {
                    /* lower face */
                    if (ijk[d] > 0)
                        flux += w[d][c] / th * (E[c - stride[d]] - E[c]);
                    else if (g->periodic[d])
                        flux += w[d][c] / th * (E[c + (size_t)(g->n[d] - 1) * stride[d]] - E[c]);
                    /* upper face */
                    if (ijk[d] < g->n[d] - 1)
                        flux += w[d][c + stride[d]] / th * (E[c + stride[d]] - E[c]);
                    else if (g->periodic[d]) {
                        size_t up = c - (size_t)(g->n[d] - 1) * stride[d];
                        flux += w[d][up] / th * (E[up] - E[c]);
                    }
                }
                for (int sd = 0; sd < 6; sd++) {
                    if (!g->dirichlet[sd]) continue;
                    long f = side_face(g->n, sd, i, j, k);
                    if (f >= 0) flux += bnd[f] / th * (g->ebc[sd] - E[c]);
                }
                b[c] = p->dt * eta[c] - p->dt * (p->c * kap + p->adot) * E[c] + flux;
            }
    return OR_OK;
}

/* ------------------------------------------------------- operator on a level */

/* Visit the (up to) six faces of cell c: weight and neighbour index. */
typedef struct { int cnt; double w[6]; size_t nb[6]; } faces6;

static void cell_faces(const or_level* L, int i, int j, int k, faces6* f) {
    const int n[3] = {L->n[0], L->n[1], L->n[2]};
    const size_t stride[3] = {1, (size_t)n[0], (size_t)n[0] * n[1]};
    const double* w[3] = {L->wx, L->wy, L->wz};
    int ijk[3] = {i, j, k};
    size_t c = i + (size_t)n[0] * (j + (size_t)n[1] * k);
    f->cnt = 0;
    for (int d = 0; d < 3; d++) {
        if (ijk[d] > 0) {
            f->w[f->cnt] = w[d][c]; f->nb[f->cnt] = c - stride[d]; f->cnt++;
        } else if (L->periodic[d]) {
            f->w[f->cnt] = w[d][c]; f->nb[f->cnt] = c + (size_t)(n[d] - 1) * stride[d]; f->cnt++;
        }
        if (ijk[d] < n[d] - 1) {
            f->w[f->cnt] = w[d][c + stride[d]]; f->nb[f->cnt] = c + stride[d]; f->cnt++;
        } else if (L->periodic[d]) {
            size_t up = c - (size_t)(n[d] - 1) * stride[d];
            f->w[f->cnt] = w[d][up]; f->nb[f->cnt] = up; f->cnt++;
        }
    }
}

/* y = A x */
static void level_apply(const or_level* L, const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < L->n[2]; k++)
        for (int j = 0; j < L->n[1]; j++)
            for (int i = 0; i < L->n[0]; i++) {
                size_t c = i + (size_t)L->n[0] * (j + (size_t)L->n[1] * k);
                faces6 f;
                cell_faces(L, i, j, k, &f);
                double s = L->m[c] * x[c];
                for (int q = 0; q < f.cnt; q++) s += f.w[q] * (x[c] - x[f.nb[q]]);
                y[c] = s;
            }
}

static double level_diag(const or_level* L, int i, int j, int k) {
    faces6 f;
    cell_faces(L, i, j, k, &f);
    size_t c = i + (size_t)L->n[0] * (j + (size_t)L->n[1] * k);
    double d = L->m[c];
    for (int q = 0; q < f.cnt; q++) d += f.w[q];
    return d;
}

static or_level fine_level(const or_grid* g, const double* m, const double* wx,
                           const double* wy, const double* wz) {
    or_level L;
    memset(&L, 0, sizeof(L));
    for (int d = 0; d < 3; d++) { L.n[d] = g->n[d]; L.periodic[d] = g->periodic[d]; }
    for (int s = 0; s < 6; s++) L.dirichlet[s] = g->dirichlet[s];
    L.m = (double*)m; L.wx = (double*)wx; L.wy = (double*)wy; L.wz = (double*)wz;
    L.owned = 0;
    L.bnd = NULL;
    return L;
}

void or_apply(const or_grid* g, const double* m, const double* wx,
              const double* wy, const double* wz, const double* x, double* y) {
    or_level L = fine_level(g, m, wx, wy, wz);
    level_apply(&L, x, y);
}

/* Dense matrix of a level, row-major n x n (n = number of cells). */
static void level_dense(const or_level* L, double* A) {
    size_t n = ncell(L->n);
    memset(A, 0, n * n * sizeof(double));
    for (int k = 0; k < L->n[2]; k++)
        for (int j = 0; j < L->n[1]; j++)
            for (int i = 0; i < L->n[0]; i++) {
                size_t c = i + (size_t)L->n[0] * (j + (size_t)L->n[1] * k);
                faces6 f;
                cell_faces(L, i, j, k, &f);
                A[c * n + c] += L->m[c];
                for (int q = 0; q < f.cnt; q++) {
                    A[c * n + c] += f.w[q];
                    A[c * n + f.nb[q]] -= f.w[q];
                }
            }
}

int or_dense_matrix(const or_grid* g, const double* m, const double* wx,
                    const double* wy, const double* wz, double* A) {
    or_level L = fine_level(g, m, wx, wy, wz);
    level_dense(&L, A);
    return OR_OK;
}

/* In-place Cholesky A = L L^T (lower triangle kept). */
static int cholesky(double* A, size_t n) {
    for (size_t j = 0; j < n; j++) {
        double s = A[j * n + j];
        for (size_t k = 0; k < j; k++) s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0)) return OR_EINVAL;
        double ljj = sqrt(s);
        A[j * n + j] = ljj;
        for (size_t i = j + 1; i < n; i++) {
            double t = A[i * n + j];
            for (size_t k = 0; k < j; k++) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / ljj;
        }
    }
    return OR_OK;
}

static void cholesky_solve(const double* Lf, size_t n, const double* b, double* x) {
    for (size_t i = 0; i < n; i++) {            /* L y = b */
        double s = b[i];
        for (size_t k = 0; k < i; k++) s -= Lf[i * n + k] * x[k];
        x[i] = s / Lf[i * n + i];
    }
    for (size_t ii = n; ii-- > 0;) {            /* L^T x = y */
        double s = x[ii];
        for (size_t k = ii + 1; k < n; k++) s -= Lf[k * n + ii] * x[k];
        x[ii] = s / Lf[ii * n + ii];
    }
}

/* Brute force: solve A x = rhs with a dense Cholesky factorisation. */
int or_dense_solve(const or_grid* g, const double* m, const double* wx,
                   const double* wy, const double* wz, const double* rhs,
                   double* x) {
    size_t n = ncell(g->n);
    double* A = (double*)malloc(n * n * sizeof(double));
    if (!A) return OR_ENOMEM;
    or_level L = fine_level(g, m, wx, wy, wz);
    level_dense(&L, A);
    int st = cholesky(A, n);
    if (st == OR_OK) cholesky_solve(A, n, rhs, x);
    free(A);
    return st;
}

/* ------------------------------------------------------ multigrid pieces */

/* Sum of the Dirichlet face weights of cell (i,j,k) of a level. */
static double cell_bnd(const or_level* L, int i, int j, int k) {
    double sum = 0.0;
    if (!L->bnd) return 0.0;
    for (int s = 0; s < 6; s++) {
        if (!L->dirichlet[s]) continue;
        long f = side_face(L->n, s, i, j, k);
        if (f >= 0) sum += L->bnd[f];
    }
    return sum;
}

/* Coarse operator by rediscretisation: every coarse face weight (interior
 * or Dirichlet boundary) is the sum of the 4 fine weights across the coarse
 * face / 16; the coarse mass term is the mean of the 8 children's mass
 * terms (their m without their boundary weights) plus the coarse cell's own
 * boundary weights. */
static void coarsen(const or_level* F, or_level* C) {
    const int cx = C->n[0], cy = C->n[1], cz = C->n[2];
    const int fx = F->n[0], fy = F->n[1];
#define FI(i, j, k) ((size_t)(i) + (size_t)fx * ((size_t)(j) + (size_t)fy * (size_t)(k)))
    if (C->bnd) {
        memset(C->bnd, 0, or_bnd_size(C->n) * sizeof(double));
        for (int s = 0; s < 6; s++) {
            if (!C->dirichlet[s]) continue;
            int d = s / 2, hi = s % 2;
            /* the two coarse axes spanning the face, and the fine layer */
            int a0 = d == 0 ? 1 : 0, a1 = d == 2 ? 1 : 2;
            for (int v = 0; v < C->n[a1]; v++)
                for (int u = 0; u < C->n[a0]; u++) {
                    int cc[3], ff[3];
                    cc[d] = hi ? C->n[d] - 1 : 0;
                    cc[a0] = u; cc[a1] = v;
                    double sum = 0.0;
                    for (int q = 0; q < 2; q++)
                        for (int r = 0; r < 2; r++) {
                            ff[d] = hi ? F->n[d] - 1 : 0;
                            ff[a0] = 2 * u + q; ff[a1] = 2 * v + r;
                            sum += F->bnd[side_face(F->n, s, ff[0], ff[1], ff[2])];
                        }
                    C->bnd[side_face(C->n, s, cc[0], cc[1], cc[2])] = sum / 16.0;
                }
        }
    }
#pragma omp parallel for schedule(static)
    for (int K = 0; K < cz; K++)
        for (int J = 0; J < cy; J++)
            for (int I = 0; I < cx; I++) {
                size_t c = I + (size_t)cx * (J + (size_t)cy * K);
                double msum = 0.0;
                for (int dk = 0; dk < 2; dk++)
                    for (int dj = 0; dj < 2; dj++)
                        for (int di = 0; di < 2; di++) {
                            int fi = 2 * I + di, fj = 2 * J + dj, fk = 2 * K + dk;
                            msum += F->m[FI(fi, fj, fk)] - cell_bnd(F, fi, fj, fk);
                        }
                C->m[c] = msum / 8.0 + cell_bnd(C, I, J, K);
                double sx = 0.0, sy = 0.0, sz = 0.0;
                for (int a = 0; a < 2; a++)
                    for (int bb = 0; bb < 2; bb++) {
                        sx += F->wx[FI(2 * I, 2 * J + a, 2 * K + bb)];
                        sy += F->wy[FI(2 * I + a, 2 * J, 2 * K + bb)];
                        sz += F->wz[FI(2 * I + a, 2 * J + bb, 2 * K)];
                    }
                C->wx[c] = sx / 16.0;
                C->wy[c] = sy / 16.0;
                C->wz[c] = sz / 16.0;
            }
#undef FI
}

/* Trilinear prolongation weights along one axis for fine index i:
 * the two coarse cells it interpolates from and their weights. */
static void prolong_axis(int i, int nc, int periodic, int* I0, int* I1,
                         double* a0, double* a1) {
    int I = i / 2;
    int J = (i % 2 == 0) ? I - 1 : I + 1;   /* the farther coarse neighbour */
    if (J < 0) J = periodic ? nc - 1 : I;   /* ghost cell */
    if (J >= nc) J = periodic ? 0 : I;
    *I0 = I; *I1 = J; *a0 = 0.75; *a1 = 0.25;
}

/* zf += P ec */
static void prolong_add(const or_level* F, const or_level* C, const double* ec,
                        double* zf) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < F->n[2]; k++)
        for (int j = 0; j < F->n[1]; j++)
            for (int i = 0; i < F->n[0]; i++) {
                int Ix[2], Iy[2], Iz[2];
                double ax[2], ay[2], az[2];
                prolong_axis(i, C->n[0], C->periodic[0], &Ix[0], &Ix[1], &ax[0], &ax[1]);
                prolong_axis(j, C->n[1], C->periodic[1], &Iy[0], &Iy[1], &ay[0], &ay[1]);
                prolong_axis(k, C->n[2], C->periodic[2], &Iz[0], &Iz[1], &az[0], &az[1]);
                double s = 0.0;
                for (int c = 0; c < 2; c++)
                    for (int b = 0; b < 2; b++)
                        for (int a = 0; a < 2; a++)
                            s += ax[a] * ay[b] * az[c] *
                                 ec[Ix[a] + (size_t)C->n[0] * (Iy[b] + (size_t)C->n[1] * Iz[c])];
                zf[i + (size_t)F->n[0] * (j + (size_t)F->n[1] * k)] += s;
            }
}

/* rc = (1/8) P^T rf : the literal transpose of prolong_add. */
static void restrict_fw(const or_level* F, const or_level* C, const double* rf,
                        double* rc) {
    memset(rc, 0, ncell(C->n) * sizeof(double));
    for (int k = 0; k < F->n[2]; k++)
        for (int j = 0; j < F->n[1]; j++)
            for (int i = 0; i < F->n[0]; i++) {
                int Ix[2], Iy[2], Iz[2];
                double ax[2], ay[2], az[2];
                prolong_axis(i, C->n[0], C->periodic[0], &Ix[0], &Ix[1], &ax[0], &ax[1]);
                prolong_axis(j, C->n[1], C->periodic[1], &Iy[0], &Iy[1], &ay[0], &ay[1]);
                prolong_axis(k, C->n[2], C->periodic[2], &Iz[0], &Iz[1], &az[0], &az[1]);
                double v = rf[i + (size_t)F->n[0] * (j + (size_t)F->n[1] * k)] / 8.0;
                for (int c = 0; c < 2; c++)
                    for (int b = 0; b < 2; b++)
                        for (int a = 0; a < 2; a++)
                            rc[Ix[a] + (size_t)C->n[0] * (Iy[b] + (size_t)C->n[1] * Iz[c])] +=
                                ax[a] * ay[b] * az[c] * v;
            }
}

/* One Gauss-Seidel half sweep over the cells of one colour:
 * z_i = (r_i + sum_f w_f z_nbr) / (m_i + sum_f w_f). */
static void gs_colour(const or_level* L, const double* r, double* z, int colour) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < L->n[2]; k++)
        for (int j = 0; j < L->n[1]; j++)
            for (int i = 0; i < L->n[0]; i++) {
                if (((i + j + k) & 1) != colour) continue;
                size_t c = i + (size_t)L->n[0] * (j + (size_t)L->n[1] * k);
                faces6 f;
                cell_faces(L, i, j, k, &f);
                double s = r[c], d = L->m[c];
                for (int q = 0; q < f.cnt; q++) { s += f.w[q] * z[f.nb[q]]; d += f.w[q]; }
                z[c] = s / d;
            }
}

/* Weighted Jacobi: z <- z + omega (r - A z) / diag (all cells at once). */
static void jacobi_sweep(const or_level* L, const double* r, double* z,
                         double omega, double* tmp) {
    size_t n = ncell(L->n);
    level_apply(L, z, tmp);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < L->n[2]; k++)
        for (int j = 0; j < L->n[1]; j++)
            for (int i = 0; i < L->n[0]; i++) {
                size_t c = i + (size_t)L->n[0] * (j + (size_t)L->n[1] * k);
                tmp[c] = z[c] + omega * (r[c] - tmp[c]) / level_diag(L, i, j, k);
            }
    memcpy(z, tmp, n * sizeof(double));
}

typedef struct {
    int nl;
    or_level lev[OR_MAX_LEVELS];
    double* chol;               /* dense factor of the coarsest operator */
    double *res[OR_MAX_LEVELS], *rc[OR_MAX_LEVELS], *zc[OR_MAX_LEVELS];
    double* tmp[OR_MAX_LEVELS];
} or_hier;

static void hier_free(or_hier* H) {
    for (int l = 0; l < H->nl; l++) {
        if (H->lev[l].owned) {
            free(H->lev[l].m); free(H->lev[l].wx); free(H->lev[l].wy); free(H->lev[l].wz);
            free(H->lev[l].bnd);
        }
        free(H->res[l]); free(H->rc[l]); free(H->zc[l]); free(H->tmp[l]);
    }
    free(H->chol);
    memset(H, 0, sizeof(*H));
}

/* Coarsening rule: halve every dimension while all are even and the
 * smallest exceeds 4. */
static int coarsenable(const int n[3]) {
    int mn = n[0] < n[1] ? n[0] : n[1];
    if (n[2] < mn) mn = n[2];
    return mn > 4 && n[0] % 2 == 0 && n[1] % 2 == 0 && n[2] % 2 == 0;
}

int or_num_levels(const int n[3], int* dims_out) {
    int d[3] = {n[0], n[1], n[2]};
    int nl = 0;
    for (;;) {
        if (dims_out) { dims_out[3 * nl] = d[0]; dims_out[3 * nl + 1] = d[1]; dims_out[3 * nl + 2] = d[2]; }
        nl++;
        if (!coarsenable(d) || nl >= OR_MAX_LEVELS) break;
        d[0] /= 2; d[1] /= 2; d[2] /= 2;
    }
    return nl;
}

static int hier_build(or_hier* H, const or_grid* g, const double* m,
                      const double* wx, const double* wy, const double* wz,
                      const double* bnd, int coarse_cap) {
    memset(H, 0, sizeof(*H));
    int dir = any_dirichlet(g->dirichlet);
    if (dir && !bnd) return OR_EINVAL;
    H->lev[0] = fine_level(g, m, wx, wy, wz);
    H->lev[0].bnd = (double*)bnd;
    H->nl = 1;
    while (coarsenable(H->lev[H->nl - 1].n) && H->nl < OR_MAX_LEVELS) {
        or_level* F = &H->lev[H->nl - 1];
        or_level* C = &H->lev[H->nl];
        for (int d = 0; d < 3; d++) { C->n[d] = F->n[d] / 2; C->periodic[d] = F->periodic[d]; }
        for (int sd = 0; sd < 6; sd++) C->dirichlet[sd] = F->dirichlet[sd];
        size_t nc = ncell(C->n);
        C->m = (double*)malloc(nc * sizeof(double));
        C->wx = (double*)malloc(nc * sizeof(double));
        C->wy = (double*)malloc(nc * sizeof(double));
        C->wz = (double*)malloc(nc * sizeof(double));
        C->bnd = dir ? (double*)malloc(or_bnd_size(C->n) * sizeof(double)) : NULL;
        C->owned = 1;
        H->nl++;
        if (!C->m || !C->wx || !C->wy || !C->wz || (dir && !C->bnd)) { hier_free(H); return OR_ENOMEM; }
        coarsen(F, C);
    }
    for (int l = 0; l < H->nl; l++) {
        size_t n = ncell(H->lev[l].n);
        H->res[l] = (double*)malloc(n * sizeof(double));
        H->rc[l] = (double*)malloc(n * sizeof(double));
        H->zc[l] = (double*)malloc(n * sizeof(double));
        H->tmp[l] = (double*)malloc(n * sizeof(double));
        if (!H->res[l] || !H->rc[l] || !H->zc[l] || !H->tmp[l]) { hier_free(H); return OR_ENOMEM; }
    }
    or_level* Lc = &H->lev[H->nl - 1];
    size_t nc = ncell(Lc->n);
    if ((long)nc > coarse_cap) { hier_free(H); return OR_EINVAL; }
    H->chol = (double*)malloc(nc * nc * sizeof(double));
    if (!H->chol) { hier_free(H); return OR_ENOMEM; }
    level_dense(Lc, H->chol);
    int st = cholesky(H->chol, nc);
    if (st != OR_OK) { hier_free(H); return st; }
    return OR_OK;
}

/* z = V-cycle(level l) applied to r. */
static void vcycle(or_hier* H, int l, const double* r, double* z,
                   const or_solver* s) {
    or_level* L = &H->lev[l];
    size_t n = ncell(L->n);
    if (l == H->nl - 1) {
        cholesky_solve(H->chol, n, r, z);
        return;
    }
    memset(z, 0, n * sizeof(double));
    for (int it = 0; it < s->pre; it++) {
        if (s->smoother == OR_SMOOTH_RBGS) { gs_colour(L, r, z, 0); gs_colour(L, r, z, 1); }
        else jacobi_sweep(L, r, z, s->omega, H->tmp[l]);
    }
    double* res = H->res[l];
    level_apply(L, z, res);
    for (size_t i = 0; i < n; i++) res[i] = r[i] - res[i];
    or_level* C = &H->lev[l + 1];
    restrict_fw(L, C, res, H->rc[l + 1]);
    vcycle(H, l + 1, H->rc[l + 1], H->zc[l + 1], s);
    prolong_add(L, C, H->zc[l + 1], z);
    for (int it = 0; it < s->post; it++) {
        if (s->smoother == OR_SMOOTH_RBGS && s->paper_order) { gs_colour(L, r, z, 0); gs_colour(L, r, z, 1); }
        else if (s->smoother == OR_SMOOTH_RBGS) { gs_colour(L, r, z, 1); gs_colour(L, r, z, 0); }
        else jacobi_sweep(L, r, z, s->omega, H->tmp[l]);
    }
}

/* One V-cycle with zero initial guess: z = B r. */
int or_vcycle(const or_grid* g, const double* m, const double* wx,
              const double* wy, const double* wz, const double* bnd,
              const double* r, double* z, const or_solver* s) {
    or_hier H;
    int st = hier_build(&H, g, m, wx, wy, wz, bnd, s->coarse_cap);
    if (st) return st;
    vcycle(&H, 0, r, z, s);
    hier_free(&H);
    return OR_OK;
}

/* Exposed pieces of the cycle, for tests of the transfer operators.
 * dirichlet may be NULL (no Dirichlet side); bnd and bndc are the packed
 * boundary weights of the fine and coarse level (used when dirichlet has a
 * side set). */
static or_level bare_level(const int n[3], const int periodic[3], const int* dirichlet) {
    or_level L;
    memset(&L, 0, sizeof(L));
    for (int d = 0; d < 3; d++) { L.n[d] = n[d]; L.periodic[d] = periodic[d]; }
    if (dirichlet)
        for (int s = 0; s < 6; s++) L.dirichlet[s] = dirichlet[s];
    return L;
}

int or_coarsen(const int nf[3], const int periodic[3], const int* dirichlet,
               const double* m, const double* wx, const double* wy, const double* wz,
               const double* bnd, double* mc, double* wxc, double* wyc, double* wzc,
               double* bndc) {
    const int nc[3] = {nf[0] / 2, nf[1] / 2, nf[2] / 2};
    or_level F = bare_level(nf, periodic, dirichlet);
    or_level C = bare_level(nc, periodic, dirichlet);
    F.m = (double*)m; F.wx = (double*)wx; F.wy = (double*)wy; F.wz = (double*)wz;
    C.m = mc; C.wx = wxc; C.wy = wyc; C.wz = wzc;
    if (dirichlet && any_dirichlet(dirichlet)) {
        if (!bnd || !bndc) return OR_EINVAL;
        F.bnd = (double*)bnd;
        C.bnd = bndc;
    }
    coarsen(&F, &C);
    return OR_OK;
}

int or_prolong_add(const int nf[3], const int periodic[3], const double* ec,
                   double* zf) {
    const int nc[3] = {nf[0] / 2, nf[1] / 2, nf[2] / 2};
    or_level F = bare_level(nf, periodic, NULL);
    or_level C = bare_level(nc, periodic, NULL);
    prolong_add(&F, &C, ec, zf);
    return OR_OK;
}

int or_restrict(const int nf[3], const int periodic[3], const double* rf,
                double* rc) {
    const int nc[3] = {nf[0] / 2, nf[1] / 2, nf[2] / 2};
    or_level F = bare_level(nf, periodic, NULL);
    or_level C = bare_level(nc, periodic, NULL);
    restrict_fw(&F, &C, rf, rc);
    return OR_OK;
}

/* ------------------------------------------------------------------- PCG */

static double dot(const double* a, const double* b, size_t n) {
    double s = 0.0;
    for (size_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* Multigrid-preconditioned CG for A x = b (Table 1).  hist, if given,
 * receives ||r_k|| / ||b|| for k = 0..iters (max_iter + 1 entries). */
int or_pcg(const or_grid* g, const double* m, const double* wx,
           const double* wy, const double* wz, const double* bnd, const double* b,
           double* x, const or_solver* s, int* iters, double* rel_res, double* hist) {
    size_t n = ncell(g->n);
    memset(x, 0, n * sizeof(double));
    *iters = 0;
    *rel_res = 0.0;
    double bnorm = sqrt(dot(b, b, n));
    if (hist) hist[0] = bnorm > 0.0 ? 1.0 : 0.0;
    if (bnorm == 0.0) return OR_OK;
    or_hier H;
    int st = hier_build(&H, g, m, wx, wy, wz, bnd, s->coarse_cap);
    if (st) return st;
    double* r = (double*)malloc(n * sizeof(double));
    double* z = (double*)malloc(n * sizeof(double));
    double* p = (double*)malloc(n * sizeof(double));
    double* q = (double*)malloc(n * sizeof(double));
    if (!r || !z || !p || !q) { free(r); free(z); free(p); free(q); hier_free(&H); return OR_ENOMEM; }
    memcpy(r, b, n * sizeof(double));
    double rho_old = 0.0;
    int conv = 0, k;
    for (k = 1; k <= s->max_iter; k++) {
        vcycle(&H, 0, r, z, s);
        double rho = dot(r, z, n);
        if (k == 1) memcpy(p, z, n * sizeof(double));
        else {
            double beta = rho / rho_old;
            for (size_t i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        }
        level_apply(&H.lev[0], p, q);
        double alpha = rho / dot(p, q, n);
        for (size_t i = 0; i < n; i++) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        rho_old = rho;
        double rr = sqrt(dot(r, r, n)) / bnorm;
        if (hist) hist[k] = rr;
        if (rr <= s->rtol) { conv = 1; break; }
    }
    *iters = conv ? k : s->max_iter;
    /* report the true residual of the returned iterate */
    level_apply(&H.lev[0], x, q);
    for (size_t i = 0; i < n; i++) q[i] = b[i] - q[i];
    *rel_res = sqrt(dot(q, q, n)) / bnorm;
    free(r); free(z); free(p); free(q);
    hier_free(&H);
    return conv ? OR_OK : OR_ENOCONV;
}

/* ------------------------------------------------------------ full step */

/* info[0] iters, [1] true ||b - A dE|| / ||b||, [2] photon imbalance
 * (photons), [3] imbalance relative to the step's photon budget,
 * [4] photons emitted in the step, [5] photons absorbed in the step,
 * [6] photons added by the E >= 0 floor, [7] relative change of the step
 * ||E^{n+1} - E^n||_2 / ||E^{n+1}||_2 (on the floored E^{n+1}),
 * [8] photons that left through Dirichlet faces (negative: entered).
 * With the theta-method every loss term is taken at
 * theta E^{n+1} + (1 - theta) E^n = E^n + theta dE, so the balance
 *   sum_i [dE_i - dt eta_i + dt (c kappa_i + adot/a)(E^n_i + theta dE_i)]
 *   + sum_b (w_b / theta)(E^n_i + theta dE_i - E_b)
 * vanishes up to the solver residual (the interior fluxes telescope). */
int or_step(const or_grid* g, const or_phys* p, const or_solver* s,
            const double* E, const double* nHI, const double* eta,
            double* E_new, double* info) {
    size_t n = ncell(g->n);
    size_t nb = any_dirichlet(g->dirichlet) ? or_bnd_size(g->n) : 0;
    double* buf = (double*)malloc((6 * n + nb) * sizeof(double));
    if (!buf) return OR_ENOMEM;
    double *m = buf, *wx = buf + n, *wy = buf + 2 * n, *wz = buf + 3 * n,
           *b = buf + 4 * n, *dE = buf + 5 * n, *bnd = nb ? buf + 6 * n : NULL;
    int st = or_assemble(g, p, E, nHI, eta, m, wx, wy, wz, b, bnd);
    if (st) { free(buf); return st; }
    int iters = 0;
    double rel = 0.0;
    st = or_pcg(g, m, wx, wy, wz, bnd, b, dE, s, &iters, &rel, NULL);
    if (st != OR_OK && st != OR_ENOCONV) { free(buf); return st; }
    const double th = p->theta;
    double V = g->h[0] * g->h[1] * g->h[2];
    double bal = 0.0, emit = 0.0, absorb = 0.0, floor_add = 0.0, dsq = 0.0, esq = 0.0;
    double out = 0.0, gross = 0.0;
    for (size_t i = 0; i < n; i++) {
        double En = E[i] + dE[i];
        double sink = p->dt * (p->c * nHI[i] * p->sigma + p->adot) * (E[i] + th * dE[i]);
        bal += dE[i] - (p->dt * eta[i] - sink);
        emit += p->dt * eta[i];
        absorb += sink;
        if (En < 0.0) floor_add -= En;
        double Ef = En < 0.0 ? 0.0 : En;
        dsq += dE[i] * dE[i];
        esq += Ef * Ef;
    }
    if (bnd)
        for (int k = 0; k < g->n[2]; k++)
            for (int j = 0; j < g->n[1]; j++)
                for (int i = 0; i < g->n[0]; i++)
                    for (int sd = 0; sd < 6; sd++) {
                        if (!g->dirichlet[sd]) continue;
                        long f = side_face(g->n, sd, i, j, k);
                        if (f < 0) continue;
                        size_t c = i + (size_t)g->n[0] * (j + (size_t)g->n[1] * k);
                        double fl = bnd[f] / th * (E[c] + th * dE[c] - g->ebc[sd]);
                        out += fl;
                        gross += fabs(fl);
                    }
    bal += out;
    if (st == OR_OK)
        for (size_t i = 0; i < n; i++) {
            double En = E[i] + dE[i];
            E_new[i] = En < 0.0 ? 0.0 : En;
        }
    double scale = V / p->hnu;
    double budget = emit > absorb ? emit : absorb;
    if (gross > budget) budget = gross;
    info[0] = iters;
    info[1] = rel;
    info[2] = bal * scale;
    info[3] = budget > 0.0 ? fabs(bal) / budget : fabs(bal);
    info[4] = emit * scale;
    info[5] = absorb * scale;
    info[6] = floor_add * scale;
    info[7] = esq > 0.0 ? sqrt(dsq / esq) : 0.0;
    info[8] = out * scale;
    free(buf);
    return st;
}

/* --------------------------------------------------- radiation subcycling */

/* Advance E over t_span in substeps (Sec. 3.3): a substep whose solve does
 * not converge is redone at 0.1 of its time step; after a successful one the
 * next time step is dt * clamp(tau_tol / change, 0.1, growth), change being
 * the relative change of the substep in the RMS norm (the estimator's
 * target tau_tol), kept within [dt_min, dt_max] (dt_max <= 0: unbounded) and
 * never past t_span.
 * out[0] substeps, [1] retries, [2] CG iterations, [3] time advanced,
 * [4] next time step. */
int or_advance(const or_grid* g, const or_phys* p0, const or_solver* s, double* E,
               const double* nHI, const double* eta, double t_span, double dt_first,
               double tau_tol, double dt_min, double dt_max, double growth,
               int max_substeps, double* out) {
    size_t n = ncell(g->n);
    double* En = (double*)malloc(n * sizeof(double));
    if (!En) return OR_ENOMEM;
    or_phys p = *p0;
    double t = 0.0, dt = dt_first;
    if (dt_max > 0.0 && dt > dt_max) dt = dt_max;
    int substeps = 0, retries = 0, iters = 0, st = OR_OK;
    while (t < t_span) {
        if (substeps + retries >= max_substeps) { st = OR_ENOCONV; break; }
        double rest = t_span - t;
        int last = dt >= rest * (1.0 - 1e-12);
        double dt_try = last ? rest : dt;
        p.dt = dt_try;
        double info[9];
        st = or_step(g, &p, s, E, nHI, eta, En, info);
        iters += (int)info[0];
        if (st == OR_ENOCONV) {
            retries++;
            dt = 0.1 * dt_try;
            if (dt < dt_min) break;
            st = OR_OK;
            continue;
        }
        if (st) break;
        memcpy(E, En, n * sizeof(double));
        t = last ? t_span : t + dt_try;
        substeps++;
        double f = info[7] > 0.0 ? tau_tol / info[7] : growth;
        dt = dt_try * (f < 0.1 ? 0.1 : (f > growth ? growth : f));
        if (dt_max > 0.0 && dt > dt_max) dt = dt_max;
        if (dt < dt_min) dt = dt_min;
    }
    out[0] = substeps; out[1] = retries; out[2] = iters; out[3] = t; out[4] = dt;
    free(En);
    return st;
}

/* ----------------------------------------------- opacity update between steps */

/* Hydrogen-only photoionisation / recombination update of the neutral
 * density after a radiation step: one linearly implicit backward-Euler
 * (Jacobi) update per cell, in the manner of the loosely coupled chemistry
 * solver (Sec. 3.2):
 *   Gamma = c sigma E / (h nu),
 *   x'    = (x + dt alpha_B n_H (1 - x)^2) / (1 + dt Gamma),  x = n_HI / n_H,
 * clamped to [1e-12, 1]; n_HI' = x' n_H. */
int or_opacity_update(size_t n, const double* E, const double* nH,
                      const double* nHI, double* nHI_out, double dt, double c,
                      double sigma, double hnu, double alpha_B) {
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)n; i++) {
        double x = nH[i] > 0.0 ? nHI[i] / nH[i] : 0.0;
        double gam = c * sigma * E[i] / hnu;
        double ion = 1.0 - x;
        double xn = (x + dt * alpha_B * nH[i] * ion * ion) / (1.0 + dt * gam);
        if (xn < 1e-12) xn = 1e-12;
        if (xn > 1.0) xn = 1.0;
        nHI_out[i] = xn * nH[i];
    }
    return OR_OK;
}
