/*
 * fld.h -- C ABI of libfld.so: one implicit grey flux-limited-diffusion (FLD)
 * radiation step on one GB300 GPU.
 *
 * The operation (Norman et al., arXiv:1306.0645):
 *   The radiation component of the operator split (Sec. 3.2, Eq. "fld"),
 *       dE/dt = div(D grad E) - (adot/a) E - c kappa E + eta,
 *   is advanced by the implicit theta-method of Sec. 3.2 (theta = 1
 *   backward Euler, the default; theta = 1/2 the trapezoidal rule) with the
 *   flux limiter D evaluated at E^n, which makes the step one linear system,
 *   posed for the correction dE = E^{n+1} - E^n.  D is the limiter of Sec. 2,
 *       D = min{ c (9 kappa_f^2 + R^2)^(-1/2), D_max },
 *       R = max{ |E_2 - E_1| / (h E_f), R_min },
 *   with face energy E_f the arithmetic mean and face opacity kappa_f the
 *   harmonic mean of the two cells, D_max = 0.006 c L_unit and
 *   R_min = 1e-20 / L_unit; or (FLD_LIMITER_LP) the Levermore-Pomraning
 *   form the paper cites (Sec. 1).  The opacity is kappa = n_HI sigma
 *   (Eq. "opacity", one species, monochromatic).  The system is solved by
 *   conjugate gradients preconditioned with a geometric multigrid V-cycle
 *   using red/black Gauss-Seidel, 1 pre- and 1 post-sweep, at most 50
 *   iterations to a relative residual of 1e-8 (Table 1).
 *
 * Discretisation (the library's reading where the paper is silent):
 *   cell-centred uniform grid, CGS units; face weight w_f = dt D_f / h_d^2;
 *   A dE = b with (A u)_i = m_i u_i + sum_f theta w_f (u_i - u_nbr),
 *   m_i = 1 + theta dt (c kappa_i + adot/a) + sum_b theta w_b,
 *   b_i = dt eta_i - dt (c kappa_i + adot/a) E_i + sum_f w_f (E_nbr - E_i)
 *         + sum_b w_b (E_b - E_i),
 *   the sums over b running over the cell's Dirichlet boundary faces.
 *   Boundaries, per face of the box (the tests of Sec. 4.1 use reflecting
 *   and outflow faces): reflecting (zero gradient) faces carry no flux;
 *   periodic axes wrap; a Dirichlet face holds E = E_b half a cell from the
 *   cell centre, its weight w_b = dt D_b / (h h/2) with D_b from the limiter
 *   at face energy (E_i + E_b)/2, normal difference |E_i - E_b| over h/2 and
 *   the cell's opacity; an outflow face is a Dirichlet face with E_b = 0,
 *   through which the limiter lets optically thin radiation stream out at
 *   |F| = c E_face.
 *   Multigrid: full 2x coarsening while all dimensions are even and the
 *   smallest exceeds 4; trilinear prolongation P, restriction P^T/8; coarse
 *   operators by rediscretisation (boundary face weights included); dense
 *   direct solve on the coarsest grid
 *   (at most fld_params.coarse_cap cells, else FLD_EINVAL).
 *
 * Conventions for every call:
 *   - Fields are contiguous FP64 arrays of nx*ny*nz cells, x fastest:
 *     idx = i + nx * (j + ny * k).  Field pointers are DEVICE pointers
 *     unless the function name ends in _host.  The caller owns them; the
 *     library never frees or retains them past the call.
 *   - The context owns its multigrid hierarchy and work buffers; they are
 *     allocated once in fld_create and reused by every step.
 *   - Work is enqueued on the stream given to fld_create.  Calls that
 *     return an fld_info synchronise that stream before returning.
 *   - No call throws across the ABI or traps on the device.  Every call
 *     returns an fld_status; fld_last_error() gives a message for the
 *     calling thread's most recent failure.
 */
#ifndef FLD_H
#define FLD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FLD_OK = 0,
    FLD_EINVAL = 1,      /* invalid argument; nothing was launched */
    FLD_ENOMEM = 2,      /* device or host allocation failed */
    FLD_ENOCONV = 3,     /* max_iter reached with ||r||/||b|| > rtol; E unchanged */
    FLD_ENONFINITE = 4,  /* NaN/Inf met in a reduction; E unchanged */
    FLD_ETIMEOUT = 5,    /* a bounded device-side wait gave up */
    FLD_ECUDA = 6        /* a CUDA runtime call failed */
} fld_status;

typedef enum { FLD_LIMITER_PAPER = 0, FLD_LIMITER_LP = 1 } fld_limiter;
typedef enum {
    FLD_BC_ZERO_GRADIENT = 0,  /* reflecting: no flux through the face */
    FLD_BC_PERIODIC = 1,       /* the axis wraps (both faces of the axis) */
    FLD_BC_DIRICHLET = 2,      /* E fixed to fld_grid.bc_value on the face */
    FLD_BC_OUTFLOW = 3         /* Dirichlet with E = 0: radiation leaves */
} fld_bc;
typedef enum { FLD_PREC_FP64 = 0, FLD_PREC_MIXED = 1 } fld_precision;
typedef enum { FLD_SMOOTH_RBGS = 0, FLD_SMOOTH_JACOBI = 1 } fld_smoother;

/* Grid: cells per axis (>= 1), cell widths in cm (> 0), boundary per face.
 * An axis is periodic when bc[a] is FLD_BC_PERIODIC, and bc_hi[a] must
 * then be FLD_BC_PERIODIC or 0.  Otherwise bc[a] governs the lower face
 * (x = 0, ...) and bc_hi[a] (not periodic) the upper face; a
 * zero-initialised bc_hi makes the upper faces reflecting. */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    int bc[3];                 /* fld_bc of the lower faces (x, y, z) */
    int bc_hi[3];              /* fld_bc of the upper faces */
    double bc_value[6];        /* E_b of Dirichlet faces, erg/cm^3, finite
                                  and >= 0, in the order x lo, x hi, y lo,
                                  y hi, z lo, z hi (others ignored) */
} fld_grid;

/* Physical and solver parameters.  fld_params_default fills the values of
 * the paper's solver (Table 1) and limiter constants (Sec. 2). */
typedef struct {
    double dt;                 /* time step, s (> 0) */
    double c;                  /* speed of light, cm/s */
    double L_unit;             /* length unit of D_max and R_min, cm */
    double dmax_coef;          /* D_max = dmax_coef * c * L_unit (0.006) */
    double rmin_coef;          /* R_min = rmin_coef / L_unit (1e-20) */
    double sigma;              /* grey cross-section, cm^2 (>= 0) */
    double adot_over_a;        /* cosmological sink adot/a, 1/s (>= 0) */
    double hnu;                /* erg per photon, for the photon balance */
    int limiter;               /* fld_limiter */
    int precision;             /* fld_precision */
    int smoother;              /* fld_smoother */
    double jacobi_omega;       /* weight of the Jacobi smoother (0.8) */
    double rtol;               /* ||b - A dE||_2 / ||b||_2 target (1e-8) */
    int max_iter;              /* CG iterations (50); in mixed mode the
                                  total of inner iterations */
    int pre, post;             /* smoothing sweeps per level (1, 1) */
    double inner_rtol;         /* mixed mode: inner FP32 solve target (1e-4) */
    int coarse_cap;            /* largest coarsest grid, cells (1024) */
    int graphs;                /* CUDA graphs (the whole CG solve as one
                                  device-side loop; per-iteration graphs in
                                  fld_step_batched): 1 on, 0 off, -1 auto
                                  (on; default).  Need a non-NULL stream:
                                  with the legacy default stream the solve
                                  launches its kernels one by one. */
    int fused_post;            /* mixed mode, RB-GS, post = 1: one fused
                                  black+red post-sweep kernel (1) or two
                                  colour sweeps (0, default, faster on
                                  GB300); same arithmetic */
    double theta;              /* time discretisation, in [1/2, 1]: 1
                                  backward Euler (default), 1/2 trapezoidal
                                  (Sec. 3.2) */
    double scale_factor;       /* cosmological expansion factor a (> 0,
                                  default 1).  Cell widths are comoving, the
                                  equation's gradients proper: the limiter
                                  and face weights use a * dx etc.  E and eta
                                  are per comoving volume (photon counts use
                                  the comoving cell volume), kappa proper. */
    int tail_cells;            /* red/black Gauss-Seidel: the levels from the
                                  first one with at most tail_cells cells
                                  down to the coarsest run as one persistent
                                  thread-block-cluster kernel per V-cycle
                                  (default 32768, at most 2^24; 0 = one
                                  launch per sweep);
                                  same arithmetic as the per-level kernels */
    int paper_order;           /* red/black Gauss-Seidel: 0 (default) post-
                                  sweeps black then red, so the V-cycle is a
                                  symmetric preconditioner; 1 red then black
                                  in the post-sweeps as in the pre-sweeps,
                                  Table 1's "nonsymmetric" relaxation */
    int persistent_cells;      /* mixed precision, red/black Gauss-Seidel: a
                                  fine grid of at most persistent_cells cells
                                  (and at most 12 levels) runs each inner
                                  FP32 MG-PCG solve as one persistent
                                  thread-block-cluster kernel (all V-cycle
                                  levels and the CG vector operations, same
                                  algorithm and stopping rule as Table 1's
                                  solver); fld_step_batched puts the inner
                                  solves of all such contexts in flight into
                                  one launch over a work list.  0 = never
                                  (default 0), at most 2^24 */
    int precond_bf16;          /* mixed precision, red/black Gauss-Seidel with
                                  one pre-sweep: 1 (default) the V-cycle
                                  smooths the fine level with its
                                  coefficients (face weights and inverse
                                  diagonal) stored as bfloat16, rounded from
                                  the FP32 operator, which halves their bytes
                                  in the smoothing and residual sweeps; the
                                  cycle stays symmetric, and the CG operator,
                                  the FP64 refinement residual and the
                                  stopping rule are unchanged, so only the
                                  preconditioner differs (by relative
                                  perturbations of its coefficients below
                                  2^-8).  0: FP32 coefficients */
} fld_params;

/* Result of one solve or step (host memory, filled on return). */
typedef struct {
    int status;                /* fld_status of the call */
    int iters;                 /* CG iterations (mixed: inner, summed) */
    int outer_iters;           /* mixed mode: refinement steps; else 0 */
    double rel_res;            /* ||b - A dE||_2 / ||b||_2 of the result,
                                  recomputed in FP64 */
    double balance_abs;        /* photons: sum_i V [dE_i - dt (eta_i -
                                  (c kappa_i + adot/a) E^theta_i)] / h nu
                                  + outflow, E^theta = E^n + theta dE */
    double balance_rel;        /* |balance_abs| / max(emitted, absorbed,
                                  photons through Dirichlet faces counted
                                  face by face in absolute value) */
    double emitted;            /* photons emitted in the step, V dt sum eta / h nu */
    double absorbed;           /* photons absorbed in the step */
    double floor_added;        /* photons added by flooring E^{n+1} at 0 */
    double rel_change;         /* ||E^{n+1} - E^n||_2 / ||E^{n+1}||_2 */
    double ms;                 /* device time of the call, ms */
    double outflow;            /* photons that left through Dirichlet and
                                  outflow faces (negative: entered) */
} fld_info;

typedef struct fld_ctx fld_ctx;

/* Fill *p with defaults: c = 2.99792458e10, dmax_coef 0.006, rmin_coef 1e-20,
 * sigma 1.6e-18, hnu 13.6 eV, PAPER limiter, FP64, RB-GS, omega 0.8,
 * rtol 1e-8, max_iter 50, pre = post = 1, inner_rtol 1e-4, coarse_cap 1024,
 * graphs -1, fused_post 0, theta 1, scale_factor 1, tail_cells 32768,
 * paper_order 0.
 * dt and L_unit are set to 1e5 yr and 6.6 kpc and should be overwritten. */
fld_status fld_params_default(fld_params* p);

/* Device bytes a context for (g, p) allocates; 0 if (g, p) is invalid.
 * Used for admission against an HBM budget. */
size_t fld_footprint_bytes(const fld_grid* g, const fld_params* p);

/* Create a context: validates g and p, builds the level shapes and
 * allocates every device buffer.  cuda_stream is a cudaStream_t (NULL for
 * the legacy default stream) on which all later work of the context is
 * enqueued.  *ctx is NULL on failure. */
fld_status fld_create(fld_ctx** ctx, const fld_grid* g, const fld_params* p,
                      void* cuda_stream);

/* Per-cell opacity, per-face limiter and coefficients, and the right-hand
 * side b of the correction system (Sec. 2 limiter; Sec. 3.2 system), then
 * the coarse operators and the coarsest-grid factorisation.  E, n_HI, eta:
 * device, FP64, finite and >= 0 (checked on the device; FLD_EINVAL if not).
 * Asynchronous except for that check. */
fld_status fld_assemble(fld_ctx* ctx, const double* E, const double* n_HI,
                        const double* eta);

/* Solve A dE = b for the last assembled system by MG-preconditioned CG
 * (Table 1), in FP64 or mixed precision per fld_params.precision.  dE:
 * device, FP64, written on success (and on FLD_ENOCONV, with the last
 * iterate).  info (may be NULL) receives iteration counts and the true
 * relative residual. */
fld_status fld_solve(fld_ctx* ctx, double* dE, fld_info* info);

/* One full step: assemble, solve, and E <- max(E + dE, 0) in place
 * (device, FP64).  The floor removes negative values of the size the
 * solver tolerance allows, so the result is a valid input of the next step;
 * info->floor_added reports what it added.  On any failure E is left
 * unchanged.  info (may be NULL) also receives the photon balance of the
 * step, evaluated on E + dE before the floor. */
fld_status fld_step(fld_ctx* ctx, double* E, const double* n_HI,
                    const double* eta, fld_info* info);

/* fld_step with HOST arrays: copies E, n_HI, eta to the context's device
 * staging buffers, steps, and copies E back.  Host arrays may be pageable
 * or pinned; pinned memory gives full copy bandwidth.  From 128^3 cells on
 * a non-periodic z axis the inputs travel in chunks of planes and each
 * chunk is assembled as soon as it has arrived, so the transfer overlaps
 * the assembly; E comes out as from fld_step (bit for bit when the
 * iteration counts agree; ||b||^2 is summed per chunk).  The call returns
 * when E is back in host memory, also on failure (no transfer from the
 * caller's buffers outlives the call). */
fld_status fld_step_host(fld_ctx* ctx, double* E, const double* n_HI,
                         const double* eta, fld_info* info);

/* Change the time step of the context (the operator depends on dt). */
fld_status fld_set_dt(fld_ctx* ctx, double dt);

/* Cosmological expansion between steps (Sec. 3.2, the adot/a term of Eq.
 * "fld" in comoving coordinates): set the scale factor a (> 0) and adot/a
 * (>= 0, 1/s) for the following steps.  The hierarchy and buffers are kept;
 * the next assembly takes the new values.  FLD_EINVAL leaves them unchanged. */
fld_status fld_set_expansion(fld_ctx* ctx, double scale_factor, double adot_over_a);

/* Radiation subcycling (Sec. 3.3): advance E over t_span in substeps.
 * A substep whose solve fails (FLD_ENOCONV or FLD_ENONFINITE) is retried at
 * 0.1 of its time step, leaving E as it was; after a successful substep the
 * next one is dt * clamp(tau_tol / rel_change, 0.1, growth) (rel_change of
 * fld_info, the relative change per step in the RMS norm), within
 * [dt_min, dt_max] and never past t_span.  Fails with the substep's status
 * when dt falls below dt_min or after max_substeps substeps. */
typedef struct {
    double tau_tol;            /* target relative change per substep (1e-4) */
    double dt_min, dt_max;     /* s; dt_max <= 0: no upper bound */
    double growth;             /* largest factor between substeps (2) */
    int max_substeps;          /* (10000) */
} fld_advance_params;

typedef struct {
    int status;
    int substeps;              /* successful substeps */
    int retries;               /* failed attempts redone at 0.1 dt */
    int iters;                 /* CG iterations summed over all attempts */
    double t_done;             /* time advanced (t_span on success) */
    double dt_next;            /* suggested first dt of the next call */
    double ms;                 /* wall time of the call, ms */
} fld_advance_info;

fld_status fld_advance(fld_ctx* ctx, double* E, const double* n_HI, const double* eta,
                       double t_span, double dt_first, const fld_advance_params* ap,
                       fld_advance_info* info);

/* Step n independent contexts whose work may overlap on the device.  Each
 * context's work runs on a private stream of the context (created on first
 * use), after the work already enqueued on the context's stream and before
 * any work enqueued there later, so contexts sharing one stream still
 * overlap; the call returns once every step has finished.  The inner solves
 * of contexts with persistent_cells set go to the device as one launch per
 * round (a work list), the others as device-side CG loops.  infos[i]
 * receives context i's result.  Returns FLD_OK if every step succeeded,
 * else the first failing status (the other steps still complete). */
fld_status fld_step_batched(int n, fld_ctx** ctxs, double** E,
                            const double** n_HI, const double** eta,
                            fld_info* infos);

/* Apply the assembled operator: y = A x (device, FP64).  For tests. */
fld_status fld_apply(fld_ctx* ctx, const double* x, double* y);

/* One multigrid V-cycle with zero initial guess, z = B r, on the assembled
 * hierarchy in the context's solver precision (device, FP64 arguments; a
 * mixed-precision context runs its FP32 cycle on r rounded to FP32, with the
 * bfloat16 smoothing coefficients where precond_bf16 gives them, and uses
 * its CG work vectors).  For tests. */
fld_status fld_vcycle(fld_ctx* ctx, const double* r, double* z);

/* Copy the assembled fine-level operator and right-hand side to caller
 * device buffers (any pointer may be NULL).  For tests. */
fld_status fld_get_system(fld_ctx* ctx, double* m, double* wx, double* wy,
                          double* wz, double* b);

/* Hydrogen-only photoionisation/recombination update of the neutral
 * density between steps, one linearly implicit backward-Euler iteration
 * per cell in the manner of the loosely coupled chemistry solver
 * (Sec. 3.2): Gamma = c sigma E / h nu,
 * x' = (x + dt alpha_B n_H (1 - x)^2) / (1 + dt Gamma), x = n_HI / n_H,
 * clamped to [1e-12, 1]; n_HI_out = x' n_H.  All arrays device FP64 of
 * n cells; n_HI_out may alias n_HI.  Enqueued on cuda_stream. */
fld_status fld_opacity_update(size_t n, const double* E, const double* n_H,
                              const double* n_HI, double* n_HI_out,
                              double dt, double c, double sigma, double hnu,
                              double alpha_B, void* cuda_stream);

/* FP64 residual r = b - A x of a 7-point operator (m, wx, wy, wz in the
 * layout of fld_get_system) and, into norms[0] and norms[1], ||r||_2^2 and
 * max |r|, for callers that cannot allocate device memory: programs whose
 * device memory is owned by another allocator, and latency-critical loops
 * where cudaMalloc may synchronise the device.  The paper has no
 * counterpart; this is a service entry point of the library.
 * Nothing is allocated: the reduction's scratch is a fixed file-scope device
 * array (about 257 KB, held by every GPU that loads the library until exit)
 * whose address the first call on each device looks up, with that device
 * current; make that first call before any stream capture.  Grids with more
 * than 4194304 cells in an x-y plane (or 2^33 cells) are rejected with
 * FLD_EINVAL.  All device pointers: m, wx, wy, wz, b, x read (nx*ny*nz
 * FP64 each), r written (may be NULL), norms written (2 FP64).  Work is
 * enqueued on cuda_stream and is asynchronous.  All calls share the scratch
 * and each clears what must start at zero; calls that overlap on the GPU
 * race. */
fld_status fld_residual_noalloc(const fld_grid* g, const double* m, const double* wx,
                                const double* wy, const double* wz, const double* b,
                                const double* x, double* r, double* norms, void* cuda_stream);

/* ---- Spectral model (Sec. 2, "Model coupling"): grey and multigroup
 * integrals of the assumed spectrum chi(nu) and the fields built from them.
 *
 * For frequency groups g = [edges[g], edges[g+1]] (a grey field is the one
 * group [nu_1, nu_max]; nu_max reads the paper's "infinity") and species
 * i = HI, HeI, HeII with thresholds nu_i, row g of the coefficient table is
 *   K_g0..2 = int sigma_i chi dnu / N_g              (Eq. "opacity")
 *   P_g0..2 = int sigma_i chi / nu dnu / N_g         (Eq. "photoionization")
 *   H_g0..2 = int sigma_i chi (1 - nu_i/nu) dnu / N_g (Eq. "photoheating")
 *   F_g     = N_g / N                                (share of the emissivity)
 * with N_g = int_g chi dnu, N = int over all groups, the species integrals
 * from max(edges[g], nu_i).  The normalisation starts at the group's lower
 * edge for all three (the paper prints nu_i in the opacity's denominator;
 * photons below nu_i are part of E but species i cannot absorb them).
 * Cross sections: sigma_0 [beta (nu/nu_i)^-s + (1-beta) (nu/nu_i)^(-s-1)],
 * nu >= nu_i (defaults: the Osterbrock 1989 fits the paper cites). */
typedef enum { FLD_SED_MONO = 0, FLD_SED_BLACKBODY = 1, FLD_SED_POWERLAW = 2 } fld_sed_kind;
#define FLD_MAX_GROUPS 16
#define FLD_SED_NCOEF 10

typedef struct {
    double nu_threshold;       /* Hz */
    double sigma0;             /* cm^2 at threshold */
    double beta, s;            /* shape of the fit */
} fld_xsec;

typedef struct {
    int kind;                  /* fld_sed_kind */
    double nu_mono;            /* Hz, line frequency (FLD_SED_MONO) */
    double T;                  /* K, blackbody chi ~ nu^3 / (exp(h nu/kT) - 1) */
    double alpha;              /* power law chi ~ nu^-alpha */
    fld_xsec species[3];       /* HI, HeI, HeII */
} fld_sed;

/* Blackbody at 1e5 K (alpha 1.5, nu_mono = nu_HI for the other kinds) with
 * the Osterbrock fits: HI (13.6 eV, 6.30e-18, 1.34, 2.99), HeI (24.6 eV,
 * 7.83e-18, 1.66, 2.05), HeII (54.4 eV, 1.58e-18, 1.34, 2.99). */
fld_status fld_sed_default(fld_sed* sed);

/* The coefficient table of `groups` groups (1 .. FLD_MAX_GROUPS; edges is a
 * HOST array of groups + 1 increasing frequencies in Hz) into the HOST
 * array coef[groups * FLD_SED_NCOEF], row g = (K_g0..2, P_g0..2, H_g0..2,
 * F_g).  Computed on the GPU (composite Simpson in ln nu, 2^14 intervals per
 * integral; a line is evaluated at its frequency) on cuda_stream, which is
 * synchronised before the call returns.  Allocates a small device scratch
 * (stream-ordered) and frees it. */
fld_status fld_sed_integrals(const fld_sed* sed, const double* edges, int groups, double* coef,
                             void* cuda_stream);

/* Group opacities and emissivities in one pass over the cells:
 * kappa[g][c] = sum_i n_i[c] K_gi and eta_out[g][c] = F_g eta[c].
 * coef: HOST table of fld_sed_integrals.  n_HI, n_HeI, n_HeII, eta: DEVICE
 * arrays of n cells (n_HeI, n_HeII may be NULL for 0; eta may be NULL when
 * eta_out is NULL).  kappa, eta_out: HOST arrays of `groups` DEVICE
 * pointers (eta_out may be NULL).  A group opacity field passed to
 * fld_step as n_HI with fld_params.sigma = 1 makes it the step's kappa.
 * Asynchronous on cuda_stream. */
fld_status fld_group_fields(size_t n, int groups, const double* coef, const double* n_HI,
                            const double* n_HeI, const double* n_HeII, const double* eta,
                            double* const* kappa, double* const* eta_out, void* cuda_stream);

/* Photoionisation and photoheating rates from the group energies:
 * gamma_i[c] = sum_g (c_light / h) P_gi E_g[c] (1/s) and
 * heating[c] = sum_g c_light E_g[c] sum_i n_i[c] H_gi / rho_b[c] (erg/s/g).
 * E: HOST array of `groups` DEVICE pointers; the density and output arrays
 * are DEVICE arrays of n cells, any output may be NULL (heating needs
 * rho_b).  Asynchronous on cuda_stream. */
fld_status fld_photo_rates(size_t n, int groups, const double* coef, const double* const* E,
                           const double* n_HI, const double* n_HeI, const double* n_HeII,
                           const double* rho_b, double c_light, double* gamma_HI, double* gamma_HeI,
                           double* gamma_HeII, double* heating, void* cuda_stream);

/* Number of levels and their shapes (dims[3*l .. 3*l+2]) for grid g. */
int fld_levels(const fld_grid* g, int* dims, int max_levels);

/* Autotuner: for each level of a mixed-precision context whose FP32 sweeps
 * run four cells per thread, time every candidate launch shape (128 or 256
 * threads per block; 608 to 9728 blocks, which sets the z-chunk each thread
 * walks; and an L2 prefetch distance of 0, 1 or 2 planes) of the
 * pre-smoothing, colour-sweep, residual, restriction, prolongation and CG
 * p/q kernels (and of the fused post-sweep when fused_post is set), reps
 * launches each, on the context's buffers and stream, and keep the
 * fastest.  No-op for FP64 contexts.
 * Discards captured CUDA graphs and the device scalars; call it after
 * fld_create and before stepping (the assembled operator is kept). */
fld_status fld_autotune(fld_ctx* ctx, int reps);

/* The tuning table: per level and kernel one record of three ints
 * (threads per block, a power of two in [32, 256]; target blocks in
 * [1, 9728]; L2 prefetch distance in planes, [0, 8]); its length
 * (3 x 7 kernels x levels), a copy, and a
 * replacement (for caching tuned shapes).  fld_set_tuning checks every
 * record and changes nothing on FLD_EINVAL; the launch shape never changes
 * a result beyond the order of the CG reductions. */
int fld_tuning_size(fld_ctx* ctx);
fld_status fld_get_tuning(fld_ctx* ctx, int* out, int n);
fld_status fld_set_tuning(fld_ctx* ctx, const int* in, int n);

/* Per-kernel-class launch statistics of one context.  bytes is the
 * algorithmic traffic of the launches (every array a kernel streams counted
 * once per cell of its level, in the array's word size); ms and timed_bytes
 * cover only the launches timed with CUDA events (see fld_profile). */
typedef struct {
    const char* name;          /* kernel class, static storage */
    long long launches;        /* launches since the last fld_profile */
    long long timed;           /* launches bracketed by events */
    double ms;                 /* summed event time of the timed launches */
    double bytes;              /* algorithmic bytes of all launches */
    double timed_bytes;        /* algorithmic bytes of the timed launches */
} fld_kernel_stat;

/* Reset the context's launch statistics and select the kernel classes
 * (bit i = class i of fld_profile_read's order) whose launches are
 * bracketed by CUDA events on the context's stream; 0 times nothing.
 * Synchronises the context's stream. */
fld_status fld_profile(fld_ctx* ctx, unsigned long long class_mask);

/* Copy up to max per-class statistics to out; returns the number of
 * classes (call with max = 0 to size out). */
int fld_profile_read(fld_ctx* ctx, fld_kernel_stat* out, int max);

/* Message of the calling thread's last failed call ("" if none). */
const char* fld_last_error(void);

/* Release every buffer of the context (NULL is ignored). */
void fld_destroy(fld_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* FLD_H */
