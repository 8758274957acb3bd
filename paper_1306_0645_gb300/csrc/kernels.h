// kernels.h -- host-side launchers of the libfld CUDA kernels.
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"
#include "df.cuh"
#include "fld.h"

namespace fld {

// Physical constants of one step, precomputed on the host.  theta is the
// time discretisation of the theta-method: the operator A carries theta
// times the face weights and loss rates, the right-hand side the full ones.
struct PhysDev {
    double dt, c, Dmax, Rmin, sigma, adot;
    double h[3];        // cell widths
    double dt_h2[3];    // theta dt / h^2 (face weights of A per unit D)
    double wmax[3];     // theta dt D_max / h^2, the weight of a capped face
    double dtcs;        // dt c sigma (right-hand side and photon balance)
    double one_dta;     // 1 + theta dt adot/a (mass term of A)
    double dta;         // dt adot/a
    double mdtcs;       // theta dt c sigma (mass term of A)
    double theta, inv_theta;
    double ebc[6];      // E_b of the Dirichlet faces: x lo, x hi, y lo, ...
    int dmask;          // bit s set: side s (2 axis + upper) is Dirichlet
    float wmax32[3];    // FP32 copy of wmax
    float sigmaL32;     // sigma L_unit
    float twoL_h32[3];  // 2 L_unit / h
    float thr32;        // screen threshold on 9 (kappa_f L)^2 + (R L)^2
    int limiter;        // 0 paper, 1 Levermore-Pomraning
    // double-float constants of the mixed-precision kernels (k_mixed.cu)
    df sigh[3];         // sigma h: optical depth of a cell per unit n_HI
    df cw[3];           // theta dt c / h: a face weight is cw K S / sqrt(X)
    df rminh[3];        // R_min h
    df wmaxd[3];        // wmax (hi = wmax32)
    df one_dta_d, mdtcs_d;   // mass term m = one_dta + mdtcs n_HI
    df dtcs_d, dta_d;        // loss rate dt (c sigma n_HI + adot/a)
    df dtm_d;                // dt = dtm 2^dt_exp, dtm in [1, 2)
    df ith_d;                // 1 / theta
    int dt_exp;
    int df_limiter;     // the df limiter's constants lie in the FP32 range
};

// Operator of one level: mass term m, lower-face weights, inverse diagonal.
template <class T>
struct Op {
    T *m, *wx, *wy, *wz, *invd;
};

// Weights of the Dirichlet faces of a level (theta-scaled, on the diagonal
// of A), packed by side in the order x lo, x hi, y lo, y hi, z lo, z hi; the
// face of cell (i,j,k) on an x side has index j + ny k, on a y side
// i + nx k, on a z side i + nx j.  w == nullptr: no Dirichlet face.
struct Bnd {
    double* w;
    int mask;           // Dirichlet sides, bit 2 axis + upper
};

__host__ __device__ inline long long bnd_side_size(const Dims& d, int s) {
    const int a = s >> 1;
    return a == 0 ? (long long)d.ny * d.nz : (a == 1 ? (long long)d.nx * d.nz : (long long)d.nx * d.ny);
}
__host__ __device__ inline long long bnd_offset(const Dims& d, int s) {
    long long o = 0;
    for (int q = 0; q < s; q++) o += bnd_side_size(d, q);
    return o;
}

// Per-block lists of the faces the FP32 screen could not settle, finished
// by a compacted FP64 pass.  entries == nullptr disables the lists.
struct FaceList {
    unsigned* entries;   // block b owns entries[b * cap, (b + 1) * cap)
    unsigned* counts;    // entries used per block
    int cap;
};

// ---- assembly (k_assemble.cu)
// The assembly kernels walk the planes in nzb z-blocks of kch planes each
// (grid sh); a launch covers the z-blocks [zb0, zb0 + nzb) (nzb < 0: all),
// so the assembly of a grid can follow its planes as they arrive.  The
// face lists belong to the blocks of this decomposition.
struct AsmShape {
    ColShape sh;
    int kch, nzb;
};
AsmShape asm_shape(const Dims& d);
// Pass 1: opacity, face limiter and weights (FP64, plus FP32 copies of the
// weights and mass term when op32.m != nullptr); flags invalid inputs.
// Reads E and n_HI of planes zb0 * kch - 1 .. (zb0 + nzb) * kch - 1.
void launch_assemble_faces(const Dims& d, const PhysDev& p, const double* E, const double* nHI,
                           const double* eta, Op<double> op, Op<float> op32, double* sc,
                           FaceList fl, cudaStream_t s, int zb0 = 0, int nzb = -1);
// FP64 limiter for the listed faces of those z-blocks (one block per list
// segment).
void launch_assemble_fix(const Dims& d, const PhysDev& p, const double* E, const double* nHI,
                         Op<double> op, Op<float> op32, FaceList fl, cudaStream_t s, int zb0 = 0,
                         int nzb = -1);
// Size of the face lists for a level: blocks of the faces launch and
// entries per block (0 when lists are not used).
void face_list_shape(const Dims& d, int limiter, long long* blocks, int* cap);
// Pass 2: right-hand side b, inverse diagonals (FP64 if op.invd, FP32 if
// op32.invd), the FP64 diagonal if diag64, ||b||^2 into slot0 and max |b|
// into slot1.  Cells on a Dirichlet face (p.dmask) also get the face's
// limiter weight: stored in bnd, added to m (FP64 and FP32) and its flux
// to b.  Needs the weights of the planes one past its z-blocks (upper
// z faces) and E of the planes on either side.
void launch_assemble_rhs(const Dims& d, const PhysDev& p, const double* E, const double* nHI,
                         const double* eta, Op<double> op, Op<float> op32, double* b, double* diag64,
                         Bnd bnd, const RedArgs& ra, cudaStream_t s, int zb0 = 0, int nzb = -1);
// Photons through the Dirichlet faces of side s over the step (before the
// finalisation overwrites E): sum of w_b (inv_theta (E - E_b) + dE) into
// slot S_OUT0 + s and the sum of its absolute values into S_OUTABS0 + s
// (reduction ra with op R_STORE2).
void launch_bnd_outflow(const Dims& d, const PhysDev& p, int s, Bnd bnd, const double* E,
                        const double* dE, const RedArgs& ra, cudaStream_t st);

// ---- mixed-precision step on the FP32 pipe in double-float arithmetic
// (k_mixed.cu).  The fine operator is (A, L): the FP32 operator of the
// V-cycles and the low parts of m and the weights.
// Pass 1: m and the face weights (df), input validation into sc[S_BAD], the
// maxima of E, n_HI and eta into sc[S_EMAX], sc[S_NMAX], sc[S_ETAMAX] (the
// caller zeroes them with the other slots before the assembly).
// Faces the FP32 screen does not settle go to the per-block lists fl (when
// fl.entries is set), finished by launch_asm_fix_mx.
void launch_asm_faces_mx(const Dims& d, const PhysDev& p, const double* E, const double* nHI, const double* eta,
                         Op<float> A, Op<float> L, double* sc, FaceList fl, cudaStream_t s, int zb0 = 0,
                         int nzb = -1);
// The df limiter for the listed faces of those z-blocks.
void launch_asm_fix_mx(const Dims& d, const PhysDev& p, const double* E, const double* nHI, Op<float> A,
                       Op<float> L, FaceList fl, cudaStream_t s, int zb0 = 0, int nzb = -1);
// Pass 2: b (FP64), ||b||^2 and max |b| (reduction ra, R_STORE_SUM_MAX), the
// FP32 inverse diagonal A.invd, Dirichlet face weights into bnd and m; scg:
// the slots of pass 1's maxima.  Needs pass 1 of its z-blocks and the one
// above.
// Bf: where its pointers are set, also the bfloat16 copies (nearest) of the
// FP32 weights wx, wy, wz and of the FP32 inverse diagonal.
void launch_asm_rhs_mx(const Dims& d, const PhysDev& p, const double* E, const double* nHI, const double* eta,
                       Op<float> A, Op<float> L, double* b, Bnd bnd, const RedArgs& ra, const double* scg,
                       cudaStream_t s, int zb0 = 0, int nzb = -1, Op<unsigned short> Bf = {});
// r32 = b 2^-ks (nearest float); ||r32||^2, max |r32| (R_IRRES).
void launch_ir_scale_b(long long n, const double* b, int ks, float* r32, const RedArgs& ra, cudaStream_t s);
// The refinement unknown x (dE) of the mixed solver is a df pair per cell
// (float2), scaled by 2^-K with K the step's scale exponent (from the
// maxima in scg, the context's slots).
// x += 2^ks x32 (assign: x = 2^ks x32); p_last (optional): x32 still lacks
// the last CG iteration's update, x32 + sc[S_ALPHA] p_last in FP32 is used
void launch_ir_update_mx(long long n, void* x, const float* x32, const double* sc, bool assign, int ks,
                         const float* p_last, const double* scg, int dt_exp, cudaStream_t s);
// r = b - m x - sum_f w_f (x - x_nbr) in df; ||r32||^2, max |r32| of r32 =
// r 2^-ks (nearest float) (R_IRRES), r32 itself only with write.
void launch_ir_residual(const Dims& d, Op<float> A, Op<float> L, const double* b, const void* x, int ks,
                        float* r32, bool write, const RedArgs& ra, const double* scg, int dt_exp, cudaStream_t s);
ColShape ir_residual_shape(const Dims& d);
// E_out = max(E + dE, 0) and the photon-balance sums as launch_finalize,
// summed in df relative to the scales of the maxima in scg; dE the df x.
void launch_finalize_mx(long long n, const PhysDev& p, const double* E, const void* dE, const double* nHI,
                        const double* eta, double* E_out, const RedArgs& ra, const double* scg, cudaStream_t s);
// launch_bnd_outflow with dE the df x
void launch_bnd_outflow_mx(const Dims& d, const PhysDev& p, int s, Bnd bnd, const double* E, const void* dE,
                           const RedArgs& ra, const double* scg, cudaStream_t st);
// the df x as FP64 values (fld_solve's output)
void launch_dE_to_f64(long long n, const void* x, double* out, const double* scg, int dt_exp, cudaStream_t s);
// out = h + l in FP64 (inspection hooks)
void launch_df_to_f64(long long n, const float* h, const float* l, double* out, cudaStream_t s);
// y = A x with the df operator, in FP64 (test hook)
void launch_apply_mx(const Dims& d, Op<float> A, Op<float> L, const double* x, double* y, cudaStream_t s);

// ---- multigrid (k_mg.cu), T = float or double
template <class T>
void launch_coarsen(const Dims& f, const Dims& c, Op<T> F, Op<T> C, cudaStream_t s);
// Coarse Dirichlet face weights of side s (sum of the 4 fine ones / 16);
// the coarse mass term, which k_coarsen took as the mean of the children's
// full m, gives back the difference: m_c -= w_c.  After launch_coarsen.
template <class T>
void launch_coarsen_bnd(const Dims& f, const Dims& c, int s, Bnd F, Bnd C, Op<T> CA,
                        cudaStream_t st);
template <class T>
void launch_invd(const Dims& d, Op<T> A, const Op<T>& src, cudaStream_t s);
template <class T>
void launch_smooth_zero(const Dims& d, Op<T> A, const T* r, T* z, cudaStream_t s);
template <class T>
void launch_rb_colour(const Dims& d, Op<T> A, const T* r, T* z, int colour, cudaStream_t s);
template <class T>
void launch_jacobi(const Dims& d, Op<T> A, const T* r, const T* z, T* out, double omega,
                   bool zero_guess, cudaStream_t s);
template <class T>
void launch_residual(const Dims& d, Op<T> A, const T* r, const T* z, T* res, cudaStream_t s);
template <class T>
void launch_restrict(const Dims& f, const Dims& c, const T* rf, T* rc, cudaStream_t s);
template <class T>
void launch_prolong_add(const Dims& f, const Dims& c, const T* ec, T* zf, cudaStream_t s);
// Coarsest grid: dense matrix, Cholesky, explicit inverse (one CTA; in
// shared memory and in FP32 when fp32 and the matrix fits, else FP64).
template <class T>
void launch_coarse_setup(const Dims& d, Op<T> A, double* dense, double* ainv, double* sc, bool fp32,
                         cudaStream_t s);
template <class T>
void launch_coarse_apply(int n, const double* ainv, const T* r, T* z, cudaStream_t s);

// ---- Krylov and refinement (k_cg.cu)
template <class T>
void launch_dot(long long n, const T* a, const T* b, const RedArgs& ra, cudaStream_t s);
template <class T>
void launch_cg_p_matvec(const Dims& d, Op<T> A, const T* z, const T* p_in, T* p_out, T* q,
                        const RedArgs& ra, cudaStream_t s);
template <class T>
void launch_cg_update(long long n, T* x, T* r, const T* p, const T* q, const RedArgs& ra,
                      cudaStream_t s);
template <class T>
void launch_apply(const Dims& d, Op<T> A, const T* x, T* y, cudaStream_t s);
// element-wise precision conversions (test hooks)
void launch_f64_to_f32(long long n, const double* a, float* b, cudaStream_t s);
void launch_f32_to_f64(long long n, const float* a, double* b, cudaStream_t s);
// Device-side CG convergence test: sc[S_KITER] += 1 and the conditional h
// set to continue while sc[S_RR] > sc[S_THRESH], S_KITER < S_MAXIT and no
// non-finite reduction (one thread).
// Slots of a reduction done in chunks (at most 8).
struct SlotList {
    int n;
    int s[8];
};
// sc[slot] = the chunks' slot summed in chunk order, for each listed slot,
// and the non-finite flag of any chunk.
void launch_combine_sums(const double* chunk_sc, int nch, double* sc, const SlotList& sl, cudaStream_t s);
// Reductions done in nch chunks, each into its own block of NUM_SLOTS
// slots: sc[s_sum] = the chunks' s_sum summed in chunk order, sc[s_max] =
// their s_max maximised, and the non-finite flag of any chunk.
void launch_combine_chunks(const double* chunk_sc, int nch, double* sc, int s_sum, int s_max, cudaStream_t s);
void launch_cg_check(cudaGraphConditionalHandle h, double* sc, cudaStream_t s,
                     const cudaGraphConditionalHandle* h2 = nullptr);
// The launch shape of launch_residual64 (callers that size reduction
// scratch for it check its block count).
ColShape residual64_shape(const Dims& d);
// r64 = b - A x (FP64); ||r64||^2 -> slot0, max|r64| -> slot1.  diag (may
// be null) is the stored FP64 diagonal.
void launch_residual64(const Dims& d, Op<double> A, const double* diag, const double* b, const double* x,
                       double* r, const RedArgs& ra, cudaStream_t s);
// E_out = max(E + dE, 0); sums for the photon balance into S_BAL (dE),
// S_EMIT (eta), S_ABSORB (n_HI E^theta), S_ESUM (E^theta), the floor's
// energy into S_FLOOR, sum dE^2 into S_DE2, sum E_out^2 into S_EN2
// (reduction R_STORE7_FIN).
void launch_finalize(long long n, const PhysDev& p, const double* E, const double* dE,
                     const double* nHI, const double* eta, double* E_out, const RedArgs& ra,
                     cudaStream_t s);
void launch_opacity_update(long long n, const double* E, const double* nH, const double* nHI,
                           double* out, double dt, double c, double sigma, double hnu,
                           double alpha_B, cudaStream_t s);

// ---- persistent coarse tail of the V-cycle (k_tail.cu): levels L[0] (the
// first level at or below the size threshold) to L[nlev - 1] (the coarsest)
// in one launch of one cluster of `cluster` CTAs.  L[0].r is the input,
// L[0].z the output; the other r, z, t are the levels' work vectors.
constexpr int TAIL_MAX_LEVELS = 12;
// small levels of the tail run in one CTA with their vectors (r, z, t) in
// shared memory: from the first level with at most this many cells, when
// their vectors fit TAIL_SMEM_MAX bytes
constexpr long long TAIL_SMALL_CELLS = 512;
constexpr size_t TAIL_SMEM_MAX = 160 * 1024;
template <class T>
struct TailLevel {
    Dims d;
    Op<T> A;
    T *r, *z, *t;
};
template <class T>
struct TailArgs {
    int nlev, pre, post;
    int paper_order;  // post-sweeps red then black (else black then red)
    int small_from;   // first level run by one CTA in shared memory (nlev: none)
    const double* ainv;
    TailLevel<T> L[TAIL_MAX_LEVELS];
};
template <class T>
cudaError_t launch_vtail(const TailArgs<T>& a, int cluster, cudaStream_t s);
// the cluster size to launch the tail with (16 or 8 CTAs), 0 if no cluster
// of the tail kernel can be resident on this device
template <class T>
int vtail_cluster();

// ---- persistent inner solves over a work list (k_tail.cu, mixed
// precision): each cluster takes requests by ticket and runs a request's
// whole FP32 MG-PCG solve (V-cycles over all its levels and the CG vector
// operations) to ||r||^2 <= sc[S_THRESH] or sc[S_MAXIT] iterations.
struct PsReq {
    TailArgs<float> v;   // all levels; L[0].r is the CG residual (in: the
                         // right-hand side, x = 0), L[0].z the preconditioned one
    float *x, *p, *q;    // fine-level CG vectors
    double* sc;          // the request's scalar slots: S_THRESH, S_MAXIT in;
                         // S_KITER, S_RR, S_RHO.., S_NONFINITE out
    int cta;             // 1: solved by one CTA with every vector in its
                         // shared memory (psolve_cta_bytes fits), else by a cluster
    int pad_;
};
constexpr int PS_MAX_BATCH = 256;
constexpr int PS_CLUSTER = 8;
// the most dynamic shared memory of a persistent launch
constexpr size_t PS_SMEM_MAX = 200 * 1024;
struct PsBatch {
    int n;          // requests: [0, ncl) by clusters, [ncl, n) by single CTAs
    int ncl;
    unsigned* ticket;                 // two counters, set to 0 by launch_psolve
    const PsReq* req[PS_MAX_BATCH];   // device descriptors, in work-list order
};
struct PsShape {
    int cluster;    // CTAs per cluster
    int clusters;   // clusters resident at once
};
PsShape psolve_shape();
// shared memory of a single-CTA solve: r, z, t of every level and p, q, x
size_t psolve_cta_bytes(const TailArgs<float>& v);
size_t psolve_smem_bytes(const PsReq& r);
// one launch: min(n, resident clusters) clusters drain the work list; smem
// is the largest psolve_smem_bytes of the batch
cudaError_t launch_psolve(const PsBatch& b, size_t smem, cudaStream_t s);

// Sets the calling thread's fld_last_error message (fld_api.cu).
void record_error(const char* msg);
// The per-face boundary conditions of g are consistent (fld_create's rule);
// otherwise false with the reason in msg (fld_api.cu).
bool bc_valid(const fld_grid* g, char* msg, size_t len);

// Launch shape of a four-cells-per-thread sweep: threads per block (a
// power of two up to 256, x lanes first) and the total blocks aimed at (the
// z-chunk length follows).  Chosen per level and kernel by fld_autotune.
struct Tune {
    int threads = 256;
    int target = 152 * 8;
    int pf = 1;             // L2 prefetch distance in planes (0: none; FP32 sweeps)
};
constexpr int TUNE_FIELDS = 3;      // entries of one tuning-table record
constexpr int TUNE_PF_MAX = 8;

// ---- FP32 four-cells-per-thread sweeps (k_fine4.cu); need nx % 4 == 0
bool fine4_ok(const Dims& d);
// x (optional): also x += alpha_prev p_in, the previous iteration's update
// of x (see launch_cg_update4 with x null)
void launch_cg_p_matvec4(const Dims& d, Op<float> A, const float* z, const float* p_in, float* p_out,
                         float* q, const RedArgs& ra, cudaStream_t s, const Tune& tn = Tune{},
                         float* x = nullptr);
// after_zero_sweep: z comes from one red/black sweep from z = 0 (black
// last), so the residual is sum_f w_f z_nbr at red cells and 0 at black
// ones; red_compressed (with after_zero_sweep, where red_compress_ok):
// stored red-compressed, res[l >> 1] for red cell l
void launch_residual4(const Dims& d, Op<float> A, const float* r, const float* z, float* res,
                      cudaStream_t s, const Tune& tn = Tune{}, bool after_zero_sweep = false,
                      bool red_compressed = false);
bool red_compress_ok(const Dims& f);
void launch_smooth_zero4(const Dims& d, Op<float> A, const float* r, float* z, cudaStream_t s,
                         const Tune& tn = Tune{});
void launch_rb_colour4(const Dims& d, Op<float> A, const float* r, float* z, int colour,
                       cudaStream_t s, const Tune& tn = Tune{});
// The same sweeps with the smoothing operator's coefficients (wx, wy, wz,
// invd; m unused) stored as bfloat16 (the upper 16 bits of the FP32
// values, rounded to nearest); the residual only in its zero-guess form.
void launch_smooth_zero4(const Dims& d, Op<unsigned short> A, const float* r, float* z, cudaStream_t s,
                         const Tune& tn = Tune{});
void launch_rb_colour4(const Dims& d, Op<unsigned short> A, const float* r, float* z, int colour,
                       cudaStream_t s, const Tune& tn = Tune{});
void launch_rb_colour4_dot(const Dims& d, Op<unsigned short> A, const float* r, float* z, int colour,
                           const RedArgs& ra, cudaStream_t s, const Tune& tn = Tune{});
void launch_residual4(const Dims& d, Op<unsigned short> A, const float* z, float* res, cudaStream_t s,
                      const Tune& tn, bool red_compressed);
// B.wx, wy, wz, invd = the bfloat16 values nearest to A's (n a multiple of 4).
void launch_op_to_bf16(long long n, Op<float> A, Op<unsigned short> B, cudaStream_t s);
void launch_dot4(long long n, const float* a, const float* b, const RedArgs& ra, cudaStream_t s);
// one colour of a sweep followed by <r, z> of the result (reduction ra)
void launch_rb_colour4_dot(const Dims& d, Op<float> A, const float* r, float* z, int colour,
                           const RedArgs& ra, cudaStream_t s, const Tune& tn = Tune{});
// red_compressed: rf is a red-compressed residual (k_residual4 after a
// zero-guess sweep), cell l red ? rf[l >> 1] : 0
void launch_restrict4(const Dims& f, const Dims& c, const float* rf, float* rc, cudaStream_t s,
                      const Tune& tn = Tune{}, bool red_compressed = false);
// Fused post-smoothing sweep (black then red), out of place zi -> zo, with
// <r, zo> into *dot when dot is given; post4_ok tells if a level qualifies.
bool post4_ok(const Dims& d);
void launch_post_smooth4(const Dims& d, Op<float> A, const float* r, const float* zi, float* zo,
                         const RedArgs* dot, cudaStream_t s, const Tune& tn = Tune{});
// zo = z + P ec (out of place)
void launch_prolong_to4(const Dims& f, const Dims& c, const float* ec, const float* z, float* zo,
                        cudaStream_t s);
void launch_prolong_add4(const Dims& f, const Dims& c, const float* ec, float* zf, cudaStream_t s,
                         const Tune& tn = Tune{});
// x null: r -= alpha q only, the update of x deferred to the next
// launch_cg_p_matvec4 (and the last one to launch_ir_update)
void launch_cg_update4(long long n, float* x, float* r, const float* p, const float* q,
                       const RedArgs& ra, cudaStream_t s);

}  // namespace fld
