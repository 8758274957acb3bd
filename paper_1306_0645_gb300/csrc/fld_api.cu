// fld_api.cu -- the C ABI of libfld.so (declared in include/fld.h): context
// and hierarchy management, the MG-preconditioned CG driver (Table 1), the
// mixed-precision iterative-refinement driver, and the step wrapper.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "fld.h"
#include "kernels.h"

using namespace fld;

namespace {

constexpr int MAX_LEVELS = 32;
constexpr int COARSE_CAP_MAX = 4096;

thread_local std::string g_err;

fld_status set_err(fld_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CUDA_TRY(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return set_err(FLD_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

// Tuned launch shapes of a level's FP32 sweeps.
enum TuneClass { TN_SMOOTH0 = 0, TN_RB, TN_RES, TN_RESTRICT, TN_PROLONG, TN_PMATVEC, TN_POST, NTUNE };

struct Level {
    Dims d;
    Op<double> A64;
    Op<float> A32;
    Op<float> Alo;     // mixed fine level: low parts of m and w (df with A32)
    Op<unsigned short> Abf;   // mixed levels: bfloat16 copies of wx, wy, wz, invd for
                              // the V-cycle's sweeps (fld_params.precond_bf16), else null
    Bnd bnd;           // Dirichlet face weights (FP64)
    void *r, *z, *t;   // level vectors in the solver precision (level 0: t only)
    Tune tune[NTUNE];
};

// Kernel classes for launch counting and optional CUDA-event timing.
enum KClass {
    K_ASM_FACES = 0, K_ASM_RHS, K_COARSEN, K_INVD, K_COARSE_SETUP, K_SMOOTH_ZERO,
    K_RB_COLOUR, K_JACOBI, K_RESIDUAL, K_RESTRICT, K_PROLONG, K_COARSE_APPLY, K_DOT,
    K_CG_PMATVEC, K_CG_UPDATE, K_RESIDUAL64, K_IR_SCALE, K_IR_UPDATE, K_FINALIZE, K_APPLY,
    K_OPACITY, K_COARSE_LEVELS, K_ASM_FIX, K_POST_FUSED, K_VTAIL, K_IR_RESID, K_PSOLVE, K_NUM
};
const char* const KNAMES[K_NUM] = {
    "assemble_faces", "assemble_rhs", "coarsen", "invd", "coarse_setup", "smooth_zero",
    "rb_colour", "jacobi", "residual", "restrict", "prolong_add", "coarse_apply", "dot",
    "cg_p_matvec", "cg_update", "residual64", "ir_scale", "ir_update", "finalize", "apply",
    "opacity_update", "coarse_levels", "assemble_fix", "post_smooth", "vtail", "ir_residual",
    "psolve"};

struct KStat {
    long long launches, timed;
    double ms, bytes, timed_bytes;
};

bool coarsenable(const int n[3]) {
    int mn = n[0] < n[1] ? n[0] : n[1];
    if (n[2] < mn) mn = n[2];
    return mn > 4 && n[0] % 2 == 0 && n[1] % 2 == 0 && n[2] % 2 == 0;
}

int level_shapes(const fld_grid* g, int dims[][3]) {
    int n[3] = {g->nx, g->ny, g->nz};
    int nl = 0;
    for (;;) {
        dims[nl][0] = n[0];
        dims[nl][1] = n[1];
        dims[nl][2] = n[2];
        nl++;
        if (!coarsenable(n) || nl >= MAX_LEVELS) break;
        n[0] /= 2;
        n[1] /= 2;
        n[2] /= 2;
    }
    return nl;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

fld_status validate(const fld_grid* g, const fld_params* p) {
    if (!g || !p) return set_err(FLD_EINVAL, "null grid or params");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1)
        return set_err(FLD_EINVAL, "grid dimensions must be >= 1 (got %d %d %d)", g->nx, g->ny, g->nz);
    if ((long long)g->nx * g->ny * g->nz > (1LL << 33))
        return set_err(FLD_EINVAL, "grid too large");
    {
        // the stencil launches tile an x-y plane with at most RED_MAX_BLOCKS
        // thread blocks (about 4.2 M cells)
        Dims d0;
        d0.nx = g->nx; d0.ny = g->ny; d0.nz = g->nz;
        d0.px = d0.py = d0.pz = 0;
        d0.n = (long long)g->nx * g->ny * g->nz;
        const ColShape sh = col_shape(d0);
        if ((long long)sh.grid.x * sh.grid.y * sh.grid.z > RED_MAX_BLOCKS)
            return set_err(FLD_EINVAL, "x-y plane too large: at most 16384 thread blocks of 256 cells");
    }
    if (!finite_pos(g->dx) || !finite_pos(g->dy) || !finite_pos(g->dz))
        return set_err(FLD_EINVAL, "cell widths must be finite and > 0");
    {
        char msg[160];
        if (!fld::bc_valid(g, msg, sizeof msg)) return set_err(FLD_EINVAL, "%s", msg);
    }
    if (!finite_pos(p->dt)) return set_err(FLD_EINVAL, "dt must be finite and > 0");
    if (!finite_pos(p->c)) return set_err(FLD_EINVAL, "c must be finite and > 0");
    if (!finite_pos(p->L_unit)) return set_err(FLD_EINVAL, "L_unit must be finite and > 0");
    if (!finite_pos(p->dmax_coef)) return set_err(FLD_EINVAL, "dmax_coef must be finite and > 0");
    if (!(std::isfinite(p->rmin_coef) && p->rmin_coef >= 0.0))
        return set_err(FLD_EINVAL, "rmin_coef must be finite and >= 0");
    if (!(std::isfinite(p->sigma) && p->sigma >= 0.0))
        return set_err(FLD_EINVAL, "sigma must be finite and >= 0");
    if (!(std::isfinite(p->adot_over_a) && p->adot_over_a >= 0.0))
        return set_err(FLD_EINVAL, "adot_over_a must be finite and >= 0");
    if (!finite_pos(p->hnu)) return set_err(FLD_EINVAL, "hnu must be finite and > 0");
    if (!(p->theta >= 0.5 && p->theta <= 1.0))
        return set_err(FLD_EINVAL, "theta must lie in [1/2, 1] (1 backward Euler, 1/2 trapezoidal)");
    if (!(std::isfinite(p->scale_factor) && p->scale_factor > 0.0))
        return set_err(FLD_EINVAL, "scale_factor must be finite and > 0");
    if (p->limiter != FLD_LIMITER_PAPER && p->limiter != FLD_LIMITER_LP)
        return set_err(FLD_EINVAL, "unknown limiter %d", p->limiter);
    if (p->precision != FLD_PREC_FP64 && p->precision != FLD_PREC_MIXED)
        return set_err(FLD_EINVAL, "unknown precision %d", p->precision);
    if (p->smoother != FLD_SMOOTH_RBGS && p->smoother != FLD_SMOOTH_JACOBI)
        return set_err(FLD_EINVAL, "unknown smoother %d", p->smoother);
    if (p->smoother == FLD_SMOOTH_JACOBI && !(p->jacobi_omega > 0.0 && p->jacobi_omega < 2.0))
        return set_err(FLD_EINVAL, "jacobi_omega must lie in (0, 2)");
    if (!(p->rtol > 0.0 && p->rtol < 1.0)) return set_err(FLD_EINVAL, "rtol must lie in (0, 1)");
    if (p->max_iter < 1 || p->max_iter > 100000) return set_err(FLD_EINVAL, "max_iter out of range");
    if (p->pre < 0 || p->post < 0 || p->pre > 16 || p->post > 16 || p->pre + p->post < 1)
        return set_err(FLD_EINVAL, "pre/post sweeps must be in [0, 16] with at least one sweep");
    if (p->precision == FLD_PREC_MIXED && !(p->inner_rtol > 0.0 && p->inner_rtol < 1.0))
        return set_err(FLD_EINVAL, "inner_rtol must lie in (0, 1)");
    if (p->coarse_cap < 1 || p->coarse_cap > COARSE_CAP_MAX)
        return set_err(FLD_EINVAL, "coarse_cap must lie in [1, %d]", COARSE_CAP_MAX);
    if (p->tail_cells < 0 || p->tail_cells > (1 << 24))
        return set_err(FLD_EINVAL, "tail_cells must lie in [0, 2^24]");
    if (p->paper_order != 0 && p->paper_order != 1) return set_err(FLD_EINVAL, "paper_order must be 0 or 1");
    if (p->persistent_cells < 0 || p->persistent_cells > (1 << 24))
        return set_err(FLD_EINVAL, "persistent_cells must lie in [0, 2^24]");
    if (p->precond_bf16 != 0 && p->precond_bf16 != 1) return set_err(FLD_EINVAL, "precond_bf16 must be 0 or 1");
    int dims[MAX_LEVELS][3];
    int nl = level_shapes(g, dims);
    long long nc = (long long)dims[nl - 1][0] * dims[nl - 1][1] * dims[nl - 1][2];
    if (nc > p->coarse_cap)
        return set_err(FLD_EINVAL,
                       "coarsest grid %dx%dx%d has %lld cells > coarse_cap %d (coarsening stops at "
                       "the first odd dimension or a dimension <= 4)",
                       dims[nl - 1][0], dims[nl - 1][1], dims[nl - 1][2], nc, p->coarse_cap);
    return FLD_OK;
}

}  // namespace

namespace fld {
// The per-face boundary conditions of a grid: known kinds, a periodic axis
// periodic at both faces (an upper face left at 0, zero gradient, counts as
// periodic too), and finite non-negative Dirichlet values.  On failure msg
// says why.
bool bc_valid(const fld_grid* g, char* msg, size_t len) {
    for (int a = 0; a < 3; a++) {
        const int lo = g->bc[a], hi = g->bc_hi[a];
        if (lo < FLD_BC_ZERO_GRADIENT || lo > FLD_BC_OUTFLOW || hi < FLD_BC_ZERO_GRADIENT || hi > FLD_BC_OUTFLOW) {
            snprintf(msg, len, "unknown boundary condition (%d, %d) on axis %d", lo, hi, a);
            return false;
        }
        if (lo == FLD_BC_PERIODIC && hi != FLD_BC_PERIODIC && hi != FLD_BC_ZERO_GRADIENT) {
            snprintf(msg, len, "axis %d is periodic but its upper face is %d", a, hi);
            return false;
        }
        if (lo != FLD_BC_PERIODIC && hi == FLD_BC_PERIODIC) {
            snprintf(msg, len, "axis %d: periodic upper face needs a periodic lower face", a);
            return false;
        }
        for (int u = 0; u < 2; u++)
            if ((u ? hi : lo) == FLD_BC_DIRICHLET && lo != FLD_BC_PERIODIC &&
                !(std::isfinite(g->bc_value[2 * a + u]) && g->bc_value[2 * a + u] >= 0.0)) {
                snprintf(msg, len, "Dirichlet value of face %d must be finite and >= 0", 2 * a + u);
                return false;
            }
    }
    return true;
}
}  // namespace fld

namespace {

// Sides (bit 2 axis + upper) held at a fixed E: Dirichlet and outflow faces.
int dirichlet_mask(const fld_grid* g) {
    int m = 0;
    for (int a = 0; a < 3; a++) {
        if (g->bc[a] == FLD_BC_PERIODIC) continue;
        if (g->bc[a] == FLD_BC_DIRICHLET || g->bc[a] == FLD_BC_OUTFLOW) m |= 1 << (2 * a);
        if (g->bc_hi[a] == FLD_BC_DIRICHLET || g->bc_hi[a] == FLD_BC_OUTFLOW) m |= 1 << (2 * a + 1);
    }
    return m;
}

// Whether a context runs its inner solves as persistent cluster kernels
// (fld_params.persistent_cells): mixed precision, red/black Gauss-Seidel, a
// small enough fine grid and at most TAIL_MAX_LEVELS levels.
bool ps_wanted(const fld_params* p, size_t n0, int nl) {
    return p->precision == FLD_PREC_MIXED && p->smoother == FLD_SMOOTH_RBGS && p->persistent_cells > 0 &&
           n0 <= (size_t)p->persistent_cells && nl >= 2 && nl <= TAIL_MAX_LEVELS;
}

// Whether the V-cycle sweeps of level l (nx by n cells; the fine level has
// n0) read bfloat16 copies of its coefficients (fld_params.precond_bf16):
// mixed precision, red/black Gauss-Seidel with one pre-sweep (the
// zero-guess residual, which needs no m) and separate colour sweeps,
// four-cell sweeps on a level above the coarsest one and outside the
// persistent coarse tail, and inner solves launched kernel by kernel.
bool bf16_wanted(const fld_params* p, int l, int nx, size_t n, size_t n0, int nl) {
    return p->precision == FLD_PREC_MIXED && p->precond_bf16 == 1 && p->smoother == FLD_SMOOTH_RBGS &&
           p->pre == 1 && p->fused_post == 0 && l < nl - 1 && nx % 4 == 0 && nx >= 16 &&
           !(p->tail_cells > 0 && n <= (size_t)p->tail_cells) && !ps_wanted(p, n0, nl);
}

// Enumerates every device buffer a context needs, in a fixed order; the
// same walk sizes the footprint and performs the allocation.
template <class F>
void plan(const fld_grid* g, const fld_params* p, F&& buf) {
    int dims[MAX_LEVELS][3];
    const int nl = level_shapes(g, dims);
    const bool mixed = p->precision == FLD_PREC_MIXED;
    const size_t ts = mixed ? sizeof(float) : sizeof(double);
    for (int l = 0; l < nl; l++) {
        const size_t n = (size_t)dims[l][0] * dims[l][1] * dims[l][2];
        // the coarse levels serve only the cycle, FP32 on every level of the
        // mixed solver: FP64 operators there for the FP64 solver only (the
        // fine level keeps its FP64 operator for the refinement residual)
        // the fine operator of the mixed solver is double-float: the FP32
        // operator of its V-cycles plus low parts (k_mixed.cu)
        if (!mixed)
            for (int q = 0; q < 5; q++) buf(l, "A64", q, n * sizeof(double));
        if (mixed)
            for (int q = 0; q < 5; q++) buf(l, "A32", q, n * sizeof(float));
        if (mixed && l == 0)
            for (int q = 0; q < 4; q++) buf(l, "Alo", q, n * sizeof(float));
        if (bf16_wanted(p, l, dims[l][0], n, (size_t)g->nx * g->ny * g->nz, nl))
            for (int q = 0; q < 4; q++) buf(l, "Abf", q, n * sizeof(unsigned short));
        if (l > 0) {
            buf(l, "vec", 0, n * ts);
            buf(l, "vec", 1, n * ts);
        }
        buf(l, "vec", 2, n * ts);
        if (dirichlet_mask(g)) {
            const size_t nb = 2 * ((size_t)dims[l][1] * dims[l][2] + (size_t)dims[l][0] * dims[l][2] +
                                   (size_t)dims[l][0] * dims[l][1]);
            buf(l, "bnd", 0, nb * sizeof(double));
        }
    }
    const size_t n0 = (size_t)g->nx * g->ny * g->nz;
    buf(0, "b", 0, n0 * sizeof(double));
    buf(0, "dE", 0, n0 * sizeof(double));
    {
        Dims d0;
        d0.nx = g->nx; d0.ny = g->ny; d0.nz = g->nz;
        d0.px = d0.py = d0.pz = 0;
        d0.n = (long long)n0;
        long long blocks = 0;
        int cap = 0;
        face_list_shape(d0, p->limiter, &blocks, &cap);
        if (cap > 0) {
            buf(0, "flist", 0, (size_t)blocks * cap * sizeof(unsigned));
            buf(0, "flist", 1, (size_t)blocks * sizeof(unsigned));
        }
    }
    for (int q = 0; q < 6; q++) buf(0, "cg", q, n0 * ts);
    if (ps_wanted(p, n0, nl)) buf(0, "ps", 0, sizeof(PsReq));
    const size_t nc = (size_t)dims[nl - 1][0] * dims[nl - 1][1] * dims[nl - 1][2];
    buf(0, "dense", 0, nc * nc * sizeof(double));
    buf(0, "dense", 1, nc * nc * sizeof(double));
    buf(0, "red", 0, 8 * RED_MAX_BLOCKS * sizeof(double));
    buf(0, "red", 1, 256);
    buf(0, "red", 2, NUM_SLOTS * sizeof(double));
}

}  // namespace

constexpr int MAX_CHUNKS = 16;

struct fld_ctx {
    fld_grid g;
    fld_params p;
    cudaStream_t s;
    bool mixed;
    int nl;
    Level L[MAX_LEVELS];
    double* b;
    // refinement unknown: FP64, or (mixed mode) a double-float pair per cell
    // scaled by the step's power of two (k_mixed.cu)
    double* dE;
    int ks;           // mixed mode: the inner solve's scale 2^ks
    FaceList flist;   // faces left by the FP32 limiter screen
    void* cg[6];   // r, z, p0, p1, q, x
    int nc;
    double *dense, *ainv;
    double* partials;
    unsigned* counter;
    double* sc;
    double* h_sc;  // pinned mirror of sc
    double *stage[3];
    cudaEvent_t e0, e1;
    PhysDev pd;
    bool assembled;
    std::vector<void*> allocs;
    // launch accounting and optional per-class event timing
    unsigned long long tmask;
    KStat kstat[K_NUM];
    struct Pend { int cls; double bytes; cudaEvent_t a, b; };
    std::vector<Pend> pend;
    std::vector<cudaEvent_t> pool;
    size_t pool_used;
    // CUDA graphs of one CG iteration, per solver precision (0 FP64, 1 FP32)
    // and p-buffer parity; the launches each graph holds, for accounting
    bool use_graphs;
    bool capturing;
    bool graphs_broken;
    cudaGraphExec_t gexec[2][2];
    cudaGraph_t graph[2][2];       // the captured iterations (children of batch graphs)
    unsigned long long id;         // unique per context, keys batch graphs
    unsigned graph_gen;            // bumped whenever the iteration graphs change
    cudaEvent_t ev_join;           // orders this stream with a batch stream
    // fld_step_batched: the context's work runs on a private stream (so the
    // contexts of a batch overlap even when they share one caller stream),
    // ordered after earlier and before later work on the caller's stream
    cudaStream_t bstream;
    cudaStream_t user_s;
    // state of the CG run in progress (see pcg_begin / pcg_after)
    struct Run {
        double thresh;
        int max_iter, k, cur;
        bool conv, done;
    } run;
    std::vector<std::pair<int, double>> glaunch[2][2];
    std::vector<std::pair<int, double>>* grec;   // launch list being captured
    double* h_one;   // pinned: [0] = 1.0 to raise S_FIRST, [1..3] loop slots
    // persistent inner solves (k_psolve): the device descriptor, its host
    // copy and whether this context uses them
    PsReq* ps_req;
    PsReq ps_host;
    bool ps;
    int tail_from;   // first level of the persistent coarse tail (-1: none)
    int tail_cluster;   // CTAs of the tail's cluster
    // device-side CG loop per solver precision: a while-node graph whose
    // body is one iteration, the p copy and the convergence test
    cudaGraph_t loop_graph[2];
    cudaGraphExec_t loop_exec[2];
    std::vector<std::pair<int, double>> loop_launch[2];
    // host-buffer steps: side streams that split the copies over several
    // copy engines, forked from and joined to the context's stream
    cudaStream_t cstream[4];
    cudaEvent_t cfork, cjoin[4];
    // overlapped host-buffer steps: one event per plane chunk and the
    // chunks' reduction slots (MAX_CHUNKS x NUM_SLOTS)
    cudaEvent_t chunk_ev[MAX_CHUNKS];
    double* chunk_sc;
};

namespace {

RedArgs red(fld_ctx* c, int op, int slot0 = 0, int slot1 = 0, int first = 0) {
    RedArgs r;
    r.partials = c->partials;
    r.counter = c->counter;
    r.sc = c->sc;
    r.op = op;
    r.slot0 = slot0;
    r.slot1 = slot1;
    r.first = first;
    return r;
}

cudaEvent_t pool_event(fld_ctx* c) {
    if (c->pool_used == c->pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        c->pool.push_back(e);
    }
    return c->pool[c->pool_used++];
}

// Counts one kernel launch of class cls moving `bytes` of algorithmic
// traffic; when the class is selected for timing, brackets it with events.
struct KScope {
    fld_ctx* c;
    int cls;
    double bytes;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t st;   // the stream of the launch (the context's by default)
    KScope(fld_ctx* c_, int cls_, double bytes_, cudaStream_t s_ = nullptr)
        : c(c_), cls(cls_), bytes(bytes_), st(s_ ? s_ : c_->s) {
        if (c->capturing) {   // counted each time the graph is launched
            c->grec->push_back({cls, bytes});
            return;
        }
        c->kstat[cls].launches++;
        c->kstat[cls].bytes += bytes;
        if ((c->tmask >> cls) & 1ULL) {
            a = pool_event(c);
            b = pool_event(c);
            if (a && b) cudaEventRecord(a, st); else a = b = nullptr;
        }
    }
    ~KScope() {
        if (a) {
            cudaEventRecord(b, st);
            c->pend.push_back({cls, bytes, a, b});
        }
    }
};

// Called once the stream has drained: turn pending event pairs into times.
void harvest(fld_ctx* c) {
    for (auto& p : c->pend) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            c->kstat[p.cls].ms += ms;
            c->kstat[p.cls].timed++;
            c->kstat[p.cls].timed_bytes += p.bytes;
        } else {
            cudaGetLastError();
        }
    }
    c->pend.clear();
    c->pool_used = 0;
}

fld_status read_scalars(fld_ctx* c) {
    CUDA_TRY(cudaMemcpyAsync(c->h_sc, c->sc, NUM_SLOTS * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    CUDA_TRY(cudaStreamSynchronize(c->s));
    harvest(c);
    return FLD_OK;
}

template <class T>
Op<T> op_of(Level& L);
template <>
Op<double> op_of<double>(Level& L) { return L.A64; }
template <>
Op<float> op_of<float>(Level& L) { return L.A32; }

// FP32 sweeps on levels with nx % 4 == 0 use the four-cells-per-thread
// kernels; everything else the scalar ones.
template <class T>
bool use4(const Dims& d) {
    return std::is_same<T, float>::value && fine4_ok(d);
}
template <class T>
void smooth_zero_any(const Dims& d, Op<T> A, const T* r, T* z, cudaStream_t s, const Tune& tn) {
    if constexpr (std::is_same<T, float>::value) {
        if (fine4_ok(d)) return launch_smooth_zero4(d, A, r, z, s, tn);
    }
    launch_smooth_zero<T>(d, A, r, z, s);
}
template <class T>
void rb_colour_any(const Dims& d, Op<T> A, const T* r, T* z, int colour, cudaStream_t s, const Tune& tn) {
    if constexpr (std::is_same<T, float>::value) {
        if (fine4_ok(d)) return launch_rb_colour4(d, A, r, z, colour, s, tn);
    }
    launch_rb_colour<T>(d, A, r, z, colour, s);
}
template <class T>
void residual_any(const Dims& d, Op<T> A, const T* r, const T* z, T* res, cudaStream_t s, const Tune& tn,
                  bool after_zero_sweep, bool red_compressed) {
    if constexpr (std::is_same<T, float>::value) {
        if (fine4_ok(d)) return launch_residual4(d, A, r, z, res, s, tn, after_zero_sweep, red_compressed);
    }
    launch_residual<T>(d, A, r, z, res, s);
}

// red_compressed (FP32 levels where red_compress_ok): rf as k_residual4
// stores it after a zero-guess sweep
template <class T>
void restrict_any(const Dims& f, const Dims& c, const T* rf, T* rc, cudaStream_t s, const Tune& tn,
                  bool red_compressed) {
    if constexpr (std::is_same<T, float>::value) {
        if (fine4_ok(f)) return launch_restrict4(f, c, rf, rc, s, tn, red_compressed);
    }
    launch_restrict<T>(f, c, rf, rc, s);
}
template <class T>
void prolong_any(const Dims& f, const Dims& c, const T* ec, T* zf, cudaStream_t s, const Tune& tn) {
    if constexpr (std::is_same<T, float>::value) {
        if (fine4_ok(f)) return launch_prolong_add4(f, c, ec, zf, s, tn);
    }
    launch_prolong_add<T>(f, c, ec, zf, s);
}

// z = B r on level l (zero initial guess).  If dot is given and the last
// post-smoothing sweep of this level can carry it, <r, z> goes there (with
// reduction *dot) and *dot_done is set.
template <class T>
void vcycle(fld_ctx* c, int l, const T* r, T* z, const RedArgs* dot = nullptr, bool* dot_done = nullptr) {
    Level& L = c->L[l];
    cudaStream_t s = c->s;
    const double n = (double)L.d.n, ts = sizeof(T);
    // launches on levels below the finest are accounted as one class
    auto kc = [&](int cls) { return l == 0 ? cls : (int)K_COARSE_LEVELS; };
    if (l == c->nl - 1) {
        KScope k(c, kc(K_COARSE_APPLY), n * n * 8.0 + 2.0 * n * ts);
        launch_coarse_apply<T>((int)L.d.n, c->ainv, r, z, s);
        return;
    }
    if (l == c->tail_from) {
        // this level and all coarser ones in one cluster launch
        TailArgs<T> ta{};
        ta.nlev = c->nl - l;
        ta.pre = c->p.pre;
        ta.post = c->p.post;
        ta.paper_order = c->p.paper_order;
        ta.ainv = c->ainv;
        double bytes = 0.0;
        for (int q = 0; q < ta.nlev; q++) {
            Level& Q = c->L[l + q];
            TailLevel<T>& t = ta.L[q];
            t.d = Q.d;
            t.A = op_of<T>(Q);
            t.r = q == 0 ? const_cast<T*>(r) : (T*)Q.r;
            t.z = q == 0 ? z : (T*)Q.z;
            t.t = (T*)Q.t;
            // smoothing, residual, transfers: about 30 words per cell
            bytes += 30.0 * (double)Q.d.n * ts;
        }
        // the small levels in one CTA's shared memory, if their vectors fit
        ta.small_from = ta.nlev;
        for (int q = 0; q < ta.nlev; q++)
            if (ta.L[q].d.n <= TAIL_SMALL_CELLS) {
                size_t cells = 0;
                for (int u = q; u < ta.nlev; u++) cells += (size_t)ta.L[u].d.n;
                if (3 * cells * sizeof(T) <= TAIL_SMEM_MAX) ta.small_from = q;
                break;
            }
        KScope k(c, K_VTAIL, bytes);
        launch_vtail<T>(ta, c->tail_cluster, s);
        return;
    }
    Op<T> A = op_of<T>(L);
    T* t = (T*)L.t;
    const fld_params& p = c->p;
    // the levels of a mixed context may sweep with bfloat16 copies of their
    // coefficients (allocated only where bf16_wanted holds): half the bytes
    // of the face weights and the inverse diagonal
    const bool bf = std::is_same<T, float>::value && L.Abf.wx != nullptr;
    const double cw = bf ? 0.5 : 1.0;
    if (p.smoother == FLD_SMOOTH_RBGS) {
        if (p.pre >= 1) {
            KScope k(c, kc(K_SMOOTH_ZERO), (2.0 + 4.0 * cw) * n * ts);
            if constexpr (std::is_same<T, float>::value) {
                if (bf) launch_smooth_zero4(L.d, L.Abf, r, z, s, L.tune[TN_SMOOTH0]);
                else smooth_zero_any<T>(L.d, A, r, z, s, L.tune[TN_SMOOTH0]);
            } else {
                smooth_zero_any<T>(L.d, A, r, z, s, L.tune[TN_SMOOTH0]);
            }
        }
        for (int it = 1; it < p.pre; it++)
            for (int colour = 0; colour < 2; colour++) {
                KScope k(c, kc(K_RB_COLOUR), 6.5 * n * ts);
                rb_colour_any<T>(L.d, A, r, z, colour, s, L.tune[TN_RB]);
            }
        if (p.pre < 1) {
            cudaMemsetAsync(z, 0, L.d.n * sizeof(T), s);
        }
    } else {
        if (p.pre >= 1) {
            { KScope k(c, kc(K_JACOBI), 3.0 * n * ts); launch_jacobi<T>(L.d, A, r, z, z, p.jacobi_omega, true, s); }
            for (int it = 1; it < p.pre; it++) {
                { KScope k(c, kc(K_JACOBI), 8.0 * n * ts); launch_jacobi<T>(L.d, A, r, z, t, p.jacobi_omega, false, s); }
                cudaMemcpyAsync(z, t, L.d.n * sizeof(T), cudaMemcpyDeviceToDevice, s);
            }
        } else {
            cudaMemsetAsync(z, 0, L.d.n * sizeof(T), s);
        }
    }
    Level& C = c->L[l + 1];
    const double nc = (double)C.d.n;
    // one red/black sweep from zero (black last) leaves a residual that
    // needs neither r nor m and vanishes at black cells; where the x extent
    // allows it is stored red-compressed (see k_residual4)
    const bool zg = p.smoother == FLD_SMOOTH_RBGS && p.pre == 1 && std::is_same<T, float>::value &&
                    fine4_ok(L.d);
    const bool cmp = zg && red_compress_ok(L.d);
    {
        KScope k(c, kc(K_RESIDUAL), (cmp ? 1.5 + 3.0 * cw : (zg ? 2.0 + 3.0 * cw : 7.0)) * n * ts);
        if constexpr (std::is_same<T, float>::value) {
            if (bf) launch_residual4(L.d, L.Abf, z, t, s, L.tune[TN_RES], cmp);
            else residual_any<T>(L.d, A, r, z, t, s, L.tune[TN_RES], zg, cmp);
        } else {
            residual_any<T>(L.d, A, r, z, t, s, L.tune[TN_RES], zg, cmp);
        }
    }
    { KScope k(c, kc(K_RESTRICT), ((cmp ? 0.5 : 1.0) * n + nc) * ts);
      restrict_any<T>(L.d, C.d, t, (T*)C.r, s, L.tune[TN_RESTRICT], cmp); }
    vcycle<T>(c, l + 1, (const T*)C.r, (T*)C.z);
    if constexpr (std::is_same<T, float>::value) {
        // one fused post-sweep: t = z + P e_c, then black and red from t into z
        if (p.fused_post && !p.paper_order && p.smoother == FLD_SMOOTH_RBGS && p.post == 1 && post4_ok(L.d)) {
            { KScope k(c, kc(K_PROLONG), (2.0 * n + nc) * ts);
              launch_prolong_to4(L.d, C.d, (const float*)C.z, z, t, s); }
            KScope k(c, kc(K_POST_FUSED), 7.0 * n * ts);
            launch_post_smooth4(L.d, A, r, t, z, dot, s, L.tune[TN_POST]);
            if (dot) *dot_done = true;
            return;
        }
    }
    { KScope k(c, kc(K_PROLONG), (2.0 * n + nc) * ts); prolong_any<T>(L.d, C.d, (const T*)C.z, z, s, L.tune[TN_PROLONG]); }
    // post-sweeps black then red (symmetric cycle), or red then black as
    // the pre-sweeps (Table 1's order, paper_order)
    const int first = p.paper_order ? 0 : 1;
    for (int it = 0; it < p.post; it++) {
        if (p.smoother == FLD_SMOOTH_RBGS) {
            for (int q = 0; q < 2; q++) {
                const int colour = q == 0 ? first : 1 - first;
                const bool last = it == p.post - 1 && q == 1;
                KScope k(c, kc(K_RB_COLOUR), (2.5 + 4.0 * cw) * n * ts);
                if constexpr (std::is_same<T, float>::value) {
                    if (last && dot && use4<T>(L.d)) {
                        if (bf) launch_rb_colour4_dot(L.d, L.Abf, r, z, colour, *dot, s, L.tune[TN_RB]);
                        else launch_rb_colour4_dot(L.d, A, r, z, colour, *dot, s, L.tune[TN_RB]);
                        *dot_done = true;
                        continue;
                    }
                    if (bf) {
                        launch_rb_colour4(L.d, L.Abf, r, z, colour, s, L.tune[TN_RB]);
                        continue;
                    }
                }
                rb_colour_any<T>(L.d, A, r, z, colour, s, L.tune[TN_RB]);
            }
        } else {
            { KScope k(c, kc(K_JACOBI), 8.0 * n * ts); launch_jacobi<T>(L.d, A, r, z, t, p.jacobi_omega, false, s); }
            cudaMemcpyAsync(z, t, L.d.n * sizeof(T), cudaMemcpyDeviceToDevice, s);
        }
    }
}

// One CG iteration on the fine level in precision T (p parity cur): the
// V-cycle, <r,z>, p and q = A p, the x and r updates, and the scalars to the
// pinned host mirror.
// Whether the CG of precision T defers each update of x to the next
// iteration (FP32 four-cell kernels): the last one is then applied by
// launch_ir_update with the p of the last iteration, p[run.cur].
template <class T>
bool defers_x(fld_ctx* c) {
    return std::is_same<T, float>::value && use4<T>(c->L[0].d) && !c->ps;
}

template <class T>
void pcg_iteration(fld_ctx* c, int cur, bool mirror = true) {
    T* r = (T*)c->cg[0];
    T* z = (T*)c->cg[1];
    T* p[2] = {(T*)c->cg[2], (T*)c->cg[3]};
    T* q = (T*)c->cg[4];
    T* x = (T*)c->cg[5];
    Level& L0 = c->L[0];
    Op<T> A = op_of<T>(L0);
    const long long n = L0.d.n;
    const RedArgs dra = red(c, R_RHO);
    bool dot_done = false;
    vcycle<T>(c, 0, r, z, &dra, &dot_done);
    const double ts = sizeof(T);
    if (!dot_done) {
        KScope ks(c, K_DOT, 2.0 * n * ts);
        if constexpr (std::is_same<T, float>::value) {
            if (use4<T>(L0.d)) launch_dot4(n, r, z, red(c, R_RHO), c->s);
            else launch_dot<T>(n, r, z, red(c, R_RHO), c->s);
        } else {
            launch_dot<T>(n, r, z, red(c, R_RHO), c->s);
        }
    }
    // the FP32 four-cell kernels defer x += alpha p to the next iteration's
    // p/q kernel, which reads that p anyway (see defers_x)
    const bool defer = defers_x<T>(c);
    {
        KScope ks(c, K_CG_PMATVEC, (defer ? 10.0 : 8.0) * n * ts);
        if constexpr (std::is_same<T, float>::value) {
            if (defer)
                launch_cg_p_matvec4(L0.d, A, z, p[cur], p[cur ^ 1], q, red(c, R_ALPHA), c->s, L0.tune[TN_PMATVEC], x);
            else launch_cg_p_matvec<T>(L0.d, A, z, p[cur], p[cur ^ 1], q, red(c, R_ALPHA), c->s);
        } else {
            launch_cg_p_matvec<T>(L0.d, A, z, p[cur], p[cur ^ 1], q, red(c, R_ALPHA), c->s);
        }
    }
    {
        KScope ks(c, K_CG_UPDATE, (defer ? 3.0 : 6.0) * n * ts);
        if constexpr (std::is_same<T, float>::value) {
            if (defer) launch_cg_update4(n, nullptr, r, p[cur ^ 1], q, red(c, R_STORE1, S_RR), c->s);
            else launch_cg_update<T>(n, x, r, p[cur ^ 1], q, red(c, R_STORE1, S_RR), c->s);
        } else {
            launch_cg_update<T>(n, x, r, p[cur ^ 1], q, red(c, R_STORE1, S_RR), c->s);
        }
    }
    if (mirror) cudaMemcpyAsync(c->h_sc, c->sc, NUM_SLOTS * sizeof(double), cudaMemcpyDeviceToHost, c->s);
}

void drop_graphs(fld_ctx* c) {
    for (int a = 0; a < 2; a++) {
        for (int b = 0; b < 2; b++) {
            if (c->gexec[a][b]) cudaGraphExecDestroy(c->gexec[a][b]);
            if (c->graph[a][b]) cudaGraphDestroy(c->graph[a][b]);
            c->gexec[a][b] = nullptr;
            c->graph[a][b] = nullptr;
        }
        if (c->loop_exec[a]) cudaGraphExecDestroy(c->loop_exec[a]);
        if (c->loop_graph[a]) cudaGraphDestroy(c->loop_graph[a]);
        c->loop_exec[a] = nullptr;
        c->loop_graph[a] = nullptr;
    }
    c->graph_gen++;
}

// The device-side CG loop of precision T (built on first use), or null when
// graphs are off or unavailable.  Its body, captured into the while node,
// is one iteration at p parity 0 and its convergence test, then an IF node
// holding the iteration at p parity 1 and its test; the tests set the
// conditions.  One launch runs the whole solve, and the host synchronises
// once instead of per iteration.
template <class T>
cudaGraphExec_t loop_graph(fld_ctx* c) {
    const int prec = std::is_same<T, float>::value ? 1 : 0;
    if (!(c->use_graphs && !c->graphs_broken && c->tmask == 0)) return nullptr;
    cudaGraphExec_t& ge = c->loop_exec[prec];
    if (ge) return ge;
    cudaGraph_t g = nullptr;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
    cudaGraphConditionalHandle h = 0;
    cudaGraph_t body = nullptr;
    if (ok) ok = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
        if (ok) body = np.conditional.phGraph_out[0];
    }
    // the body holds two iterations, p parity 0 then (under an IF node whose
    // condition the first test sets as well) parity 1, so the new p never
    // has to be copied into the old one
    cudaGraphConditionalHandle hi = 0;
    if (ok) ok = cudaGraphConditionalHandleCreate(&hi, body, 0, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) ok = cudaStreamBeginCaptureToGraph(c->s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                 cudaSuccess;
    if (ok) {
        c->loop_launch[prec].clear();
        c->grec = &c->loop_launch[prec];
        c->capturing = true;
        pcg_iteration<T>(c, 0, false);
        launch_cg_check(h, c->sc, c->s, &hi);
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        const cudaGraphEdgeData* ed = nullptr;
        size_t nd = 0;
        ok = cudaStreamGetCaptureInfo(c->s, &cs, nullptr, &cg, &deps, &ed, &nd) == cudaSuccess &&
             cs == cudaStreamCaptureStatusActive;
        cudaGraphNode_t ifnode = nullptr;
        cudaGraph_t ifbody = nullptr;
        if (ok) {
            cudaGraphNodeParams ip = {};
            ip.type = cudaGraphNodeTypeConditional;
            ip.conditional.handle = hi;
            ip.conditional.type = cudaGraphCondTypeIf;
            ip.conditional.size = 1;
            ok = cudaGraphAddNode(&ifnode, cg, deps, ed, nd, &ip) == cudaSuccess;
            if (ok) ifbody = ip.conditional.phGraph_out[0];
        }
        if (ok)
            ok = cudaStreamUpdateCaptureDependencies(c->s, &ifnode, nullptr, 1, cudaStreamSetCaptureDependencies) ==
                 cudaSuccess;
        c->capturing = false;
        cudaGraph_t out = nullptr;
        const bool ended = cudaStreamEndCapture(c->s, &out) == cudaSuccess;
        ok = ok && ended;
        if (ok) ok = cudaStreamBeginCaptureToGraph(c->s, ifbody, nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            // its launches are the same as the first iteration's, which the
            // host counts once per executed iteration
            std::vector<std::pair<int, double>> second;
            c->grec = &second;
            c->capturing = true;
            pcg_iteration<T>(c, 1, false);
            launch_cg_check(h, c->sc, c->s);
            c->capturing = false;
            c->grec = nullptr;
            cudaGraph_t out2 = nullptr;
            ok = cudaStreamEndCapture(c->s, &out2) == cudaSuccess;
        }
    }
    if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
    if (!ok) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        ge = nullptr;
        c->graphs_broken = true;
        return nullptr;
    }
    c->loop_graph[prec] = g;
    return ge;
}

// The captured and instantiated iteration of precision T and parity cur
// (capturing it on first use), or null when graphs are off or unavailable.
template <class T>
cudaGraphExec_t pcg_graph(fld_ctx* c, int cur) {
    const int prec = std::is_same<T, float>::value ? 1 : 0;
    if (!(c->use_graphs && !c->graphs_broken && c->tmask == 0)) return nullptr;
    cudaGraphExec_t& ge = c->gexec[prec][cur];
    if (!ge) {
        // capture (records, does not run) and instantiate this parity
        c->glaunch[prec][cur].clear();
        c->grec = &c->glaunch[prec][cur];
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            c->capturing = true;
            pcg_iteration<T>(c, cur);
            c->capturing = false;
            ok = cudaStreamEndCapture(c->s, &g) == cudaSuccess && g;
        }
        if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
        if (!ok) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            ge = nullptr;
            c->graphs_broken = true;
            return nullptr;
        }
        c->graph[prec][cur] = g;
        c->graph_gen++;
    }
    return ge;
}

// Count the launches a graph of this context holds, once per replay.
void count_graph_launches(fld_ctx* c, int prec, int cur) {
    for (auto& e : c->glaunch[prec][cur]) {
        c->kstat[e.first].launches++;
        c->kstat[e.first].bytes += e.second;
    }
}

// Start preconditioned CG in precision T: r holds the initial residual
// (x = 0), r0sq = ||r||^2; it stops when ||r||^2 <= rtol^2 r0sq.
template <class T>
fld_status pcg_begin(fld_ctx* c, double r0sq, double rtol, int max_iter) {
    if (!(std::is_same<T, float>::value && c->ps)) {
        CUDA_TRY(cudaMemsetAsync(c->cg[2], 0, c->L[0].d.n * sizeof(T), c->s));
        // beta = 0 in the first iteration, signalled on the device so that
        // every iteration launches the same work; alpha = 0 before it, so
        // that a deferred update of x adds nothing there (the persistent
        // solve keeps these in registers)
        CUDA_TRY(cudaMemcpyAsync(c->sc + S_FIRST, c->h_one, sizeof(double), cudaMemcpyHostToDevice, c->s));
        CUDA_TRY(cudaMemsetAsync(c->sc + S_ALPHA, 0, sizeof(double), c->s));
        if (std::is_same<T, float>::value) {
            // the FP32 solve starts from x = 0: the first p/q kernel writes
            // it where the update of x is deferred to that kernel, else here
            // (the FP64 solve's caller clears its x)
            if (defers_x<T>(c))
                CUDA_TRY(cudaMemcpyAsync(c->sc + S_XZERO, c->h_one, sizeof(double), cudaMemcpyHostToDevice, c->s));
            else
                CUDA_TRY(cudaMemsetAsync(c->cg[5], 0, c->L[0].d.n * sizeof(T), c->s));
        }
    }
    c->run.thresh = rtol * rtol * r0sq;
    c->run.max_iter = max_iter;
    c->run.k = 0;
    c->run.cur = 0;
    c->run.conv = false;
    c->run.done = max_iter < 1;
    return FLD_OK;
}

// Enqueue the next iteration: the captured graph, or the launches.
template <class T>
fld_status pcg_enqueue(fld_ctx* c) {
    const int prec = std::is_same<T, float>::value ? 1 : 0;
    cudaGraphExec_t ge = pcg_graph<T>(c, c->run.cur);
    if (ge) {
        CUDA_TRY(cudaGraphLaunch(ge, c->s));
        count_graph_launches(c, prec, c->run.cur);
    } else {
        pcg_iteration<T>(c, c->run.cur);
    }
    CUDA_TRY(cudaGetLastError());
    return FLD_OK;
}

// After an iteration has completed (its scalars are in the host mirror).
fld_status pcg_after(fld_ctx* c) {
    harvest(c);
    auto& R = c->run;
    R.k++;
    R.cur ^= 1;
    if (c->h_sc[S_NONFINITE] != 0.0) {
        R.done = true;
        return set_err(FLD_ENONFINITE, "non-finite value in a CG reduction at iteration %d", R.k);
    }
    if (c->h_sc[S_RR] <= R.thresh) {
        R.conv = true;
        R.done = true;
    } else if (R.k >= R.max_iter) {
        R.done = true;
    }
    return FLD_OK;
}

// The threshold, iteration cap and iteration counter of a whole inner solve
// run on the device (loop graph or persistent kernel) to their slots.
fld_status whole_slots(fld_ctx* c) {
    c->h_one[1] = c->run.thresh;
    c->h_one[2] = (double)c->run.max_iter;
    c->h_one[3] = 0.0;
    CUDA_TRY(cudaMemcpyAsync(c->sc + S_THRESH, c->h_one + 1, 3 * sizeof(double), cudaMemcpyHostToDevice, c->s));
    return FLD_OK;
}

// One launch of the persistent inner solves of contexts cs (all with ps
// set and their slots written) on stream s: the work list in decreasing
// grid size, so the largest solves start first.
fld_status ps_enqueue(std::vector<fld_ctx*> cs, cudaStream_t s) {
    if (cs.empty()) return FLD_OK;
    if ((int)cs.size() > PS_MAX_BATCH) return set_err(FLD_EINVAL, "more than %d persistent solves in one launch", PS_MAX_BATCH);
    // cluster requests first, then the single-CTA ones, each largest first
    std::stable_sort(cs.begin(), cs.end(), [](fld_ctx* a, fld_ctx* b) {
        if (a->ps_host.cta != b->ps_host.cta) return a->ps_host.cta < b->ps_host.cta;
        return a->L[0].d.n > b->L[0].d.n;
    });
    PsBatch pb{};
    pb.n = (int)cs.size();
    pb.ncl = 0;
    while (pb.ncl < pb.n && !cs[pb.ncl]->ps_host.cta) pb.ncl++;
    pb.ticket = cs[0]->counter + 32;
    size_t smem = 0;
    for (int i = 0; i < pb.n; i++) {
        pb.req[i] = cs[i]->ps_req;
        const size_t b = psolve_smem_bytes(cs[i]->ps_host);
        if (b > smem) smem = b;
    }
    {
        KScope k(cs[0], K_PSOLVE, 0.0, s);
        CUDA_TRY(launch_psolve(pb, smem, s));
    }
    return FLD_OK;
}

// After a whole inner solve has completed and its scalars are in the host
// mirror: the run state as after its last iteration.
fld_status whole_after(fld_ctx* c, int prec, bool graph) {
    const int k = (int)c->h_sc[S_KITER];
    if (graph)
        for (int q = 0; q < k; q++)
            for (auto& e : c->loop_launch[prec]) {
                c->kstat[e.first].launches++;
                c->kstat[e.first].bytes += e.second;
            }
    c->run.k = k;
    c->run.cur = k & 1;   // as after k single iterations: the last p is p[cur]
    c->run.done = true;
    if (c->h_sc[S_NONFINITE] != 0.0)
        return set_err(FLD_ENONFINITE, "non-finite value in a CG reduction at iteration %d", k);
    c->run.conv = c->h_sc[S_RR] <= c->run.thresh;
    return FLD_OK;
}

template <class T>
fld_status pcg(fld_ctx* c, double r0sq, double rtol, int max_iter, int* iters, bool* converged) {
    fld_status st = pcg_begin<T>(c, r0sq, rtol, max_iter);
    if (st) return st;
    if (std::is_same<T, float>::value && c->ps && !c->run.done) {
        // the whole solve in one persistent launch
        if ((st = whole_slots(c))) return st;
        if ((st = ps_enqueue({c}, c->s))) return st;
        if ((st = read_scalars(c))) return st;
        if ((st = whole_after(c, 1, false))) return st;
        *iters = c->run.k;
        *converged = c->run.conv;
        return FLD_OK;
    }
    cudaGraphExec_t le = c->run.done ? nullptr : loop_graph<T>(c);
    if (le) {
        // the whole loop on the device: threshold, iteration cap and counter
        // to their slots, one graph launch, one synchronisation
        const int prec = std::is_same<T, float>::value ? 1 : 0;
        if ((st = whole_slots(c))) return st;
        CUDA_TRY(cudaGraphLaunch(le, c->s));
        CUDA_TRY(cudaGetLastError());
        if ((st = read_scalars(c))) return st;
        if ((st = whole_after(c, prec, true))) return st;
        *iters = c->run.k;
        *converged = c->run.conv;
        return FLD_OK;
    }
    while (!c->run.done) {
        if ((st = pcg_enqueue<T>(c))) return st;
        CUDA_TRY(cudaStreamSynchronize(c->s));
        if ((st = pcg_after(c))) return st;
    }
    *iters = c->run.k;
    *converged = c->run.conv;
    return FLD_OK;
}

fld_status alloc_ctx(fld_ctx* c) {
    int li = -1;
    fld_status st = FLD_OK;
    plan(&c->g, &c->p, [&](int l, const char* kind, int q, size_t bytes) {
        if (st != FLD_OK) return;
        void* ptr = nullptr;
        cudaError_t e = cudaMalloc(&ptr, bytes < 256 ? 256 : bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            st = set_err(FLD_ENOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
            return;
        }
        c->allocs.push_back(ptr);
        Level& L = c->L[l];
        (void)li;
        if (!strcmp(kind, "A64")) {
            double* d = (double*)ptr;
            if (q == 0) L.A64.m = d; else if (q == 1) L.A64.wx = d; else if (q == 2) L.A64.wy = d;
            else if (q == 3) L.A64.wz = d; else L.A64.invd = d;
        } else if (!strcmp(kind, "A32")) {
            float* f = (float*)ptr;
            if (q == 0) L.A32.m = f; else if (q == 1) L.A32.wx = f; else if (q == 2) L.A32.wy = f;
            else if (q == 3) L.A32.wz = f; else L.A32.invd = f;
        } else if (!strcmp(kind, "Abf")) {
            unsigned short* h = (unsigned short*)ptr;
            if (q == 0) L.Abf.wx = h; else if (q == 1) L.Abf.wy = h; else if (q == 2) L.Abf.wz = h;
            else L.Abf.invd = h;
        } else if (!strcmp(kind, "Alo")) {
            float* f = (float*)ptr;
            if (q == 0) L.Alo.m = f; else if (q == 1) L.Alo.wx = f; else if (q == 2) L.Alo.wy = f;
            else L.Alo.wz = f;
        } else if (!strcmp(kind, "vec")) {
            if (q == 0) L.r = ptr; else if (q == 1) L.z = ptr; else L.t = ptr;
        } else if (!strcmp(kind, "bnd")) {
            L.bnd.w = (double*)ptr;
        } else if (!strcmp(kind, "b")) c->b = (double*)ptr;
        else if (!strcmp(kind, "dE")) c->dE = (double*)ptr;
        else if (!strcmp(kind, "flist")) {
            if (q == 0) c->flist.entries = (unsigned*)ptr;
            else c->flist.counts = (unsigned*)ptr;
        }
        else if (!strcmp(kind, "cg")) c->cg[q] = ptr;
        else if (!strcmp(kind, "ps")) c->ps_req = (PsReq*)ptr;
        else if (!strcmp(kind, "dense")) { if (q == 0) c->dense = (double*)ptr; else c->ainv = (double*)ptr; }
        else if (!strcmp(kind, "red")) {
            if (q == 0) c->partials = (double*)ptr;
            else if (q == 1) c->counter = (unsigned*)ptr;
            else c->sc = (double*)ptr;
        }
    });
    return st;
}

void free_ctx(fld_ctx* c) {
    if (!c) return;
    if (c->s) cudaStreamSynchronize(c->s);
    for (void* p : c->allocs) cudaFree(p);
    for (int q = 0; q < 3; q++)
        if (c->stage[q]) cudaFree(c->stage[q]);
    if (c->h_sc) cudaFreeHost(c->h_sc);
    for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
    drop_graphs(c);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->bstream) cudaStreamDestroy(c->bstream);
    for (int q = 0; q < 4; q++) {
        if (c->cstream[q]) cudaStreamDestroy(c->cstream[q]);
        if (c->cjoin[q]) cudaEventDestroy(c->cjoin[q]);
    }
    if (c->cfork) cudaEventDestroy(c->cfork);
    for (int q = 0; q < MAX_CHUNKS; q++)
        if (c->chunk_ev[q]) cudaEventDestroy(c->chunk_ev[q]);
    if (c->chunk_sc) cudaFree(c->chunk_sc);
    if (c->h_one) cudaFreeHost(c->h_one);
    if (c->e0) cudaEventDestroy(c->e0);
    if (c->e1) cudaEventDestroy(c->e1);
    delete c;
}

// ---- mixed-precision refinement (kernels in k_mixed.cu)

RedArgs red_irres(fld_ctx* c, int ks) {
    RedArgs r = red(c, R_IRRES);
    r.aux = std::ldexp(1.0, ks);
    return r;
}

// The first refinement's right-hand side: r32 = b / 2^ks with 2^ks the
// power of two above max |b| (in the host mirror after the assembly).
void scale_rhs_enqueue(fld_ctx* c) {
    const long long n = c->L[0].d.n;
    c->ks = exp_above(c->h_sc[S_RMAX]);
    KScope k(c, K_IR_SCALE, 12.0 * n);
    launch_ir_scale_b(n, c->b, c->ks, (float*)c->cg[0], red_irres(c, c->ks), c->s);
}

// x64 += 2^ks (x32 + alpha p_last) after an inner solve (x64 = ... after
// the first one).
void update_enqueue(fld_ctx* c, bool assign) {
    const long long n = c->L[0].d.n;
    const bool defer = defers_x<float>(c);
    KScope k(c, K_IR_UPDATE, ((assign ? 12.0 : 20.0) + (defer ? 4.0 : 0.0)) * n);
    launch_ir_update_mx(n, c->dE, (const float*)c->cg[5], c->sc, assign, c->ks,
                        defer ? (const float*)c->cg[2 + c->run.cur] : nullptr, c->sc, c->pd.dt_exp, c->s);
}

// The scale of the next inner solve, predicted from the one just done: its
// residual fell from ||r32_0|| to ||r32|| (S_RR), so the new residual's
// largest entry is about 2^ks ||r32||.
int next_scale(fld_ctx* c) {
    const double rr = c->h_sc[S_RR];
    return rr > 0.0 && std::isfinite(rr) ? c->ks + exp_above(std::sqrt(rr)) : c->ks - 30;
}

// The refinement residual with the scale 2^ks; write: also the next inner
// solve's right-hand side r32 (else only its norms, for a residual that is
// expected to meet the tolerance).
void residual_enqueue(fld_ctx* c, int ks, bool write) {
    Level& L0 = c->L[0];
    KScope k(c, K_IR_RESID, (write ? 52.0 : 48.0) * L0.d.n);
    launch_ir_residual(L0.d, L0.A32, L0.Alo, c->b, c->dE, ks, (float*)c->cg[0], write, red_irres(c, ks), c->sc,
                       c->pd.dt_exp, c->s);
}

// After a residual launched with scale 2^ks has reported its largest entry:
// 0 if it stays well inside the FP32 range (or is 0), 1 with ks corrected
// for a relaunch, -1 if it stays non-finite after a few corrections.
int scale_fix(fld_ctx* c, int& ks, int attempt) {
    const double mx = c->h_sc[S_RMAX];
    const bool nonfinite = c->h_sc[S_NONFINITE] != 0.0 || !std::isfinite(mx);
    if (!nonfinite && (mx == 0.0 || (mx >= 0x1p-40 && mx <= 0x1p40))) return 0;
    if (attempt >= 3) return nonfinite ? -1 : 0;
    ks += nonfinite ? 100 : exp_above(mx);
    return 1;
}

// Whether the refinement residual after the inner solve just done is
// expected to meet the tolerance (with a factor 2 of margin): the inner
// solve's final ||r32|| scaled by 2^ks against ||b||.  Its residual is then
// launched for its norms only.
bool expect_converged(fld_ctx* c, double bb, double rtol) {
    const double rr = c->h_sc[S_RR];
    return rr >= 0.0 && std::isfinite(rr) && bb > 0.0 && std::ldexp(std::sqrt(rr), c->ks) <= 0.5 * rtol * std::sqrt(bb);
}

// ||b - A x|| / ||b|| from the scaled residual's norm.
double scaled_rel_res(fld_ctx* c, double bb) {
    return std::ldexp(std::sqrt(c->h_sc[S_R0]), c->ks) / std::sqrt(bb);
}

fld_status solve_impl(fld_ctx* c, fld_info* info) {
    const long long n = c->L[0].d.n;
    const double bb = c->h_sc[S_BB];
    fld_info inf{};
    if (bb == 0.0) {
        CUDA_TRY(cudaMemsetAsync(c->dE, 0, n * sizeof(double), c->s));
        if (info) *info = inf;
        return FLD_OK;
    }
    const double rtol = c->p.rtol;
    fld_status st = FLD_OK;
    bool conv = false;
    if (!c->mixed) {
        CUDA_TRY(cudaMemcpyAsync(c->cg[0], c->b, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
        CUDA_TRY(cudaMemsetAsync(c->cg[5], 0, n * sizeof(double), c->s));
        int it = 0;
        st = pcg<double>(c, bb, rtol, c->p.max_iter, &it, &conv);
        inf.iters = it;
        if (st) return st;
        CUDA_TRY(cudaMemcpyAsync(c->dE, c->cg[5], n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
        { KScope k(c, K_RESIDUAL64, 48.0 * n);
          launch_residual64(c->L[0].d, c->L[0].A64, nullptr, c->b, c->dE, nullptr,
                            red(c, R_STORE_SUM_MAX, S_TRUE_RR, S_RMAX), c->s); }
        if ((st = read_scalars(c))) return st;
        inf.rel_res = std::sqrt(c->h_sc[S_TRUE_RR] / bb);
    } else {
        // Iterative refinement: the residual in double-float arithmetic, the
        // FP32 inner MG-PCG on it scaled by a power of two 2^ks, the FP64
        // update.  The first residual is b itself (x = 0), scaled by the
        // power of two above max |b|, which the assembly reduced.
        int inner_total = 0, outer = 0;
        inf.rel_res = 1.0;
        scale_rhs_enqueue(c);
        if ((st = read_scalars(c))) return st;
        if (c->h_sc[S_NONFINITE] != 0.0) return set_err(FLD_ENONFINITE, "non-finite scaled right-hand side");
        for (;;) {
            int it = 0;
            bool iconv = false;
            // the inner solve need not reduce its residual further than the
            // outer target requires (with a factor 2 of margin)
            double irtol = 0.5 * rtol / inf.rel_res;
            if (irtol < c->p.inner_rtol) irtol = c->p.inner_rtol;
            if (irtol > 0.5) irtol = 0.5;
            st = pcg<float>(c, c->h_sc[S_R0], irtol, c->p.max_iter - inner_total, &it, &iconv);
            if (st) return st;
            inner_total += it;
            update_enqueue(c, outer == 0);
            outer++;
            const bool write = !expect_converged(c, bb, rtol);
            int ks = next_scale(c);
            for (int attempt = 0;; attempt++) {
                residual_enqueue(c, ks, write);
                if ((st = read_scalars(c))) return st;
                const int fix = scale_fix(c, ks, attempt);
                if (fix == 0) break;
                if (fix < 0) return set_err(FLD_ENONFINITE, "non-finite refinement residual after %d refinements", outer);
                CUDA_TRY(cudaMemsetAsync(c->sc + S_NONFINITE, 0, sizeof(double), c->s));
            }
            c->ks = ks;
            inf.rel_res = scaled_rel_res(c, bb);
            if (inf.rel_res <= rtol) { conv = true; break; }
            if (inner_total >= c->p.max_iter) break;
            if (!write) {
                // expected to converge and did not: the right-hand side of
                // the next inner solve (same scale, same norms)
                residual_enqueue(c, ks, true);
                if ((st = read_scalars(c))) return st;
            }
        }
        inf.iters = inner_total;
        inf.outer_iters = outer;
    }
    inf.status = conv ? FLD_OK : FLD_ENOCONV;
    if (info) *info = inf;
    if (!conv)
        return set_err(FLD_ENOCONV, "no convergence: relative residual %.3e > rtol %.3e after %d iterations",
                       inf.rel_res, rtol, inf.iters);
    return FLD_OK;
}

// Assembly (Sec. 2 limiter, Sec. 3.2 system) and multigrid setup.
//
// Fine-level faces over the z-blocks [zb0, zb0 + nzb) of the assembly
// decomposition (nzb < 0: all): limiter and weights, then the FP64 pass over
// the faces the screen listed.  frac: the share of the cells, for the
// launch statistics.
void assemble_faces_range(fld_ctx* c, const double* E, const double* nHI, const double* eta, int zb0,
                          int nzb, double frac) {
    Level& L0 = c->L[0];
    const double n0 = (double)L0.d.n * frac;
    if (c->mixed) {
        // double-float limiter in place (k_mixed.cu): reads E, n_HI, eta,
        // writes m and the three weights as float pairs
        { KScope k(c, K_ASM_FACES, n0 * 56.0);
          launch_asm_faces_mx(L0.d, c->pd, E, nHI, eta, L0.A32, L0.Alo, c->sc, c->flist, c->s, zb0, nzb); }
        if (c->flist.entries) {
            KScope k(c, K_ASM_FIX, 0.0);
            launch_asm_fix_mx(L0.d, c->pd, E, nHI, L0.A32, L0.Alo, c->flist, c->s, zb0, nzb);
        }
        return;
    }
    Op<float> op32{};
    { KScope k(c, K_ASM_FACES, n0 * 56.0);
      launch_assemble_faces(L0.d, c->pd, E, nHI, eta, L0.A64, op32, c->sc, c->flist, c->s, zb0, nzb); }
    if (c->flist.entries) {
        KScope k(c, K_ASM_FIX, 0.0);
        launch_assemble_fix(L0.d, c->pd, E, nHI, L0.A64, op32, c->flist, c->s, zb0, nzb);
    }
}

// Right-hand side over z-blocks (it needs the faces of the z-block above).
void assemble_rhs_range(fld_ctx* c, const double* E, const double* nHI, const double* eta, int zb0, int nzb,
                        double frac, const RedArgs& ra) {
    Level& L0 = c->L[0];
    if (c->mixed) {
        // reads E, n_HI, eta, the df weights and the FP32 mass term; writes
        // b and the FP32 inverse diagonal
        KScope k(c, K_ASM_RHS, (double)L0.d.n * frac * 64.0);
        launch_asm_rhs_mx(L0.d, c->pd, E, nHI, eta, L0.A32, L0.Alo, c->b, L0.bnd, ra, c->sc, c->s, zb0, nzb,
                          L0.Abf);
        return;
    }
    KScope k(c, K_ASM_RHS, (double)L0.d.n * frac * 72.0);
    launch_assemble_rhs(L0.d, c->pd, E, nHI, eta, L0.A64, Op<float>{}, c->b, nullptr, L0.bnd, ra, c->s, zb0, nzb);
}

// The coarse levels, the coarsest-grid setup, then the scalars to the host
// mirror (assemble_finish reads them).
fld_status assemble_coarse(fld_ctx* c) {
    cudaStream_t s = c->s;
    // the mixed solver's coarse operators are formed in FP32 from the FP32
    // operator of the level above (its FP32 cycle is their only reader)
    for (int l = 1; l < c->nl; l++) {
        Level& F = c->L[l - 1];
        Level& C = c->L[l];
        const double nf = (double)F.d.n, nc = (double)C.d.n;
        if (c->mixed) {
            { KScope k(c, K_COARSEN, 16.0 * (nf + nc)); launch_coarsen<float>(F.d, C.d, F.A32, C.A32, s); }
            for (int sd = 0; sd < 6; sd++)
                if ((C.bnd.mask >> sd) & 1) {
                    KScope k(c, K_COARSEN, 0.0);
                    launch_coarsen_bnd<float>(F.d, C.d, sd, F.bnd, C.bnd, C.A32, s);
                }
            { KScope k(c, K_INVD, 20.0 * nc); launch_invd<float>(C.d, C.A32, C.A32, s); }
            if (C.Abf.wx) {
                KScope k(c, K_INVD, 24.0 * nc);
                launch_op_to_bf16(C.d.n, C.A32, C.Abf, s);
            }
        } else {
            { KScope k(c, K_COARSEN, 32.0 * (nf + nc)); launch_coarsen<double>(F.d, C.d, F.A64, C.A64, s); }
            for (int sd = 0; sd < 6; sd++)
                if ((C.bnd.mask >> sd) & 1) {
                    KScope k(c, K_COARSEN, 0.0);
                    launch_coarsen_bnd<double>(F.d, C.d, sd, F.bnd, C.bnd, C.A64, s);
                }
            { KScope k(c, K_INVD, 40.0 * nc); launch_invd<double>(C.d, C.A64, C.A64, s); }
        }
    }
    Level& Lc = c->L[c->nl - 1];
    { const double nc = (double)Lc.d.n;
      KScope k(c, K_COARSE_SETUP, 16.0 * nc * nc);
      // the mixed solver's cycle is FP32 throughout, also on a one-level grid
      if (c->mixed) launch_coarse_setup<float>(Lc.d, Lc.A32, c->dense, c->ainv, c->sc, true, s);
      else launch_coarse_setup<double>(Lc.d, Lc.A64, c->dense, c->ainv, c->sc, false, s); }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(c->h_sc, c->sc, NUM_SLOTS * sizeof(double), cudaMemcpyDeviceToHost, s));
    return FLD_OK;
}

// Enqueue the whole assembly: fine-level faces, limiter and right-hand
// side, coarse levels and coarsest-grid setup, then the scalars to the host
// mirror; assemble_finish reads them.
fld_status assemble_enqueue(fld_ctx* c, const double* E, const double* nHI, const double* eta) {
    if (!c) return set_err(FLD_EINVAL, "null context");
    if (!E || !nHI || !eta) return set_err(FLD_EINVAL, "null field pointer");
    c->assembled = false;
    CUDA_TRY(cudaMemsetAsync(c->sc, 0, NUM_SLOTS * sizeof(double), c->s));
    assemble_faces_range(c, E, nHI, eta, 0, -1, 1.0);
    assemble_rhs_range(c, E, nHI, eta, 0, -1, 1.0, red(c, R_STORE_SUM_MAX, S_BB, S_RMAX));
    return assemble_coarse(c);
}

// After the assembly's scalars arrived: input checks.
fld_status assemble_finish(fld_ctx* c) {
    harvest(c);
    if (c->h_sc[S_BAD] == 1.0)
        return set_err(FLD_EINVAL, "E, n_HI and eta must be finite and >= 0");
    if (c->h_sc[S_BAD] == 2.0)
        return set_err(FLD_ENONFINITE, "coarsest-grid operator is not positive definite");
    if (c->h_sc[S_NONFINITE] != 0.0 || !std::isfinite(c->h_sc[S_BB]))
        return set_err(FLD_ENONFINITE, "non-finite right-hand side");
    c->assembled = true;
    return FLD_OK;
}

fld_status assemble_impl(fld_ctx* c, const double* E, const double* nHI, const double* eta) {
    fld_status st = assemble_enqueue(c, E, nHI, eta);
    if (st) return st;
    CUDA_TRY(cudaStreamSynchronize(c->s));
    return assemble_finish(c);
}


// Device constants of a step with time step dt (the operator depends on dt
// through the face weights and the mass term).
void fill_physdev(fld_ctx* c, double dt) {
    const fld_params* p = &c->p;
    const fld_grid* g = &c->g;
    PhysDev& pd = c->pd;
    c->p.dt = dt;
    pd.dt = dt;
    pd.c = p->c;
    pd.Dmax = p->dmax_coef * p->c * p->L_unit;
    pd.Rmin = p->rmin_coef / p->L_unit;
    pd.sigma = p->sigma;
    pd.adot = p->adot_over_a;
    // the equation's gradients are proper: widths a * (comoving width)
    pd.h[0] = p->scale_factor * g->dx;
    pd.h[1] = p->scale_factor * g->dy;
    pd.h[2] = p->scale_factor * g->dz;
    pd.theta = p->theta;
    pd.inv_theta = 1.0 / p->theta;
    for (int a = 0; a < 3; a++) {
        pd.dt_h2[a] = p->theta * dt / (pd.h[a] * pd.h[a]);
        pd.wmax[a] = pd.dt_h2[a] * pd.Dmax;
        pd.wmax32[a] = (float)pd.wmax[a];
        pd.twoL_h32[a] = (float)(2.0 * p->L_unit / pd.h[a]);
    }
    pd.dtcs = dt * p->c * p->sigma;
    pd.dta = dt * p->adot_over_a;
    pd.mdtcs = p->theta * pd.dtcs;
    pd.one_dta = 1.0 + p->theta * pd.dta;
    pd.dmask = dirichlet_mask(g);
    for (int sd = 0; sd < 6; sd++) {
        const int kind = (sd & 1) ? g->bc_hi[sd >> 1] : g->bc[sd >> 1];
        pd.ebc[sd] = kind == FLD_BC_DIRICHLET ? g->bc_value[sd] : 0.0;
    }
    pd.sigmaL32 = (float)(p->sigma * p->L_unit);
    // D = D_max exactly when 9 (kappa_f L)^2 + (R L)^2 <= (c L / D_max)^2;
    // the FP32 screen accepts a face only 1e-3 inside that bound
    pd.thr32 = (float)((1.0 / (p->dmax_coef * p->dmax_coef)) * (1.0 - 1e-3));
    // the FP32 error of (R L)^2 grows with L / h; beyond 1e5 the screen is off
    for (int a = 0; a < 3; a++)
        if (!(pd.twoL_h32[a] < 2e5f)) pd.thr32 = -1.0f;
    pd.limiter = p->limiter;
    // double-float constants of the mixed kernels (high part the nearest
    // float, low part the nearest float to the rest)
    auto to_df = [](double v) {
        df r;
        r.h = (float)v;
        r.l = (float)(v - (double)r.h);
        return r;
    };
    auto in_range = [](double v) {
        const double a = std::fabs(v);
        return std::isfinite(v) && (a == 0.0 || (a > 1e-36 && a < 1e36));
    };
    bool lim_ok = true;
    for (int a = 0; a < 3; a++) {
        const double sh = p->sigma * pd.h[a], cw = p->theta * dt * p->c / pd.h[a], rm = pd.Rmin * pd.h[a];
        pd.sigh[a] = to_df(sh);
        pd.cw[a] = to_df(cw);
        pd.rminh[a] = to_df(rm);
        pd.wmaxd[a].h = pd.wmax32[a];
        pd.wmaxd[a].l = (float)(pd.wmax[a] - (double)pd.wmax32[a]);
        lim_ok = lim_ok && in_range(sh) && in_range(cw) && in_range(rm) && in_range(pd.wmax[a]);
    }
    pd.df_limiter = lim_ok ? 1 : 0;
    pd.one_dta_d = to_df(pd.one_dta);
    pd.mdtcs_d = to_df(pd.mdtcs);
    pd.dtcs_d = to_df(pd.dtcs);
    pd.dta_d = to_df(pd.dta);
    int e2 = 0;
    const double fr = std::frexp(dt, &e2);   // dt = fr 2^e2, fr in [1/2, 1)
    pd.dt_exp = e2 - 1;
    pd.dtm_d = to_df(2.0 * fr);
    pd.ith_d = to_df(pd.inv_theta);
}

// E = max(E + dE, 0) over n cells from E with the photon-balance sums:
// FP64 sums (FP64 solver), or df sums on the FP32 pipe (mixed solver,
// k_mixed.cu; its scales come from the assembly's maxima in c->sc).
void finalize_any(fld_ctx* c, long long n, double* E, const double* dE, const double* nHI, const double* eta,
                  const RedArgs& ra) {
    if (c->mixed) launch_finalize_mx(n, c->pd, E, dE, nHI, eta, E, ra, c->sc, c->s);
    else launch_finalize(n, c->pd, E, dE, nHI, eta, E, ra, c->s);
}

// Photons through the Dirichlet faces of side sd (before E is overwritten).
void bnd_outflow_any(fld_ctx* c, int sd, const double* E) {
    const RedArgs ra = red(c, R_STORE2, S_OUT0 + sd, S_OUTABS0 + sd);
    if (c->mixed) launch_bnd_outflow_mx(c->L[0].d, c->pd, sd, c->L[0].bnd, E, c->dE, ra, c->sc, c->s);
    else launch_bnd_outflow(c->L[0].d, c->pd, sd, c->L[0].bnd, E, c->dE, ra, c->s);
}

void finalize_enqueue(fld_ctx* c, double* E, const double* nHI, const double* eta) {
    const long long n = c->L[0].d.n;
    // the flux through Dirichlet faces needs E^n, before the update below
    for (int sd = 0; sd < 6; sd++)
        if ((c->L[0].bnd.mask >> sd) & 1) {
            KScope k(c, K_FINALIZE, 0.0);
            bnd_outflow_any(c, sd, E);
        }
    { KScope k(c, K_FINALIZE, 40.0 * n); finalize_any(c, n, E, c->dE, nHI, eta, red(c, R_STORE7_FIN)); }
    cudaEventRecord(c->e1, c->s);
    cudaMemcpyAsync(c->h_sc, c->sc, NUM_SLOTS * sizeof(double), cudaMemcpyDeviceToHost, c->s);
}

// The side streams and events of the host-buffer transfers (created on
// first use).
fld_status copy_streams(fld_ctx* c) {
    if (!c->cstream[0]) {
        for (int q = 0; q < 4; q++) {
            CUDA_TRY(cudaStreamCreateWithFlags(&c->cstream[q], cudaStreamNonBlocking));
            CUDA_TRY(cudaEventCreateWithFlags(&c->cjoin[q], cudaEventDisableTiming));
        }
        CUDA_TRY(cudaEventCreateWithFlags(&c->cfork, cudaEventDisableTiming));
    }
    return FLD_OK;
}

// finalize_enqueue for a host-buffer step: the finalisation runs in plane
// chunks and each chunk's E^{n+1} goes back to the host (E_host) on a side
// stream as soon as it is final, so the transfer overlaps the rest of the
// finalisation.  The chunks' balance sums are added in chunk order; the
// context's stream waits for the last transfer.
fld_status finalize_enqueue_host(fld_ctx* c, double* E, const double* nHI, const double* eta, double* E_host) {
    const Dims& d = c->L[0].d;
    const long long nxy = (long long)d.nx * d.ny;
    for (int sd = 0; sd < 6; sd++)
        if ((c->L[0].bnd.mask >> sd) & 1) {
            KScope k(c, K_FINALIZE, 0.0);
            bnd_outflow_any(c, sd, E);
        }
    const int nch = std::min(8, d.nz);
    if (fld_status st = copy_streams(c)) return st;
    for (int q = 0; q < nch; q++)
        if (!c->chunk_ev[q]) CUDA_TRY(cudaEventCreateWithFlags(&c->chunk_ev[q], cudaEventDisableTiming));
    if (!c->chunk_sc) CUDA_TRY(cudaMalloc(&c->chunk_sc, MAX_CHUNKS * NUM_SLOTS * sizeof(double)));
    cudaStream_t cs = c->cstream[0];
    CUDA_TRY(cudaMemsetAsync(c->chunk_sc, 0, (size_t)nch * NUM_SLOTS * sizeof(double), c->s));
    for (int q = 0; q < nch; q++) {
        const long long c0 = (long long)d.nz * q / nch * nxy, c1 = (long long)d.nz * (q + 1) / nch * nxy;
        RedArgs ra = red(c, R_STORE7_FIN);
        ra.sc = c->chunk_sc + (size_t)q * NUM_SLOTS;
        { KScope k(c, K_FINALIZE, 40.0 * (c1 - c0));
          finalize_any(c, c1 - c0, E + c0, c->dE + c0, nHI + c0, eta + c0, ra); }
        CUDA_TRY(cudaEventRecord(c->chunk_ev[q], c->s));
        CUDA_TRY(cudaStreamWaitEvent(cs, c->chunk_ev[q], 0));
        CUDA_TRY(cudaMemcpyAsync(E_host + c0, E + c0, (size_t)(c1 - c0) * sizeof(double), cudaMemcpyDeviceToHost, cs));
    }
    const SlotList sl{7, {S_BAL, S_EMIT, S_ABSORB, S_FLOOR, S_DE2, S_EN2, S_ESUM, 0}};
    launch_combine_sums(c->chunk_sc, nch, c->sc, sl, c->s);
    CUDA_TRY(cudaEventRecord(c->e1, c->s));
    CUDA_TRY(cudaMemcpyAsync(c->h_sc, c->sc, NUM_SLOTS * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    CUDA_TRY(cudaEventRecord(c->cjoin[0], cs));
    CUDA_TRY(cudaStreamWaitEvent(c->s, c->cjoin[0], 0));
    return FLD_OK;
}

// The photon balance and relative change from the host mirror.
void finalize_info(fld_ctx* c, fld_info* inf) {
    harvest(c);
    const double V = c->g.dx * c->g.dy * c->g.dz;
    const double scale = V / c->p.hnu;
    double out = 0.0, gross = 0.0;
    for (int sd = 0; sd < 6; sd++)
        if ((c->L[0].bnd.mask >> sd) & 1) {
            out += c->h_sc[S_OUT0 + sd];
            gross += c->h_sc[S_OUTABS0 + sd];
        }
    // the finalisation sums dE, eta, n_HI E^theta and E^theta over the cells
    // (E^theta = E^n + theta dE); emission and absorption follow by the
    // step's constants
    const double emit = c->pd.dt * c->h_sc[S_EMIT];
    const double absorb = c->pd.dtcs * c->h_sc[S_ABSORB] + c->pd.dta * c->h_sc[S_ESUM];
    inf->outflow = out * scale;
    inf->balance_abs = ((c->h_sc[S_BAL] - emit) + absorb + out) * scale;
    inf->emitted = emit * scale;
    inf->absorbed = absorb * scale;
    inf->floor_added = c->h_sc[S_FLOOR] * scale;
    inf->rel_change = c->h_sc[S_EN2] > 0.0 ? std::sqrt(c->h_sc[S_DE2] / c->h_sc[S_EN2]) : 0.0;
    double budget = inf->emitted > inf->absorbed ? inf->emitted : inf->absorbed;
    if (gross * scale > budget) budget = gross * scale;
    inf->balance_rel = budget > 0.0 ? std::fabs(inf->balance_abs) / budget : std::fabs(inf->balance_abs);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->e0, c->e1);
    inf->ms = ms;
}

// The step after its assembly has been enqueued (assembly status st).
// E_host: a host-buffer step whose finalisation also returns E^{n+1} to it.
fld_status step_after_assembly(fld_ctx* c, fld_status st, double* E, const double* nHI, const double* eta,
                               fld_info* info, double* E_host = nullptr) {
    fld_info inf{};
    if (!st) {
        if (cudaStreamSynchronize(c->s) != cudaSuccess) st = set_err(FLD_ECUDA, "%s", cudaGetErrorString(cudaGetLastError()));
        else st = assemble_finish(c);
    }
    if (st) {
        inf.status = st;
        if (info) *info = inf;
        return st;
    }
    st = solve_impl(c, &inf);
    if (st) {
        inf.status = st;
        if (info) *info = inf;
        return st;
    }
    if (E_host) {
        if ((st = finalize_enqueue_host(c, E, nHI, eta, E_host))) {
            inf.status = st;
            if (info) *info = inf;
            return st;
        }
    } else {
        finalize_enqueue(c, E, nHI, eta);
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(c->s));
    finalize_info(c, &inf);
    inf.status = FLD_OK;
    if (info) *info = inf;
    return FLD_OK;
}

fld_status step_impl(fld_ctx* c, double* E, const double* nHI, const double* eta, fld_info* info) {
    CUDA_TRY(cudaEventRecord(c->e0, c->s));
    return step_after_assembly(c, assemble_enqueue(c, E, nHI, eta), E, nHI, eta, info);
}


// ------------------------------------------------------- batched stepping
//
// Independent contexts advance in lockstep rounds.  In a round every
// context enqueues its next piece of work on its own stream (assembly,
// refinement residual, scaling, update, finalise); the contexts inside CG
// contribute their captured iteration graphs as independent branches of one
// batch graph, so all their iterations, whatever the grid sizes, go to the
// device in a single graph launch.  One synchronisation per round, then each
// context takes its next state from its scalars.  Each context runs exactly
// the kernels of a single fld_step, so results match it bit for bit.

enum BState { BS_ASM, BS_SCALE, BS_ITER, BS_RESID, BS_TRUE_RES, BS_FINAL, BS_DONE };

struct BItem {
    fld_ctx* c;
    double* E;
    const double* nHI;
    const double* eta;
    fld_info inf;
    fld_status st;
    int state;
    int prec;            // CG precision in progress (0 FP64, 1 FP32)
    double bb;
    int inner_total, outer;
    int ks, attempt;     // mixed: scale of the residual in flight, relaunches
    bool write;          // mixed: the residual in flight writes the next right-hand side
    int whole;           // the inner solve in flight runs whole on the device:
                         // 0 no (one round per iteration), 1 persistent
                         // kernel, 2 device-side loop graph
    bool conv;
    std::string err;
};

std::mutex g_batch_lock;
std::map<std::vector<unsigned long long>, cudaGraphExec_t> g_batch_graphs;
unsigned long long g_next_ctx_id = 1;

thread_local cudaStream_t tl_bs = nullptr;
thread_local cudaEvent_t tl_bev = nullptr;
thread_local int tl_dev = -1;

fld_status batch_stream(cudaStream_t* bs, cudaEvent_t* bev) {
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (!tl_bs || tl_dev != dev) {
        CUDA_TRY(cudaStreamCreateWithFlags(&tl_bs, cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&tl_bev, cudaEventDisableTiming));
        tl_dev = dev;
    }
    *bs = tl_bs;
    *bev = tl_bev;
    return FLD_OK;
}

// One graph holding the current CG iteration of every item as a branch.
cudaGraphExec_t batch_graph(const std::vector<BItem*>& its) {
    std::vector<unsigned long long> key;
    for (BItem* b : its) {
        key.push_back(b->c->id);
        key.push_back((unsigned long long)(b->prec * 2 + b->c->run.cur));
        key.push_back(b->c->graph_gen);
    }
    std::lock_guard<std::mutex> lock(g_batch_lock);
    auto it = g_batch_graphs.find(key);
    if (it != g_batch_graphs.end()) return it->second;
    if (g_batch_graphs.size() >= 64) {
        for (auto& kv : g_batch_graphs) cudaGraphExecDestroy(kv.second);
        g_batch_graphs.clear();
    }
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    bool ok = true;
    for (BItem* b : its) {
        cudaGraphNode_t node;
        cudaGraph_t child = b->c->graph[b->prec][b->c->run.cur];
        if (!child || cudaGraphAddChildGraphNode(&node, g, nullptr, 0, child) != cudaSuccess) { ok = false; break; }
    }
    cudaGraphExec_t ge = nullptr;
    if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
    cudaGraphDestroy(g);
    if (!ok) { cudaGetLastError(); return nullptr; }
    g_batch_graphs[key] = ge;
    return ge;
}

// Forget batch graphs holding this context's iterations (it is going away).
void forget_batch_graphs(unsigned long long id) {
    std::lock_guard<std::mutex> lock(g_batch_lock);
    for (auto it = g_batch_graphs.begin(); it != g_batch_graphs.end();) {
        bool uses = false;
        for (size_t q = 0; q < it->first.size(); q += 3) uses = uses || it->first[q] == id;
        if (uses) {
            cudaGraphExecDestroy(it->second);
            it = g_batch_graphs.erase(it);
        } else {
            ++it;
        }
    }
}

void bfail(BItem& b, fld_status st) {
    b.st = st;
    b.inf.status = st;
    b.err = g_err;
    b.state = BS_DONE;
}

// What a context does after the round's synchronisation.
void batch_after(BItem& b) {
    fld_ctx* c = b.c;
    const long long n = c->L[0].d.n;
    const double rtol = c->p.rtol;
    fld_status st = FLD_OK;
    switch (b.state) {
    case BS_ASM: {
        if ((st = assemble_finish(c))) return bfail(b, st);
        b.bb = c->h_sc[S_BB];
        if (b.bb == 0.0) {
            cudaMemsetAsync(c->dE, 0, n * sizeof(double), c->s);
            finalize_enqueue(c, b.E, b.nHI, b.eta);
            b.conv = true;
            b.state = BS_FINAL;
        } else if (!c->mixed) {
            cudaMemcpyAsync(c->cg[0], c->b, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s);
            cudaMemsetAsync(c->cg[5], 0, n * sizeof(double), c->s);
            b.prec = 0;
            if ((st = pcg_begin<double>(c, b.bb, rtol, c->p.max_iter))) return bfail(b, st);
            b.state = BS_ITER;
        } else {
            // the first refinement residual is b itself (x = 0)
            b.inf.rel_res = 1.0;
            scale_rhs_enqueue(c);
            cudaMemcpyAsync(c->h_sc, c->sc, NUM_SLOTS * sizeof(double), cudaMemcpyDeviceToHost, c->s);
            b.state = BS_SCALE;
        }
        return;
    }
    case BS_SCALE: {
        harvest(c);
        if (c->h_sc[S_NONFINITE] != 0.0) {
            set_err(FLD_ENONFINITE, "non-finite scaled right-hand side");
            return bfail(b, FLD_ENONFINITE);
        }
        double irtol = 0.5 * rtol / b.inf.rel_res;
        if (irtol < c->p.inner_rtol) irtol = c->p.inner_rtol;
        if (irtol > 0.5) irtol = 0.5;
        b.prec = 1;
        if ((st = pcg_begin<float>(c, c->h_sc[S_R0], irtol, c->p.max_iter - b.inner_total))) return bfail(b, st);
        b.state = BS_ITER;
        return;
    }
    case BS_ITER: {
        if (b.whole) {
            harvest(c);
            st = whole_after(c, b.prec, b.whole == 2);
            b.whole = 0;
            if (st) return bfail(b, st);
        } else if ((st = pcg_after(c))) {
            return bfail(b, st);
        }
        if (!c->run.done) return;
        if (!c->mixed) {
            b.inf.iters = c->run.k;
            b.conv = c->run.conv;
            cudaMemcpyAsync(c->dE, c->cg[5], n * sizeof(double), cudaMemcpyDeviceToDevice, c->s);
            { KScope k(c, K_RESIDUAL64, 48.0 * n);
              launch_residual64(c->L[0].d, c->L[0].A64, nullptr, c->b, c->dE, nullptr,
                                red(c, R_STORE_SUM_MAX, S_TRUE_RR, S_RMAX), c->s); }
            cudaMemcpyAsync(c->h_sc, c->sc, NUM_SLOTS * sizeof(double), cudaMemcpyDeviceToHost, c->s);
            b.state = BS_TRUE_RES;
        } else {
            b.inner_total += c->run.k;
            update_enqueue(c, b.outer == 0);
            b.outer++;
            b.write = !expect_converged(c, b.bb, rtol);
            b.ks = next_scale(c);
            b.attempt = 0;
            residual_enqueue(c, b.ks, b.write);
            cudaMemcpyAsync(c->h_sc, c->sc, NUM_SLOTS * sizeof(double), cudaMemcpyDeviceToHost, c->s);
            b.state = BS_RESID;
        }
        return;
    }
    case BS_RESID: {
        harvest(c);
        const int fix = scale_fix(c, b.ks, b.attempt);
        if (fix < 0) {
            set_err(FLD_ENONFINITE, "non-finite refinement residual after %d refinements", b.outer);
            return bfail(b, FLD_ENONFINITE);
        }
        if (fix > 0) {
            // the predicted scale left the FP32 range: again with the scale the
            // residual reported
            b.attempt++;
            cudaMemsetAsync(c->sc + S_NONFINITE, 0, sizeof(double), c->s);
            residual_enqueue(c, b.ks, b.write);
            cudaMemcpyAsync(c->h_sc, c->sc, NUM_SLOTS * sizeof(double), cudaMemcpyDeviceToHost, c->s);
            return;
        }
        c->ks = b.ks;
        b.inf.rel_res = scaled_rel_res(c, b.bb);
        b.inf.iters = b.inner_total;
        b.inf.outer_iters = b.outer;
        if (b.inf.rel_res <= rtol) {
            b.conv = true;
            finalize_enqueue(c, b.E, b.nHI, b.eta);
            b.state = BS_FINAL;
        } else if (b.inner_total >= c->p.max_iter) {
            set_err(FLD_ENOCONV, "no convergence: relative residual %.3e > rtol %.3e after %d iterations",
                    b.inf.rel_res, rtol, b.inner_total);
            return bfail(b, FLD_ENOCONV);
        } else if (!b.write) {
            // expected to converge and did not: the same residual again,
            // now writing the next inner solve's right-hand side
            b.write = true;
            residual_enqueue(c, b.ks, true);
            cudaMemcpyAsync(c->h_sc, c->sc, NUM_SLOTS * sizeof(double), cudaMemcpyDeviceToHost, c->s);
        } else {
            // the residual kernel left the next inner solve's scaled
            // right-hand side and its norm: straight to the inner solve
            double irtol = 0.5 * rtol / b.inf.rel_res;
            if (irtol < c->p.inner_rtol) irtol = c->p.inner_rtol;
            if (irtol > 0.5) irtol = 0.5;
            b.prec = 1;
            if ((st = pcg_begin<float>(c, c->h_sc[S_R0], irtol, c->p.max_iter - b.inner_total))) return bfail(b, st);
            b.state = BS_ITER;
        }
        return;
    }
    case BS_TRUE_RES: {
        harvest(c);
        b.inf.rel_res = std::sqrt(c->h_sc[S_TRUE_RR] / b.bb);
        if (!b.conv) {
            set_err(FLD_ENOCONV, "no convergence: relative residual %.3e > rtol %.3e after %d iterations",
                    b.inf.rel_res, rtol, b.inf.iters);
            return bfail(b, FLD_ENOCONV);
        }
        finalize_enqueue(c, b.E, b.nHI, b.eta);
        b.state = BS_FINAL;
        return;
    }
    case BS_FINAL: {
        finalize_info(c, &b.inf);
        b.inf.status = FLD_OK;
        b.st = FLD_OK;
        b.state = BS_DONE;
        return;
    }
    default:
        return;
    }
}

fld_status step_batched_impl(int n, fld_ctx** cs, double** E, const double** nHI, const double** eta,
                             fld_info* infos) {
    cudaStream_t bs = nullptr;
    cudaEvent_t bev = nullptr;
    fld_status st = batch_stream(&bs, &bev);
    if (st) return st;
    // each context onto its private stream, after the caller's work
    for (int i = 0; i < n; i++) {
        fld_ctx* c = cs[i];
        if (!c->bstream && cudaStreamCreateWithFlags(&c->bstream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            c->bstream = nullptr;
            for (int q = 0; q < i; q++) cs[q]->s = cs[q]->user_s;
            return set_err(FLD_ECUDA, "stream creation for batch item %d failed", i);
        }
        c->user_s = c->s;
        cudaEventRecord(c->ev_join, c->s);
        cudaStreamWaitEvent(c->bstream, c->ev_join, 0);
        c->s = c->bstream;
    }
    std::vector<BItem> items(n);
    for (int i = 0; i < n; i++) {
        BItem& b = items[i];
        b.c = cs[i];
        b.E = E[i];
        b.nHI = nHI[i];
        b.eta = eta[i];
        b.inf = fld_info{};
        b.st = FLD_OK;
        b.prec = 0;
        b.bb = 0.0;
        b.inner_total = b.outer = 0;
        b.whole = 0;
        b.write = true;
        b.conv = false;
        b.state = BS_ASM;
        cudaEventRecord(b.c->e0, b.c->s);
        if ((st = assemble_enqueue(b.c, b.E, b.nHI, b.eta))) bfail(b, st);
    }
    for (;;) {
        // contexts entering an inner solve: the persistent ones all in one
        // launch over a work list, the others with a device-side loop graph
        // on their own streams; both run the whole solve in this round
        std::vector<fld_ctx*> psc;
        std::vector<BItem*> iter, direct;
        for (BItem& b : items) {
            if (b.state != BS_ITER || b.c->run.k != 0 || b.c->run.done) continue;
            fld_ctx* c = b.c;
            if (b.prec == 1 && c->ps) {
                if ((st = whole_slots(c))) { bfail(b, st); continue; }
                cudaEventRecord(c->ev_join, c->s);
                cudaStreamWaitEvent(bs, c->ev_join, 0);
                psc.push_back(c);
                b.whole = 1;
                continue;
            }
            cudaGraphExec_t le = b.prec ? loop_graph<float>(c) : loop_graph<double>(c);
            if (le) {
                if ((st = whole_slots(c))) { bfail(b, st); continue; }
                if (cudaGraphLaunch(le, c->s) != cudaSuccess) {
                    cudaGetLastError();
                    bfail(b, set_err(FLD_ECUDA, "launch of the device-side CG loop failed"));
                    continue;
                }
                cudaMemcpyAsync(c->h_sc, c->sc, NUM_SLOTS * sizeof(double), cudaMemcpyDeviceToHost, c->s);
                b.whole = 2;
            }
        }
        if (!psc.empty()) {
            st = ps_enqueue(psc, bs);
            cudaEventRecord(bev, bs);
            for (BItem& b : items)
                if (b.whole == 1) {
                    cudaStreamWaitEvent(b.c->s, bev, 0);
                    cudaMemcpyAsync(b.c->h_sc, b.c->sc, NUM_SLOTS * sizeof(double), cudaMemcpyDeviceToHost, b.c->s);
                    if (st) bfail(b, st);
                }
        }
        // the other contexts inside CG: their iterations as one batch-graph
        // launch per round
        for (BItem& b : items)
            if (b.state == BS_ITER && !b.whole) {
                const bool g = b.prec ? pcg_graph<float>(b.c, b.c->run.cur) != nullptr
                                      : pcg_graph<double>(b.c, b.c->run.cur) != nullptr;
                (g ? iter : direct).push_back(&b);
            }
        cudaGraphExec_t ge = iter.size() > 1 ? batch_graph(iter) : nullptr;
        if (ge) {
            for (BItem* b : iter) {
                cudaEventRecord(b->c->ev_join, b->c->s);
                cudaStreamWaitEvent(bs, b->c->ev_join, 0);
            }
            cudaGraphLaunch(ge, bs);
            cudaEventRecord(bev, bs);
            for (BItem* b : iter) {
                cudaStreamWaitEvent(b->c->s, bev, 0);
                count_graph_launches(b->c, b->prec, b->c->run.cur);
            }
        } else {
            for (BItem* b : iter) direct.push_back(b);
        }
        for (BItem* b : direct) {
            st = b->prec ? pcg_enqueue<float>(b->c) : pcg_enqueue<double>(b->c);
            if (st) bfail(*b, st);
        }
        bool any = false;
        for (BItem& b : items) {
            if (b.state == BS_DONE) continue;
            any = true;
            cudaError_t e = cudaStreamSynchronize(b.c->s);
            if (e != cudaSuccess) {
                set_err(FLD_ECUDA, "stream synchronisation failed: %s", cudaGetErrorString(e));
                bfail(b, FLD_ECUDA);
            }
        }
        if (!any) break;
        for (BItem& b : items)
            if (b.state != BS_DONE) batch_after(b);
    }
    // back to the caller's streams, which wait for the private ones
    for (int i = 0; i < n; i++) {
        fld_ctx* c = cs[i];
        cudaEventRecord(c->ev_join, c->bstream);
        c->s = c->user_s;
        cudaStreamWaitEvent(c->s, c->ev_join, 0);
    }
    fld_status first = FLD_OK;
    std::string msg;
    for (int i = 0; i < n; i++) {
        infos[i] = items[i].inf;
        infos[i].status = items[i].st;
        if (items[i].st && !first) {
            first = items[i].st;
            msg = "batch item " + std::to_string(i) + ": " + items[i].err;
        }
    }
    if (first) g_err = msg;
    return first;
}

}  // namespace

namespace fld {
// Lets other translation units of the library set fld_last_error's message.
void record_error(const char* msg) { g_err = msg ? msg : ""; }
}  // namespace fld

extern "C" {

fld_status fld_params_default(fld_params* p) {
    if (!p) return set_err(FLD_EINVAL, "null params");
    memset(p, 0, sizeof(*p));
    p->dt = 1e5 * 3.15576e7;
    p->c = 2.99792458e10;
    p->L_unit = 6.6 * 3.0856776e21;
    p->dmax_coef = 0.006;
    p->rmin_coef = 1e-20;
    p->sigma = 1.6e-18;
    p->adot_over_a = 0.0;
    p->hnu = 13.6 * 1.602176634e-12;
    p->limiter = FLD_LIMITER_PAPER;
    p->precision = FLD_PREC_FP64;
    p->smoother = FLD_SMOOTH_RBGS;
    p->jacobi_omega = 0.8;
    p->rtol = 1e-8;
    p->max_iter = 50;
    p->pre = 1;
    p->post = 1;
    p->inner_rtol = 1e-4;
    p->coarse_cap = 1024;
    p->graphs = -1;
    p->fused_post = 0;
    p->paper_order = 0;
    p->persistent_cells = 0;
    p->precond_bf16 = 1;
    p->theta = 1.0;
    p->scale_factor = 1.0;
    p->tail_cells = 32768;
    return FLD_OK;
}

size_t fld_footprint_bytes(const fld_grid* g, const fld_params* p) {
    if (validate(g, p) != FLD_OK) return 0;
    size_t total = 0;
    plan(g, p, [&](int, const char*, int, size_t bytes) { total += (bytes + 511) / 512 * 512; });
    return total;
}

int fld_levels(const fld_grid* g, int* dims, int max_levels) {
    if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1) return 0;
    int d[MAX_LEVELS][3];
    int nl = level_shapes(g, d);
    for (int l = 0; l < nl && l < max_levels; l++)
        for (int a = 0; a < 3; a++) dims[3 * l + a] = d[l][a];
    return nl;
}

fld_status fld_create(fld_ctx** out, const fld_grid* g, const fld_params* p, void* stream) {
    if (!out) return set_err(FLD_EINVAL, "null output pointer");
    *out = nullptr;
    fld_status st = validate(g, p);
    if (st) return st;
    fld_ctx* c = new (std::nothrow) fld_ctx();
    if (!c) return set_err(FLD_ENOMEM, "host allocation failed");
    c->g = *g;
    c->p = *p;
    c->s = (cudaStream_t)stream;
    c->mixed = p->precision == FLD_PREC_MIXED;
    int dims[MAX_LEVELS][3];
    c->nl = level_shapes(g, dims);
    for (int l = 0; l < c->nl; l++) {
        Dims& d = c->L[l].d;
        d.nx = dims[l][0];
        d.ny = dims[l][1];
        d.nz = dims[l][2];
        d.px = g->bc[0] == FLD_BC_PERIODIC;
        d.py = g->bc[1] == FLD_BC_PERIODIC;
        d.pz = g->bc[2] == FLD_BC_PERIODIC;
        d.n = (long long)d.nx * d.ny * d.nz;
    }
    c->nc = (int)c->L[c->nl - 1].d.n;
    st = alloc_ctx(c);
    if (st) { free_ctx(c); return st; }
    for (int l = 0; l < c->nl; l++) c->L[l].bnd.mask = c->L[l].bnd.w ? dirichlet_mask(g) : 0;
    // persistent coarse tail: from the first level with at most tail_cells
    // cells (red/black Gauss-Seidel only), if at least one level lies above
    // the coarsest one and a cluster of the tail kernel fits on the device
    c->tail_from = -1;
    if (p->tail_cells > 0 && p->smoother == FLD_SMOOTH_RBGS && c->nl >= 2) {
        int l0 = 0;
        while (l0 < c->nl - 1 && c->L[l0].d.n > p->tail_cells) l0++;
        c->tail_cluster = c->mixed ? vtail_cluster<float>() : vtail_cluster<double>();
        if (l0 < c->nl - 1 && c->nl - l0 <= TAIL_MAX_LEVELS && c->tail_cluster > 0) c->tail_from = l0;
    }
    // persistent inner solves: the V-cycle over every level with the fine
    // level's CG vectors, written once to the context's device descriptor
    c->ps = false;
    if (c->ps_req && psolve_shape().cluster > 0) {
        PsReq& R = c->ps_host;
        memset(&R, 0, sizeof(R));
        TailArgs<float>& ta = R.v;
        ta.nlev = c->nl;
        ta.pre = p->pre;
        ta.post = p->post;
        ta.paper_order = p->paper_order;
        for (int q = 0; q < c->nl; q++) {
            Level& Q = c->L[q];
            TailLevel<float>& t = ta.L[q];
            t.d = Q.d;
            t.A = Q.A32;
            t.r = (float*)(q == 0 ? c->cg[0] : Q.r);
            t.z = (float*)(q == 0 ? c->cg[1] : Q.z);
            t.t = (float*)Q.t;
        }
        ta.small_from = ta.nlev;
        for (int q = 0; q < ta.nlev; q++)
            if (ta.L[q].d.n <= TAIL_SMALL_CELLS) {
                size_t cells = 0;
                for (int u = q; u < ta.nlev; u++) cells += (size_t)ta.L[u].d.n;
                if (3 * cells * sizeof(float) <= TAIL_SMEM_MAX) ta.small_from = q;
                break;
            }
        ta.ainv = c->ainv;   // filled by every assembly
        R.cta = psolve_cta_bytes(ta) <= PS_SMEM_MAX ? 1 : 0;
        R.x = (float*)c->cg[5];
        R.p = (float*)c->cg[2];
        R.q = (float*)c->cg[4];
        R.sc = c->sc;
        if (cudaMemcpy(c->ps_req, &R, sizeof(R), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            free_ctx(c);
            return set_err(FLD_ECUDA, "copy of the persistent-solve descriptor failed");
        }
        c->ps = true;
    }
    {
        long long blocks = 0;
        int cap = 0;
        face_list_shape(c->L[0].d, p->limiter, &blocks, &cap);
        c->flist.cap = cap;
        if (cap == 0) c->flist.entries = c->flist.counts = nullptr;
    }
    if (cudaMallocHost(&c->h_sc, NUM_SLOTS * sizeof(double)) != cudaSuccess ||
        cudaEventCreate(&c->e0) != cudaSuccess || cudaEventCreate(&c->e1) != cudaSuccess) {
        cudaGetLastError();
        free_ctx(c);
        return set_err(FLD_ENOMEM, "pinned scalar buffer or event creation failed");
    }
    memset(c->h_sc, 0, NUM_SLOTS * sizeof(double));
    if (cudaMallocHost(&c->h_one, 4 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        free_ctx(c);
        return set_err(FLD_ENOMEM, "pinned allocation failed");
    }
    *c->h_one = 1.0;
    if (cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        free_ctx(c);
        return set_err(FLD_ECUDA, "event creation failed");
    }
    {
        std::lock_guard<std::mutex> lock(g_batch_lock);
        c->id = g_next_ctx_id++;
    }
    // graphs need a capturable (non-legacy) stream; "auto" uses them at any
    // size (the device-side CG loop saves the host round trip per iteration)
    c->use_graphs = c->s != nullptr && p->graphs != 0;
    if (cudaMemsetAsync(c->counter, 0, 256, c->s) != cudaSuccess ||
        cudaMemsetAsync(c->sc, 0, NUM_SLOTS * sizeof(double), c->s) != cudaSuccess) {
        free_ctx(c);
        return set_err(FLD_ECUDA, "initial memset failed");
    }
    fill_physdev(c, p->dt);
    *out = c;
    return FLD_OK;
}

void fld_destroy(fld_ctx* c) {
    if (c) forget_batch_graphs(c->id);
    free_ctx(c);
}

fld_status fld_assemble(fld_ctx* c, const double* E, const double* nHI, const double* eta) {
    return assemble_impl(c, E, nHI, eta);
}

fld_status fld_solve(fld_ctx* c, double* dE, fld_info* info) {
    if (!c) return set_err(FLD_EINVAL, "null context");
    if (!dE) return set_err(FLD_EINVAL, "null dE");
    if (!c->assembled) return set_err(FLD_EINVAL, "fld_solve before a successful fld_assemble");
    if (cudaEventRecord(c->e0, c->s) != cudaSuccess) return set_err(FLD_ECUDA, "event record failed");
    fld_info inf{};
    fld_status st = solve_impl(c, &inf);
    if (st == FLD_OK || st == FLD_ENOCONV) {
        // the mixed solver keeps dE as a double-float pair scaled by the
        // step's power of two
        if (c->mixed) launch_dE_to_f64(c->L[0].d.n, c->dE, dE, c->sc, c->pd.dt_exp, c->s);
        else CUDA_TRY(cudaMemcpyAsync(dE, c->dE, c->L[0].d.n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
        CUDA_TRY(cudaEventRecord(c->e1, c->s));
        CUDA_TRY(cudaStreamSynchronize(c->s));
        harvest(c);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->e0, c->e1);
        inf.ms = ms;
    }
    inf.status = st;
    if (info) *info = inf;
    return st;
}

fld_status fld_step(fld_ctx* c, double* E, const double* nHI, const double* eta, fld_info* info) {
    if (!c) return set_err(FLD_EINVAL, "null context");
    return step_impl(c, E, nHI, eta, info);
}

// Copies of host-buffer steps: each array in chunks spread over the side
// streams (several copy engines share the host link), ordered after the
// context stream's work so far and joined back into it.
fld_status split_copies(fld_ctx* c, int narr, void* const* dst, const void* const* src, size_t bytes,
                        cudaMemcpyKind kind) {
    constexpr int NS = 4;
    if (fld_status st = copy_streams(c)) return st;
    CUDA_TRY(cudaEventRecord(c->cfork, c->s));
    for (int q = 0; q < NS; q++) CUDA_TRY(cudaStreamWaitEvent(c->cstream[q], c->cfork, 0));
    const size_t chunk = ((bytes + NS - 1) / NS + 255) / 256 * 256;
    int k = 0;
    for (int a = 0; a < narr; a++)
        for (size_t off = 0; off < bytes; off += chunk, k++) {
            const size_t len = bytes - off < chunk ? bytes - off : chunk;
            CUDA_TRY(cudaMemcpyAsync((char*)dst[a] + off, (const char*)src[a] + off, len, kind, c->cstream[k % NS]));
        }
    for (int q = 0; q < NS; q++) {
        CUDA_TRY(cudaEventRecord(c->cjoin[q], c->cstream[q]));
        CUDA_TRY(cudaStreamWaitEvent(c->s, c->cjoin[q], 0));
    }
    return FLD_OK;
}

// Whether the host-buffer step overlaps its input transfer with the
// assembly: the faces of plane 0 need plane nz - 1 on a periodic z axis
// (the last chunk), and small grids gain nothing.
bool overlap_host_step(const fld_ctx* c) {
    const Dims& d = c->L[0].d;
    return !d.pz && d.n >= (1LL << 21) && asm_shape(d).nzb >= 2;
}

// Enqueue the input transfer of a host-buffer step overlapped with the
// fine-level assembly.  The planes travel in chunks of whole z-blocks of
// the assembly decomposition on one side stream, in order; the faces of a
// chunk are formed as soon as it has arrived, its right-hand side once the
// next chunk's faces exist (it needs the z faces above it).  Each chunk's
// right-hand-side reductions go to slots of their own, summed (||b||^2) and
// maximised (max |b|) in chunk order afterwards.  Then the coarse levels.
fld_status assemble_host_overlapped(fld_ctx* c, const double* E, const double* nHI, const double* eta) {
    Level& L0 = c->L[0];
    const Dims& d = L0.d;
    const AsmShape a = asm_shape(d);
    const int zbc = std::max((a.nzb + MAX_CHUNKS - 1) / MAX_CHUNKS, (a.nzb + 7) / 8);   // z-blocks per chunk
    const int nch = (a.nzb + zbc - 1) / zbc;
    if (fld_status st = copy_streams(c)) return st;
    for (int q = 0; q < nch; q++)
        if (!c->chunk_ev[q]) CUDA_TRY(cudaEventCreateWithFlags(&c->chunk_ev[q], cudaEventDisableTiming));
    if (!c->chunk_sc) CUDA_TRY(cudaMalloc(&c->chunk_sc, MAX_CHUNKS * NUM_SLOTS * sizeof(double)));
    cudaStream_t s = c->s, cs = c->cstream[0];
    c->assembled = false;
    CUDA_TRY(cudaMemsetAsync(c->sc, 0, NUM_SLOTS * sizeof(double), s));
    CUDA_TRY(cudaMemsetAsync(c->chunk_sc, 0, (size_t)nch * NUM_SLOTS * sizeof(double), s));
    // the staging buffers are free once the context's stream has reached here
    CUDA_TRY(cudaEventRecord(c->cfork, s));
    CUDA_TRY(cudaStreamWaitEvent(cs, c->cfork, 0));
    const long long nxy = (long long)d.nx * d.ny;
    const double* src[3] = {E, nHI, eta};
    int p0[MAX_CHUNKS + 1];
    for (int q = 0; q <= nch; q++) p0[q] = std::min(d.nz, q * zbc * a.kch);
    for (int q = 0; q < nch; q++) {
        const size_t off = (size_t)p0[q] * nxy, len = (size_t)(p0[q + 1] - p0[q]) * nxy * sizeof(double);
        for (int v = 0; v < 3; v++)
            CUDA_TRY(cudaMemcpyAsync(c->stage[v] + off, src[v] + off, len, cudaMemcpyHostToDevice, cs));
        CUDA_TRY(cudaEventRecord(c->chunk_ev[q], cs));
    }
    auto chunk_red = [&](int q) {
        RedArgs r = red(c, R_STORE_SUM_MAX, S_BB, S_RMAX);
        r.sc = c->chunk_sc + (size_t)q * NUM_SLOTS;
        return r;
    };
    auto frac = [&](int q) { return (double)(p0[q + 1] - p0[q]) / d.nz; };
    const double *Es = c->stage[0], *ns = c->stage[1], *es = c->stage[2];
    for (int q = 0; q < nch; q++) {
        CUDA_TRY(cudaStreamWaitEvent(s, c->chunk_ev[q], 0));
        assemble_faces_range(c, Es, ns, es, q * zbc, zbc, frac(q));
        if (q > 0) assemble_rhs_range(c, Es, ns, es, (q - 1) * zbc, zbc, frac(q - 1), chunk_red(q - 1));
    }
    assemble_rhs_range(c, Es, ns, es, (nch - 1) * zbc, zbc, frac(nch - 1), chunk_red(nch - 1));
    launch_combine_chunks(c->chunk_sc, nch, c->sc, S_BB, S_RMAX, s);
    return assemble_coarse(c);
}

fld_status fld_step_host(fld_ctx* c, double* E, const double* nHI, const double* eta, fld_info* info) {
    if (!c) return set_err(FLD_EINVAL, "null context");
    if (!E || !nHI || !eta) return set_err(FLD_EINVAL, "null field pointer");
    const size_t bytes = c->L[0].d.n * sizeof(double);
    for (int q = 0; q < 3; q++)
        if (!c->stage[q]) {
            if (cudaMalloc(&c->stage[q], bytes) != cudaSuccess) {
                cudaGetLastError();
                c->stage[q] = nullptr;
                return set_err(FLD_ENOMEM, "staging allocation failed");
            }
        }
    fld_status st;
    if (overlap_host_step(c)) {
        CUDA_TRY(cudaEventRecord(c->e0, c->s));
        st = assemble_host_overlapped(c, E, nHI, eta);
        // no transfer from the caller's buffers may outlive a failed call
        if (st && c->cstream[0]) cudaStreamSynchronize(c->cstream[0]);
        st = step_after_assembly(c, st, c->stage[0], c->stage[1], c->stage[2], info, E);
        if (!st) return FLD_OK;   // E is back: the finalisation returned it chunk by chunk
    } else {
        void* dst[3] = {c->stage[0], c->stage[1], c->stage[2]};
        const void* src[3] = {E, nHI, eta};
        if ((st = split_copies(c, 3, dst, src, bytes, cudaMemcpyHostToDevice))) return st;
        st = step_impl(c, c->stage[0], c->stage[1], c->stage[2], info);
    }
    if (st) {
        // no transfer from the caller's buffers may outlive a failed call
        for (int q = 0; q < 4; q++)
            if (c->cstream[q]) cudaStreamSynchronize(c->cstream[q]);
        return st;
    }
    {
        void* dst[1] = {E};
        const void* src[1] = {c->stage[0]};
        if ((st = split_copies(c, 1, dst, src, bytes, cudaMemcpyDeviceToHost))) return st;
    }
    CUDA_TRY(cudaStreamSynchronize(c->s));
    return FLD_OK;
}

fld_status fld_set_dt(fld_ctx* c, double dt) {
    if (!c) return set_err(FLD_EINVAL, "null context");
    if (!(std::isfinite(dt) && dt > 0.0)) return set_err(FLD_EINVAL, "dt must be finite and > 0");
    fill_physdev(c, dt);
    return FLD_OK;
}

fld_status fld_set_expansion(fld_ctx* c, double a, double adot_over_a) {
    if (!c) return set_err(FLD_EINVAL, "null context");
    if (!(std::isfinite(a) && a > 0.0)) return set_err(FLD_EINVAL, "scale factor must be finite and > 0");
    if (!(std::isfinite(adot_over_a) && adot_over_a >= 0.0))
        return set_err(FLD_EINVAL, "adot_over_a must be finite and >= 0");
    c->p.scale_factor = a;
    c->p.adot_over_a = adot_over_a;
    fill_physdev(c, c->p.dt);
    return FLD_OK;
}

fld_status fld_advance(fld_ctx* c, double* E, const double* nHI, const double* eta, double t_span,
                       double dt_first, const fld_advance_params* ap, fld_advance_info* info) {
    if (!c || !ap) return set_err(FLD_EINVAL, "null argument");
    if (!(t_span > 0.0) || !(dt_first > 0.0) || !(ap->tau_tol > 0.0) || !(ap->growth >= 1.0) ||
        !(ap->dt_min > 0.0) || ap->max_substeps < 1)
        return set_err(FLD_EINVAL, "invalid subcycling parameters");
    const auto t0 = std::chrono::steady_clock::now();
    fld_advance_info ai{};
    const double dt_orig = c->p.dt;
    double t = 0.0, dt = dt_first;
    if (ap->dt_max > 0.0 && dt > ap->dt_max) dt = ap->dt_max;
    fld_status st = FLD_OK;
    while (t < t_span) {
        if (ai.substeps + ai.retries >= ap->max_substeps) {
            st = set_err(FLD_ENOCONV, "subcycling stopped after %d substeps", ap->max_substeps);
            break;
        }
        const double rest = t_span - t;
        const bool last = dt >= rest * (1.0 - 1e-12);
        const double dt_try = last ? rest : dt;
        fill_physdev(c, dt_try);
        fld_info inf{};
        st = step_impl(c, E, nHI, eta, &inf);
        ai.iters += inf.iters;
        if (st == FLD_ENOCONV || st == FLD_ENONFINITE) {
            ai.retries++;
            dt = 0.1 * dt_try;
            if (dt < ap->dt_min) {
                set_err(st, "substep of %.3e s failed and 0.1 dt is below dt_min", dt_try);
                break;
            }
            st = FLD_OK;
            continue;
        }
        if (st) break;
        t = last ? t_span : t + dt_try;
        ai.substeps++;
        const double f = inf.rel_change > 0.0 ? ap->tau_tol / inf.rel_change : ap->growth;
        dt = dt_try * (f < 0.1 ? 0.1 : (f > ap->growth ? ap->growth : f));
        if (ap->dt_max > 0.0 && dt > ap->dt_max) dt = ap->dt_max;
        if (dt < ap->dt_min) dt = ap->dt_min;
    }
    fill_physdev(c, dt_orig);
    ai.status = st;
    ai.t_done = t;
    ai.dt_next = dt;
    ai.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = ai;
    return st;
}

fld_status fld_step_batched(int n, fld_ctx** ctxs, double** E, const double** nHI,
                            const double** eta, fld_info* infos) {
    if (n < 0 || (n > 0 && (!ctxs || !E || !nHI || !eta || !infos)))
        return set_err(FLD_EINVAL, "invalid batch arguments");
    for (int i = 0; i < n; i++)
        if (!ctxs[i]) return set_err(FLD_EINVAL, "null context %d in batch", i);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < i; j++)
            if (ctxs[i] == ctxs[j]) return set_err(FLD_EINVAL, "context %d appears twice in the batch", i);
    return step_batched_impl(n, ctxs, E, nHI, eta, infos);
}

fld_status fld_apply(fld_ctx* c, const double* x, double* y) {
    if (!c || !x || !y) return set_err(FLD_EINVAL, "null argument");
    if (!c->assembled) return set_err(FLD_EINVAL, "fld_apply before fld_assemble");
    {
        KScope k(c, K_APPLY, 48.0 * c->L[0].d.n);
        if (c->mixed) launch_apply_mx(c->L[0].d, c->L[0].A32, c->L[0].Alo, x, y, c->s);
        else launch_apply<double>(c->L[0].d, c->L[0].A64, x, y, c->s);
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(c->s));
    harvest(c);
    return FLD_OK;
}

fld_status fld_vcycle(fld_ctx* c, const double* r, double* z) {
    if (!c || !r || !z) return set_err(FLD_EINVAL, "null argument");
    if (!c->assembled) return set_err(FLD_EINVAL, "fld_vcycle before fld_assemble");
    if (c->mixed) {
        // the FP32 cycle of the mixed solver on r rounded to FP32 (the CG
        // work vectors r and z serve as its input and output)
        const long long n = c->L[0].d.n;
        float* r32 = (float*)c->cg[0];
        float* z32 = (float*)c->cg[1];
        launch_f64_to_f32(n, r, r32, c->s);
        vcycle<float>(c, 0, r32, z32);
        launch_f32_to_f64(n, z32, z, c->s);
    } else {
        vcycle<double>(c, 0, r, z);
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(c->s));
    harvest(c);
    return FLD_OK;
}

fld_status fld_get_system(fld_ctx* c, double* m, double* wx, double* wy, double* wz, double* b) {
    if (!c) return set_err(FLD_EINVAL, "null context");
    if (!c->assembled) return set_err(FLD_EINVAL, "fld_get_system before fld_assemble");
    const long long n = c->L[0].d.n;
    const size_t bytes = n * sizeof(double);
    double* dst[5] = {m, wx, wy, wz, b};
    if (c->mixed) {
        // the double-float operator as FP64 values
        const Level& L = c->L[0];
        const float* hi[4] = {L.A32.m, L.A32.wx, L.A32.wy, L.A32.wz};
        const float* lo[4] = {L.Alo.m, L.Alo.wx, L.Alo.wy, L.Alo.wz};
        for (int q = 0; q < 4; q++)
            if (dst[q]) launch_df_to_f64(n, hi[q], lo[q], dst[q], c->s);
        if (b) CUDA_TRY(cudaMemcpyAsync(b, c->b, bytes, cudaMemcpyDeviceToDevice, c->s));
        CUDA_TRY(cudaGetLastError());
    } else {
        const double* src[5] = {c->L[0].A64.m, c->L[0].A64.wx, c->L[0].A64.wy, c->L[0].A64.wz, c->b};
        for (int q = 0; q < 5; q++)
            if (dst[q]) CUDA_TRY(cudaMemcpyAsync(dst[q], src[q], bytes, cudaMemcpyDeviceToDevice, c->s));
    }
    CUDA_TRY(cudaStreamSynchronize(c->s));
    return FLD_OK;
}

fld_status fld_opacity_update(size_t n, const double* E, const double* nH, const double* nHI,
                              double* out, double dt, double c, double sigma, double hnu,
                              double alpha_B, void* stream) {
    if (!E || !nH || !nHI || !out) return set_err(FLD_EINVAL, "null argument");
    if (!(dt > 0.0) || !(c > 0.0) || !(sigma >= 0.0) || !(hnu > 0.0) || !(alpha_B >= 0.0))
        return set_err(FLD_EINVAL, "invalid opacity-update constants");
    if (n == 0) return FLD_OK;
    launch_opacity_update((long long)n, E, nH, nHI, out, dt, c, sigma, hnu, alpha_B,
                          (cudaStream_t)stream);
    CUDA_TRY(cudaGetLastError());
    return FLD_OK;
}

fld_status fld_autotune(fld_ctx* c, int reps) {
    if (!c) return set_err(FLD_EINVAL, "null context");
    if (reps < 1 || reps > 100) return set_err(FLD_EINVAL, "reps must lie in [1, 100]");
    if (!c->mixed) return FLD_OK;   // FP64 sweeps have a single launch shape
    cudaStream_t s = c->s;
    CUDA_TRY(cudaStreamSynchronize(s));
    // captured graphs hold the old launch shapes
    drop_graphs(c);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    const int threads_c[] = {128, 256};
    const int target_c[] = {152 * 4, 152 * 8, 152 * 16, 152 * 32, 152 * 64};
    const int pf_c[] = {0, 1, 2};
    constexpr int NCAND = 2 * 5 * 3;
    // the residual and restriction forms the V-cycle will launch
    const bool zg_cfg = c->p.smoother == FLD_SMOOTH_RBGS && c->p.pre == 1;
    fld_status st = FLD_OK;
    for (int l = 0; l + 1 < c->nl && !st; l++) {
        Level& L = c->L[l];
        Level& C = c->L[l + 1];
        if (!fine4_ok(L.d)) continue;
        const size_t nb = L.d.n * sizeof(float), ncb = C.d.n * sizeof(float);
        float* r = l == 0 ? (float*)c->cg[0] : (float*)L.r;
        float* z = l == 0 ? (float*)c->cg[1] : (float*)L.z;
        float* t = (float*)L.t;
        // sweep inputs need finite values only; results are discarded
        cudaMemsetAsync(r, 0, nb, s);
        cudaMemsetAsync(z, 0, nb, s);
        cudaMemsetAsync(t, 0, nb, s);
        cudaMemsetAsync(C.t, 0, ncb, s);
        cudaMemsetAsync(C.z, 0, ncb, s);
        if (!c->assembled) {
            cudaMemsetAsync(L.A32.m, 0, nb, s);
            cudaMemsetAsync(L.A32.wx, 0, nb, s);
            cudaMemsetAsync(L.A32.wy, 0, nb, s);
            cudaMemsetAsync(L.A32.wz, 0, nb, s);
            cudaMemsetAsync(L.A32.invd, 0, nb, s);
            if (L.Abf.wx) {
                cudaMemsetAsync(L.Abf.wx, 0, nb / 2, s);
                cudaMemsetAsync(L.Abf.wy, 0, nb / 2, s);
                cudaMemsetAsync(L.Abf.wz, 0, nb / 2, s);
                cudaMemsetAsync(L.Abf.invd, 0, nb / 2, s);
            }
        }
        if (l == 0) {
            cudaMemsetAsync(c->cg[2], 0, nb, s);
            cudaMemsetAsync(c->cg[3], 0, nb, s);
        }
        for (int k = 0; k < NTUNE && !st; k++) {
            if (k == TN_PMATVEC && l != 0) continue;
            if (k == TN_POST && !(c->p.fused_post && post4_ok(L.d))) continue;
            auto run = [&](const Tune& tn) {
                switch (k) {
                // the sweeps the V-cycle launches: bfloat16 coefficients where
                // the level has them
                case TN_SMOOTH0:
                    if (L.Abf.wx) launch_smooth_zero4(L.d, L.Abf, r, t, s, tn);
                    else launch_smooth_zero4(L.d, L.A32, r, t, s, tn);
                    break;
                case TN_RB:
                    if (L.Abf.wx) launch_rb_colour4(L.d, L.Abf, r, t, 0, s, tn);
                    else launch_rb_colour4(L.d, L.A32, r, t, 0, s, tn);
                    break;
                case TN_RES:
                    if (L.Abf.wx) launch_residual4(L.d, L.Abf, z, t, s, tn, red_compress_ok(L.d));
                    else launch_residual4(L.d, L.A32, r, z, t, s, tn, zg_cfg, zg_cfg && red_compress_ok(L.d));
                    break;
                case TN_RESTRICT:
                    launch_restrict4(L.d, C.d, t, (float*)C.t, s, tn, zg_cfg && red_compress_ok(L.d));
                    break;
                case TN_PROLONG: launch_prolong_add4(L.d, C.d, (const float*)C.z, t, s, tn); break;
                case TN_POST: launch_post_smooth4(L.d, L.A32, r, z, t, nullptr, s, tn); break;
                case TN_PMATVEC:
                    launch_cg_p_matvec4(L.d, L.A32, z, (const float*)c->cg[2], (float*)c->cg[3],
                                        (float*)c->cg[4], red(c, R_ALPHA), s, tn);
                    break;
                }
            };
            float best = 1e30f;
            for (int q = 0; q < NCAND && !st; q++) {
                Tune tn;
                tn.threads = threads_c[q % 2];
                tn.target = target_c[(q / 2) % 5];
                tn.pf = pf_c[q / 10];
                if (k == TN_POST && tn.threads != 256) continue;   // fixed block of 32 x 8
                run(tn);
                cudaEventRecord(e0, s);
                for (int rep = 0; rep < reps; rep++) run(tn);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    st = set_err(FLD_ECUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    L.tune[k] = tn;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the timing launches left scalars behind
    cudaMemsetAsync(c->sc, 0, NUM_SLOTS * sizeof(double), s);
    cudaMemsetAsync(c->counter, 0, 256, s);
    CUDA_TRY(cudaStreamSynchronize(s));
    return st;
}

int fld_tuning_size(fld_ctx* c) { return c ? TUNE_FIELDS * NTUNE * c->nl : 0; }

fld_status fld_get_tuning(fld_ctx* c, int* out, int n) {
    if (!c || !out || n < TUNE_FIELDS * NTUNE * c->nl) return set_err(FLD_EINVAL, "buffer too small");
    for (int l = 0; l < c->nl; l++)
        for (int k = 0; k < NTUNE; k++) {
            int* e = out + TUNE_FIELDS * (l * NTUNE + k);
            e[0] = c->L[l].tune[k].threads;
            e[1] = c->L[l].tune[k].target;
            e[2] = c->L[l].tune[k].pf;
        }
    return FLD_OK;
}

fld_status fld_set_tuning(fld_ctx* c, const int* in, int n) {
    if (!c || !in || n != TUNE_FIELDS * NTUNE * c->nl)
        return set_err(FLD_EINVAL, "tuning table of the wrong size");
    for (int q = 0; q < n; q += TUNE_FIELDS) {
        const int th = in[q], tg = in[q + 1], pf = in[q + 2];
        if (th < 32 || th > 256 || (th & (th - 1)) || tg < 1 || tg > RED_MAX_BLOCKS || pf < 0 || pf > TUNE_PF_MAX)
            return set_err(FLD_EINVAL, "invalid launch shape in tuning table");
    }
    for (int l = 0; l < c->nl; l++)
        for (int k = 0; k < NTUNE; k++) {
            const int* e = in + TUNE_FIELDS * (l * NTUNE + k);
            c->L[l].tune[k].threads = e[0];
            c->L[l].tune[k].target = e[1];
            c->L[l].tune[k].pf = e[2];
        }
    drop_graphs(c);
    return FLD_OK;
}

fld_status fld_profile(fld_ctx* c, unsigned long long class_mask) {
    if (!c) return set_err(FLD_EINVAL, "null context");
    if (c->s) cudaStreamSynchronize(c->s);
    harvest(c);
    c->tmask = class_mask;
    for (int k = 0; k < K_NUM; k++) c->kstat[k] = KStat{};
    return FLD_OK;
}

int fld_profile_read(fld_ctx* c, fld_kernel_stat* out, int max) {
    if (!c) return 0;
    for (int k = 0; k < K_NUM && k < max; k++) {
        out[k].name = KNAMES[k];
        out[k].launches = c->kstat[k].launches;
        out[k].timed = c->kstat[k].timed;
        out[k].ms = c->kstat[k].ms;
        out[k].bytes = c->kstat[k].bytes;
        out[k].timed_bytes = c->kstat[k].timed_bytes;
    }
    return K_NUM;
}

const char* fld_last_error(void) { return g_err.c_str(); }

}  // extern "C"
