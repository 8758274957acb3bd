// common.cuh -- shared device helpers of libfld: grid shapes, device scalar
// slots and the deterministic two-level FP64 reduction.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fld {

// Shape of one level of the hierarchy.
struct Dims {
    int nx, ny, nz;
    int px, py, pz;   // 1 = periodic axis
    long long n;      // nx * ny * nz
};

// Device-resident scalars of the solver, one double slot each.
enum Slot {
    S_BB = 0,     // ||b||^2 (FP64 fine system)
    S_RHO,        // <r, z>
    S_RHO_OLD,
    S_BETA,
    S_PQ,         // <p, q>
    S_ALPHA,
    S_RR,         // ||r||^2 of the current (inner) solve
    S_R0,         // ||r_0||^2 of the current inner solve
    S_XZERO,      // != 0: the next CG p/q kernel starts x at 0 (its reduction clears it)
    S_RMAX,       // max |r64|
    S_SCALE,      // inner-solve scale s (mixed mode)
    S_BAL,        // photon balance partial sums
    S_EMIT,
    S_ABSORB,
    S_BAD,        // > 0: invalid input seen by the assembly
    S_NONFINITE,  // > 0: a reduction produced NaN/Inf
    S_TRUE_RR,    // ||b - A x||^2 recomputed
    S_FLOOR,      // energy density added by the E >= 0 floor (after S_ABSORB)
    S_FIRST,      // 1 before the first CG iteration (beta = 0), then 0
    S_DE2,        // sum dE^2 of the step
    S_EN2,        // sum (E^{n+1})^2
    S_OUT0,       // photons out through the Dirichlet faces of side 0..5
    S_OUT5 = S_OUT0 + 5,
    S_OUTABS0,    // the same summed in absolute value per face, side 0..5
    S_OUTABS5 = S_OUTABS0 + 5,
    S_ESUM,       // sum of the loss-weighted energies E^n + theta dE (finalise)
    S_THRESH,     // device-side CG loop: stop when ||r||^2 <= this,
    S_MAXIT,      //   or after this many iterations;
    S_KITER,      //   iterations done
    S_EMAX,       // mixed assembly: max E, max n_HI, max eta (bit patterns of
    S_NMAX,       //   non-negative doubles, so they are maximised as integers;
    S_ETAMAX,     //   the low word is cleared), the scales of the df arithmetic
    NUM_SLOTS = 40
};

// What the last block of a reduction does with the finished sums.
enum RedOp {
    R_STORE1 = 0,   // sc[slot0] = v0
    R_RHO,          // rho = v0; beta = first ? 0 : rho/rho_old; rho_old = rho
    R_ALPHA,        // alpha = rho / v0
    R_STORE2,       // sc[slot0] = v0, sc[slot1] = v1
    R_STORE3,       // sc[slot0..2] = v0..v2 (slots consecutive from slot0)
    R_STORE7_FIN,   // sc[S_BAL], [S_EMIT], [S_ABSORB], [S_FLOOR], [S_DE2], [S_EN2], [S_ESUM] = v0..v6
    R_STORE_SUM_MAX, // sc[slot0] = v0 (sum), sc[slot1] = v1 (max)
    R_IRRES         // scaled refinement residual: sc[S_R0] = sc[S_RR] = v0,
                    // sc[S_RMAX] = v1 (max), sc[S_SCALE] = aux
};

struct RedArgs {
    double* partials;     // >= 8 * RED_MAX_BLOCKS doubles
    unsigned* counter;    // one counter, 0 between reductions
    double* sc;           // scalar slots
    int op;
    int slot0, slot1;
    int first;            // R_RHO: first iteration
    double aux;           // R_IRRES: the scale stored in S_SCALE
};

constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 16384;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide reduction of NV values in a fixed order; result valid in
// thread 0.  ismax[k] selects max instead of sum for value k.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], const bool (&ismax)[NV]) {
    __shared__ double sh[NV][32];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (nthr + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        v[k] = ismax[k] ? warp_max(v[k]) : warp_sum(v[k]);
        if (lane == 0) sh[k][warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) {
            double t = lane < nwarps ? sh[k][lane] : (ismax[k] ? -INFINITY : 0.0);
            v[k] = ismax[k] ? warp_max(t) : warp_sum(t);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void red_finalize(const RedArgs& ra, const double* v) {
    double* sc = ra.sc;
    bool bad = false;
    switch (ra.op) {
    case R_STORE1:
        sc[ra.slot0] = v[0];
        bad = !isfinite(v[0]);
        break;
    case R_RHO: {
        double rho = v[0];
        const bool first = ra.first || sc[S_FIRST] != 0.0;
        sc[S_FIRST] = 0.0;
        sc[S_BETA] = first ? 0.0 : rho / sc[S_RHO_OLD];
        sc[S_RHO] = rho;
        sc[S_RHO_OLD] = rho;
        bad = !isfinite(rho);
        break;
    }
    case R_ALPHA:
        sc[S_PQ] = v[0];
        sc[S_ALPHA] = sc[S_RHO] / v[0];
        sc[S_XZERO] = 0.0;   // every block has read it (the last block runs this)
        bad = !isfinite(sc[S_ALPHA]);
        break;
    case R_STORE2:
    case R_STORE_SUM_MAX:
        sc[ra.slot0] = v[0];
        sc[ra.slot1] = v[1];
        bad = !isfinite(v[0]) || !isfinite(v[1]);
        break;
    case R_STORE7_FIN:
        sc[S_BAL] = v[0];
        sc[S_EMIT] = v[1];
        sc[S_ABSORB] = v[2];
        sc[S_FLOOR] = v[3];
        sc[S_DE2] = v[4];
        sc[S_EN2] = v[5];
        sc[S_ESUM] = v[6];
        for (int q = 0; q < 7; q++) bad = bad || !isfinite(v[q]);
        break;
    case R_IRRES:
        sc[S_R0] = v[0];
        sc[S_RR] = v[0];
        sc[S_RMAX] = v[1];
        sc[S_SCALE] = ra.aux;
        bad = !isfinite(v[0]) || !isfinite(v[1]);
        break;
    case R_STORE3:
        sc[ra.slot0] = v[0];
        sc[ra.slot0 + 1] = v[1];
        sc[ra.slot0 + 2] = v[2];
        bad = !isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2]);
        break;
    }
    if (bad) sc[S_NONFINITE] = 1.0;
}

// Deterministic grid reduction: each block writes its partials; the last
// block to arrive (atomic ticket, no waiting) sums all partials in block
// order and runs the finaliser.  The order of the additions depends only on
// the launch shape, never on block scheduling.
template <int NV>
__device__ __forceinline__ void grid_reduce(double (&v)[NV], const bool (&ismax)[NV],
                                            const RedArgs& ra) {
    block_reduce<NV>(v, ismax);
    __shared__ bool last;
    const int G = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) ra.partials[k * RED_MAX_BLOCKS + bid] = v[k];
        __threadfence();
        unsigned t = atomicAdd(ra.counter, 1u);
        last = (t == (unsigned)(G - 1));
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double w[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) w[k] = ismax[k] ? -INFINITY : 0.0;
    // the partials b = tid, tid + nthr, ... of every value, U of them per
    // step with their loads issued together (the same order of additions
    // as one at a time)
    constexpr int U = NV <= 2 ? 8 : (NV <= 4 ? 4 : 2);
    int b = tid;
    for (; b + (U - 1) * nthr < G; b += U * nthr) {
        double p[U][NV];
#pragma unroll
        for (int u = 0; u < U; u++)
#pragma unroll
            for (int k = 0; k < NV; k++) p[u][k] = __ldcg(&ra.partials[k * RED_MAX_BLOCKS + b + u * nthr]);
#pragma unroll
        for (int u = 0; u < U; u++)
#pragma unroll
            for (int k = 0; k < NV; k++) w[k] = ismax[k] ? fmax(w[k], p[u][k]) : w[k] + p[u][k];
    }
    for (; b < G; b += nthr)
#pragma unroll
        for (int k = 0; k < NV; k++) {
            const double p = __ldcg(&ra.partials[k * RED_MAX_BLOCKS + b]);
            w[k] = ismax[k] ? fmax(w[k], p) : w[k] + p;
        }
    block_reduce<NV>(w, ismax);
    if (tid == 0) {
        red_finalize(ra, w);
        *ra.counter = 0u;
    }
}

// Per-thread accumulator of a dot product.  FP64 data accumulate with FMA.
// FP32 data keep FP64-level accuracy without FP64 arithmetic per element
// (the FP64 pipe of this GPU is 1/64 of the FP32 one): each product is split
// exactly into p + e (p = fl(a b), e = fma(a, b, -p)), and the products are
// summed in a compensated pair (Knuth's two-sum).  Only the per-thread
// result goes to FP64.  The _rn intrinsics keep the compiler from fusing
// the error-free steps.
template <class T>
struct DotAcc;
template <>
struct DotAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);
        const float t = __fadd_rn(hi, p);
        const float bp = __fsub_rn(t, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        hi = t;
        lo = __fadd_rn(lo, __fadd_rn(err, e));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

constexpr int FLAT_MAX_BLOCKS = 152 * 16;

// Grid-stride loop over [0, n).
#define GRID_LOOP(c, n) \
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < (n); c += (long long)gridDim.x * blockDim.x)

// Blocks of a flat reduction over n items: 16 items per thread (fewer
// partial sums for the last block to add on small grids), but two blocks
// per SM while the items allow one per thread, and at most FLAT_MAX_BLOCKS.
inline int red_blocks(long long n, int threads = RED_THREADS) {
    long long b = (n + 16LL * threads - 1) / (16LL * threads);
    if (b < 152 * 2) {
        const long long one = (n + threads - 1) / threads;
        b = one < 152 * 2 ? one : 152 * 2;
    }
    if (b > FLAT_MAX_BLOCKS) b = FLAT_MAX_BLOCKS;
    if (b < 1) b = 1;
    return (int)b;
}

inline int grid_blocks(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    const long long cap = 152LL * 64;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// Launch shape of a stencil sweep over one level: a 2-D thread block tiles
// (x, y), the grid covers the (x, y) tiles times z chunks, and every thread
// walks k through its chunk (no integer division per cell).
struct ColShape {
    dim3 grid, block;
};

inline int pow2ceil(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

inline ColShape col_shape(const Dims& d, int threads = 256, int target_blocks = 152 * 8) {
    int bx = pow2ceil(d.nx) < 32 ? pow2ceil(d.nx) : 32;
    int by = threads / bx;
    if (by > pow2ceil(d.ny)) by = pow2ceil(d.ny);
    const int gx = (d.nx + bx - 1) / bx, gy = (d.ny + by - 1) / by;
    long long xy = (long long)gx * gy;
    long long gz = (target_blocks + xy - 1) / xy;
    if (gz > d.nz) gz = d.nz;
    if (xy * gz > RED_MAX_BLOCKS) gz = RED_MAX_BLOCKS / xy;
    if (gz < 1) gz = 1;
    ColShape s;
    s.block = dim3(bx, by, 1);
    s.grid = dim3(gx, gy, (unsigned)gz);
    return s;
}

// Per-thread column walk: defines i, j and loops k over the thread's chunk.
#define COL_BEGIN(d)                                                                    \
    const int i = blockIdx.x * blockDim.x + threadIdx.x;                                \
    const int j = blockIdx.y * blockDim.y + threadIdx.y;                                \
    const int kch_ = ((d).nz + (int)gridDim.z - 1) / (int)gridDim.z;                   \
    const int k0_ = (int)blockIdx.z * kch_;                                             \
    const int k1_ = min((d).nz, k0_ + kch_);                                            \
    const bool inb_ = i < (d).nx && j < (d).ny;                                         \
    const long long nxy_ = (long long)(d).nx * (d).ny;                                  \
    for (int k = inb_ ? k0_ : k1_; k < k1_; k++) {                                      \
        const long long c = (long long)k * nxy_ + (long long)j * (d).nx + i;
#define COL_END }

// The same walk over z-blocks zb0 .. zb0 + gridDim.z - 1 of a decomposition
// of the planes into blocks of kch planes (a launch that covers a range of
// whole z-blocks of a larger grid; zb0 = 0 and kch = ceil(nz / gridDim.z)
// is COL_BEGIN).
#define COL_BEGIN_ZB(d, zb0, kch)                                                       \
    const int i = blockIdx.x * blockDim.x + threadIdx.x;                                \
    const int j = blockIdx.y * blockDim.y + threadIdx.y;                                \
    const int k0_ = ((zb0) + (int)blockIdx.z) * (kch);                                  \
    const int k1_ = min((d).nz, k0_ + (kch));                                           \
    const bool inb_ = i < (d).nx && j < (d).ny;                                         \
    const long long nxy_ = (long long)(d).nx * (d).ny;                                  \
    for (int k = inb_ ? k0_ : k1_; k < k1_; k++) {                                      \
        const long long c = (long long)k * nxy_ + (long long)j * (d).nx + i;

// Decompose a flat cell index.
__device__ __forceinline__ void cell_ijk(long long c, const Dims& d, int& i, int& j, int& k) {
    long long t = c / d.nx;
    i = (int)(c - t * d.nx);
    k = (int)(t / d.ny);
    j = (int)(t - (long long)k * d.ny);
}

}  // namespace fld
