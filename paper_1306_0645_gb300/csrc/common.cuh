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
    S_R64,        // ||r64||^2 (outer FP64 residual)
    S_RMAX,       // max |r64|
    S_SCALE,      // inner-solve scale s (mixed mode)
    S_BAL,        // photon balance partial sums
    S_EMIT,
    S_ABSORB,
    S_BAD,        // > 0: invalid input seen by the assembly
    S_NONFINITE,  // > 0: a reduction produced NaN/Inf
    S_TRUE_RR,    // ||b - A x||^2 recomputed
    NUM_SLOTS = 32
};

// What the last block of a reduction does with the finished sums.
enum RedOp {
    R_STORE1 = 0,   // sc[slot0] = v0
    R_RHO,          // rho = v0; beta = first ? 0 : rho/rho_old; rho_old = rho
    R_ALPHA,        // alpha = rho / v0
    R_STORE2,       // sc[slot0] = v0, sc[slot1] = v1
    R_STORE3,       // sc[slot0..2] = v0..v2 (slots consecutive from slot0)
    R_STORE_SUM_MAX // sc[slot0] = v0 (sum), sc[slot1] = v1 (max)
};

struct RedArgs {
    double* partials;     // >= 3 * max_blocks doubles
    unsigned* counter;    // one counter, 0 between reductions
    double* sc;           // scalar slots
    int op;
    int slot0, slot1;
    int first;            // R_RHO: first iteration
};

constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 152 * 8;

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
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
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
        sc[S_BETA] = ra.first ? 0.0 : rho / sc[S_RHO_OLD];
        sc[S_RHO] = rho;
        sc[S_RHO_OLD] = rho;
        bad = !isfinite(rho);
        break;
    }
    case R_ALPHA:
        sc[S_PQ] = v[0];
        sc[S_ALPHA] = sc[S_RHO] / v[0];
        bad = !isfinite(sc[S_ALPHA]);
        break;
    case R_STORE2:
    case R_STORE_SUM_MAX:
        sc[ra.slot0] = v[0];
        sc[ra.slot1] = v[1];
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
    const int G = gridDim.x;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) ra.partials[k * RED_MAX_BLOCKS + blockIdx.x] = v[k];
        __threadfence();
        unsigned t = atomicAdd(ra.counter, 1u);
        last = (t == (unsigned)(G - 1));
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double w[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double acc = ismax[k] ? -INFINITY : 0.0;
        for (int b = threadIdx.x; b < G; b += blockDim.x) {
            double p = __ldcg(&ra.partials[k * RED_MAX_BLOCKS + b]);
            acc = ismax[k] ? fmax(acc, p) : acc + p;
        }
        w[k] = acc;
    }
    block_reduce<NV>(w, ismax);
    if (threadIdx.x == 0) {
        red_finalize(ra, w);
        *ra.counter = 0u;
    }
}

inline int red_blocks(long long n, int threads = RED_THREADS) {
    long long b = (n + threads - 1) / threads;
    if (b > RED_MAX_BLOCKS) b = RED_MAX_BLOCKS;
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

// Decompose a flat cell index.
__device__ __forceinline__ void cell_ijk(long long c, const Dims& d, int& i, int& j, int& k) {
    long long t = c / d.nx;
    i = (int)(c - t * d.nx);
    k = (int)(t / d.ny);
    j = (int)(t - (long long)k * d.ny);
}

}  // namespace fld
