// walk4.cuh -- the thread geometry of the four-cells-per-thread stencil
// sweeps: a thread owns four consecutive cells along x (one float4 of an
// FP32 array), a row j, and walks k through its chunk of planes; the x
// neighbours of its four cells come from the adjacent lanes.
#pragma once
#include "kernels.h"

namespace fld {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float4 ld4(const float* __restrict__ p, long long i) {
    return *reinterpret_cast<const float4*>(p + i);
}
__device__ __forceinline__ void st4(float* p, long long i, float4 v) {
    *reinterpret_cast<float4*>(p + i) = v;
}
// Prefetch of the line holding p + i into L2.  The sweeps issue it for the
// plane pf ahead of the one they compute, so that plane's loads hit L2:
// bytes are requested from HBM without holding registers or scoreboard
// entries while the current plane waits on its own loads.
template <class T>
__device__ __forceinline__ void pf2(const T* p, long long i) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(p + i)));
}

// Geometry of one 4-cell vector on one plane.  Indices of missing
// neighbours (zero-gradient boundary) point at the cell itself; the matching
// face weights are zero, so those values never contribute.
struct Geo {
    long long c;            // first cell of the vector
    long long ym, yp;       // first cell of the y-neighbour vectors
    long long xl, xr;       // left neighbour of element 0, right of element 3
    long long xr_w;         // weight index of the upper x face of element 3
    bool has_xr, has_yp;    // upper faces exist
    bool load_l, load_r;    // x neighbour not held by the adjacent lane
};

struct Walk {
    int i4, j, k0, k1, nx4;
    bool valid;             // owns real cells (else computes on clamped ones)
    long long nxy;
};

__device__ __forceinline__ Walk walk_of(const Dims& d) {
    Walk w;
    w.nx4 = d.nx >> 2;
    const int i4 = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    w.valid = i4 < w.nx4 && j < d.ny;
    w.i4 = min(i4, w.nx4 - 1);
    w.j = min(j, d.ny - 1);
    const int kch = (d.nz + (int)gridDim.z - 1) / (int)gridDim.z;
    w.k0 = (int)blockIdx.z * kch;
    w.k1 = min(d.nz, w.k0 + kch);
    w.nxy = (long long)d.nx * d.ny;
    return w;
}

__device__ __forceinline__ Geo geo_of(const Dims& d, const Walk& w, int k) {
    Geo g;
    const int i0 = 4 * w.i4;
    const long long row = (long long)k * w.nxy + (long long)w.j * d.nx;
    g.c = row + i0;
    // y
    if (w.j > 0) g.ym = g.c - d.nx;
    else g.ym = d.py ? g.c + (long long)(d.ny - 1) * d.nx : g.c;
    g.has_yp = w.j < d.ny - 1 || d.py;
    g.yp = (w.j < d.ny - 1) ? g.c + d.nx : (d.py ? g.c - (long long)(d.ny - 1) * d.nx : g.c);
    // x: left of element 0, right of element 3
    g.xl = (i0 > 0) ? g.c - 1 : (d.px ? row + d.nx - 1 : g.c);
    g.has_xr = (i0 + 4 < d.nx) || d.px;
    g.xr = (i0 + 4 < d.nx) ? g.c + 4 : (d.px ? row : g.c + 3);
    g.xr_w = (i0 + 4 < d.nx) ? g.c + 4 : row;   // weight of that face (periodic: cell 0's lower face)
    // the adjacent lane holds the neighbouring vector unless this lane is
    // the first / last of its block row or the row ends
    g.load_l = threadIdx.x == 0 || i0 == 0;
    g.load_r = threadIdx.x == blockDim.x - 1 || i0 + 4 >= d.nx;
    return g;
}

// z-neighbour plane offsets (missing: own plane, weight 0)
__device__ __forceinline__ long long zdn(const Dims& d, int k, long long nxy) {
    return k > 0 ? -nxy : (d.pz ? (long long)(d.nz - 1) * nxy : 0);
}
__device__ __forceinline__ long long zup(const Dims& d, int k, long long nxy) {
    return k < d.nz - 1 ? nxy : (d.pz ? -(long long)(d.nz - 1) * nxy : 0);
}

}  // namespace

}  // namespace fld
