// k_tail.cu -- the coarse tail of the multigrid V-cycle (Table 1's
// preconditioner) as one persistent kernel: every level at or below a size
// threshold, from the first such level down to the dense coarsest grid and
// back up, runs in a single launch of one thread-block cluster.
//
// Below ~32^3 cells a level's sweeps are latency-bound: each launch costs a
// few microseconds whatever its size, and a V-cycle has about seven of them
// per level.  Here the phases of those levels (pre-smoothing, residual,
// restriction, coarsest solve, prolongation, post-smoothing) are separated
// by the cluster barrier instead of kernel boundaries.  The barrier is the
// hardware one of the cluster (all CTAs of a cluster are co-scheduled), so
// no software spin is involved.  Values written inside the kernel are read
// back with L1-bypassing loads (.cg), so no CTA sees a stale line of
// another's writes.  From the first level of at most TAIL_SMALL_CELLS cells
// down, CTA 0 works alone with the levels' vectors in its shared memory
// and block barriers between the phases (a phase then costs a fraction of
// a microsecond); the other CTAs wait at the next cluster barrier.
//
// The arithmetic of every phase is that of the scalar level kernels of
// k_mg.cu (red/black Gauss-Seidel from a zero guess, colour sweeps, r - A z,
// full-weighting restriction, trilinear prolongation, dense inverse on the
// coarsest grid), so the tail gives the V-cycle those kernels give.
#include <cooperative_groups.h>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace fld {

namespace {

constexpr int TAIL_THREADS = 1024;

// Vectors written inside the kernel: in cluster mode they live in global
// memory and are read through L2 (.cg); in single-CTA mode they live in
// shared memory and are read directly.
template <bool CG, class T>
__device__ __forceinline__ T ldw(const T* p, long long i) {
    if constexpr (CG) return __ldcg(p + i);
    else return p[i];
}

// sum_f w_f u_nbr and sum_f w_f of cell c
template <bool CG, class T>
__device__ __forceinline__ void tail_nbr_sums(const Dims& d, const Op<T>& A, long long c, int i, int j,
                                              int k, const T* u, T& swu, T& sw) {
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    T a = T(0), s = T(0);
    {
        const T wl = A.wx[c];
        if (i > 0) { a += wl * ldw<CG>(u, c - 1); s += wl; }
        else if (d.px) { a += wl * ldw<CG>(u, c + d.nx - 1); s += wl; }
        if (i < d.nx - 1) { const T wu = A.wx[c + 1]; a += wu * ldw<CG>(u, c + 1); s += wu; }
        else if (d.px) { const long long up = c - (d.nx - 1); const T wu = A.wx[up]; a += wu * ldw<CG>(u, up); s += wu; }
    }
    {
        const T wl = A.wy[c];
        if (j > 0) { a += wl * ldw<CG>(u, c - sy); s += wl; }
        else if (d.py) { a += wl * ldw<CG>(u, c + (long long)(d.ny - 1) * sy); s += wl; }
        if (j < d.ny - 1) { const T wu = A.wy[c + sy]; a += wu * ldw<CG>(u, c + sy); s += wu; }
        else if (d.py) { const long long up = c - (long long)(d.ny - 1) * sy; const T wu = A.wy[up]; a += wu * ldw<CG>(u, up); s += wu; }
    }
    {
        const T wl = A.wz[c];
        if (k > 0) { a += wl * ldw<CG>(u, c - sz); s += wl; }
        else if (d.pz) { a += wl * ldw<CG>(u, c + (long long)(d.nz - 1) * sz); s += wl; }
        if (k < d.nz - 1) { const T wu = A.wz[c + sz]; a += wu * ldw<CG>(u, c + sz); s += wu; }
        else if (d.pz) { const long long up = c - (long long)(d.nz - 1) * sz; const T wu = A.wz[up]; a += wu * ldw<CG>(u, up); s += wu; }
    }
    swu = a;
    sw = s;
}

// sum_f w_f u_nbr v_nbr (the red neighbours r * invd of a zero-guess sweep)
template <bool CG, class T>
__device__ __forceinline__ T tail_nbr_sum_prod(const Dims& d, const Op<T>& A, long long c, int i, int j,
                                               int k, const T* u, const T* v) {
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    T a = T(0);
    if (i > 0) a += A.wx[c] * ldw<CG>(u, c - 1) * v[c - 1];
    else if (d.px) a += A.wx[c] * ldw<CG>(u, c + d.nx - 1) * v[c + d.nx - 1];
    if (i < d.nx - 1) a += A.wx[c + 1] * ldw<CG>(u, c + 1) * v[c + 1];
    else if (d.px) { const long long up = c - (d.nx - 1); a += A.wx[up] * ldw<CG>(u, up) * v[up]; }
    if (j > 0) a += A.wy[c] * ldw<CG>(u, c - sy) * v[c - sy];
    else if (d.py) { const long long lo = c + (long long)(d.ny - 1) * sy; a += A.wy[c] * ldw<CG>(u, lo) * v[lo]; }
    if (j < d.ny - 1) a += A.wy[c + sy] * ldw<CG>(u, c + sy) * v[c + sy];
    else if (d.py) { const long long up = c - (long long)(d.ny - 1) * sy; a += A.wy[up] * ldw<CG>(u, up) * v[up]; }
    if (k > 0) a += A.wz[c] * ldw<CG>(u, c - sz) * v[c - sz];
    else if (d.pz) { const long long lo = c + (long long)(d.nz - 1) * sz; a += A.wz[c] * ldw<CG>(u, lo) * v[lo]; }
    if (k < d.nz - 1) a += A.wz[c + sz] * ldw<CG>(u, c + sz) * v[c + sz];
    else if (d.pz) { const long long up = c - (long long)(d.nz - 1) * sz; a += A.wz[up] * ldw<CG>(u, up) * v[up]; }
    return a;
}

// Cell coordinates by 32-bit unsigned division (tail levels hold fewer
// than 2^24 cells; 64-bit division would cost far more than the sweep).
__device__ __forceinline__ void tail_ijk(long long c, const Dims& d, int& i, int& j, int& k) {
    const unsigned cu = (unsigned)c, nx = (unsigned)d.nx, nxy = (unsigned)d.nx * (unsigned)d.ny;
    const unsigned kk = cu / nxy;
    const unsigned rem = cu - kk * nxy;
    const unsigned jj = rem / nx;
    k = (int)kk;
    j = (int)jj;
    i = (int)(rem - jj * nx);
}

__device__ __forceinline__ int tail_fine_tap(int I, int t, int nf, int periodic) {
    int f = 2 * I - 1 + t;
    if (f < 0) f = periodic ? f + nf : 0;
    if (f >= nf) f = periodic ? f - nf : nf - 1;
    return f;
}

__device__ __forceinline__ void tail_coarse_pair(int i, int nc, int periodic, int& I0, int& I1) {
    I0 = i >> 1;
    int J = (i & 1) ? I0 + 1 : I0 - 1;
    if (J < 0) J = periodic ? nc - 1 : I0;
    if (J >= nc) J = periodic ? 0 : I0;
    I1 = J;
}

// The vectors of one level as a phase sees them (global or shared memory).
template <class T>
struct Vec {
    T *r, *z, *t;
};

// Phase loops: the participating threads stride over the level's cells.
#define TAIL_LOOP(c, n) for (long long c = tid; c < (n); c += nth)

// Down-leg phases of level L into the coarse right-hand side rc:
// smoothing from zero (and further pre-sweeps), t = r - A z, rc = R t.
template <bool CG, class T, class Sync>
__device__ void tail_down(const TailLevel<T>& L, Vec<T> v, const Dims& cd, T* rc, int pre, long long tid,
                          long long nth, Sync sync) {
    const Dims& d = L.d;
    const Op<T>& A = L.A;
    const T* r = v.r;
    T* z = v.z;
    if (pre >= 1) {
        TAIL_LOOP(c, d.n) {
            int i, j, k;
            tail_ijk(c, d, i, j, k);
            const T rcv = ldw<CG>(r, c);
            if (((i + j + k) & 1) == 0) z[c] = rcv * A.invd[c];
            else z[c] = A.invd[c] * (rcv + tail_nbr_sum_prod<CG, T>(d, A, c, i, j, k, r, A.invd));
        }
        sync();
        for (int it = 1; it < pre; it++)
            for (int colour = 0; colour < 2; colour++) {
                TAIL_LOOP(c, d.n) {
                    int i, j, k;
                    tail_ijk(c, d, i, j, k);
                    if (((i + j + k) & 1) != colour) continue;
                    T swu, sw;
                    tail_nbr_sums<CG, T>(d, A, c, i, j, k, z, swu, sw);
                    z[c] = A.invd[c] * (ldw<CG>(r, c) + swu);
                }
                sync();
            }
    } else {
        TAIL_LOOP(c, d.n) z[c] = T(0);
        sync();
    }
    TAIL_LOOP(c, d.n) {
        int i, j, k;
        tail_ijk(c, d, i, j, k);
        T swu, sw;
        tail_nbr_sums<CG, T>(d, A, c, i, j, k, z, swu, sw);
        const T zc = ldw<CG>((const T*)z, c);
        v.t[c] = ldw<CG>(r, c) - (A.m[c] * zc + sw * zc - swu);
    }
    sync();
    const T wt[4] = {T(0.25), T(0.75), T(0.75), T(0.25)};
    TAIL_LOOP(cc, cd.n) {
        int I, J, K;
        tail_ijk(cc, cd, I, J, K);
        int fi[4], fj[4], fk[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
            fi[t] = tail_fine_tap(I, t, d.nx, d.px);
            fj[t] = tail_fine_tap(J, t, d.ny, d.py);
            fk[t] = tail_fine_tap(K, t, d.nz, d.pz);
        }
        T acc = T(0);
#pragma unroll
        for (int tk = 0; tk < 4; tk++) {
            T acc_j = T(0);
#pragma unroll
            for (int tj = 0; tj < 4; tj++) {
                const long long row = (long long)d.nx * (fj[tj] + (long long)d.ny * fk[tk]);
                T acc_i = T(0);
#pragma unroll
                for (int ti = 0; ti < 4; ti++) acc_i += wt[ti] * ldw<CG>((const T*)v.t, row + fi[ti]);
                acc_j += wt[tj] * acc_i;
            }
            acc += wt[tk] * acc_j;
        }
        rc[cc] = acc * T(0.125);
    }
    sync();
}

// Up-leg phases of level L: z += P zc, then the post-sweeps.
template <bool CG, class T, class Sync>
__device__ void tail_up(const TailLevel<T>& L, Vec<T> v, const Dims& cd, const T* zc, int post, int first,
                        long long tid,
                        long long nth, Sync sync) {
    const Dims& d = L.d;
    const Op<T>& A = L.A;
    T* z = v.z;
    const T w2[2] = {T(0.75), T(0.25)};
    TAIL_LOOP(c, d.n) {
        int i, j, k;
        tail_ijk(c, d, i, j, k);
        int Ix[2], Iy[2], Iz[2];
        tail_coarse_pair(i, cd.nx, cd.px, Ix[0], Ix[1]);
        tail_coarse_pair(j, cd.ny, cd.py, Iy[0], Iy[1]);
        tail_coarse_pair(k, cd.nz, cd.pz, Iz[0], Iz[1]);
        T acc = T(0);
#pragma unroll
        for (int b = 0; b < 2; b++) {
            T acc_j = T(0);
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const long long row = (long long)cd.nx * (Iy[q] + (long long)cd.ny * Iz[b]);
                acc_j += w2[q] * (w2[0] * ldw<CG>(zc, row + Ix[0]) + w2[1] * ldw<CG>(zc, row + Ix[1]));
            }
            acc += w2[b] * acc_j;
        }
        z[c] = ldw<CG>((const T*)z, c) + acc;
    }
    sync();
    // first: the colour the post-sweep starts with (1 black: symmetric cycle)
    for (int it = 0; it < post; it++)
        for (int q = 0; q < 2; q++) {
            const int colour = q == 0 ? first : 1 - first;
            TAIL_LOOP(c, d.n) {
                int i, j, k;
                tail_ijk(c, d, i, j, k);
                if (((i + j + k) & 1) != colour) continue;
                T swu, sw;
                tail_nbr_sums<CG, T>(d, A, c, i, j, k, z, swu, sw);
                z[c] = A.invd[c] * (ldw<CG>((const T*)v.r, c) + swu);
            }
            sync();
        }
}

// z = A^-1 r on the coarsest grid with the stored explicit inverse.
template <bool CG, class T, class Sync>
__device__ void tail_coarsest(int n, const double* ainv, Vec<T> v, long long tid, long long nth, Sync sync) {
    TAIL_LOOP(row, n) {
        double acc = 0.0;
        for (int q = 0; q < n; q++) acc += ainv[(long long)q * n + row] * (double)ldw<CG>((const T*)v.r, q);
        v.z[row] = (T)acc;
    }
    sync();
}

#undef TAIL_LOOP

template <class T>
__global__ void __launch_bounds__(TAIL_THREADS) k_vtail(TailArgs<T> a) {
    extern __shared__ __align__(16) unsigned char tail_smem[];
    cg::cluster_group cl = cg::this_cluster();
    const long long gthreads = (long long)TAIL_THREADS * cl.num_blocks();
    const long long gtid = (long long)cl.block_rank() * TAIL_THREADS + threadIdx.x;
    const int nl = a.nlev, ls = a.small_from;
    auto csync = [&]() { cl.sync(); };
    auto bsync = []() { __syncthreads(); };
    // ---- down, cluster mode: levels 0 .. ls-1
    for (int l = 0; l < ls && l < nl - 1; l++) {
        const TailLevel<T>& L = a.L[l];
        tail_down<true, T>(L, Vec<T>{L.r, L.z, L.t}, a.L[l + 1].d, a.L[l + 1].r, a.pre, gtid, gthreads, csync);
    }
    if (ls < nl) {
        // ---- the small levels in CTA 0 alone, vectors in shared memory
        if (cl.block_rank() == 0) {
            const long long tid = threadIdx.x, nth = TAIL_THREADS;
            Vec<T> sv[TAIL_MAX_LEVELS];
            T* base = reinterpret_cast<T*>(tail_smem);
            for (int l = ls; l < nl; l++) {
                const long long n = a.L[l].d.n;
                sv[l] = Vec<T>{base, base + n, base + 2 * n};
                base += 3 * n;
            }
            for (long long c = tid; c < a.L[ls].d.n; c += nth) sv[ls].r[c] = __ldcg(a.L[ls].r + c);
            __syncthreads();
            for (int l = ls; l < nl - 1; l++)
                tail_down<false, T>(a.L[l], sv[l], a.L[l + 1].d, sv[l + 1].r, a.pre, tid, nth, bsync);
            tail_coarsest<false, T>((int)a.L[nl - 1].d.n, a.ainv, sv[nl - 1], tid, nth, bsync);
            for (int l = nl - 2; l >= ls; l--)
                tail_up<false, T>(a.L[l], sv[l], a.L[l + 1].d, sv[l + 1].z, a.post, a.paper_order ? 0 : 1, tid, nth,
                                  bsync);
            for (long long c = tid; c < a.L[ls].d.n; c += nth) a.L[ls].z[c] = sv[ls].z[c];
        }
        cl.sync();
    } else {
        tail_coarsest<true, T>((int)a.L[nl - 1].d.n, a.ainv, Vec<T>{a.L[nl - 1].r, a.L[nl - 1].z, a.L[nl - 1].t},
                               gtid, gthreads, csync);
    }
    // ---- up, cluster mode: levels ls-1 .. 0
    for (int l = (ls < nl ? ls : nl - 1) - 1; l >= 0; l--) {
        const TailLevel<T>& L = a.L[l];
        tail_up<true, T>(L, Vec<T>{L.r, L.z, L.t}, a.L[l + 1].d, a.L[l + 1].z, a.post, a.paper_order ? 0 : 1, gtid,
                         gthreads, csync);
    }
}

}  // namespace

namespace {

cudaLaunchConfig_t tail_config(int cluster, cudaStream_t s, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster, 1, 1);
    cfg.blockDim = dim3(TAIL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

}  // namespace

template <class T>
size_t vtail_smem_bytes(const TailArgs<T>& a) {
    size_t cells = 0;
    for (int l = a.small_from; l < a.nlev; l++) cells += (size_t)a.L[l].d.n;
    return 3 * cells * sizeof(T);
}

template <class T>
cudaError_t launch_vtail(const TailArgs<T>& a, int cluster, cudaStream_t s) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = tail_config(cluster, s, attr);
    cfg.dynamicSmemBytes = vtail_smem_bytes(a);
    return cudaLaunchKernelEx(&cfg, k_vtail<T>, a);
}

// The largest cluster (16 CTAs, a non-portable size, else the portable 8)
// of which at least one can be resident; 0 if none.
template <class T>
int vtail_cluster() {
    if (cudaFuncSetAttribute(k_vtail<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        cudaGetLastError();
    if (cudaFuncSetAttribute(k_vtail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TAIL_SMEM_MAX) !=
        cudaSuccess)
        cudaGetLastError();
    for (int cluster : {16, 8}) {
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = tail_config(cluster, nullptr, attr);
        cfg.dynamicSmemBytes = TAIL_SMEM_MAX;
        int n = 0;
        const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, k_vtail<T>, &cfg);
        if (e != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (n > 0) return cluster;
    }
    return 0;
}

template cudaError_t launch_vtail<float>(const TailArgs<float>&, int, cudaStream_t);
template cudaError_t launch_vtail<double>(const TailArgs<double>&, int, cudaStream_t);
template int vtail_cluster<float>();
template int vtail_cluster<double>();

}  // namespace fld
