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
// another's writes.
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

template <class T>
__device__ __forceinline__ T ldw(const T* p, long long i) { return __ldcg(p + i); }

// sum_f w_f u_nbr and sum_f w_f of cell c (u read through L2)
template <class T>
__device__ __forceinline__ void tail_nbr_sums(const Dims& d, const Op<T>& A, long long c, int i, int j,
                                              int k, const T* u, T& swu, T& sw) {
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    T a = T(0), s = T(0);
    {
        const T wl = A.wx[c];
        if (i > 0) { a += wl * ldw(u, c - 1); s += wl; }
        else if (d.px) { a += wl * ldw(u, c + d.nx - 1); s += wl; }
        if (i < d.nx - 1) { const T wu = A.wx[c + 1]; a += wu * ldw(u, c + 1); s += wu; }
        else if (d.px) { const long long up = c - (d.nx - 1); const T wu = A.wx[up]; a += wu * ldw(u, up); s += wu; }
    }
    {
        const T wl = A.wy[c];
        if (j > 0) { a += wl * ldw(u, c - sy); s += wl; }
        else if (d.py) { a += wl * ldw(u, c + (long long)(d.ny - 1) * sy); s += wl; }
        if (j < d.ny - 1) { const T wu = A.wy[c + sy]; a += wu * ldw(u, c + sy); s += wu; }
        else if (d.py) { const long long up = c - (long long)(d.ny - 1) * sy; const T wu = A.wy[up]; a += wu * ldw(u, up); s += wu; }
    }
    {
        const T wl = A.wz[c];
        if (k > 0) { a += wl * ldw(u, c - sz); s += wl; }
        else if (d.pz) { a += wl * ldw(u, c + (long long)(d.nz - 1) * sz); s += wl; }
        if (k < d.nz - 1) { const T wu = A.wz[c + sz]; a += wu * ldw(u, c + sz); s += wu; }
        else if (d.pz) { const long long up = c - (long long)(d.nz - 1) * sz; const T wu = A.wz[up]; a += wu * ldw(u, up); s += wu; }
    }
    swu = a;
    sw = s;
}

// sum_f w_f u_nbr v_nbr (the red neighbours r * invd of a zero-guess sweep)
template <class T>
__device__ __forceinline__ T tail_nbr_sum_prod(const Dims& d, const Op<T>& A, long long c, int i, int j,
                                               int k, const T* u, const T* v) {
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    T a = T(0);
    if (i > 0) a += A.wx[c] * ldw(u, c - 1) * v[c - 1];
    else if (d.px) a += A.wx[c] * ldw(u, c + d.nx - 1) * v[c + d.nx - 1];
    if (i < d.nx - 1) a += A.wx[c + 1] * ldw(u, c + 1) * v[c + 1];
    else if (d.px) { const long long up = c - (d.nx - 1); a += A.wx[up] * ldw(u, up) * v[up]; }
    if (j > 0) a += A.wy[c] * ldw(u, c - sy) * v[c - sy];
    else if (d.py) { const long long lo = c + (long long)(d.ny - 1) * sy; a += A.wy[c] * ldw(u, lo) * v[lo]; }
    if (j < d.ny - 1) a += A.wy[c + sy] * ldw(u, c + sy) * v[c + sy];
    else if (d.py) { const long long up = c - (long long)(d.ny - 1) * sy; a += A.wy[up] * ldw(u, up) * v[up]; }
    if (k > 0) a += A.wz[c] * ldw(u, c - sz) * v[c - sz];
    else if (d.pz) { const long long lo = c + (long long)(d.nz - 1) * sz; a += A.wz[c] * ldw(u, lo) * v[lo]; }
    if (k < d.nz - 1) a += A.wz[c + sz] * ldw(u, c + sz) * v[c + sz];
    else if (d.pz) { const long long up = c - (long long)(d.nz - 1) * sz; a += A.wz[up] * ldw(u, up) * v[up]; }
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

// Phase loops: the cluster's threads stride over the level's cells.
#define TAIL_LOOP(c, n) for (long long c = gtid; c < (n); c += gthreads)

template <class T>
__global__ void __launch_bounds__(TAIL_THREADS) k_vtail(TailArgs<T> a) {
    cg::cluster_group cl = cg::this_cluster();
    const long long gthreads = (long long)TAIL_THREADS * cl.num_blocks();
    const long long gtid = (long long)cl.block_rank() * TAIL_THREADS + threadIdx.x;
    const int nl = a.nlev;
    // ---- down: smooth from zero, residual, restrict
    for (int l = 0; l < nl - 1; l++) {
        const TailLevel<T>& L = a.L[l];
        const Dims& d = L.d;
        const Op<T>& A = L.A;
        const T* r = L.r;
        T* z = L.z;
        if (a.pre >= 1) {
            TAIL_LOOP(c, d.n) {
                int i, j, k;
                tail_ijk(c, d, i, j, k);
                const T rc = ldw(r, c);
                if (((i + j + k) & 1) == 0) z[c] = rc * A.invd[c];
                else z[c] = A.invd[c] * (rc + tail_nbr_sum_prod<T>(d, A, c, i, j, k, r, A.invd));
            }
            cl.sync();
            for (int it = 1; it < a.pre; it++)
                for (int colour = 0; colour < 2; colour++) {
                    TAIL_LOOP(c, d.n) {
                        int i, j, k;
                        tail_ijk(c, d, i, j, k);
                        if (((i + j + k) & 1) != colour) continue;
                        T swu, sw;
                        tail_nbr_sums<T>(d, A, c, i, j, k, z, swu, sw);
                        z[c] = A.invd[c] * (ldw(r, c) + swu);
                    }
                    cl.sync();
                }
        } else {
            TAIL_LOOP(c, d.n) z[c] = T(0);
            cl.sync();
        }
        // t = r - A z
        TAIL_LOOP(c, d.n) {
            int i, j, k;
            tail_ijk(c, d, i, j, k);
            T swu, sw;
            tail_nbr_sums<T>(d, A, c, i, j, k, z, swu, sw);
            const T zc = ldw(z, c);
            L.t[c] = ldw(r, c) - (A.m[c] * zc + sw * zc - swu);
        }
        cl.sync();
        // r_{l+1} = R t
        const TailLevel<T>& C = a.L[l + 1];
        const T wt[4] = {T(0.25), T(0.75), T(0.75), T(0.25)};
        TAIL_LOOP(cc, C.d.n) {
            int I, J, K;
            tail_ijk(cc, C.d, I, J, K);
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
                    for (int ti = 0; ti < 4; ti++) acc_i += wt[ti] * ldw((const T*)L.t, row + fi[ti]);
                    acc_j += wt[tj] * acc_i;
                }
                acc += wt[tk] * acc_j;
            }
            C.r[cc] = acc * T(0.125);
        }
        cl.sync();
    }
    // ---- coarsest: z = A^-1 r with the stored explicit inverse
    {
        const TailLevel<T>& L = a.L[nl - 1];
        const int n = (int)L.d.n;
        TAIL_LOOP(row, n) {
            double acc = 0.0;
            for (int q = 0; q < n; q++) acc += a.ainv[(long long)q * n + row] * (double)ldw((const T*)L.r, q);
            L.z[row] = (T)acc;
        }
        cl.sync();
    }
    // ---- up: prolongate and correct, post-smooth
    for (int l = nl - 2; l >= 0; l--) {
        const TailLevel<T>& L = a.L[l];
        const TailLevel<T>& C = a.L[l + 1];
        const Dims& d = L.d;
        const Op<T>& A = L.A;
        T* z = L.z;
        const T w2[2] = {T(0.75), T(0.25)};
        TAIL_LOOP(c, d.n) {
            int i, j, k;
            tail_ijk(c, d, i, j, k);
            int Ix[2], Iy[2], Iz[2];
            tail_coarse_pair(i, C.d.nx, C.d.px, Ix[0], Ix[1]);
            tail_coarse_pair(j, C.d.ny, C.d.py, Iy[0], Iy[1]);
            tail_coarse_pair(k, C.d.nz, C.d.pz, Iz[0], Iz[1]);
            T acc = T(0);
#pragma unroll
            for (int b = 0; b < 2; b++) {
                T acc_j = T(0);
#pragma unroll
                for (int q = 0; q < 2; q++) {
                    const long long row = (long long)C.d.nx * (Iy[q] + (long long)C.d.ny * Iz[b]);
                    acc_j += w2[q] * (w2[0] * ldw((const T*)C.z, row + Ix[0]) + w2[1] * ldw((const T*)C.z, row + Ix[1]));
                }
                acc += w2[b] * acc_j;
            }
            z[c] = ldw((const T*)z, c) + acc;
        }
        cl.sync();
        for (int it = 0; it < a.post; it++)
            for (int colour = 1; colour >= 0; colour--) {
                TAIL_LOOP(c, d.n) {
                    int i, j, k;
                    tail_ijk(c, d, i, j, k);
                    if (((i + j + k) & 1) != colour) continue;
                    T swu, sw;
                    tail_nbr_sums<T>(d, A, c, i, j, k, z, swu, sw);
                    z[c] = A.invd[c] * (ldw(L.r, c) + swu);
                }
                cl.sync();
            }
    }
}

#undef TAIL_LOOP

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
cudaError_t launch_vtail(const TailArgs<T>& a, int cluster, cudaStream_t s) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = tail_config(cluster, s, attr);
    return cudaLaunchKernelEx(&cfg, k_vtail<T>, a);
}

// The largest cluster (16 CTAs, a non-portable size, else the portable 8)
// of which at least one can be resident; 0 if none.
template <class T>
int vtail_cluster() {
    if (cudaFuncSetAttribute(k_vtail<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        cudaGetLastError();
    for (int cluster : {16, 8}) {
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = tail_config(cluster, nullptr, attr);
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
