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
//
// The same phases also serve k_psolve, which runs whole inner MG-PCG solves
// of small grids (every level, then the CG vector operations) for a work
// list of requests in one launch (see the section below).
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
__device__ __forceinline__ T ldw(const T* p, int i) {
    if constexpr (CG) return __ldcg(p + i);
    else return p[i];
}

// Cell offsets within a level are 32-bit: tail and persistent-solve levels
// hold fewer than 2^31 cells (the size limits of fld_params bound them).

// sum_f w_f u_nbr and sum_f w_f of cell c
template <bool CG, class T>
__device__ __forceinline__ void tail_nbr_sums(const Dims& d, const Op<T>& A, int c, int i, int j, int k,
                                              const T* u, T& swu, T& sw) {
    const int sy = d.nx, sz = d.nx * d.ny;
    T a = T(0), s = T(0);
    {
        const T wl = A.wx[c];
        if (i > 0) { a += wl * ldw<CG>(u, c - 1); s += wl; }
        else if (d.px) { a += wl * ldw<CG>(u, c + d.nx - 1); s += wl; }
        if (i < d.nx - 1) { const T wu = A.wx[c + 1]; a += wu * ldw<CG>(u, c + 1); s += wu; }
        else if (d.px) { const int up = c - (d.nx - 1); const T wu = A.wx[up]; a += wu * ldw<CG>(u, up); s += wu; }
    }
    {
        const T wl = A.wy[c];
        if (j > 0) { a += wl * ldw<CG>(u, c - sy); s += wl; }
        else if (d.py) { a += wl * ldw<CG>(u, c + (d.ny - 1) * sy); s += wl; }
        if (j < d.ny - 1) { const T wu = A.wy[c + sy]; a += wu * ldw<CG>(u, c + sy); s += wu; }
        else if (d.py) { const int up = c - (d.ny - 1) * sy; const T wu = A.wy[up]; a += wu * ldw<CG>(u, up); s += wu; }
    }
    {
        const T wl = A.wz[c];
        if (k > 0) { a += wl * ldw<CG>(u, c - sz); s += wl; }
        else if (d.pz) { a += wl * ldw<CG>(u, c + (d.nz - 1) * sz); s += wl; }
        if (k < d.nz - 1) { const T wu = A.wz[c + sz]; a += wu * ldw<CG>(u, c + sz); s += wu; }
        else if (d.pz) { const int up = c - (d.nz - 1) * sz; const T wu = A.wz[up]; a += wu * ldw<CG>(u, up); s += wu; }
    }
    swu = a;
    sw = s;
}

// sum_f w_f u_nbr v_nbr (the red neighbours r * invd of a zero-guess sweep)
template <bool CG, class T>
__device__ __forceinline__ T tail_nbr_sum_prod(const Dims& d, const Op<T>& A, int c, int i, int j, int k,
                                               const T* u, const T* v) {
    const int sy = d.nx, sz = d.nx * d.ny;
    T a = T(0);
    if (i > 0) a += A.wx[c] * ldw<CG>(u, c - 1) * v[c - 1];
    else if (d.px) a += A.wx[c] * ldw<CG>(u, c + d.nx - 1) * v[c + d.nx - 1];
    if (i < d.nx - 1) a += A.wx[c + 1] * ldw<CG>(u, c + 1) * v[c + 1];
    else if (d.px) { const int up = c - (d.nx - 1); a += A.wx[up] * ldw<CG>(u, up) * v[up]; }
    if (j > 0) a += A.wy[c] * ldw<CG>(u, c - sy) * v[c - sy];
    else if (d.py) { const int lo = c + (d.ny - 1) * sy; a += A.wy[c] * ldw<CG>(u, lo) * v[lo]; }
    if (j < d.ny - 1) a += A.wy[c + sy] * ldw<CG>(u, c + sy) * v[c + sy];
    else if (d.py) { const int up = c - (d.ny - 1) * sy; a += A.wy[up] * ldw<CG>(u, up) * v[up]; }
    if (k > 0) a += A.wz[c] * ldw<CG>(u, c - sz) * v[c - sz];
    else if (d.pz) { const int lo = c + (d.nz - 1) * sz; a += A.wz[c] * ldw<CG>(u, lo) * v[lo]; }
    if (k < d.nz - 1) a += A.wz[c + sz] * ldw<CG>(u, c + sz) * v[c + sz];
    else if (d.pz) { const int up = c - (d.nz - 1) * sz; a += A.wz[up] * ldw<CG>(u, up) * v[up]; }
    return a;
}

// Cell coordinates by 32-bit unsigned division.
__device__ __forceinline__ void tail_ijk(int c, const Dims& d, int& i, int& j, int& k) {
    const unsigned cu = (unsigned)c, nx = (unsigned)d.nx, nxy = (unsigned)d.nx * (unsigned)d.ny;
    const unsigned kk = cu / nxy;
    const unsigned rem = cu - kk * nxy;
    const unsigned jj = rem / nx;
    k = (int)kk;
    j = (int)jj;
    i = (int)(rem - jj * nx);
}

// A thread's strided walk c = c0, c0 + s, ... over a level's cells with the
// coordinates kept incrementally: the stride is split once into (di, dj, dk)
// in the level's mixed radix, so a step costs a few adds and compares
// instead of two divisions (i + di < 2 nx and j + dj + 1 < 2 ny, so one
// carry each suffices).
struct Walk {
    int c, s, n;
    int i, j, k, di, dj, dk, nx, ny;
    __device__ __forceinline__ Walk(const Dims& d, int c0, int stride)
        : c(c0), s(stride), n((int)d.n), nx(d.nx), ny(d.ny) {
        tail_ijk(c0 < n ? c0 : 0, d, i, j, k);
        const unsigned su = (unsigned)stride, nxu = (unsigned)d.nx, nyu = (unsigned)d.ny;
        const unsigned t = su / nxu;
        di = (int)(su - t * nxu);
        dk = (int)(t / nyu);
        dj = (int)(t - (unsigned)dk * nyu);
    }
    __device__ __forceinline__ bool more() const { return c < n; }
    __device__ __forceinline__ void next() {
        c += s;
        i += di;
        if (i >= nx) { i -= nx; j++; }
        j += dj;
        if (j >= ny) { j -= ny; k++; }
        k += dk;
    }
};

// The same walk over the cells of one colour, (i + j + k) % 2 == col, of a
// level with an even x extent: half-index h over the n / 2 cells of that
// colour, x position 2 t + ((col + j + k) & 1), so no lane of a warp idles
// on a cell of the other colour.
struct WalkC {
    int h, s, n2;
    int t, j, k, dt, dj, dk, nx2, ny, nx, col;
    __device__ __forceinline__ WalkC(const Dims& d, int colour, int h0, int stride)
        : h(h0), s(stride), n2((int)(d.n >> 1)), nx2(d.nx >> 1), ny(d.ny), nx(d.nx), col(colour) {
        const unsigned hu = (unsigned)(h0 < n2 ? h0 : 0), n2x = (unsigned)nx2, nyu = (unsigned)d.ny;
        const unsigned r = hu / n2x;
        t = (int)(hu - r * n2x);
        k = (int)(r / nyu);
        j = (int)(r - (unsigned)k * nyu);
        const unsigned su = (unsigned)stride;
        const unsigned q = su / n2x;
        dt = (int)(su - q * n2x);
        dk = (int)(q / nyu);
        dj = (int)(q - (unsigned)dk * nyu);
    }
    __device__ __forceinline__ bool more() const { return h < n2; }
    __device__ __forceinline__ int i() const { return 2 * t + ((col + j + k) & 1); }
    __device__ __forceinline__ int c() const { return i() + nx * (j + ny * k); }
    __device__ __forceinline__ void next() {
        h += s;
        t += dt;
        if (t >= nx2) { t -= nx2; j++; }
        j += dj;
        if (j >= ny) { j -= ny; k++; }
        k += dk;
    }
};

// f(c, i, j, k) for every cell of colour col in this thread's share: the
// colour walk where nx is even, else the plain walk with the other colour
// skipped.  The cells are independent, so the order does not matter.
template <class F>
__device__ __forceinline__ void for_colour(const Dims& d, int col, int tid, int nth, F f) {
    if ((d.nx & 1) == 0) {
        for (WalkC w(d, col, tid, nth); w.more(); w.next()) f(w.c(), w.i(), w.j, w.k);
    } else {
        for (Walk w(d, tid, nth); w.more(); w.next())
            if (((w.i + w.j + w.k) & 1) == col) f(w.c, w.i, w.j, w.k);
    }
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
#define TAIL_LOOP(c, n) for (int c = tid; c < (int)(n); c += nth)

// Down-leg phases of level L into the coarse right-hand side rc:
// smoothing from zero (and further pre-sweeps), t = r - A z, rc = R t.
template <bool CG, class T, class Sync>
__device__ void tail_down(const TailLevel<T>& L, Vec<T> v, const Dims& cd, T* rc, int pre, int tid, int nth,
                          Sync sync) {
    const Dims& d = L.d;
    const Op<T>& A = L.A;
    const T* r = v.r;
    T* z = v.z;
    if (pre >= 1) {
        // red cells r / diag, black cells from the red ones' r / diag (the
        // two colours independent, so in one phase)
        for_colour(d, 0, tid, nth, [&](int c, int, int, int) { z[c] = ldw<CG>(r, c) * A.invd[c]; });
        for_colour(d, 1, tid, nth, [&](int c, int i, int j, int k) {
            z[c] = A.invd[c] * (ldw<CG>(r, c) + tail_nbr_sum_prod<CG, T>(d, A, c, i, j, k, r, A.invd));
        });
        sync();
        for (int it = 1; it < pre; it++)
            for (int colour = 0; colour < 2; colour++) {
                for_colour(d, colour, tid, nth, [&](int c, int i, int j, int k) {
                    T swu, sw;
                    tail_nbr_sums<CG, T>(d, A, c, i, j, k, z, swu, sw);
                    z[c] = A.invd[c] * (ldw<CG>(r, c) + swu);
                });
                sync();
            }
    } else {
        TAIL_LOOP(c, d.n) z[c] = T(0);
        sync();
    }
    for (Walk w(d, tid, nth); w.more(); w.next()) {
        const int c = w.c;
        T swu, sw;
        tail_nbr_sums<CG, T>(d, A, c, w.i, w.j, w.k, z, swu, sw);
        const T zc = ldw<CG>((const T*)z, c);
        v.t[c] = ldw<CG>(r, c) - (A.m[c] * zc + sw * zc - swu);
    }
    sync();
    const T wt[4] = {T(0.25), T(0.75), T(0.75), T(0.25)};
    for (Walk w(cd, tid, nth); w.more(); w.next()) {
        int fi[4], fj[4], fk[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
            fi[t] = tail_fine_tap(w.i, t, d.nx, d.px);
            fj[t] = tail_fine_tap(w.j, t, d.ny, d.py);
            fk[t] = tail_fine_tap(w.k, t, d.nz, d.pz);
        }
        T acc = T(0);
#pragma unroll
        for (int tk = 0; tk < 4; tk++) {
            T acc_j = T(0);
#pragma unroll
            for (int tj = 0; tj < 4; tj++) {
                const int row = d.nx * (fj[tj] + d.ny * fk[tk]);
                T acc_i = T(0);
#pragma unroll
                for (int ti = 0; ti < 4; ti++) acc_i += wt[ti] * ldw<CG>((const T*)v.t, row + fi[ti]);
                acc_j += wt[tj] * acc_i;
            }
            acc += wt[tk] * acc_j;
        }
        rc[w.c] = acc * T(0.125);
    }
    sync();
}

// Up-leg phases of level L: z += P zc, then the post-sweeps.
template <bool CG, class T, class Sync>
__device__ void tail_up(const TailLevel<T>& L, Vec<T> v, const Dims& cd, const T* zc, int post, int first, int tid,
                        int nth, Sync sync) {
    const Dims& d = L.d;
    const Op<T>& A = L.A;
    T* z = v.z;
    const T w2[2] = {T(0.75), T(0.25)};
    for (Walk w(d, tid, nth); w.more(); w.next()) {
        const int c = w.c;
        int Ix[2], Iy[2], Iz[2];
        tail_coarse_pair(w.i, cd.nx, cd.px, Ix[0], Ix[1]);
        tail_coarse_pair(w.j, cd.ny, cd.py, Iy[0], Iy[1]);
        tail_coarse_pair(w.k, cd.nz, cd.pz, Iz[0], Iz[1]);
        T acc = T(0);
#pragma unroll
        for (int b = 0; b < 2; b++) {
            T acc_j = T(0);
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const int row = cd.nx * (Iy[q] + cd.ny * Iz[b]);
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
            for_colour(d, colour, tid, nth, [&](int c, int i, int j, int k) {
                T swu, sw;
                tail_nbr_sums<CG, T>(d, A, c, i, j, k, z, swu, sw);
                z[c] = A.invd[c] * (ldw<CG>((const T*)v.r, c) + swu);
            });
            sync();
        }
}

// z = A^-1 r on the coarsest grid with the stored explicit inverse.
template <bool CG, class T, class Sync>
__device__ void tail_coarsest(int n, const double* ainv, Vec<T> v, int tid, int nth, Sync sync) {
    TAIL_LOOP(row, n) {
        double acc = 0.0;
        for (int q = 0; q < n; q++) acc += ainv[q * n + row] * (double)ldw<CG>((const T*)v.r, q);
        v.z[row] = (T)acc;
    }
    sync();
}

#undef TAIL_LOOP

// One V-cycle from the tail's first level down and back up, run by every
// thread of the calling cluster (smem: the dynamic shared memory of the
// small levels); it ends with a cluster barrier, so L[0].z is complete and
// visible to the whole cluster on return.
template <class T>
__device__ __forceinline__ void tail_cycle(const TailArgs<T>& a, cg::cluster_group& cl, unsigned char* smem) {
    const int gthreads = TAIL_THREADS * (int)cl.num_blocks();
    const int gtid = (int)cl.block_rank() * TAIL_THREADS + (int)threadIdx.x;
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
            const int tid = threadIdx.x, nth = TAIL_THREADS;
            Vec<T> sv[TAIL_MAX_LEVELS];
            T* base = reinterpret_cast<T*>(smem);
            for (int l = ls; l < nl; l++) {
                const long long n = a.L[l].d.n;
                sv[l] = Vec<T>{base, base + n, base + 2 * n};
                base += 3 * n;
            }
            for (int c = tid; c < (int)a.L[ls].d.n; c += nth) sv[ls].r[c] = __ldcg(a.L[ls].r + c);
            __syncthreads();
            for (int l = ls; l < nl - 1; l++)
                tail_down<false, T>(a.L[l], sv[l], a.L[l + 1].d, sv[l + 1].r, a.pre, tid, nth, bsync);
            tail_coarsest<false, T>((int)a.L[nl - 1].d.n, a.ainv, sv[nl - 1], tid, nth, bsync);
            for (int l = nl - 2; l >= ls; l--)
                tail_up<false, T>(a.L[l], sv[l], a.L[l + 1].d, sv[l + 1].z, a.post, a.paper_order ? 0 : 1, tid, nth,
                                  bsync);
            for (int c = tid; c < (int)a.L[ls].d.n; c += nth) a.L[ls].z[c] = sv[ls].z[c];
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

template <class T>
__global__ void __launch_bounds__(TAIL_THREADS) k_vtail(TailArgs<T> a) {
    extern __shared__ __align__(16) unsigned char tail_smem[];
    cg::cluster_group cl = cg::this_cluster();
    tail_cycle<T>(a, cl, tail_smem);
}

// ---------------------------------------------------------------------------
// Persistent inner solves over a work list (mixed precision).
//
// Each cluster takes a ticket, solves that request's FP32 system A x = r by
// MG-preconditioned CG (Table 1's solver: the V-cycle over all of the
// request's levels, then the CG vector operations) to its threshold or
// iteration cap, and takes the next ticket; the requests may have any grid
// sizes.  Phases are separated by the hardware cluster barrier and the dot
// products are summed in a fixed order (per thread in its cell order with
// error-free FP32 products, per CTA by warps, then the CTAs' partials in
// rank order, read by every CTA from distributed shared memory), so every
// CTA computes the same scalars and a request's result depends only on the
// cluster shape, never on the other requests or on which cluster took it.

// Sum of v over the cluster, the same in every thread of every CTA.  part:
// a __shared__ slot of this CTA, not written again before the next cluster
// barrier that follows this call.
__device__ __forceinline__ double ps_cluster_sum(double v, double* part, cg::cluster_group& cl) {
    __shared__ double wsum[TAIL_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = wsum[lane];
        t = warp_sum(t);
        if (lane == 0) *part = t;
    }
    cl.sync();
    double tot = 0.0;
    const unsigned nb = cl.num_blocks();
    for (unsigned b = 0; b < nb; b++) tot += *cl.map_shared_rank(part, b);
    return tot;
}

// The inner solve of one request: r holds the scaled residual, x = 0.
__device__ void ps_solve(const PsReq& R, cg::cluster_group& cl, unsigned char* smem, double* part) {
    const TailArgs<float>& a = R.v;
    const Dims& d = a.L[0].d;
    const Op<float>& A = a.L[0].A;
    float* r = a.L[0].r;
    float* z = a.L[0].z;
    float* p = R.p;
    float* q = R.q;
    float* x = R.x;
    const int nth = TAIL_THREADS * (int)cl.num_blocks();
    const int tid = (int)cl.block_rank() * TAIL_THREADS + (int)threadIdx.x;
    const int n = (int)d.n;
    const double thresh = __ldcg(R.sc + S_THRESH);
    const int maxit = (int)__ldcg(R.sc + S_MAXIT);
    double rho = 0.0, rho_old = 0.0, beta = 0.0, pq = 0.0, alpha = 0.0, rr = __ldcg(R.sc + S_RR);
    int k = 0, slot = 0;
    bool bad = false;
    while (k < maxit) {
        tail_cycle<float>(a, cl, smem);   // z = M r
        DotAcc<float> arz;
        for (int c = tid; c < n; c += nth) arz.add(__ldcg(r + c), __ldcg(z + c));
        rho = ps_cluster_sum(arz.value(), part + slot, cl);
        slot = (slot + 1) & 3;
        beta = k == 0 ? 0.0 : rho / rho_old;
        rho_old = rho;
        const float bf = (float)beta;
        if (k == 0)
            for (int c = tid; c < n; c += nth) p[c] = __ldcg(z + c);
        else
            for (int c = tid; c < n; c += nth) p[c] = fmaf(bf, __ldcg(p + c), __ldcg(z + c));
        cl.sync();
        // q = A p and <p, q>
        DotAcc<float> apq;
        for (Walk w(d, tid, nth); w.more(); w.next()) {
            const int c = w.c;
            float swu, sw;
            tail_nbr_sums<true, float>(d, A, c, w.i, w.j, w.k, p, swu, sw);
            const float pc = __ldcg(p + c);
            const float qc = A.m[c] * pc + sw * pc - swu;
            q[c] = qc;
            apq.add(pc, qc);
        }
        pq = ps_cluster_sum(apq.value(), part + slot, cl);
        slot = (slot + 1) & 3;
        alpha = rho / pq;
        const float af = (float)alpha;
        // x += alpha p, r -= alpha q, ||r||^2
        DotAcc<float> arr;
        for (int c = tid; c < n; c += nth) {
            // x starts at 0 (the caller's x32 is not cleared)
            x[c] = k == 0 ? af * __ldcg(p + c) : fmaf(af, __ldcg(p + c), __ldcg(x + c));
            const float rn = fmaf(-af, __ldcg(q + c), __ldcg(r + c));
            r[c] = rn;
            arr.add(rn, rn);
        }
        rr = ps_cluster_sum(arr.value(), part + slot, cl);
        slot = (slot + 1) & 3;
        k++;
        if (!isfinite(rho) || !isfinite(alpha) || !isfinite(rr)) {
            bad = true;
            break;
        }
        if (rr <= thresh) break;
    }
    if (cl.block_rank() == 0 && threadIdx.x == 0) {
        double* sc = R.sc;
        sc[S_RHO] = rho;
        sc[S_RHO_OLD] = rho_old;
        sc[S_BETA] = beta;
        sc[S_PQ] = pq;
        sc[S_ALPHA] = alpha;
        sc[S_RR] = rr;
        sc[S_KITER] = (double)k;
        sc[S_FIRST] = 0.0;
        if (bad) sc[S_NONFINITE] = 1.0;
    }
}

// Sum of v over the CTA, the same in every thread (fixed order).
__device__ __forceinline__ double ps_block_sum(double v) {
    __shared__ double wsum[TAIL_THREADS / 32];
    __shared__ double tot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = wsum[lane];
        t = warp_sum(t);
        if (lane == 0) tot = t;
    }
    __syncthreads();
    const double out = tot;
    __syncthreads();
    return out;
}

// The inner solve of a small request by one CTA: the vectors of every
// level and the CG vectors live in shared memory (block barriers between
// the phases, no L2 round trip); the operator comes from global memory
// (read-only here, so cached in L1).  r is read from and x written back to
// the request's global vectors.
__device__ void ps_solve_cta(const PsReq& R, unsigned char* smem) {
    const TailArgs<float>& a = R.v;
    const int nl = a.nlev;
    const int tid = threadIdx.x, nth = TAIL_THREADS;
    auto bsync = []() { __syncthreads(); };
    Vec<float> sv[TAIL_MAX_LEVELS];
    float* base = reinterpret_cast<float*>(smem);
    for (int l = 0; l < nl; l++) {
        const long long n = a.L[l].d.n;
        sv[l] = Vec<float>{base, base + n, base + 2 * n};
        base += 3 * n;
    }
    const Dims& d = a.L[0].d;
    const Op<float>& A = a.L[0].A;
    const int n0 = (int)d.n;
    float* r = sv[0].r;
    float* z = sv[0].z;
    float* p = base;
    float* q = base + n0;
    float* x = base + 2 * n0;
    for (int c = tid; c < n0; c += nth) {
        r[c] = __ldcg(a.L[0].r + c);
        x[c] = 0.0f;
    }
    __syncthreads();
    const double thresh = __ldcg(R.sc + S_THRESH);
    const int maxit = (int)__ldcg(R.sc + S_MAXIT);
    double rho = 0.0, rho_old = 0.0, beta = 0.0, pq = 0.0, alpha = 0.0, rr = __ldcg(R.sc + S_RR);
    int k = 0;
    bool bad = false;
    while (k < maxit) {
        // z = M r: the V-cycle over every level in shared memory
        for (int l = 0; l < nl - 1; l++)
            tail_down<false, float>(a.L[l], sv[l], a.L[l + 1].d, sv[l + 1].r, a.pre, tid, nth, bsync);
        tail_coarsest<false, float>((int)a.L[nl - 1].d.n, a.ainv, sv[nl - 1], tid, nth, bsync);
        for (int l = nl - 2; l >= 0; l--)
            tail_up<false, float>(a.L[l], sv[l], a.L[l + 1].d, sv[l + 1].z, a.post, a.paper_order ? 0 : 1, tid, nth,
                                  bsync);
        DotAcc<float> arz;
        for (int c = tid; c < n0; c += nth) arz.add(r[c], z[c]);
        rho = ps_block_sum(arz.value());
        beta = k == 0 ? 0.0 : rho / rho_old;
        rho_old = rho;
        const float bf = (float)beta;
        if (k == 0)
            for (int c = tid; c < n0; c += nth) p[c] = z[c];
        else
            for (int c = tid; c < n0; c += nth) p[c] = fmaf(bf, p[c], z[c]);
        __syncthreads();
        DotAcc<float> apq;
        for (Walk w(d, tid, nth); w.more(); w.next()) {
            const int c = w.c;
            float swu, sw;
            tail_nbr_sums<false, float>(d, A, c, w.i, w.j, w.k, p, swu, sw);
            const float pc = p[c];
            const float qc = A.m[c] * pc + sw * pc - swu;
            q[c] = qc;
            apq.add(pc, qc);
        }
        pq = ps_block_sum(apq.value());
        alpha = rho / pq;
        const float af = (float)alpha;
        DotAcc<float> arr;
        for (int c = tid; c < n0; c += nth) {
            x[c] = fmaf(af, p[c], x[c]);
            const float rn = fmaf(-af, q[c], r[c]);
            r[c] = rn;
            arr.add(rn, rn);
        }
        rr = ps_block_sum(arr.value());
        k++;
        if (!isfinite(rho) || !isfinite(alpha) || !isfinite(rr)) {
            bad = true;
            break;
        }
        if (rr <= thresh) break;
    }
    for (int c = tid; c < n0; c += nth) R.x[c] = x[c];
    if (threadIdx.x == 0) {
        double* sc = R.sc;
        sc[S_RHO] = rho;
        sc[S_RHO_OLD] = rho_old;
        sc[S_BETA] = beta;
        sc[S_PQ] = pq;
        sc[S_ALPHA] = alpha;
        sc[S_RR] = rr;
        sc[S_KITER] = (double)k;
        sc[S_FIRST] = 0.0;
        if (bad) sc[S_NONFINITE] = 1.0;
    }
}

__global__ void __launch_bounds__(TAIL_THREADS) k_psolve(const __grid_constant__ PsBatch b) {
    extern __shared__ __align__(16) unsigned char ps_smem[];
    __shared__ __align__(16) PsReq R;
    __shared__ double part[4];
    __shared__ int item;
    cg::cluster_group cl = cg::this_cluster();
    for (;;) {
        if (cl.block_rank() == 0 && threadIdx.x == 0) item = (int)atomicAdd(b.ticket, 1u);
        cl.sync();
        const int it = *cl.map_shared_rank(&item, 0);
        // every CTA has read the ticket before CTA 0 may draw the next one
        // or exit (its shared memory must outlive the remote reads)
        cl.sync();
        if (it >= b.ncl) break;
        const unsigned* src = reinterpret_cast<const unsigned*>(b.req[it]);
        unsigned* dst = reinterpret_cast<unsigned*>(&R);
        for (int w = threadIdx.x; w < (int)(sizeof(PsReq) / 4); w += TAIL_THREADS) dst[w] = __ldcg(src + w);
        __syncthreads();
        ps_solve(R, cl, ps_smem, part);
        // the last reduction's remote reads are done before the next request
        cl.sync();
    }
    // then the small requests, each CTA on its own (no remote accesses
    // follow, so the CTAs may finish independently)
    for (;;) {
        if (threadIdx.x == 0) item = b.ncl + (int)atomicAdd(b.ticket + 1, 1u);
        __syncthreads();
        const int it = item;
        __syncthreads();
        if (it >= b.n) break;
        const unsigned* src = reinterpret_cast<const unsigned*>(b.req[it]);
        unsigned* dst = reinterpret_cast<unsigned*>(&R);
        for (int w = threadIdx.x; w < (int)(sizeof(PsReq) / 4); w += TAIL_THREADS) dst[w] = __ldcg(src + w);
        __syncthreads();
        ps_solve_cta(R, ps_smem);
        __syncthreads();
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

size_t psolve_cta_bytes(const TailArgs<float>& v) {
    size_t cells = 0;
    for (int l = 0; l < v.nlev; l++) cells += (size_t)v.L[l].d.n;
    return (3 * cells + 3 * (size_t)v.L[0].d.n) * sizeof(float);
}

size_t psolve_smem_bytes(const PsReq& r) { return r.cta ? psolve_cta_bytes(r.v) : vtail_smem_bytes(r.v); }

// Cluster size of the persistent solves (fixed per device, so a request's
// arithmetic never depends on the launch that carries it) and how many such
// clusters can be resident at once; {0, 0} if none fits.
PsShape psolve_shape() {
    static thread_local int dev = -1;
    static thread_local PsShape shape{0, 0};
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) {
        cudaGetLastError();
        return PsShape{0, 0};
    }
    if (d == dev) return shape;
    dev = d;
    shape = PsShape{0, 0};
    if (cudaFuncSetAttribute(k_psolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PS_SMEM_MAX) !=
        cudaSuccess)
        cudaGetLastError();
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = tail_config(PS_CLUSTER, nullptr, attr);
    cfg.dynamicSmemBytes = PS_SMEM_MAX;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_psolve, &cfg) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    if (n > 0) shape = PsShape{PS_CLUSTER, n};
    return shape;
}

cudaError_t launch_psolve(const PsBatch& b, size_t smem, cudaStream_t s) {
    const PsShape sh = psolve_shape();
    if (sh.cluster == 0) return cudaErrorNotSupported;
    if (b.n < 1) return cudaSuccess;
    // enough clusters for the cluster requests and for one CTA per small one
    const int ncta = b.n - b.ncl;
    int clusters = b.ncl > (ncta + sh.cluster - 1) / sh.cluster ? b.ncl : (ncta + sh.cluster - 1) / sh.cluster;
    if (clusters > sh.clusters) clusters = sh.clusters;
    cudaError_t e = cudaMemsetAsync(b.ticket, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = tail_config(sh.cluster, s, attr);
    cfg.gridDim = dim3(sh.cluster * clusters, 1, 1);
    cfg.dynamicSmemBytes = smem;
    return cudaLaunchKernelEx(&cfg, k_psolve, b);
}

template cudaError_t launch_vtail<float>(const TailArgs<float>&, int, cudaStream_t);
template cudaError_t launch_vtail<double>(const TailArgs<double>&, int, cudaStream_t);
template int vtail_cluster<float>();
template int vtail_cluster<double>();

}  // namespace fld
