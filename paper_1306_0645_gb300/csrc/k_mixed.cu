// k_mixed.cu -- the FP64-accurate kernels of the mixed-precision step,
// computed on the FP32 pipe in double-float arithmetic (df.cuh):
//
//   * assembly (Sec. 2 limiter, Sec. 3.2 theta-method system): the mass term
//     m and the face weights w stored as a pair of floats (the FP32 operator
//     of the V-cycles is the high part), and the right-hand side
//     b = dt eta - dt (c kappa + adot/a) E + sum_f (w_f / theta)(E_nbr - E);
//   * the refinement update x += 2^ks x32 and the residual
//     r = b - m x - sum_f w_f (x - x_nbr), written as the FP32 right-hand
//     side of the next inner solve, scaled by a power of two, with its norms;
//   * the finalisation E^{n+1} = max(E^n + x, 0) with the sums of the photon
//     balance.
//
// E, n_HI, eta and b stay FP64 in memory; their values enter the df
// arithmetic through integer conversions (split64) relative to a
// power-of-two scale 2^K, where K bounds the step's E and dt eta from above
// (the faces kernel reduces their maxima into slots).  The refinement
// unknown x = dE is kept as a df pair scaled by 2^-K.  The flux through a
// face is written with the difference of the two values formed before any
// rounding that could cancel (an FP64 subtraction for E, an error-free df
// subtraction for x), so the right-hand side and the residual keep their
// accuracy where neighbouring values nearly cancel: the residual's error is
// of order 2^-47 (|b| + m |x| + sum_f w_f |x - x_nbr|), and the refinement
// converges as an FP64 one would.
//
// On levels whose x extent is a multiple of 4 the right-hand side, the
// refinement residual and the update run four cells per thread (walk4.cuh),
// with the same operations per cell as the one-cell kernels; the right-hand
// side also writes the bfloat16 copies of the V-cycle's smoothing
// coefficients where the context keeps them.
#include "limiter.cuh"
#include "walk4.cuh"
#include <cuda_bf16.h>

namespace fld {

namespace {

// The high word of v without its sign bit.  Taken as a 32-bit word first:
// clearing the sign of the 64-bit pattern is compiled as an FP64 absolute
// value, an instruction of the FP64 pipe.
__device__ __forceinline__ unsigned hiword(double v) { return (unsigned)__double2hiint(v) & 0x7FFFFFFFu; }

// The bfloat16 nearest to v, as its 16 bits.
__device__ __forceinline__ unsigned short bf16_bits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
// Four of them packed in storage order.
__device__ __forceinline__ uint2 bf16_pack4(float a, float b, float c, float d) {
    return make_uint2((unsigned)bf16_bits(a) | ((unsigned)bf16_bits(b) << 16),
                      (unsigned)bf16_bits(c) | ((unsigned)bf16_bits(d) << 16));
}

// L2 prefetch of the line holding p (a streamed array's element one or more
// planes ahead): its bytes are requested from HBM without holding a
// register or a scoreboard entry, so the walk's loads of that plane hit L2.
template <class T>
__device__ __forceinline__ void pfl2(const T* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(p)));
}

// planes ahead that the z-walks prefetch (measured at 512^3: 0, 1 and 2
// planes gave 4.9, 3.96 and 3.82 ms per step for the two residuals)
constexpr int PF_PLANES = 2;

// The step's scale exponent: 2^K >= max E and >= dt max eta (the slots
// hold the maxima the faces kernel reduced).
__device__ __forceinline__ int step_scale(const double* sc, int dt_exp) {
    const int ke = exp_above(sc[S_EMAX]);
    const int kq = exp_above(sc[S_ETAMAX]) + dt_exp + 1;
    const int K = ke > kq ? ke : kq;
    return K < -1000 ? 0 : K;
}

// v * 2^e for a float v and any integer e, by two exact power-of-two
// products (each factor within the FP32 range); underflow rounds to a
// subnormal or 0 as IEEE multiplication does.
__device__ __forceinline__ float ldexp2(float v, int e) {
    e = e > 250 ? 250 : (e < -250 ? -250 : e);
    const int e1 = e / 2, e2 = e - e1;
    return __fmul_rn(__fmul_rn(v, __uint_as_float((unsigned)(127 + e1) << 23)),
                     __uint_as_float((unsigned)(127 + e2) << 23));
}

// FP64 value to df with a round-to-nearest high part (FP64 instructions;
// only the faces whose limiter leaves the df range take this).
__device__ __forceinline__ df d2df_rn(double v) {
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}

// Sec. 2 limiter in df for the face between cells 1 and 2 (energies E1, E2,
// neutral densities n1, n2) along axis a, as its theta-scaled weight
// w = theta dt D / h^2.  With t = n sigma h (optical depths), P = 2 t1 t2,
// K = t1 + t2 (kappa_f h = P / K; P = 0, K = 1 if either t is 0),
// S = E1 + E2 and A = max(2 |E2 - E1|, R_min h S) (R h = A / S):
//     w = theta dt c / h * K S / sqrt(9 P^2 S^2 + A^2 K^2),  capped at wmax.
// E1 and E2 enter relative to the larger one's exponent, so the ratio is
// scale free; their difference is formed in FP64.  Returns false where a
// value leaves the FP32 range.
__device__ bool limiter_paper_df(double E1, double E2, double n1, double n2, int a, const PhysDev& p, df& w) {
    const unsigned h1 = hiword(E1), h2 = hiword(E2);
    const int emax = (int)((h1 > h2 ? h1 : h2) >> 20);
    df S, A;
    if (emax == 0) {
        // both energies zero: R = R_min
        S = {1.0f, 0.0f};
        A = p.rminh[a];
    } else {
        const int K = emax - 1023;
        S = df_add(split64(E1, K), split64(E2, K));
        // |E2 - E1|: split64 truncates toward zero, so both parts carry the sign
        const df dd = split64(E2 - E1, K);
        A = {2.0f * fabsf(dd.h), 2.0f * fabsf(dd.l)};
        const df amin = df_mul(p.rminh[a], S);
        if (df_lt(A, amin)) A = amin;
    }
    const df t1 = df_mul(split64(n1, 0), p.sigh[a]);
    const df t2 = df_mul(split64(n2, 0), p.sigh[a]);
    const bool nz1 = (hiword(n1) | (unsigned)__double2loint(n1)) != 0u;
    const bool nz2 = (hiword(n2) | (unsigned)__double2loint(n2)) != 0u;
    if ((nz1 && t1.h == 0.0f) || (nz2 && t2.h == 0.0f)) return false;
    df P = {0.0f, 0.0f}, Kk = {1.0f, 0.0f};
    if (t1.h > 0.0f && t2.h > 0.0f) {
        P = df_mul(t1, t2);
        P.h *= 2.0f;
        P.l *= 2.0f;
        Kk = df_add(t1, t2);
    }
    const df PS = df_mul(P, S), AK = df_mul(A, Kk);
    const df X = df_add(df_mul_f(df_mul(PS, PS), 9.0f), df_mul(AK, AK));
    if (!(X.h >= 0x1p-120f && X.h <= 0x1p120f)) return false;
    df r = df_mul(df_mul(p.cw[a], df_mul(Kk, S)), df_rsqrt(X));
    if (!(r.h < 0x1p126f)) return false;
    if (!df_lt(r, p.wmaxd[a])) r = p.wmaxd[a];
    w = r;
    return true;
}

// Weight of the face between cells 1 (lower) and 2 along axis a: the df
// limiter, or the FP64 one (the Levermore-Pomraning form, and the paper's
// form outside the df range).
__device__ __forceinline__ df face_w_mx(double E1, double E2, double n1, double n2, int a, const PhysDev& p) {
    if (p.limiter == 0 && p.df_limiter) {
        df w;
        if (limiter_paper_df(E1, E2, n1, n2, a, p, w)) return w;
    }
    const double D = face_D(E1, E2, n1 * p.sigma, n2 * p.sigma, p.h[a], p);
    return d2df_rn(p.dt_h2[a] * D);
}

// A field as the flux walk reads it: an FP64 array (E) whose differences
// are formed in FP64 and split at scale 2^K ...
struct F64Field {
    const double* u;
    int K;
    using V = double;
    __device__ __forceinline__ V at(long long c) const { return u[c]; }
    __device__ __forceinline__ df diff(V nb, V uc) const { return split64(nb - uc, K); }
};
// ... or a df array (the refinement unknown), differences error-free in df.
struct DFField {
    const float2* u;
    using V = df;
    __device__ __forceinline__ V at(long long c) const {
        const float2 v = u[c];
        return {v.x, v.y};
    }
    __device__ __forceinline__ df diff(V nb, V uc) const { return df_sub(nb, uc); }
};

// Sum over the faces of cell c of w_f (u_nbr - u_c) (w the theta-scaled df
// weights), accumulated into F, for a thread walking z with its x
// neighbour in the next lane.  The flux through a face is formed once: the
// x-upper face's comes from the next lane (its x-lower face) where that
// lane holds the next cell of the row, the z-lower face's is the previous
// plane's z-upper face (carried in fz; valid when have_z).  wsum32 gets the
// FP32 weights of the faces in the order x lo, x hi, y lo, y hi, z lo,
// z hi (the FP32 diagonal of the V-cycle).
template <class Field>
struct FluxWalk {
    Dims d;
    Op<float> A, L;
    Field u;
    unsigned wmask;
    bool xnext;   // the next lane holds cell (i + 1, j, k)

    // w (u_nbr - u_c) through the face with weight index wi of axis a
    __device__ __forceinline__ df face(int a, long long wi, long long nb, typename Field::V uc) const {
        const float* h = a == 0 ? A.wx : (a == 1 ? A.wy : A.wz);
        const float* l = a == 0 ? L.wx : (a == 1 ? L.wy : L.wz);
        return df_mul_raw({h[wi], l[wi]}, u.diff(u.at(nb), uc));
    }

    // inb: the thread's cell exists
    __device__ __forceinline__ void plane(bool inb, int i, int j, int k, long long c, typename Field::V uc,
                                          Acc2& F, float& wsum32, df& fz, bool& have_z) const {
        const long long sy = d.nx, sz = (long long)d.nx * d.ny;
        df fxl = {0.0f, 0.0f};
        float wxl = 0.0f;
        if (inb && (i > 0 || d.px)) {
            fxl = face(0, c, i > 0 ? c - 1 : c + d.nx - 1, uc);
            wxl = A.wx[c];
        }
        // the next lane's x-lower flux is this cell's x-upper flux, negated
        const float nh = __shfl_down_sync(wmask, fxl.h, 1);
        const float nl = __shfl_down_sync(wmask, fxl.l, 1);
        const float nw = __shfl_down_sync(wmask, wxl, 1);
        if (!inb) return;
        df fxu = {0.0f, 0.0f};
        float wxu = 0.0f;
        if (i < d.nx - 1) {
            if (xnext) {
                fxu = {-nh, -nl};
                wxu = nw;
            } else {
                fxu = face(0, c + 1, c + 1, uc);
                wxu = A.wx[c + 1];
            }
        } else if (d.px) {
            fxu = face(0, c - (d.nx - 1), c - (d.nx - 1), uc);
            wxu = A.wx[c - (d.nx - 1)];
        }
        df fyl = {0.0f, 0.0f}, fyu = {0.0f, 0.0f};
        float wyl = 0.0f, wyu = 0.0f;
        if (j > 0 || d.py) {
            fyl = face(1, c, j > 0 ? c - sy : c + (long long)(d.ny - 1) * sy, uc);
            wyl = A.wy[c];
        }
        if (j < d.ny - 1) {
            fyu = face(1, c + sy, c + sy, uc);
            wyu = A.wy[c + sy];
        } else if (d.py) {
            const long long o = c - (long long)(d.ny - 1) * sy;
            fyu = face(1, o, o, uc);
            wyu = A.wy[o];
        }
        df fzl = {0.0f, 0.0f};
        float wzl = 0.0f;
        if (k > 0 || d.pz) {
            wzl = A.wz[c];
            fzl = have_z ? fz : face(2, c, k > 0 ? c - sz : c + (long long)(d.nz - 1) * sz, uc);
        }
        df fzu = {0.0f, 0.0f};
        float wzu = 0.0f;
        if (k < d.nz - 1) {
            fzu = face(2, c + sz, c + sz, uc);
            wzu = A.wz[c + sz];
        } else if (d.pz) {
            const long long o = c - (long long)(d.nz - 1) * sz;
            fzu = face(2, o, o, uc);
            wzu = A.wz[o];
        }
        fz = df_neg(fzu);
        have_z = true;
        F.add(fxl);
        F.add(fxu);
        F.add(fyl);
        F.add(fyu);
        F.add(fzl);
        F.add(fzu);
        // the FP32 diagonal's weights in the FP32 operator's order
        if (i > 0 || d.px) wsum32 += wxl;
        if (i < d.nx - 1 || d.px) wsum32 += wxu;
        if (j > 0 || d.py) wsum32 += wyl;
        if (j < d.ny - 1 || d.py) wsum32 += wyu;
        if (k > 0 || d.pz) wsum32 += wzl;
        if (k < d.nz - 1 || d.pz) wsum32 += wzu;
    }
};

}  // namespace

// ---------------------------------------------------------------- assembly

// Pass 1 of the mixed assembly: mass term and face weights in df (high parts
// into A, low parts into L), the exact FP32 screen for capped faces, input
// validation, and the maxima of E, n_HI and eta (S_EMAX, S_NMAX, S_ETAMAX).
// A face the screen does not settle goes to the block's list for the
// compacted pass k_asm_fix_mx (whole warps on the df limiter); a block whose
// list is full computes the rest in place.
__global__ void __launch_bounds__(256, 4) k_asm_faces_mx(Dims d, PhysDev p, const double* __restrict__ E,
                                                     const double* __restrict__ nHI,
                                                     const double* __restrict__ eta, Op<float> A, Op<float> L,
                                                     double* sc, FaceList fl, int zb0, int kch) {
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    bool bad = false;
    unsigned mE = 0u, mN = 0u, mQ = 0u;
    const bool screen = p.limiter == 0;
    __shared__ unsigned s_cnt;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const long long bid = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * (zb0 + blockIdx.z));
    if (tid == 0) s_cnt = 0u;
    __syncthreads();
    unsigned* seg = fl.entries ? fl.entries + bid * fl.cap : nullptr;
    COL_BEGIN_ZB(d, zb0, kch)
        if (PF_PLANES > 0 && k + PF_PLANES < k1_) {
            const long long cp = c + PF_PLANES * sz;
            pfl2(E + cp);
            pfl2(nHI + cp);
            pfl2(eta + cp);
        }
        const double Ec = E[c], nc = nHI[c], qc = eta[c];
        bad |= !valid_bits(Ec) || !valid_bits(nc) || !valid_bits(qc);
        mE = max(mE, hiword(Ec));
        mN = max(mN, hiword(nc));
        mQ = max(mQ, hiword(qc));
        const df m = df_add(p.one_dta_d, df_mul(p.mdtcs_d, split64(nc, 0)));
        bool okc = true;
        const float kL32 = f32_trunc(nc, okc) * p.sigmaL32;
        df w[3];
        const int ijk[3] = {i, j, k};
        const int nn[3] = {d.nx, d.ny, d.nz};
        const int per[3] = {d.px, d.py, d.pz};
        const long long st[3] = {1, sy, sz};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            long long lo;
            if (ijk[a] > 0) lo = c - st[a];
            else if (per[a]) lo = c + (long long)(nn[a] - 1) * st[a];
            else { w[a] = {0.0f, 0.0f}; continue; }
            const double El = E[lo], nl = nHI[lo];
            bool ok = okc;
            float el32, e32;
            pair32(El, Ec, el32, e32, ok);
            const float kLl = f32_trunc(nl, ok) * p.sigmaL32;
            if (screen && ok && capped32(el32, e32, kLl, kL32, p.twoL_h32[a], p.thr32)) {
                w[a] = p.wmaxd[a];
                continue;
            }
            if (seg) {
                const unsigned pos = atomicAdd(&s_cnt, 1u);
                if (pos < (unsigned)fl.cap) {
                    seg[pos] = ((unsigned)c << 2) | (unsigned)a;
                    w[a] = {0.0f, 0.0f};
                    continue;
                }
            }
            w[a] = face_w_mx(El, Ec, nl, nc, a, p);
        }
        A.m[c] = m.h;
        L.m[c] = m.l;
        A.wx[c] = w[0].h;
        L.wx[c] = w[0].l;
        A.wy[c] = w[1].h;
        L.wy[c] = w[1].l;
        A.wz[c] = w[2].h;
        L.wz[c] = w[2].l;
    }
    if (bad) sc[S_BAD] = 1.0;
    // block maxima, one atomic per block and value
    __shared__ unsigned smax[3];
    if (tid < 3) smax[tid] = 0u;
    __syncthreads();
    const unsigned wm = __activemask();
    mE = __reduce_max_sync(wm, mE);
    mN = __reduce_max_sync(wm, mN);
    mQ = __reduce_max_sync(wm, mQ);
    if ((tid & 31) == 0) {
        atomicMax(&smax[0], mE);
        atomicMax(&smax[1], mN);
        atomicMax(&smax[2], mQ);
    }
    __syncthreads();
    if (tid < 3 && smax[tid] != 0u)
        atomicMax((unsigned long long*)&sc[S_EMAX + tid], (unsigned long long)smax[tid] << 32);
    if (tid == 0 && seg) fl.counts[bid] = s_cnt < (unsigned)fl.cap ? s_cnt : (unsigned)fl.cap;
}

// The faces pass 1 listed: the df limiter with whole warps busy.  Entry =
// (cell << 2) | axis; the face couples the cell with its lower neighbour
// along the axis (wrapping on a periodic axis).
__global__ void __launch_bounds__(256) k_asm_fix_mx(Dims d, PhysDev p, const double* __restrict__ E,
                                                   const double* __restrict__ nHI, Op<float> A, Op<float> L,
                                                   FaceList fl) {
    const unsigned cnt = fl.counts[blockIdx.x];
    const unsigned* seg = fl.entries + (long long)blockIdx.x * fl.cap;
    const unsigned nx = (unsigned)d.nx, ny = (unsigned)d.ny, nz = (unsigned)d.nz;
    const unsigned nxy = nx * ny;
    for (unsigned t = threadIdx.x; t < cnt; t += blockDim.x) {
        const unsigned e = seg[t];
        const unsigned cu = e >> 2;
        const int a = (int)(e & 3u);
        const long long c = cu;
        long long lo;
        if (a == 0) lo = (cu % nx) > 0 ? c - 1 : c + (nx - 1);
        else if (a == 1) lo = ((cu / nx) % ny) > 0 ? c - nx : c + (long long)(ny - 1) * nx;
        else lo = (cu / nxy) > 0 ? c - nxy : c + (long long)(nz - 1) * nxy;
        const df w = face_w_mx(E[lo], E[c], nHI[lo], nHI[c], a, p);
        float* Wh = a == 0 ? A.wx : (a == 1 ? A.wy : A.wz);
        float* Wl = a == 0 ? L.wx : (a == 1 ? L.wy : L.wz);
        Wh[c] = w.h;
        Wl[c] = w.l;
    }
}

// Pass 2 of the mixed assembly: right-hand side b (FP64), ||b||^2 and max|b|
// (reduction ra, R_STORE_SUM_MAX), the FP32 inverse diagonal of the V-cycle
// and, on Dirichlet faces (DIR), their weights (bnd, FP64) added to m.
// BE: theta = 1.  scg: the slots holding the maxima of pass 1.
template <bool BE, bool DIR>
__global__ void __launch_bounds__(256) k_asm_rhs_mx(Dims d, PhysDev p, const double* __restrict__ E,
                                                   const double* __restrict__ nHI,
                                                   const double* __restrict__ eta, Op<float> A, Op<float> L,
                                                   double* __restrict__ b, Bnd bnd, RedArgs ra, const double* scg,
                                                   int zb0, int kch, Op<unsigned short> Bf) {
    const int K = step_scale(scg, p.dt_exp);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = (zb0 + (int)blockIdx.z) * kch;
    const int k1 = min(d.nz, k0 + kch);
    const bool inb = i < d.nx && j < d.ny;
    const long long nxy = (long long)d.nx * d.ny;
    FluxWalk<F64Field> fw;
    fw.d = d;
    fw.A = A;
    fw.L = L;
    fw.u = F64Field{E, K};
    fw.wmask = __activemask();
    fw.xnext = threadIdx.x + 1 < blockDim.x;
    double bb = 0.0;
    float bmax = 0.0f;
    df fz = {0.0f, 0.0f};
    bool have_z = false;
    for (int k = k0; k < k1; k++) {
        const long long c = (long long)k * nxy + (long long)j * d.nx + i;
        if (PF_PLANES > 0 && inb && k + PF_PLANES < k1) {
            const long long cp = c + PF_PLANES * nxy;
            pfl2(E + cp);
            pfl2(nHI + cp);
            pfl2(eta + cp);
            pfl2(A.wx + cp);
            pfl2(L.wx + cp);
            pfl2(A.wy + cp);
            pfl2(L.wy + cp);
            pfl2(A.wz + cp);
            pfl2(L.wz + cp);
            pfl2(A.m + cp);
        }
        const double Ec = inb ? E[c] : 0.0;
        Acc2 F;
        float wsum32 = 0.0f;
        fw.plane(inb, i, j, k, c, Ec, F, wsum32, fz, have_z);
        if (!inb) continue;
        const double nc = nHI[c];
        Acc2 B;
        if (DIR) {
            // Dirichlet faces of the box touching this cell: E_b half a cell out
            const int ijk[3] = {i, j, k};
            const int nn[3] = {d.nx, d.ny, d.nz};
            const double kc = nc * p.sigma;
            df wb_sum = {0.0f, 0.0f};
            bool any = false;
#pragma unroll
            for (int sd = 0; sd < 6; sd++) {
                const int a = sd >> 1;
                if (!((p.dmask >> sd) & 1) || ijk[a] != ((sd & 1) ? nn[a] - 1 : 0)) continue;
                const double Eb = p.ebc[sd];
                const double wb = 2.0 * p.dt_h2[a] * face_D(Eb, Ec, kc, kc, 0.5 * p.h[a], p);
                const long long f = a == 0 ? j + (long long)d.ny * k
                                           : (a == 1 ? i + (long long)d.nx * k : i + (long long)d.nx * j);
                bnd.w[bnd_offset(d, sd) + f] = wb;
                const df wbd = d2df_rn(wb);
                F.add(df_mul_raw(wbd, split64(Eb - Ec, K)));
                wb_sum = df_add(wb_sum, wbd);
                any = true;
            }
            if (any) {
                const df m = df_add({A.m[c], L.m[c]}, wb_sum);
                A.m[c] = m.h;
                L.m[c] = m.l;
            }
        }
        // b = dt eta - dt (c sigma n_HI + adot/a) E + flux / theta
        B.add(df_mul_raw(split64(eta[c], K - p.dt_exp), p.dtm_d));
        const df loss = df_add(df_mul(p.dtcs_d, split64(nc, 0)), p.dta_d);
        B.submul(loss, split64(Ec, K));
        if (BE) {
            B.add(F.s);
            B.c = __fadd_rn(B.c, F.c);
        } else {
            B.add(df_mul_raw(F.value(), p.ith_d));
        }
        const df bd = B.value();
        const double b64 = df2d(bd, K);
        b[c] = b64;
        bb = fma(b64, b64, bb);
        bmax = fmaxf(bmax, fabsf(bd.h));
        const float iv = 1.0f / (A.m[c] + wsum32);
        A.invd[c] = iv;
        if (Bf.invd) {
            Bf.wx[c] = bf16_bits(A.wx[c]);
            Bf.wy[c] = bf16_bits(A.wy[c]);
            Bf.wz[c] = bf16_bits(A.wz[c]);
            Bf.invd[c] = bf16_bits(iv);
        }
    }
    double acc[2] = {bb, f2d(bmax, K)};
    const bool ismax[2] = {false, true};
    grid_reduce<2>(acc, ismax, ra);
}

// Four consecutive doubles (c a multiple of 4: 32-byte aligned).
__device__ __forceinline__ void ld_d4(const double* __restrict__ u, long long c, double v[4]) {
    const double2 a = *reinterpret_cast<const double2*>(u + c);
    const double2 e = *reinterpret_cast<const double2*>(u + c + 2);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = e.x;
    v[3] = e.y;
}
// Four consecutive df weights from their high and low arrays.
__device__ __forceinline__ void ld_w4(const float* __restrict__ h, const float* __restrict__ l, long long c,
                                      df w[4]) {
    const float4 a = ld4(h, c), e = ld4(l, c);
    w[0] = {a.x, e.x};
    w[1] = {a.y, e.y};
    w[2] = {a.z, e.z};
    w[3] = {a.w, e.w};
}

// k_asm_rhs_mx without Dirichlet faces, for levels whose x extent is a
// multiple of 4 (at least 16): a thread owns four consecutive cells of a row
// (walk4.cuh) and walks a part of one z-block of the assembly decomposition
// (blockIdx.z = z-block * zs + part).  Every flux is FluxWalk's df operation
// and every cell adds its terms in FluxWalk's order, as do the FP32
// diagonal's weights, so b and invd equal k_asm_rhs_mx's bit for bit (only
// the order of the sums of ||b||^2 differs).  The x-lower flux of a cell,
// negated, is its left neighbour's x-upper flux; a missing face (a
// zero-gradient boundary) is the flux of a cell with itself, 0, and adds a
// zero weight.
template <bool BE>
__global__ void __launch_bounds__(256, 2) k_asm_rhs4_mx(Dims d, PhysDev p, const double* __restrict__ E,
                                                     const double* __restrict__ nHI,
                                                     const double* __restrict__ eta, Op<float> A, Op<float> L,
                                                     double* __restrict__ b, RedArgs ra, const double* scg,
                                                     int zb0, int kch, int zs, Op<unsigned short> Bf) {
    const int K = step_scale(scg, p.dt_exp);
    const unsigned wm = __activemask();
    Walk w = walk_of(d);
    {
        const int zb = zb0 + (int)blockIdx.z / zs;
        const int part = (kch + zs - 1) / zs;
        w.k0 = zb * kch + ((int)blockIdx.z % zs) * part;
        w.k1 = min(min(d.nz, (zb + 1) * kch), w.k0 + part);
    }
    double bb = 0.0;
    float bmax = 0.0f;
    if (w.k0 < w.k1) {
        Geo g = geo_of(d, w, w.k0);
        double ec[4];
        ld_d4(E, g.c, ec);
        df fz[4];
        float wzc[4];
        {
            // the z-lower fluxes and weights of the part's first plane
            double ed[4];
            df wd[4];
            ld_d4(E, g.c + zdn(d, w.k0, w.nxy), ed);
            ld_w4(A.wz, L.wz, g.c, wd);
#pragma unroll
            for (int e = 0; e < 4; e++) {
                fz[e] = df_mul_raw(wd[e], split64(ed[e] - ec[e], K));
                wzc[e] = wd[e].h;
            }
        }
        for (int k = w.k0; k < w.k1; k++) {
            if (k > w.k0) g = geo_of(d, w, k);
            if (PF_PLANES > 0 && k + PF_PLANES < w.k1) {
                const long long cp = g.c + PF_PLANES * w.nxy;
                pfl2(E + cp);
                pfl2(nHI + cp);
                pfl2(eta + cp);
                pfl2(A.wx + cp);
                pfl2(L.wx + cp);
                pfl2(A.wy + cp);
                pfl2(L.wy + cp);
                pfl2(A.wz + cp);
                pfl2(L.wz + cp);
                pfl2(A.m + cp);
            }
            Acc2 F[4];
            float ws[4];
            float wxl[4], wyl[4], wzl[4];   // the lower faces' FP32 weights
            // x faces
            {
                df wx[4];
                ld_w4(A.wx, L.wx, g.c, wx);
#pragma unroll
                for (int e = 0; e < 4; e++) wxl[e] = wx[e].h;
                const double el_sh = __shfl_up_sync(wm, ec[3], 1);
                const double el = g.load_l ? E[g.xl] : el_sh;
                df fl[4];
                fl[0] = df_mul_raw(wx[0], split64(el - ec[0], K));
#pragma unroll
                for (int e = 1; e < 4; e++) fl[e] = df_mul_raw(wx[e], split64(ec[e - 1] - ec[e], K));
                const float nh = __shfl_down_sync(wm, fl[0].h, 1);
                const float nl = __shfl_down_sync(wm, fl[0].l, 1);
                const float nw = __shfl_down_sync(wm, wx[0].h, 1);
                df fu3 = {-nh, -nl};
                float wu3 = nw;
                if (g.load_r) {
                    const float wh = A.wx[g.xr_w];
                    fu3 = df_mul_raw({wh, L.wx[g.xr_w]}, split64(E[g.xr] - ec[3], K));
                    wu3 = wh;
                }
                if (!g.has_xr) wu3 = 0.0f;
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    F[e].add(fl[e]);
                    F[e].add(e < 3 ? df_neg(fl[e + 1]) : fu3);
                    ws[e] = wx[e].h;
                    ws[e] += e < 3 ? wx[e + 1].h : wu3;
                }
            }
            // y faces (the upper face's weight is the lower weight of the row above)
            {
                double em[4];
                df wl[4];
                ld_d4(E, g.ym, em);
                ld_w4(A.wy, L.wy, g.c, wl);
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    F[e].add(df_mul_raw(wl[e], split64(em[e] - ec[e], K)));
                    ws[e] += wl[e].h;
                    wyl[e] = wl[e].h;
                }
            }
            {
                double ep[4];
                df wu[4];
                ld_d4(E, g.yp, ep);
                ld_w4(A.wy, L.wy, g.yp, wu);
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    F[e].add(df_mul_raw(wu[e], split64(ep[e] - ec[e], K)));
                    ws[e] += g.has_yp ? wu[e].h : 0.0f;
                }
            }
            // z faces: the carried lower flux, the upper one formed here
            double eu[4];
            {
                const long long up = zup(d, k, w.nxy);
                const bool has_zu = k < d.nz - 1 || d.pz;
                df wu[4];
                ld_d4(E, g.c + up, eu);
                ld_w4(A.wz, L.wz, g.c + up, wu);
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    F[e].add(fz[e]);
                    const df f = df_mul_raw(wu[e], split64(eu[e] - ec[e], K));
                    F[e].add(f);
                    fz[e] = df_neg(f);
                    ws[e] += wzc[e];
                    ws[e] += has_zu ? wu[e].h : 0.0f;
                    wzl[e] = wzc[e];
                    wzc[e] = wu[e].h;
                }
            }
            // b = dt eta - dt (c sigma n_HI + adot/a) E + flux / theta
            {
                double nc[4], qc[4];
                ld_d4(nHI, g.c, nc);
                ld_d4(eta, g.c, qc);
                const float4 m4 = ld4(A.m, g.c);
                const float mv[4] = {m4.x, m4.y, m4.z, m4.w};
                double bo[4];
                float iv[4];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    Acc2 B;
                    B.add(df_mul_raw(split64(qc[e], K - p.dt_exp), p.dtm_d));
                    const df loss = df_add(df_mul(p.dtcs_d, split64(nc[e], 0)), p.dta_d);
                    B.submul(loss, split64(ec[e], K));
                    if (BE) {
                        B.add(F[e].s);
                        B.c = __fadd_rn(B.c, F[e].c);
                    } else {
                        B.add(df_mul_raw(F[e].value(), p.ith_d));
                    }
                    const df bd = B.value();
                    bo[e] = df2d(bd, K);
                    iv[e] = 1.0f / (mv[e] + ws[e]);
                    if (w.valid) {
                        bb = fma(bo[e], bo[e], bb);
                        bmax = fmaxf(bmax, fabsf(bd.h));
                    }
                }
                if (w.valid) {
                    *reinterpret_cast<double2*>(b + g.c) = make_double2(bo[0], bo[1]);
                    *reinterpret_cast<double2*>(b + g.c + 2) = make_double2(bo[2], bo[3]);
                    st4(A.invd, g.c, make_float4(iv[0], iv[1], iv[2], iv[3]));
                    if (Bf.invd) {
                        *reinterpret_cast<uint2*>(Bf.wx + g.c) = bf16_pack4(wxl[0], wxl[1], wxl[2], wxl[3]);
                        *reinterpret_cast<uint2*>(Bf.wy + g.c) = bf16_pack4(wyl[0], wyl[1], wyl[2], wyl[3]);
                        *reinterpret_cast<uint2*>(Bf.wz + g.c) = bf16_pack4(wzl[0], wzl[1], wzl[2], wzl[3]);
                        *reinterpret_cast<uint2*>(Bf.invd + g.c) = bf16_pack4(iv[0], iv[1], iv[2], iv[3]);
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 4; e++) ec[e] = eu[e];
        }
    }
    double acc[2] = {bb, f2d(bmax, K)};
    const bool ismax[2] = {false, true};
    grid_reduce<2>(acc, ismax, ra);
}

// -------------------------------------------------------------- refinement

// The first refinement's right-hand side, r = b (x = 0): r32 = b * 2^-Ks
// rounded to FP32, ||r32||^2 and max |r32| (reduction R_IRRES with aux =
// 2^Ks).  The inner solve starts its x32 at 0 itself.
__global__ void __launch_bounds__(RED_THREADS) k_ir_scale_b(long long n, const double* __restrict__ b, int Ks,
                                                           float* __restrict__ r32, RedArgs ra) {
    DotAcc<float> da;
    float mx = 0.0f;
    GRID_LOOP(c, n) {
        const float v = round64(b[c], Ks);
        r32[c] = v;
        da.add(v, v);
        mx = fmaxf(mx, fabsf(v));
    }
    double acc[2] = {da.value(), (double)mx};
    const bool ismax[2] = {false, true};
    grid_reduce<2>(acc, ismax, ra);
}

// x += 2^ks (x32 + alpha p_last) with x a df pair scaled by 2^-K (assign:
// x = ..., the first refinement from x = 0).  p_last: the inner solve
// deferred its last update of x32; the FP32 operation the update kernel
// would have done, x32 + alpha p_last, takes its place.
__global__ void k_ir_update_mx(long long n, float2* __restrict__ x, const float* __restrict__ x32,
                               const double* __restrict__ sc, int assign, int ks, const float* __restrict__ p_last,
                               const double* scg, int dt_exp) {
    const int K = step_scale(scg, dt_exp);
    const float alpha = (float)sc[S_ALPHA];
    GRID_LOOP(c, n) {
        const float xf = p_last ? fmaf(alpha, p_last[c], x32[c]) : x32[c];
        const float u = ldexp2(xf, ks - K);
        if (assign) {
            x[c] = make_float2(u, 0.0f);
        } else {
            const float2 o = x[c];
            df s = two_sum(o.x, u);
            s.l = __fadd_rn(s.l, o.y);
            s = fast_two_sum(s.h, s.l);
            x[c] = make_float2(s.h, s.l);
        }
    }
}

// k_ir_update_mx four cells per thread (n a multiple of 4): the same
// operations on each cell, with 16-byte loads and stores.
__global__ void k_ir_update4_mx(long long n4, float4* __restrict__ x, const float4* __restrict__ x32,
                                const double* __restrict__ sc, int assign, int ks, const float4* __restrict__ p_last,
                                const double* scg, int dt_exp) {
    const int K = step_scale(scg, dt_exp);
    const float alpha = (float)sc[S_ALPHA];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4;
         q += (long long)gridDim.x * blockDim.x) {
        float4 xf = x32[q];
        if (p_last) {
            const float4 pv = p_last[q];
            xf.x = fmaf(alpha, pv.x, xf.x);
            xf.y = fmaf(alpha, pv.y, xf.y);
            xf.z = fmaf(alpha, pv.z, xf.z);
            xf.w = fmaf(alpha, pv.w, xf.w);
        }
        const float u[4] = {ldexp2(xf.x, ks - K), ldexp2(xf.y, ks - K), ldexp2(xf.z, ks - K), ldexp2(xf.w, ks - K)};
        if (assign) {
            x[2 * q] = make_float4(u[0], 0.0f, u[1], 0.0f);
            x[2 * q + 1] = make_float4(u[2], 0.0f, u[3], 0.0f);
        } else {
            const float4 o0 = x[2 * q], o1 = x[2 * q + 1];
            const float oh[4] = {o0.x, o0.z, o1.x, o1.z}, ol[4] = {o0.y, o0.w, o1.y, o1.w};
            float h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                df t = two_sum(oh[e], u[e]);
                t.l = __fadd_rn(t.l, ol[e]);
                t = fast_two_sum(t.h, t.l);
                h[e] = t.h;
                l[e] = t.l;
            }
            x[2 * q] = make_float4(h[0], l[0], h[1], l[1]);
            x[2 * q + 1] = make_float4(h[2], l[2], h[3], l[3]);
        }
    }
}

// Refinement residual r = b - m x - sum_f w_f (x - x_nbr) of the df iterate
// x: ||r32||^2 and max |r32| of r32 = r * 2^-Ks rounded to FP32 (reduction
// R_IRRES) and, with WRITE, r32 itself (the next inner solve's right-hand
// side; without it the launch only measures the residual).
template <bool WRITE>
__global__ void __launch_bounds__(256) k_ir_residual(Dims d, Op<float> A, Op<float> L,
                                                    const double* __restrict__ b, const float2* __restrict__ x,
                                                    int Ks, float* __restrict__ r32, RedArgs ra, const double* scg,
                                                    int dt_exp) {
    const int K = step_scale(scg, dt_exp);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int kch = (d.nz + (int)gridDim.z - 1) / (int)gridDim.z;
    const int k0 = (int)blockIdx.z * kch;
    const int k1 = min(d.nz, k0 + kch);
    const bool inb = i < d.nx && j < d.ny;
    const long long nxy = (long long)d.nx * d.ny;
    FluxWalk<DFField> fw;
    fw.d = d;
    fw.A = A;
    fw.L = L;
    fw.u = DFField{x};
    fw.wmask = __activemask();
    fw.xnext = threadIdx.x + 1 < blockDim.x;
    DotAcc<float> da;
    float mx = 0.0f;
    df fz = {0.0f, 0.0f};
    bool have_z = false;
    for (int k = k0; k < k1; k++) {
        const long long c = (long long)k * nxy + (long long)j * d.nx + i;
        if (PF_PLANES > 0 && inb && k + PF_PLANES < k1) {
            const long long cp = c + PF_PLANES * nxy;
            pfl2(b + cp);
            pfl2(x + cp);
            pfl2(A.m + cp);
            pfl2(L.m + cp);
            pfl2(A.wx + cp);
            pfl2(L.wx + cp);
            pfl2(A.wy + cp);
            pfl2(L.wy + cp);
            pfl2(A.wz + cp);
            pfl2(L.wz + cp);
        }
        const df xc = inb ? fw.u.at(c) : df{0.0f, 0.0f};
        Acc2 R;
        float wsum32 = 0.0f;
        fw.plane(inb, i, j, k, c, xc, R, wsum32, fz, have_z);
        if (!inb) continue;
        R.add(split64(b[c], K));
        R.addmul({-A.m[c], -L.m[c]}, xc);
        const float v = ldexp2(R.value().h, K - Ks);
        if (WRITE) r32[c] = v;
        da.add(v, v);
        mx = fmaxf(mx, fabsf(v));
    }
    double acc[2] = {da.value(), (double)mx};
    const bool ismax[2] = {false, true};
    grid_reduce<2>(acc, ismax, ra);
}

// Four consecutive cells of a df array (c a multiple of 4: 32-byte aligned).
__device__ __forceinline__ void ld_df4(const float2* __restrict__ u, long long c, df v[4]) {
    const float4 a = *reinterpret_cast<const float4*>(u + c);
    const float4 e = *reinterpret_cast<const float4*>(u + c + 2);
    v[0] = {a.x, a.y};
    v[1] = {a.z, a.w};
    v[2] = {e.x, e.y};
    v[3] = {e.z, e.w};
}

// k_ir_residual for levels whose x extent is a multiple of 4 (at least 16):
// a thread owns four consecutive cells of a row (walk4.cuh) and walks its
// chunk of planes.  Every flux is the same df operation as in FluxWalk and
// every cell sums its terms in the same order (x lo, x hi, y lo, y hi,
// z lo, z hi, b, -m x), so r32 equals k_ir_residual's bit for bit: the
// x-lower flux of a cell, negated, is its left neighbour's x-upper flux
// (within the thread, or from the next lane for the last cell), the
// z-upper flux of a plane is the next plane's z-lower one, and a missing
// face (a zero-gradient boundary) is the flux of a cell with itself, 0.
// Vector loads and one address computation per four cells take about half
// the instructions of the one-cell form, whose issue rate bounds it.
template <bool WRITE>
__global__ void __launch_bounds__(256, 2) k_ir_residual4(Dims d, Op<float> A, Op<float> L,
                                                      const double* __restrict__ b,
                                                      const float2* __restrict__ x, int Ks,
                                                      float* __restrict__ r32, RedArgs ra, const double* scg,
                                                      int dt_exp) {
    const int K = step_scale(scg, dt_exp);
    // the lanes of this warp (a block of fewer than 32 threads has fewer)
    const unsigned wm = __activemask();
    const Walk w = walk_of(d);
    DotAcc<float> da;
    float mx = 0.0f;
    if (w.k0 < w.k1) {
        Geo g = geo_of(d, w, w.k0);
        df xc[4], fz[4];
        ld_df4(x, g.c, xc);
        {
            // the z-lower fluxes of the chunk's first plane
            df xd[4], wd[4];
            ld_df4(x, g.c + zdn(d, w.k0, w.nxy), xd);
            ld_w4(A.wz, L.wz, g.c, wd);
#pragma unroll
            for (int e = 0; e < 4; e++) fz[e] = df_mul_raw(wd[e], df_sub(xd[e], xc[e]));
        }
        for (int k = w.k0; k < w.k1; k++) {
            if (k > w.k0) g = geo_of(d, w, k);
            if (PF_PLANES > 0 && k + PF_PLANES < w.k1) {
                const long long cp = g.c + PF_PLANES * w.nxy;
                pfl2(b + cp);
                pfl2(x + cp);
                pfl2(A.m + cp);
                pfl2(L.m + cp);
                pfl2(A.wx + cp);
                pfl2(L.wx + cp);
                pfl2(A.wy + cp);
                pfl2(L.wy + cp);
                pfl2(A.wz + cp);
                pfl2(L.wz + cp);
            }
            Acc2 R[4];
            // x faces: lower fluxes of the four cells, the last cell's upper
            {
                df wx[4];
                ld_w4(A.wx, L.wx, g.c, wx);
                const float lh = __shfl_up_sync(wm, xc[3].h, 1);
                const float ll = __shfl_up_sync(wm, xc[3].l, 1);
                df xl = {lh, ll};
                if (g.load_l) {
                    const float2 v = x[g.xl];
                    xl = {v.x, v.y};
                }
                df fl[4];
                fl[0] = df_mul_raw(wx[0], df_sub(xl, xc[0]));
#pragma unroll
                for (int e = 1; e < 4; e++) fl[e] = df_mul_raw(wx[e], df_sub(xc[e - 1], xc[e]));
                const float nh = __shfl_down_sync(wm, fl[0].h, 1);
                const float nl = __shfl_down_sync(wm, fl[0].l, 1);
                df fu3 = {-nh, -nl};
                if (g.load_r) {
                    const float2 v = x[g.xr];
                    fu3 = df_mul_raw({A.wx[g.xr_w], L.wx[g.xr_w]}, df_sub({v.x, v.y}, xc[3]));
                }
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    R[e].add(fl[e]);
                    R[e].add(e < 3 ? df_neg(fl[e + 1]) : fu3);
                }
            }
            // y faces (the upper face's weight is the lower weight of the row above)
            {
                df xm[4], wl[4];
                ld_df4(x, g.ym, xm);
                ld_w4(A.wy, L.wy, g.c, wl);
#pragma unroll
                for (int e = 0; e < 4; e++) R[e].add(df_mul_raw(wl[e], df_sub(xm[e], xc[e])));
            }
            {
                df xp[4], wu[4];
                ld_df4(x, g.yp, xp);
                ld_w4(A.wy, L.wy, g.yp, wu);
#pragma unroll
                for (int e = 0; e < 4; e++) R[e].add(df_mul_raw(wu[e], df_sub(xp[e], xc[e])));
            }
            // z faces: the carried lower flux, the upper one formed here
            df xu[4];
            {
                df wu[4];
                const long long up = zup(d, k, w.nxy);
                ld_df4(x, g.c + up, xu);
                ld_w4(A.wz, L.wz, g.c + up, wu);
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    R[e].add(fz[e]);
                    const df f = df_mul_raw(wu[e], df_sub(xu[e], xc[e]));
                    R[e].add(f);
                    fz[e] = df_neg(f);
                }
            }
            // b - m x
            {
                const double2 b01 = *reinterpret_cast<const double2*>(b + g.c);
                const double2 b23 = *reinterpret_cast<const double2*>(b + g.c + 2);
                const double bv[4] = {b01.x, b01.y, b23.x, b23.y};
                const float4 mh = ld4(A.m, g.c), ml = ld4(L.m, g.c);
                const float mhv[4] = {mh.x, mh.y, mh.z, mh.w}, mlv[4] = {ml.x, ml.y, ml.z, ml.w};
                float v[4];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    R[e].add(split64(bv[e], K));
                    R[e].addmul({-mhv[e], -mlv[e]}, xc[e]);
                    v[e] = ldexp2(R[e].value().h, K - Ks);
                }
                if (w.valid) {
                    if (WRITE) st4(r32, g.c, make_float4(v[0], v[1], v[2], v[3]));
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        da.add(v[e], v[e]);
                        mx = fmaxf(mx, fabsf(v[e]));
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 4; e++) xc[e] = xu[e];
        }
    }
    double acc[2] = {da.value(), (double)mx};
    const bool ismax[2] = {false, true};
    grid_reduce<2>(acc, ismax, ra);
}

// ------------------------------------------------------------ finalisation

// E_out = max(E + dE, 0) (FP64; dE the df iterate scaled by 2^-K) and the
// sums of the photon balance: sum dE, sum eta, sum n_HI E^theta, sum
// E^theta (E^theta = E + theta dE), the energy the floor adds, sum dE^2 and
// sum E_out^2 (the last two to FP32 accuracy, for the relative change of the
// step), reduction R_STORE7_FIN.  The sums run in df relative to the scales
// of the maxima in scg.
template <bool BE>
__global__ void __launch_bounds__(RED_THREADS) k_finalize_mx(long long n, PhysDev p, const double* __restrict__ E,
                                                            const float2* __restrict__ dE,
                                                            const double* __restrict__ nHI,
                                                            const double* __restrict__ eta, double* E_out,
                                                            RedArgs ra, const double* scg) {
    const int K = step_scale(scg, p.dt_exp);
    const int Kq = exp_above(scg[S_ETAMAX]) < -1000 ? 0 : exp_above(scg[S_ETAMAX]);
    const int Kn = exp_above(scg[S_NMAX]) < -1000 ? 0 : exp_above(scg[S_NMAX]);
    Acc2 sd, sq, sn, st;
    DotAcc<float> s2d, s2e;
    double floor_e = 0.0;
    // two cells per thread and pass, their loads issued together (four
    // needed 78 registers and three blocks per SM: 1.04 against 1.00 ms per
    // 512^3 step)
    constexpr int U = 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; c0 < n; c0 += U * stride) {
        float2 dv[U];
        double Ev[U], nv[U], qv[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long c = c0 + u * stride;
            if (c < n) {
                dv[u] = dE[c];
                Ev[u] = E[c];
                nv[u] = nHI[c];
                qv[u] = eta[c];
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long c = c0 + u * stride;
            if (c >= n) break;
            const df dd = {dv[u].x, dv[u].y};
            const double d64 = f2d(dd.h, K) + f2d(dd.l, K);
            const double En = Ev[u] + d64;
            const double Et = BE ? En : fma(p.theta, d64, Ev[u]);
            const df et = split64(Et, K);
            sd.add(dd);
            st.add(et);
            sq.add(split64(qv[u], Kq));
            sn.addmul(split64(nv[u], Kn), et);
            const bool neg = __double2hiint(En) < 0;   // sign bit (also -0)
            if (neg) floor_e -= En;
            const float eo = neg ? 0.0f : (BE ? et.h : split64(En, K).h);
            s2d.add(dd.h, dd.h);
            s2e.add(eo, eo);
            E_out[c] = neg ? 0.0 : En;
        }
    }
    double acc[7] = {df2d(sd.value(), K), df2d(sq.value(), Kq), df2d(sn.value(), Kn + K), floor_e,
                     f2d(s2d.hi, 2 * K) + f2d(s2d.lo, 2 * K), f2d(s2e.hi, 2 * K) + f2d(s2e.lo, 2 * K),
                     df2d(st.value(), K)};
    const bool mx[7] = {false, false, false, false, false, false, false};
    grid_reduce<7>(acc, mx, ra);
}

// Photons through the Dirichlet faces of side sd over the step, as
// k_bnd_outflow, with dE the df iterate scaled by 2^-K.
__global__ void __launch_bounds__(RED_THREADS) k_bnd_outflow_mx(Dims d, PhysDev p, int sd, Bnd bnd,
                                                               const double* __restrict__ E,
                                                               const float2* __restrict__ dE, RedArgs ra,
                                                               const double* scg) {
    const int K = step_scale(scg, p.dt_exp);
    const int a = sd >> 1, hi = sd & 1;
    const long long nf = bnd_side_size(d, sd);
    const long long off = bnd_offset(d, sd);
    const long long nu = a == 0 ? d.ny : d.nx;
    const double Eb = p.ebc[sd];
    double acc[2] = {0.0, 0.0};
    GRID_LOOP(f, nf) {
        const long long u = f % nu, v = f / nu;
        long long i, j, k;
        if (a == 0) { i = hi ? d.nx - 1 : 0; j = u; k = v; }
        else if (a == 1) { i = u; j = hi ? d.ny - 1 : 0; k = v; }
        else { i = u; j = v; k = hi ? d.nz - 1 : 0; }
        const long long c = i + (long long)d.nx * (j + (long long)d.ny * k);
        const float2 dv = dE[c];
        const double d64 = f2d(dv.x, K) + f2d(dv.y, K);
        const double fl = bnd.w[off + f] * fma(p.inv_theta, E[c] - Eb, d64);
        acc[0] += fl;
        acc[1] += fabs(fl);
    }
    const bool mx[2] = {false, false};
    grid_reduce<2>(acc, mx, ra);
}

// ------------------------------------------------------------------ hooks

// FP64 values of a df array (test and inspection hooks).
__global__ void k_df_to_f64(long long n, const float* __restrict__ h, const float* __restrict__ l,
                            double* __restrict__ out) {
    GRID_LOOP(c, n) out[c] = (double)h[c] + (double)l[c];
}

// The df iterate dE (scaled by 2^-K) as FP64 values.
__global__ void k_dE_to_f64(long long n, const float2* __restrict__ x, double* __restrict__ out, const double* scg,
                            int dt_exp) {
    const int K = step_scale(scg, dt_exp);
    GRID_LOOP(c, n) {
        const float2 v = x[c];
        out[c] = f2d(v.x, K) + f2d(v.y, K);
    }
}

// y = A x with the df operator (FP64 arithmetic; test hook).
__global__ void k_apply_mx(Dims d, Op<float> A, Op<float> L, const double* __restrict__ x, double* __restrict__ y) {
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    auto W = [&](const float* h, const float* l, long long q) { return (double)h[q] + (double)l[q]; };
    COL_BEGIN(d)
        const double xc = x[c];
        double acc = W(A.m, L.m, c) * xc;
        if (i > 0) acc += W(A.wx, L.wx, c) * (xc - x[c - 1]); else if (d.px) acc += W(A.wx, L.wx, c) * (xc - x[c + d.nx - 1]);
        if (i < d.nx - 1) acc += W(A.wx, L.wx, c + 1) * (xc - x[c + 1]); else if (d.px) acc += W(A.wx, L.wx, c - (d.nx - 1)) * (xc - x[c - (d.nx - 1)]);
        if (j > 0) acc += W(A.wy, L.wy, c) * (xc - x[c - sy]); else if (d.py) acc += W(A.wy, L.wy, c) * (xc - x[c + (long long)(d.ny - 1) * sy]);
        if (j < d.ny - 1) acc += W(A.wy, L.wy, c + sy) * (xc - x[c + sy]); else if (d.py) acc += W(A.wy, L.wy, c - (long long)(d.ny - 1) * sy) * (xc - x[c - (long long)(d.ny - 1) * sy]);
        if (k > 0) acc += W(A.wz, L.wz, c) * (xc - x[c - sz]); else if (d.pz) acc += W(A.wz, L.wz, c) * (xc - x[c + (long long)(d.nz - 1) * sz]);
        if (k < d.nz - 1) acc += W(A.wz, L.wz, c + sz) * (xc - x[c + sz]); else if (d.pz) acc += W(A.wz, L.wz, c - (long long)(d.nz - 1) * sz) * (xc - x[c - (long long)(d.nz - 1) * sz]);
        y[c] = acc;
    }
}

// ---------------------------------------------------------------- launchers

void launch_asm_faces_mx(const Dims& d, const PhysDev& p, const double* E, const double* nHI, const double* eta,
                         Op<float> A, Op<float> L, double* sc, FaceList fl, cudaStream_t s, int zb0, int nzb) {
    const AsmShape a = asm_shape(d);
    if (nzb < 0 || zb0 + nzb > a.nzb) nzb = a.nzb - zb0;
    if (nzb <= 0) return;
    k_asm_faces_mx<<<dim3(a.sh.grid.x, a.sh.grid.y, (unsigned)nzb), a.sh.block, 0, s>>>(d, p, E, nHI, eta, A, L,
                                                                                         sc, fl, zb0, a.kch);
}

void launch_asm_fix_mx(const Dims& d, const PhysDev& p, const double* E, const double* nHI, Op<float> A,
                       Op<float> L, FaceList fl, cudaStream_t s, int zb0, int nzb) {
    if (!fl.entries) return;
    const AsmShape a = asm_shape(d);
    if (nzb < 0 || zb0 + nzb > a.nzb) nzb = a.nzb - zb0;
    if (nzb <= 0) return;
    const long long per_zb = (long long)a.sh.grid.x * a.sh.grid.y;
    FaceList f = fl;
    f.entries = fl.entries + per_zb * zb0 * fl.cap;
    f.counts = fl.counts + per_zb * zb0;
    k_asm_fix_mx<<<(unsigned)(per_zb * nzb), 256, 0, s>>>(d, p, E, nHI, A, L, f);
}

void launch_asm_rhs_mx(const Dims& d, const PhysDev& p, const double* E, const double* nHI, const double* eta,
                       Op<float> A, Op<float> L, double* b, Bnd bnd, const RedArgs& ra, const double* scg,
                       cudaStream_t s, int zb0, int nzb, Op<unsigned short> Bf) {
    const AsmShape a = asm_shape(d);
    if (nzb < 0 || zb0 + nzb > a.nzb) nzb = a.nzb - zb0;
    if (nzb <= 0) return;
    const bool be = p.theta == 1.0, dir = p.dmask != 0;
    if (!dir && fine4_ok(d)) {
        // four cells per thread; each z-block in parts of about 32 planes
        Dims h = d;
        h.nx = d.nx / 4;
        const ColShape sh = col_shape(h, 256, 1);
        const long long xy = (long long)sh.grid.x * sh.grid.y;
        int zs = (a.kch + 31) / 32;
        while (zs > 1 && xy * nzb * zs > RED_MAX_BLOCKS) zs--;
        const dim3 g4(sh.grid.x, sh.grid.y, (unsigned)(nzb * zs));
        if (be)
            k_asm_rhs4_mx<true><<<g4, sh.block, 0, s>>>(d, p, E, nHI, eta, A, L, b, ra, scg, zb0, a.kch, zs, Bf);
        else
            k_asm_rhs4_mx<false><<<g4, sh.block, 0, s>>>(d, p, E, nHI, eta, A, L, b, ra, scg, zb0, a.kch, zs, Bf);
        return;
    }
    const dim3 g(a.sh.grid.x, a.sh.grid.y, (unsigned)nzb);
    if (be && !dir)
        k_asm_rhs_mx<true, false><<<g, a.sh.block, 0, s>>>(d, p, E, nHI, eta, A, L, b, bnd, ra, scg, zb0, a.kch,
                                                             Bf);
    else if (be)
        k_asm_rhs_mx<true, true><<<g, a.sh.block, 0, s>>>(d, p, E, nHI, eta, A, L, b, bnd, ra, scg, zb0, a.kch,
                                                             Bf);
    else if (!dir)
        k_asm_rhs_mx<false, false><<<g, a.sh.block, 0, s>>>(d, p, E, nHI, eta, A, L, b, bnd, ra, scg, zb0, a.kch,
                                                             Bf);
    else
        k_asm_rhs_mx<false, true><<<g, a.sh.block, 0, s>>>(d, p, E, nHI, eta, A, L, b, bnd, ra, scg, zb0, a.kch,
                                                             Bf);
}

void launch_ir_scale_b(long long n, const double* b, int Ks, float* r32, const RedArgs& ra,
                       cudaStream_t s) {
    k_ir_scale_b<<<red_blocks(n), RED_THREADS, 0, s>>>(n, b, Ks, r32, ra);
}

void launch_ir_update_mx(long long n, void* x, const float* x32, const double* sc, bool assign, int ks,
                         const float* p_last, const double* scg, int dt_exp, cudaStream_t s) {
    if (n % 4 == 0) {
        k_ir_update4_mx<<<grid_blocks(n / 4, 256), 256, 0, s>>>(n / 4, (float4*)x, (const float4*)x32, sc,
                                                                assign ? 1 : 0, ks, (const float4*)p_last, scg,
                                                                dt_exp);
        return;
    }
    k_ir_update_mx<<<grid_blocks(n, 256), 256, 0, s>>>(n, (float2*)x, x32, sc, assign ? 1 : 0, ks, p_last, scg,
                                                       dt_exp);
}

// many short z-chunks: at 512^3 about 16 blocks per SM in several full
// waves (measured: 2.6 ms with 152 x 8 target blocks, 1.9 ms with 152 x 64)
// About 2048 cells per block (each thread walks eight planes or more), from
// 152 * 4 to 152 * 64 blocks.
ColShape ir_residual_shape(const Dims& d) {
    long long t = d.n / 2048;
    if (t < 152 * 4) t = 152 * 4;
    if (t > 152 * 64) t = 152 * 64;
    return col_shape(d, 256, (int)t);
}

// The four-cell form: 256 threads of four cells and about IR4_CELLS cells
// per block (each thread walks IR4_CELLS / 1024 planes or more).
constexpr long long IR4_CELLS = 16384;

ColShape ir_residual4_shape(const Dims& d) {
    Dims h = d;
    h.nx = d.nx / 4;
    long long t = d.n / IR4_CELLS;
    if (t < 152 * 4) t = 152 * 4;
    if (t > 152 * 64) t = 152 * 64;
    return col_shape(h, 256, (int)t);
}

void launch_ir_residual(const Dims& d, Op<float> A, Op<float> L, const double* b, const void* x, int Ks,
                        float* r32, bool write, const RedArgs& ra, const double* scg, int dt_exp, cudaStream_t s) {
    if (fine4_ok(d)) {
        const ColShape sh = ir_residual4_shape(d);
        if (write)
            k_ir_residual4<true><<<sh.grid, sh.block, 0, s>>>(d, A, L, b, (const float2*)x, Ks, r32, ra, scg, dt_exp);
        else
            k_ir_residual4<false><<<sh.grid, sh.block, 0, s>>>(d, A, L, b, (const float2*)x, Ks, r32, ra, scg,
                                                               dt_exp);
        return;
    }
    const ColShape sh = ir_residual_shape(d);
    if (write)
        k_ir_residual<true><<<sh.grid, sh.block, 0, s>>>(d, A, L, b, (const float2*)x, Ks, r32, ra, scg, dt_exp);
    else
        k_ir_residual<false><<<sh.grid, sh.block, 0, s>>>(d, A, L, b, (const float2*)x, Ks, r32, ra, scg, dt_exp);
}

void launch_finalize_mx(long long n, const PhysDev& p, const double* E, const void* dE, const double* nHI,
                        const double* eta, double* E_out, const RedArgs& ra, const double* scg, cudaStream_t s) {
    if (p.theta == 1.0)
        k_finalize_mx<true><<<red_blocks(n), RED_THREADS, 0, s>>>(n, p, E, (const float2*)dE, nHI, eta, E_out, ra,
                                                                   scg);
    else
        k_finalize_mx<false><<<red_blocks(n), RED_THREADS, 0, s>>>(n, p, E, (const float2*)dE, nHI, eta, E_out, ra,
                                                                    scg);
}

void launch_bnd_outflow_mx(const Dims& d, const PhysDev& p, int sd, Bnd bnd, const double* E, const void* dE,
                           const RedArgs& ra, const double* scg, cudaStream_t st) {
    k_bnd_outflow_mx<<<red_blocks(bnd_side_size(d, sd)), RED_THREADS, 0, st>>>(d, p, sd, bnd, E, (const float2*)dE,
                                                                              ra, scg);
}

void launch_df_to_f64(long long n, const float* h, const float* l, double* out, cudaStream_t s) {
    k_df_to_f64<<<grid_blocks(n, 256), 256, 0, s>>>(n, h, l, out);
}

void launch_dE_to_f64(long long n, const void* x, double* out, const double* scg, int dt_exp, cudaStream_t s) {
    k_dE_to_f64<<<grid_blocks(n, 256), 256, 0, s>>>(n, (const float2*)x, out, scg, dt_exp);
}

void launch_apply_mx(const Dims& d, Op<float> A, Op<float> L, const double* x, double* y, cudaStream_t s) {
    const ColShape sh = col_shape(d);
    k_apply_mx<<<sh.grid, sh.block, 0, s>>>(d, A, L, x, y);
}

}  // namespace fld
