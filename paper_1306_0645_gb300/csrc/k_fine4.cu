// k_fine4.cu -- FP32 stencil sweeps of the mixed-precision solve, each
// thread owning four consecutive cells along x (float4 loads and stores).
//
// Every sweep streams its arrays once: a thread walks k through its chunk
// of planes and keeps the z-neighbour values in registers (one new float4
// per array and plane), takes the x-neighbours of its four cells from the
// adjacent lanes with warp shuffles, and reads the y-neighbour rows (which
// the neighbouring threads of the block stream) through L1.  These are the
// same operations as the scalar kernels of k_mg.cu / k_cg.cu, restricted to
// levels whose x extent is a multiple of 4.  The V-cycle's sweeps (zero-guess
// smoothing, colour sweeps, zero-guess residual) read their coefficients from
// FP32 or from bfloat16 storage (the template parameter T), the CG's
// matrix-vector product always from the FP32 operator.
#include "walk4.cuh"
#include <cuda_bf16.h>

namespace fld {

namespace {

// x-neighbour values of the 4-vector v of array u.
__device__ __forceinline__ void xnb(const float* __restrict__ u, const Geo& g, float4 v, float& L,
                                    float& R) {
    const float l = __shfl_up_sync(FULL, v.w, 1);
    const float r = __shfl_down_sync(FULL, v.x, 1);
    L = g.load_l ? u[g.xl] : l;
    R = g.load_r ? u[g.xr] : r;
}

// Coefficients of the smoothing operator as FP32 values, from FP32 storage
// or from bfloat16 storage (the upper half of an FP32 number, so the
// conversion is exact): four consecutive ones (i a multiple of 4) or one.
__device__ __forceinline__ float4 ldw4(const float* __restrict__ p, long long i) { return ld4(p, i); }
__device__ __forceinline__ float4 ldw4(const unsigned short* __restrict__ p, long long i) {
    const uint2 v = *reinterpret_cast<const uint2*>(p + i);
    return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xFFFF0000u),
                       __uint_as_float(v.y << 16), __uint_as_float(v.y & 0xFFFF0000u));
}
__device__ __forceinline__ float ldw(const float* __restrict__ p, long long i) { return p[i]; }
__device__ __forceinline__ float ldw(const unsigned short* __restrict__ p, long long i) {
    return __uint_as_float((unsigned)p[i] << 16);
}

// Weight of the upper x face of element 3 (0 on a zero-gradient boundary).
template <class T>
__device__ __forceinline__ float wx_up(const T* __restrict__ wx, const Geo& g, float4 wv) {
    const float r = __shfl_down_sync(FULL, wv.x, 1);
    if (!g.has_xr) return 0.0f;
    return g.load_r ? ldw(wx, g.xr_w) : r;
}

struct Faces4 {      // the six face weights of each of the four cells
    float4 xl, xu, yl, yu, zl, zu;
};

template <class T>
__device__ __forceinline__ Faces4 faces_of(const Op<T>& A, const Geo& g, float4 wxc, float4 wzc,
                                           float4 wzu, bool has_zu) {
    Faces4 f;
    f.xl = wxc;
    const float xu3 = wx_up(A.wx, g, wxc);
    f.xu = make_float4(wxc.y, wxc.z, wxc.w, xu3);
    f.yl = ldw4(A.wy, g.c);
    f.yu = g.has_yp ? ldw4(A.wy, g.yp) : make_float4(0.f, 0.f, 0.f, 0.f);
    f.zl = wzc;
    f.zu = has_zu ? wzu : make_float4(0.f, 0.f, 0.f, 0.f);
    return f;
}

}  // namespace

// ------------------------------------------------------------------ p, q

// p_out = z + beta p_in;  q = A p_out;  <p_out, q>.  With x: also the
// previous iteration's solution update x += alpha_prev p_in (alpha_prev is
// the alpha slot when the kernel starts; its own reduction replaces it only
// after every block has read it), which k_cg_update4 then leaves out.
__global__ void __launch_bounds__(256, 4) k_cg_p_matvec4(Dims d, Op<float> A, const float* __restrict__ z,
                                                      const float* __restrict__ p_in,
                                                      float* __restrict__ p_out, float* __restrict__ q,
                                                      float* __restrict__ x, RedArgs ra, int pf) {
    const float beta = (float)ra.sc[S_BETA];
    const float alpha_prev = x ? (float)ra.sc[S_ALPHA] : 0.0f;
    // the first iteration of a solve starts x at 0 instead of updating it
    const bool x_zero = x && ra.sc[S_XZERO] != 0.0;
    const Walk w = walk_of(d);
    DotAcc<float> da;
    auto P = [&](long long i) {
        const float4 a = ld4(z, i), b = ld4(p_in, i);
        return make_float4(fmaf(beta, b.x, a.x), fmaf(beta, b.y, a.y), fmaf(beta, b.z, a.z),
                           fmaf(beta, b.w, a.w));
    };
    auto Ps = [&](long long i) { return fmaf(beta, p_in[i], z[i]); };
    if (w.k0 < w.k1) {
        Geo g = geo_of(d, w, w.k0);
        float4 pc = P(g.c);
        float4 pd = P(g.c + zdn(d, w.k0, w.nxy));
        float4 wzc = ld4(A.wz, g.c);
        for (int k = w.k0; k < w.k1; k++) {
            if (k > w.k0) g = geo_of(d, w, k);
            if (pf > 0 && k + pf < w.k1) {
                const long long o = g.c + (long long)pf * w.nxy;
                pf2(z, o);
                pf2(p_in, o);
                pf2(A.m, o);
                pf2(A.wx, o);
                pf2(A.wy, o);
                pf2(A.wz, o);
            }
            const long long up = zup(d, k, w.nxy);
            const bool has_zu = k < d.nz - 1 || d.pz;
            const float4 pu = P(g.c + up);
            const float4 wzu = ld4(A.wz, g.c + (k < d.nz - 1 ? w.nxy : -(long long)(d.nz - 1) * w.nxy * (d.pz ? 1 : 0)));
            const float4 wxc = ld4(A.wx, g.c);
            const Faces4 f = faces_of(A, g, wxc, wzc, wzu, has_zu);
            // x neighbours of p
            const float lsh = __shfl_up_sync(FULL, pc.w, 1);
            const float rsh = __shfl_down_sync(FULL, pc.x, 1);
            const float L = g.load_l ? Ps(g.xl) : lsh;
            const float R = g.load_r ? Ps(g.xr) : rsh;
            const float4 pym = P(g.ym), pyp = P(g.yp);
            const float4 m = ld4(A.m, g.c);
            float4 qv;
#define Q1(X, LX, RX)                                                                   \
            qv.X = m.X * pc.X + f.xl.X * (pc.X - (LX)) + f.xu.X * (pc.X - (RX)) +       \
                   f.yl.X * (pc.X - pym.X) + f.yu.X * (pc.X - pyp.X) +                 \
                   f.zl.X * (pc.X - pd.X) + f.zu.X * (pc.X - pu.X);
            Q1(x, L, pc.y)
            Q1(y, pc.x, pc.z)
            Q1(z, pc.y, pc.w)
            Q1(w, pc.z, R)
#undef Q1
            if (w.valid) {
                st4(p_out, g.c, pc);
                st4(q, g.c, qv);
                if (x_zero) {
                    st4(x, g.c, make_float4(0.f, 0.f, 0.f, 0.f));
                } else if (x) {
                    // p_in of this plane was read one plane ago (L1)
                    const float4 pv = ld4(p_in, g.c);
                    float4 xv = ld4(x, g.c);
                    xv.x = fmaf(alpha_prev, pv.x, xv.x); xv.y = fmaf(alpha_prev, pv.y, xv.y);
                    xv.z = fmaf(alpha_prev, pv.z, xv.z); xv.w = fmaf(alpha_prev, pv.w, xv.w);
                    st4(x, g.c, xv);
                }
                da.add(pc.x, qv.x);
                da.add(pc.y, qv.y);
                da.add(pc.z, qv.z);
                da.add(pc.w, qv.w);
            }
            pd = pc;
            pc = pu;
            wzc = wzu;
        }
    }
    double acc[1] = {da.value()};
    const bool mx[1] = {false};
    grid_reduce<1>(acc, mx, ra);
}

// ---------------------------------------------------------------- residual

// res = r - A z.  ZG: z is the result of one red/black sweep from z = 0
// (k_smooth_zero4), black cells last.  Then, in exact arithmetic, the
// residual vanishes at black cells (their update solved their own row) and
// at a red cell, where d z = r, it is the weighted sum of the black
// neighbours, sum_f w_f z_nbr: neither r nor m is read, and the result
// differs from r - A z only by rounding (20 instead of 28 bytes per cell).
// CMP: only the red values are stored, red-compressed: every pair of cells
// (2m, 2m + 1) along x holds one red cell, whose residual goes to res[m],
// so cell l has residual res[l >> 1] if it is red and 0 if it is black
// (18 bytes per cell; k_restrict_red4 reads this form).
template <class T, bool ZG, bool CMP>
__global__ void __launch_bounds__(256, 4) k_residual4(Dims d, Op<T> A, const float* __restrict__ r,
                                                   const float* __restrict__ z, float* __restrict__ res, int pf) {
    const Walk w = walk_of(d);
    if (w.k0 >= w.k1) return;
    Geo g = geo_of(d, w, w.k0);
    float4 zc = ld4(z, g.c);
    float4 zd = ld4(z, g.c + zdn(d, w.k0, w.nxy));
    float4 wzc = ldw4(A.wz, g.c);
    for (int k = w.k0; k < w.k1; k++) {
        if (k > w.k0) g = geo_of(d, w, k);
        if (pf > 0 && k + pf < w.k1) {
            const long long o = g.c + (long long)pf * w.nxy;
            pf2(z, o);
            if (!ZG) {
                pf2(r, o);
                pf2(A.m, o);
            }
            pf2(A.wx, o);
            pf2(A.wy, o);
            pf2(A.wz, o);
        }
        const bool has_zu = k < d.nz - 1 || d.pz;
        const float4 zu = ld4(z, g.c + zup(d, k, w.nxy));
        const float4 wzu = ldw4(A.wz, g.c + (k < d.nz - 1 ? w.nxy : (d.pz ? -(long long)(d.nz - 1) * w.nxy : 0)));
        const float4 wxc = ldw4(A.wx, g.c);
        const Faces4 f = faces_of(A, g, wxc, wzc, wzu, has_zu);
        float L, R;
        xnb(z, g, zc, L, R);
        const float4 zym = ld4(z, g.ym), zyp = ld4(z, g.yp);
        if (ZG) {
            // red = (i + j + k) even; element 0 has i even
            const bool e0_red = ((w.j + k) & 1) == 0;
#define S1(X, LX, RX)                                                                    \
            (f.xl.X * (LX) + f.xu.X * (RX) + f.yl.X * zym.X + f.yu.X * zyp.X + f.zl.X * zd.X + \
             f.zu.X * zu.X)
            float2 h;
            if (e0_red) {
                h.x = S1(x, L, zc.y);
                h.y = S1(z, zc.y, zc.w);
            } else {
                h.x = S1(y, zc.x, zc.z);
                h.y = S1(w, zc.z, R);
            }
#undef S1
            if (w.valid) {
                if (CMP) *reinterpret_cast<float2*>(res + (g.c >> 1)) = h;
                else st4(res, g.c, e0_red ? make_float4(h.x, 0.f, h.y, 0.f) : make_float4(0.f, h.x, 0.f, h.y));
            }
        } else {
            const float4 m = ldw4(A.m, g.c), rc = ld4(r, g.c);
            float4 o;
#define R1(X, LX, RX)                                                                   \
            o.X = rc.X - (m.X * zc.X + f.xl.X * (zc.X - (LX)) + f.xu.X * (zc.X - (RX)) +    \
                          f.yl.X * (zc.X - zym.X) + f.yu.X * (zc.X - zyp.X) +               \
                          f.zl.X * (zc.X - zd.X) + f.zu.X * (zc.X - zu.X));
            R1(x, L, zc.y)
            R1(y, zc.x, zc.z)
            R1(z, zc.y, zc.w)
            R1(w, zc.z, R)
#undef R1
            if (w.valid) st4(res, g.c, o);
        }
        zd = zc;
        zc = zu;
        wzc = wzu;
    }
}

// ------------------------------------------------------------- smoothers

// First red/black Gauss-Seidel sweep from z = 0 (see k_smooth_zero): red
// cells r / diag; black cells (r + sum_f w_f r_nbr / diag_nbr) / diag.
template <class T>
__global__ void __launch_bounds__(256, 4) k_smooth_zero4(Dims d, Op<T> A, const float* __restrict__ r,
                                                      float* __restrict__ z, int pf) {
    const Walk w = walk_of(d);
    if (w.k0 >= w.k1) return;
    auto U = [&](long long i) {
        const float4 a = ld4(r, i), b = ldw4(A.invd, i);
        return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
    };
    auto Us = [&](long long i) { return r[i] * ldw(A.invd, i); };
    Geo g = geo_of(d, w, w.k0);
    float4 uc = U(g.c);
    float4 ud = U(g.c + zdn(d, w.k0, w.nxy));
    float4 wzc = ldw4(A.wz, g.c);
    for (int k = w.k0; k < w.k1; k++) {
        if (k > w.k0) g = geo_of(d, w, k);
        if (pf > 0 && k + pf < w.k1) {
            const long long o = g.c + (long long)pf * w.nxy;
            pf2(r, o);
            pf2(A.invd, o);
            pf2(A.wx, o);
            pf2(A.wy, o);
            pf2(A.wz, o);
        }
        const bool has_zu = k < d.nz - 1 || d.pz;
        const float4 uu = U(g.c + zup(d, k, w.nxy));
        const float4 wzu = ldw4(A.wz, g.c + (k < d.nz - 1 ? w.nxy : (d.pz ? -(long long)(d.nz - 1) * w.nxy : 0)));
        const float4 wxc = ldw4(A.wx, g.c);
        const Faces4 f = faces_of(A, g, wxc, wzc, wzu, has_zu);
        const float lsh = __shfl_up_sync(FULL, uc.w, 1);
        const float rsh = __shfl_down_sync(FULL, uc.x, 1);
        const float L = g.load_l ? Us(g.xl) : lsh;
        const float R = g.load_r ? Us(g.xr) : rsh;
        const float4 uym = U(g.ym), uyp = U(g.yp);
        const float4 rc = ld4(r, g.c), iv = ldw4(A.invd, g.c);
        // parity of element 0: red = (i + j + k) even, i0 = 4 i4 is even
        const bool e0_red = ((w.j + k) & 1) == 0;
        float4 o;
#define B1(X, LX, RX)                                                                       \
        (iv.X * (rc.X + f.xl.X * (LX) + f.xu.X * (RX) + f.yl.X * uym.X + f.yu.X * uyp.X +  \
                 f.zl.X * ud.X + f.zu.X * uu.X))
        if (e0_red) {
            o.x = uc.x;
            o.y = B1(y, uc.x, uc.z);
            o.z = uc.z;
            o.w = B1(w, uc.z, R);
        } else {
            o.x = B1(x, L, uc.y);
            o.y = uc.y;
            o.z = B1(z, uc.y, uc.w);
            o.w = uc.w;
        }
#undef B1
        if (w.valid) st4(z, g.c, o);
        ud = uc;
        uc = uu;
        wzc = wzu;
    }
}

// One colour of a red/black Gauss-Seidel sweep, in place: the cells of the
// other colour are read, never written, so the in-place update is exact.
// With dot (the last sweep of a V-cycle's post-smoothing on the finest
// level) it also forms <r, z> of the finished z for CG.
template <class T, bool DOT>
__global__ void __launch_bounds__(256, 4) k_rb_colour4(Dims d, Op<T> A, const float* __restrict__ r,
                                                    float* z, int colour, RedArgs ra, int pf) {
    const Walk w = walk_of(d);
    DotAcc<float> da;
    if (w.k0 < w.k1) {
        Geo g = geo_of(d, w, w.k0);
        float4 zc = ld4(z, g.c);
        float4 zd = ld4(z, g.c + zdn(d, w.k0, w.nxy));
        float4 wzc = ldw4(A.wz, g.c);
        for (int k = w.k0; k < w.k1; k++) {
            if (k > w.k0) g = geo_of(d, w, k);
            if (pf > 0 && k + pf < w.k1) {
                const long long o = g.c + (long long)pf * w.nxy;
                pf2(z, o);
                pf2(r, o);
                pf2(A.invd, o);
                pf2(A.wx, o);
                pf2(A.wy, o);
                pf2(A.wz, o);
            }
            const bool has_zu = k < d.nz - 1 || d.pz;
            const float4 zu = ld4(z, g.c + zup(d, k, w.nxy));
            const float4 wzu = ldw4(A.wz, g.c + (k < d.nz - 1 ? w.nxy : (d.pz ? -(long long)(d.nz - 1) * w.nxy : 0)));
            const float4 wxc = ldw4(A.wx, g.c);
            const Faces4 f = faces_of(A, g, wxc, wzc, wzu, has_zu);
            float L, R;
            xnb(z, g, zc, L, R);
            const float4 zym = ld4(z, g.ym), zyp = ld4(z, g.yp);
            const float4 rc = ld4(r, g.c), iv = ldw4(A.invd, g.c);
            const bool e0_mine = ((w.j + k + colour) & 1) == 0;
            float4 o = zc;
#define U1(X, LX, RX)                                                                       \
            (iv.X * (rc.X + f.xl.X * (LX) + f.xu.X * (RX) + f.yl.X * zym.X + f.yu.X * zyp.X +  \
                     f.zl.X * zd.X + f.zu.X * zu.X))
            if (e0_mine) {
                o.x = U1(x, L, zc.y);
                o.z = U1(z, zc.y, zc.w);
            } else {
                o.y = U1(y, zc.x, zc.z);
                o.w = U1(w, zc.z, R);
            }
#undef U1
            // z-neighbour values are of the other colour in the planes k +- 1
            // and are not modified by this sweep, so rotating the loaded
            // values is exact
            if (w.valid) {
                st4(z, g.c, o);
                if (DOT) {
                    da.add(rc.x, o.x);
                    da.add(rc.y, o.y);
                    da.add(rc.z, o.z);
                    da.add(rc.w, o.w);
                }
            }
            zd = o;
            zc = zu;
            wzc = wzu;
        }
    }
    if (DOT) {
        double acc[1] = {da.value()};
        const bool mx[1] = {false};
        grid_reduce<1>(acc, mx, ra);
    }
}

// ------------------------------------------------ fused post-smoothing sweep

// One post-smoothing sweep, black then red (see k_rb_colour4), in a single
// pass and out of place: zi holds the pre-smoothed z plus the coarse
// correction, zo receives the smoothed z.  A block is 32 lanes (4 cells
// each) by PBY + 2 rows.  Lanes 0 and 31 and the first and last rows are
// halo threads that only form black values: every red cell of the inner
// lanes and rows then finds its black neighbours in the block (x by warp
// shuffle, y in shared memory, z in registers), and no cell is formed
// twice by one thread.  A block walks its chunk of planes with a one-plane
// lag: at plane p it forms the black values of plane p + 1 (from zi, which
// nothing writes) and the red values of plane p.  The black values are
// double-buffered in shared memory, so one barrier per plane suffices.
// Reading only zi keeps blocks independent, so the result equals the two
// separate colour sweeps.
constexpr int PBY = 6;
constexpr int PLANES_X = 30;   // inner lanes of a block row

namespace {

__device__ __forceinline__ int wrapc(int v, int n, int periodic) {
    if (v < 0) return periodic ? v + n : 0;
    if (v >= n) return periodic ? v - n : n - 1;
    return v;
}

// plane index of plane q with the boundary rule of the z axis
__device__ __forceinline__ int plane_of(int q, const Dims& d) { return wrapc(q, d.nz, d.pz); }

}  // namespace

template <bool DOT>
__global__ void __launch_bounds__(256, 3) k_post_smooth4(Dims d, Op<float> A, const float* __restrict__ r,
                                                      const float* __restrict__ zi, float* __restrict__ zo,
                                                      RedArgs ra, int pf) {
    __shared__ float4 sB[2][PBY + 2][32];
    const int nx4 = d.nx >> 2;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i4raw = (int)blockIdx.x * PLANES_X - 1 + tx;
    const int i4 = wrapc(i4raw, nx4, d.px);
    const int i0 = 4 * i4;
    const int jraw = (int)blockIdx.y * PBY - 1 + ty;
    const int j = wrapc(jraw, d.ny, d.py);
    const bool inner = tx >= 1 && tx <= PLANES_X && ty >= 1 && ty <= PBY && i4raw < nx4 && jraw < d.ny;
    const long long nxy = (long long)d.nx * d.ny;
    const long long rowoff = (long long)j * d.nx;
    const int jd = wrapc(j - 1, d.ny, d.py), ju = wrapc(j + 1, d.ny, d.py);
    const bool has_yp = j < d.ny - 1 || d.py;
    // the halo lanes take their outer x-neighbour from memory
    const bool load_l = tx == 0;
    const bool load_r = tx == 31;
    const bool has_xr = i0 + 4 < d.nx || d.px;
    const int xl = i0 > 0 ? i0 - 1 : (d.px ? d.nx - 1 : 0);
    const int xr = i0 + 4 < d.nx ? i0 + 4 : (d.px ? 0 : d.nx - 1);
    const int kch = (d.nz + (int)gridDim.z - 1) / (int)gridDim.z;
    const int k0 = (int)blockIdx.z * kch, k1 = min(d.nz, k0 + kch);
    DotAcc<float> da;

    // face weights of the four cells of this thread on plane q
    auto faces = [&](int q, Faces4& f) {
        const long long c = (long long)q * nxy + rowoff + i0;
        const float4 wxc = ld4(A.wx, c);
        const float rsh = __shfl_down_sync(FULL, wxc.x, 1);
        const float xu3 = !has_xr ? 0.0f : (load_r ? A.wx[(long long)q * nxy + rowoff + (i0 + 4 < d.nx ? i0 + 4 : 0)] : rsh);
        f.xl = wxc;
        f.xu = make_float4(wxc.y, wxc.z, wxc.w, xu3);
        f.yl = ld4(A.wy, c);
        f.yu = has_yp ? ld4(A.wy, (long long)q * nxy + (long long)ju * d.nx + i0) : make_float4(0.f, 0.f, 0.f, 0.f);
        f.zl = ld4(A.wz, c);
        const bool has_zu = q < d.nz - 1 || d.pz;
        f.zu = has_zu ? ld4(A.wz, (long long)plane_of(q + 1, d) * nxy + rowoff + i0) : make_float4(0.f, 0.f, 0.f, 0.f);
    };

    // black values of plane q (cells of the other colour copied) from zi;
    // cd, cc, cu: zi of planes q-1, q, q+1 at this thread's cells
    auto black = [&](int q, float4 cd, float4 cc, float4 cu) {
        Faces4 f;
        faces(q, f);
        const long long c = (long long)q * nxy + rowoff + i0;
        const float lsh = __shfl_up_sync(FULL, cc.w, 1);
        const float rsh = __shfl_down_sync(FULL, cc.x, 1);
        const float L = load_l ? zi[(long long)q * nxy + rowoff + xl] : lsh;
        const float R = load_r ? zi[(long long)q * nxy + rowoff + xr] : rsh;
        const float4 ym = ld4(zi, (long long)q * nxy + (long long)jd * d.nx + i0);
        const float4 yp = ld4(zi, (long long)q * nxy + (long long)ju * d.nx + i0);
        const float4 rc = ld4(r, c), iv = ld4(A.invd, c);
        const bool e0_black = ((j + q) & 1) == 1;
        float4 o = cc;
#define U1(X, LX, RX)                                                                      \
        (iv.X * (rc.X + f.xl.X * (LX) + f.xu.X * (RX) + f.yl.X * ym.X + f.yu.X * yp.X +   \
                 f.zl.X * cd.X + f.zu.X * cu.X))
        if (e0_black) {
            o.x = U1(x, L, cc.y);
            o.z = U1(z, cc.y, cc.w);
        } else {
            o.y = U1(y, cc.x, cc.z);
            o.w = U1(w, cc.z, R);
        }
#undef U1
        return o;
    };

    if (k0 < k1) {
        // zi at planes p, p+1, p+2 (rolling) and black values at p-1, p, p+1
        const int pm1 = plane_of(k0 - 1, d), pm2 = plane_of(k0 - 2, d);
        float4 zq0 = ld4(zi, (long long)pm2 * nxy + rowoff + i0);   // plane k0-2
        float4 zq1 = ld4(zi, (long long)pm1 * nxy + rowoff + i0);   // plane k0-1
        float4 zq2 = ld4(zi, (long long)k0 * nxy + rowoff + i0);    // plane k0
        float4 Bd = black(pm1, zq0, zq1, zq2);                      // B_{k0-1}
        float4 zq3 = ld4(zi, (long long)plane_of(k0 + 1, d) * nxy + rowoff + i0);
        float4 Bc = black(k0, zq1, zq2, zq3);                       // B_{k0}
        sB[k0 & 1][ty][tx] = Bc;
        __syncthreads();
        // now zq2 = z_{k0}, zq3 = z_{k0+1}
        for (int p = k0; p < k1; p++) {
            const int pu = plane_of(p + 1, d);
            // the black front reads zi of plane p + 2 and the operator of
            // plane p + 1: prefetch those pf planes further on
            if (pf > 0 && p + 2 + pf < d.nz && p + 1 + pf <= k1) {
                const long long o = (long long)(p + 1 + pf) * nxy + rowoff + i0;
                pf2(zi, o + nxy);
                pf2(r, o);
                pf2(A.invd, o);
                pf2(A.wx, o);
                pf2(A.wy, o);
                pf2(A.wz, o + nxy);
            }
            const float4 zq4 = ld4(zi, (long long)plane_of(p + 2, d) * nxy + rowoff + i0);
            const float4 Bu = black(pu, zq2, zq3, zq4);             // B_{p+1}
            // buffer (p+1) & 1 was last read in the previous plane, before
            // the barrier that ended it
            sB[(p + 1) & 1][ty][tx] = Bu;
            // red values of plane p from the black ones (inner threads)
            Faces4 f;
            faces(p, f);
            const long long c = (long long)p * nxy + rowoff + i0;
            const float4 rc = ld4(r, c), iv = ld4(A.invd, c);
            const bool e0_red = ((j + p) & 1) == 0;
            const float L = __shfl_up_sync(FULL, Bc.w, 1);
            const float R = __shfl_down_sync(FULL, Bc.x, 1);
            const float4 ym = sB[p & 1][ty > 0 ? ty - 1 : 0][tx];
            const float4 yp = sB[p & 1][ty < PBY + 1 ? ty + 1 : PBY + 1][tx];
            float4 o = Bc;
#define V1(X, LX, RX)                                                                      \
            (iv.X * (rc.X + f.xl.X * (LX) + f.xu.X * (RX) + f.yl.X * ym.X + f.yu.X * yp.X +   \
                     f.zl.X * Bd.X + f.zu.X * Bu.X))
            if (e0_red) {
                o.x = V1(x, L, Bc.y);
                o.z = V1(z, Bc.y, Bc.w);
            } else {
                o.y = V1(y, Bc.x, Bc.z);
                o.w = V1(w, Bc.z, R);
            }
#undef V1
            if (inner) {
                st4(zo, c, o);
                if (DOT) {
                    da.add(rc.x, o.x);
                    da.add(rc.y, o.y);
                    da.add(rc.z, o.z);
                    da.add(rc.w, o.w);
                }
            }
            __syncthreads();
            Bd = Bc;
            Bc = Bu;
            zq2 = zq3;
            zq3 = zq4;
        }
    }
    if (DOT) {
        double acc[1] = {da.value()};
        const bool mx[1] = {false};
        grid_reduce<1>(acc, mx, ra);
    }
}

// The trilinear interpolation's x step for a thread's four fine cells from
// coarse cells I (c0), I + 1 (c1) and their outer neighbours I - 1 (cm) and
// I + 2 (cp): weights 3/4 for the nearer coarse cell, 1/4 for the farther.
__device__ __forceinline__ float4 xinterp(float c0, float c1, float cm, float cp) {
    return make_float4(fmaf(0.75f, c0, 0.25f * cm), fmaf(0.75f, c0, 0.25f * c1), fmaf(0.75f, c1, 0.25f * c0),
                       fmaf(0.75f, c1, 0.25f * cp));
}

// The y and z steps: rows a (nearer, 3/4) and b (farther, 1/4) of the nearer
// coarse plane (0, 3/4) and of the farther one (1, 1/4), summed in that order.
__device__ __forceinline__ float4 pcomb(float4 a0, float4 b0, float4 a1, float4 b1) {
    const float w0 = 0.75f * 0.75f, w1 = 0.25f * 0.75f, w2 = 0.75f * 0.25f, w3 = 0.25f * 0.25f;
    float4 r;
    r.x = fmaf(w3, b1.x, fmaf(w2, a1.x, fmaf(w1, b0.x, w0 * a0.x)));
    r.y = fmaf(w3, b1.y, fmaf(w2, a1.y, fmaf(w1, b0.y, w0 * a0.y)));
    r.z = fmaf(w3, b1.z, fmaf(w2, a1.z, fmaf(w1, b0.z, w0 * a0.z)));
    r.w = fmaf(w3, b1.w, fmaf(w2, a1.w, fmaf(w1, b0.w, w0 * a0.w)));
    return r;
}

// Out-of-place prolongation: zo = z + P ec (see k_prolong_add4).
__global__ void __launch_bounds__(256) k_prolong_to4(Dims f, Dims cd, const float* __restrict__ ec,
                                                     const float* __restrict__ z, float* __restrict__ zo) {
    const Walk w = walk_of(f);
    if (w.k0 >= w.k1) return;
    const int I = 2 * w.i4;
    const int xm = wrapc(I - 1, cd.nx, cd.px), xp = wrapc(I + 2, cd.nx, cd.px);
    // coarse cells I, I+1 as one float2, I-1 and I+2 from the adjacent lanes
    // (see k_prolong_add4)
    const bool load_l = threadIdx.x == 0 || I == 0;
    const bool load_r = threadIdx.x == blockDim.x - 1 || I + 2 >= cd.nx;
    const int J0 = w.j >> 1;
    const int J1 = wrapc((w.j & 1) ? J0 + 1 : J0 - 1, cd.ny, cd.py);
    const long long cxy = (long long)cd.nx * cd.ny;
    for (int k = w.k0; k < w.k1; k++) {
        const int K0 = k >> 1;
        const int K1 = wrapc((k & 1) ? K0 + 1 : K0 - 1, cd.nz, cd.pz);
        float4 X[4];   // rows (J0, K0), (J1, K0), (J0, K1), (J1, K1), x-interpolated
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int Jq = (q & 1) ? J1 : J0;
            const int Kq = (q & 2) ? K1 : K0;
            const long long row = (long long)Kq * cxy + (long long)Jq * cd.nx;
            const float2 cc = *reinterpret_cast<const float2*>(ec + row + I);
            const float lsh = __shfl_up_sync(FULL, cc.y, 1);
            const float rsh = __shfl_down_sync(FULL, cc.x, 1);
            const float cm = load_l ? ec[row + xm] : lsh;
            const float cp = load_r ? ec[row + xp] : rsh;
            X[q] = xinterp(cc.x, cc.y, cm, cp);
        }
        const float4 acc = pcomb(X[0], X[1], X[2], X[3]);
        const long long c = (long long)k * w.nxy + (long long)w.j * f.nx + 4 * w.i4;
        if (w.valid) {
            float4 v = ld4(z, c);
            v.x += acc.x;
            v.y += acc.y;
            v.z += acc.z;
            v.w += acc.w;
            st4(zo, c, v);
        }
    }
}

// ---------------------------------------------------------------- transfers

// Full-weighting restriction rc = P^T rf / 8 (see k_restrict): per axis the
// fine taps 2I-1, 2I, 2I+1, 2I+2 with weights 1/4, 3/4, 3/4, 1/4, a tap
// outside a zero-gradient boundary folding onto the boundary cell and one
// outside a periodic boundary wrapping.  A thread owns coarse cells 2t and
// 2t+1 of a row and walks coarse planes, keeping the x-y sums of the two
// fine planes it shares with the next coarse plane.
__device__ __forceinline__ int fold(int f, int n, int periodic) {
    if (f < 0) return periodic ? f + n : 0;
    if (f >= n) return periodic ? f - n : n - 1;
    return f;
}

// x-y weighted sums of fine plane fz for coarse cells (2t, J) and (2t+1, J)
__device__ __forceinline__ float2 xy_sum(const Dims& f, const float* __restrict__ rf, int t, int J,
                                         int fz, bool load_l, bool load_r) {
    const float wv[4] = {0.25f, 0.75f, 0.75f, 0.25f};
    float2 acc = make_float2(0.f, 0.f);
    const long long plane = (long long)fz * f.nx * f.ny;
    const int x0 = 4 * t;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int fy = fold(2 * J - 1 + q, f.ny, f.py);
        const long long row = plane + (long long)fy * f.nx;
        const float4 v = ld4(rf, row + x0);
        const float lsh = __shfl_up_sync(FULL, v.w, 1);
        const float rsh = __shfl_down_sync(FULL, v.x, 1);
        const float L = load_l ? rf[row + fold(x0 - 1, f.nx, f.px)] : lsh;
        const float R = load_r ? rf[row + fold(x0 + 4, f.nx, f.px)] : rsh;
        const float a = 0.25f * L + 0.75f * v.x + 0.75f * v.y + 0.25f * v.z;
        const float b = 0.25f * v.y + 0.75f * v.z + 0.75f * v.w + 0.25f * R;
        acc.x = fmaf(wv[q], a, acc.x);
        acc.y = fmaf(wv[q], b, acc.y);
    }
    return acc;
}

// Residual of fine cell `row + x` from its red-compressed form.
__device__ __forceinline__ float red_res(const float* __restrict__ rf, long long row, int x, int fy, int fz) {
    return ((x + fy + fz) & 1) == 0 ? rf[(row + x) >> 1] : 0.0f;
}

// x-y weighted sums of fine plane fz (offset pbase = fz nx ny) for coarse
// cells 4t .. 4t+3 of a coarse row, from a red-compressed residual: one
// float4 per fine row holds the red values of fine cells x0 .. x0+7 (x0 =
// 8t).  The four fine rows fy[q] (offsets ry[q] = fy[q] nx, folded at the
// boundary once per thread) are weighted 1/4, 3/4, 3/4, 1/4.  In a row
// whose even cells are red, coarse cell i takes 3/4 of its own red value
// and 1/4 of the next one (the one after the last from the next lane); with
// odd red cells, 1/4 of the previous one.  xl, xr: the folded fine cells
// x0 - 1 and x0 + 8, read directly by the lanes at a block or grid edge.
__device__ __forceinline__ float4 xy_sum_red(const float* __restrict__ rf, long long pbase, const int (&fy)[4],
                                             const int (&ry)[4], int fz, int x0, int xl, int xr, bool load_l,
                                             bool load_r) {
    const float wv[4] = {0.25f, 0.75f, 0.75f, 0.25f};
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const long long row = pbase + ry[q];
        const float4 h = ld4(rf, (row + x0) >> 1);
        const bool e = ((fy[q] + fz) & 1) == 0;   // the even cells of the row are red
        const float lsh = __shfl_up_sync(FULL, h.w, 1);
        const float rsh = __shfl_down_sync(FULL, h.x, 1);
        const float L = load_l ? red_res(rf, row, xl, fy[q], fz) : (e ? 0.f : lsh);
        const float R = load_r ? red_res(rf, row, xr, fy[q], fz) : (e ? rsh : 0.f);
        const float c0 = fmaf(0.75f, h.x, 0.25f * ((e ? h.y : 0.f) + L));
        const float c1 = fmaf(0.75f, h.y, 0.25f * (e ? h.z : h.x));
        const float c2 = fmaf(0.75f, h.z, 0.25f * (e ? h.w : h.y));
        const float c3 = fmaf(0.75f, h.w, 0.25f * ((e ? 0.f : h.z) + R));
        acc.x = fmaf(wv[q], c0, acc.x);
        acc.y = fmaf(wv[q], c1, acc.y);
        acc.z = fmaf(wv[q], c2, acc.z);
        acc.w = fmaf(wv[q], c3, acc.w);
    }
    return acc;
}

__global__ void __launch_bounds__(256) k_restrict4(Dims f, Dims cd, const float* __restrict__ rf,
                                                   float* __restrict__ rc, int pf) {
    const int ht = cd.nx >> 1;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int J0 = blockIdx.y * blockDim.y + threadIdx.y;
    const bool valid = t0 < ht && J0 < cd.ny;
    const int t = min(t0, ht - 1), J = min(J0, cd.ny - 1);
    const int kch = (cd.nz + (int)gridDim.z - 1) / (int)gridDim.z;
    const int K0 = (int)blockIdx.z * kch, K1 = min(cd.nz, K0 + kch);
    if (K0 >= K1) return;
    // the adjacent lane holds the neighbouring fine float4 of the same row
    // unless it is the first / last lane of the block row or the row ends
    const bool load_l = threadIdx.x == 0 || t == 0;
    const bool load_r = threadIdx.x == blockDim.x - 1 || t == ht - 1;
    float2 s0 = xy_sum(f, rf, t, J, fold(2 * K0 - 1, f.nz, f.pz), load_l, load_r);
    float2 s1 = xy_sum(f, rf, t, J, 2 * K0, load_l, load_r);
    for (int K = K0; K < K1; K++) {
        // this thread's own fine rows 2J, 2J + 1 of the two fine planes the
        // walk reads pf coarse planes on
        if (pf > 0 && K + pf < K1) {
            const long long o = (long long)(2 * (K + pf) + 1) * f.nx * f.ny + (long long)(2 * J) * f.nx + 4 * t;
            pf2(rf, o);
            pf2(rf, o + f.nx);
            if (2 * (K + pf) + 2 < f.nz) {
                pf2(rf, o + (long long)f.nx * f.ny);
                pf2(rf, o + (long long)f.nx * f.ny + f.nx);
            }
        }
        const float2 s2 = xy_sum(f, rf, t, J, 2 * K + 1, load_l, load_r);
        const float2 s3 = xy_sum(f, rf, t, J, fold(2 * K + 2, f.nz, f.pz), load_l, load_r);
        float2 o;
        o.x = 0.125f * (0.25f * s0.x + 0.75f * s1.x + 0.75f * s2.x + 0.25f * s3.x);
        o.y = 0.125f * (0.25f * s0.y + 0.75f * s1.y + 0.75f * s2.y + 0.25f * s3.y);
        if (valid)
            *reinterpret_cast<float2*>(rc + (long long)K * cd.nx * cd.ny + (long long)J * cd.nx + 2 * t) = o;
        s0 = s2;
        s1 = s3;
    }
}

// k_restrict4 for a red-compressed residual (k_residual4 after a
// zero-guess sweep): a thread owns coarse cells 4t .. 4t+3 of a row, one
// float4 of compressed values per fine row (fine nx a multiple of 8).
__global__ void __launch_bounds__(256) k_restrict_red4(Dims f, Dims cd, const float* __restrict__ rf,
                                                       float* __restrict__ rc, int pf) {
    const int qt = cd.nx >> 2;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int J0 = blockIdx.y * blockDim.y + threadIdx.y;
    const bool valid = t0 < qt && J0 < cd.ny;
    const int t = min(t0, qt - 1), J = min(J0, cd.ny - 1);
    const int kch = (cd.nz + (int)gridDim.z - 1) / (int)gridDim.z;
    const int K0 = (int)blockIdx.z * kch, K1 = min(cd.nz, K0 + kch);
    if (K0 >= K1) return;
    const bool load_l = threadIdx.x == 0 || t == 0;
    const bool load_r = threadIdx.x == blockDim.x - 1 || t == qt - 1;
    int fy[4], ry[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        fy[q] = fold(2 * J - 1 + q, f.ny, f.py);
        ry[q] = fy[q] * f.nx;
    }
    const int x0 = 8 * t, xl = fold(x0 - 1, f.nx, f.px), xr = fold(x0 + 8, f.nx, f.px);
    const long long nxy = (long long)f.nx * f.ny;
    auto sum = [&](int fz) { return xy_sum_red(rf, fz * nxy, fy, ry, fz, x0, xl, xr, load_l, load_r); };
    float4 s0 = sum(fold(2 * K0 - 1, f.nz, f.pz));
    float4 s1 = sum(2 * K0);
    for (int K = K0; K < K1; K++) {
        if (pf > 0 && K + pf < K1) {
            const long long o = (long long)(2 * (K + pf) + 1) * f.nx * f.ny + (long long)(2 * J) * f.nx + 8 * t;
            pf2(rf, o >> 1);
            pf2(rf, (o + f.nx) >> 1);
            if (2 * (K + pf) + 2 < f.nz) {
                pf2(rf, (o + (long long)f.nx * f.ny) >> 1);
                pf2(rf, (o + (long long)f.nx * f.ny + f.nx) >> 1);
            }
        }
        const float4 s2 = sum(2 * K + 1);
        const float4 s3 = sum(fold(2 * K + 2, f.nz, f.pz));
        float4 o;
        o.x = 0.125f * (0.25f * s0.x + 0.75f * s1.x + 0.75f * s2.x + 0.25f * s3.x);
        o.y = 0.125f * (0.25f * s0.y + 0.75f * s1.y + 0.75f * s2.y + 0.25f * s3.y);
        o.z = 0.125f * (0.25f * s0.z + 0.75f * s1.z + 0.75f * s2.z + 0.25f * s3.z);
        o.w = 0.125f * (0.25f * s0.w + 0.75f * s1.w + 0.75f * s2.w + 0.25f * s3.w);
        if (valid) st4(rc, (long long)K * cd.nx * cd.ny + (long long)J * cd.nx + 4 * t, o);
        s0 = s2;
        s1 = s3;
    }
}

// Trilinear prolongation and correction zf += P ec (see k_prolong_add): a
// thread owns four fine cells along x, which interpolate from coarse cells
// 2 i4 - 1 .. 2 i4 + 2 of two coarse rows (J0 = j / 2 and its neighbour
// towards j) in two coarse planes (K0 = k / 2 and its neighbour towards k).
// Fine planes 2K - 1 .. 2K + 2 all read coarse plane K, so the thread keeps
// the x-interpolated rows of the window of coarse planes K - 1, K, K + 1
// around K = k / 2 in registers and interpolates one new coarse plane every
// second fine plane (one coarse row per fine plane, against four).
__global__ void __launch_bounds__(256) k_prolong_add4(Dims f, Dims cd, const float* __restrict__ ec,
                                                      float* __restrict__ zf, int pf) {
    const Walk w = walk_of(f);
    if (w.k0 >= w.k1) return;
    const int I = 2 * w.i4;
    const int xm = fold(I - 1, cd.nx, cd.px), xp = fold(I + 2, cd.nx, cd.px);
    // coarse cells I, I+1 are one aligned float2 (cd.nx is even); I-1 and
    // I+2 are the neighbouring lanes' unless this lane starts or ends its
    // block row or the coarse row
    const bool load_l = threadIdx.x == 0 || I == 0;
    const bool load_r = threadIdx.x == blockDim.x - 1 || I + 2 >= cd.nx;
    const int J0 = w.j >> 1;
    const int J1 = fold((w.j & 1) ? J0 + 1 : J0 - 1, cd.ny, cd.py);
    const long long cxy = (long long)cd.nx * cd.ny;
    // rows J0 (a) and J1 (b) of coarse plane K, x-interpolated
    auto rows = [&](int K, float4& a, float4& b) {
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const long long row = (long long)K * cxy + (long long)(q ? J1 : J0) * cd.nx;
            const float2 cc = *reinterpret_cast<const float2*>(ec + row + I);
            const float lsh = __shfl_up_sync(FULL, cc.y, 1);
            const float rsh = __shfl_down_sync(FULL, cc.x, 1);
            const float cm = load_l ? ec[row + xm] : lsh;
            const float cp = load_r ? ec[row + xp] : rsh;
            const float4 v = xinterp(cc.x, cc.y, cm, cp);
            if (q) b = v;
            else a = v;
        }
    };
    int K = w.k0 >> 1;
    float4 am, bm, a0, b0, ap, bp;
    rows(fold(K - 1, cd.nz, cd.pz), am, bm);
    rows(K, a0, b0);
    rows(fold(K + 1, cd.nz, cd.pz), ap, bp);
    for (int k = w.k0; k < w.k1; k++) {
        if (k > w.k0 && (k & 1) == 0) {
            // the window moves up one coarse plane
            K = k >> 1;
            am = a0;
            bm = b0;
            a0 = ap;
            b0 = bp;
            rows(fold(K + 1, cd.nz, cd.pz), ap, bp);
        }
        if (pf > 0 && k + pf < w.k1)
            pf2(zf, (long long)(k + pf) * w.nxy + (long long)w.j * f.nx + 4 * w.i4);
        // the second coarse plane: K + 1 for odd fine planes, K - 1 for even
        const bool odd = (k & 1) != 0;
        const float4 acc = pcomb(a0, b0, odd ? ap : am, odd ? bp : bm);
        const long long c = (long long)k * w.nxy + (long long)w.j * f.nx + 4 * w.i4;
        if (w.valid) {
            float4 z = ld4(zf, c);
            z.x += acc.x;
            z.y += acc.y;
            z.z += acc.z;
            z.w += acc.w;
            st4(zf, c, z);
        }
    }
}

// ------------------------------------------------------------ flat vectors

// The bfloat16 copies of a level's smoothing coefficients (nearest, as the
// assembly writes the fine level's).
__global__ void __launch_bounds__(256) k_op_to_bf16(long long n4, Op<float> A, Op<unsigned short> B) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4;
         q += (long long)gridDim.x * blockDim.x) {
        const long long i = 4 * q;
        const float* src[4] = {A.wx, A.wy, A.wz, A.invd};
        unsigned short* dst[4] = {B.wx, B.wy, B.wz, B.invd};
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const float4 v = ld4(src[a], i);
            const unsigned lo = (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(v.x)) |
                                ((unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(v.y)) << 16);
            const unsigned hi = (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(v.z)) |
                                ((unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(v.w)) << 16);
            *reinterpret_cast<uint2*>(dst[a] + i) = make_uint2(lo, hi);
        }
    }
}

__global__ void __launch_bounds__(RED_THREADS) k_dot4(long long n4, const float* __restrict__ a,
                                                      const float* __restrict__ b, RedArgs ra) {
    DotAcc<float> da;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n4;
         c += (long long)gridDim.x * blockDim.x) {
        const float4 x = ld4(a, 4 * c), y = ld4(b, 4 * c);
        da.add(x.x, y.x);
        da.add(x.y, y.y);
        da.add(x.z, y.z);
        da.add(x.w, y.w);
    }
    double acc[1] = {da.value()};
    const bool mx[1] = {false};
    grid_reduce<1>(acc, mx, ra);
}

// x += alpha p;  r -= alpha q;  ||r||^2
// x += alpha p (X; without it the update of x is deferred to the next
// k_cg_p_matvec4), r -= alpha q, ||r||^2.
template <bool X>
__global__ void __launch_bounds__(RED_THREADS) k_cg_update4(long long n4, float* __restrict__ x,
                                                            float* __restrict__ r, const float* __restrict__ p,
                                                            const float* __restrict__ q, RedArgs ra) {
    const float alpha = (float)ra.sc[S_ALPHA];
    DotAcc<float> da;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n4;
         c += (long long)gridDim.x * blockDim.x) {
        float4 rv = ld4(r, 4 * c);
        const float4 qv = ld4(q, 4 * c);
        if (X) {
            float4 xv = ld4(x, 4 * c);
            const float4 pv = ld4(p, 4 * c);
            xv.x = fmaf(alpha, pv.x, xv.x); xv.y = fmaf(alpha, pv.y, xv.y);
            xv.z = fmaf(alpha, pv.z, xv.z); xv.w = fmaf(alpha, pv.w, xv.w);
            st4(x, 4 * c, xv);
        }
        rv.x = fmaf(-alpha, qv.x, rv.x); rv.y = fmaf(-alpha, qv.y, rv.y);
        rv.z = fmaf(-alpha, qv.z, rv.z); rv.w = fmaf(-alpha, qv.w, rv.w);
        st4(r, 4 * c, rv);
        da.add(rv.x, rv.x);
        da.add(rv.y, rv.y);
        da.add(rv.z, rv.z);
        da.add(rv.w, rv.w);
    }
    double acc[1] = {da.value()};
    const bool mx[1] = {false};
    grid_reduce<1>(acc, mx, ra);
}

// ---------------------------------------------------------------- launchers

void launch_op_to_bf16(long long n, Op<float> A, Op<unsigned short> B, cudaStream_t s) {
    k_op_to_bf16<<<grid_blocks(n / 4, 256), 256, 0, s>>>(n / 4, A, B);
}

void launch_dot4(long long n, const float* a, const float* b, const RedArgs& ra, cudaStream_t s) {
    k_dot4<<<red_blocks(n / 4), RED_THREADS, 0, s>>>(n / 4, a, b, ra);
}
void launch_cg_update4(long long n, float* x, float* r, const float* p, const float* q,
                       const RedArgs& ra, cudaStream_t s) {
    if (x) k_cg_update4<true><<<red_blocks(n / 4), RED_THREADS, 0, s>>>(n / 4, x, r, p, q, ra);
    else k_cg_update4<false><<<red_blocks(n / 4), RED_THREADS, 0, s>>>(n / 4, x, r, p, q, ra);
}

static ColShape shape4(const Dims& d, const Tune& tn = Tune{}) {
    Dims h = d;
    h.nx = d.nx / 4;
    ColShape s = col_shape(h, tn.threads, tn.target);
    return s;
}

// Blocks of 32 lanes (30 inner) by PBY + 2 rows (PBY inner); the z chunk
// follows from the target number of blocks.
static ColShape shape_post4(const Dims& d, int target = 152 * 8) {
    const int nx4 = d.nx / 4;
    ColShape s;
    const int gx = (nx4 + PLANES_X - 1) / PLANES_X, gy = (d.ny + PBY - 1) / PBY;
    long long xy = (long long)gx * gy;
    long long gz = (target + xy - 1) / xy;
    if (gz > d.nz) gz = d.nz;
    if (xy * gz > RED_MAX_BLOCKS) gz = RED_MAX_BLOCKS / xy;
    if (gz < 1) gz = 1;
    s.block = dim3(32, PBY + 2, 1);
    s.grid = dim3(gx, gy, (unsigned)gz);
    return s;
}

// the fused sweep needs full warps of lanes: at least 32 float4 columns
bool post4_ok(const Dims& d) {
    const int nx4 = d.nx / 4;
    return fine4_ok(d) && nx4 >= 32 &&
           (long long)((nx4 + PLANES_X - 1) / PLANES_X) * ((d.ny + PBY - 1) / PBY) <= RED_MAX_BLOCKS;
}

void launch_post_smooth4(const Dims& d, Op<float> A, const float* r, const float* zi, float* zo,
                         const RedArgs* dot, cudaStream_t s, const Tune& tn) {
    ColShape sh = shape_post4(d, tn.target);
    if (dot) k_post_smooth4<true><<<sh.grid, sh.block, 0, s>>>(d, A, r, zi, zo, *dot, tn.pf);
    else k_post_smooth4<false><<<sh.grid, sh.block, 0, s>>>(d, A, r, zi, zo, RedArgs{}, tn.pf);
}

void launch_prolong_to4(const Dims& f, const Dims& c, const float* ec, const float* z, float* zo,
                        cudaStream_t s) {
    ColShape sh = shape4(f);
    k_prolong_to4<<<sh.grid, sh.block, 0, s>>>(f, c, ec, z, zo);
}


bool fine4_ok(const Dims& d) { return d.nx % 4 == 0 && d.nx >= 16; }

void launch_cg_p_matvec4(const Dims& d, Op<float> A, const float* z, const float* p_in, float* p_out,
                         float* q, const RedArgs& ra, cudaStream_t s, const Tune& tn, float* x) {
    ColShape sh = shape4(d, tn);
    k_cg_p_matvec4<<<sh.grid, sh.block, 0, s>>>(d, A, z, p_in, p_out, q, x, ra, tn.pf);
}
void launch_residual4(const Dims& d, Op<float> A, const float* r, const float* z, float* res,
                      cudaStream_t s, const Tune& tn, bool after_zero_sweep, bool red_compressed) {
    ColShape sh = shape4(d, tn);
    if (after_zero_sweep && red_compressed)
        k_residual4<float, true, true><<<sh.grid, sh.block, 0, s>>>(d, A, r, z, res, tn.pf);
    else if (after_zero_sweep)
        k_residual4<float, true, false><<<sh.grid, sh.block, 0, s>>>(d, A, r, z, res, tn.pf);
    else
        k_residual4<float, false, false><<<sh.grid, sh.block, 0, s>>>(d, A, r, z, res, tn.pf);
}
void launch_residual4(const Dims& d, Op<unsigned short> A, const float* z, float* res, cudaStream_t s,
                      const Tune& tn, bool red_compressed) {
    ColShape sh = shape4(d, tn);
    if (red_compressed)
        k_residual4<unsigned short, true, true><<<sh.grid, sh.block, 0, s>>>(d, A, nullptr, z, res, tn.pf);
    else
        k_residual4<unsigned short, true, false><<<sh.grid, sh.block, 0, s>>>(d, A, nullptr, z, res, tn.pf);
}
bool red_compress_ok(const Dims& f) { return fine4_ok(f) && f.nx % 8 == 0; }

void launch_restrict4(const Dims& f, const Dims& c, const float* rf, float* rc, cudaStream_t s,
                      const Tune& tn, bool red_compressed) {
    Dims h = c;
    if (red_compressed) {
        h.nx = c.nx / 4;
        ColShape sh = col_shape(h, tn.threads, tn.target);
        k_restrict_red4<<<sh.grid, sh.block, 0, s>>>(f, c, rf, rc, tn.pf);
        return;
    }
    h.nx = c.nx / 2;
    ColShape sh = col_shape(h, tn.threads, tn.target);
    k_restrict4<<<sh.grid, sh.block, 0, s>>>(f, c, rf, rc, tn.pf);
}
void launch_prolong_add4(const Dims& f, const Dims& c, const float* ec, float* zf, cudaStream_t s,
                         const Tune& tn) {
    ColShape sh = shape4(f, tn);
    k_prolong_add4<<<sh.grid, sh.block, 0, s>>>(f, c, ec, zf, tn.pf);
}
template <class T>
static void smooth_zero4_t(const Dims& d, Op<T> A, const float* r, float* z, cudaStream_t s, const Tune& tn) {
    ColShape sh = shape4(d, tn);
    k_smooth_zero4<T><<<sh.grid, sh.block, 0, s>>>(d, A, r, z, tn.pf);
}
template <class T>
static void rb_colour4_t(const Dims& d, Op<T> A, const float* r, float* z, int colour, const RedArgs* ra,
                         cudaStream_t s, const Tune& tn) {
    ColShape sh = shape4(d, tn);
    if (ra) k_rb_colour4<T, true><<<sh.grid, sh.block, 0, s>>>(d, A, r, z, colour, *ra, tn.pf);
    else k_rb_colour4<T, false><<<sh.grid, sh.block, 0, s>>>(d, A, r, z, colour, RedArgs{}, tn.pf);
}
void launch_smooth_zero4(const Dims& d, Op<float> A, const float* r, float* z, cudaStream_t s,
                         const Tune& tn) {
    smooth_zero4_t(d, A, r, z, s, tn);
}
void launch_smooth_zero4(const Dims& d, Op<unsigned short> A, const float* r, float* z, cudaStream_t s,
                         const Tune& tn) {
    smooth_zero4_t(d, A, r, z, s, tn);
}
void launch_rb_colour4(const Dims& d, Op<float> A, const float* r, float* z, int colour,
                       cudaStream_t s, const Tune& tn) {
    rb_colour4_t(d, A, r, z, colour, nullptr, s, tn);
}
void launch_rb_colour4(const Dims& d, Op<unsigned short> A, const float* r, float* z, int colour,
                       cudaStream_t s, const Tune& tn) {
    rb_colour4_t(d, A, r, z, colour, nullptr, s, tn);
}
void launch_rb_colour4_dot(const Dims& d, Op<float> A, const float* r, float* z, int colour,
                           const RedArgs& ra, cudaStream_t s, const Tune& tn) {
    rb_colour4_t(d, A, r, z, colour, &ra, s, tn);
}
void launch_rb_colour4_dot(const Dims& d, Op<unsigned short> A, const float* r, float* z, int colour,
                           const RedArgs& ra, cudaStream_t s, const Tune& tn) {
    rb_colour4_t(d, A, r, z, colour, &ra, s, tn);
}

}  // namespace fld
