// k_assemble.cu -- per-cell opacity and per-face flux-limited diffusion
// coefficients of the theta-method correction system (FP64).
//
// Flux limiter (Sec. 2): D = min{ c (9 kappa_f^2 + R^2)^(-1/2), D_max },
// R = max{ |E_2 - E_1| / (h E_f), R_min }, E_f arithmetic and kappa_f
// harmonic face means; Levermore-Pomraning alternative (Sec. 1 citation)
// with lambda(x) = (coth x - 1/x)/x, x = R/kappa_f.
// System (Sec. 3.2, residual-correction form of the theta-method with the
// limiter lagged at E^n): the operator's face weights theta dt D_f / h^2 and
// mass term 1 + theta dt (c kappa + adot/a); the right-hand side
// b = dt eta - dt (c kappa + adot/a) E + sum_f w_f (E_nbr - E) with the full
// weights w_f = dt D_f / h^2.  A Dirichlet face of the box (E = E_b half a
// cell out) adds theta w_b, w_b = dt D_b / (h h/2), to the mass term and
// w_b (E_b - E) to b, with D_b from the limiter of the half-cell face.
#include "limiter.cuh"

namespace fld {

__global__ void __launch_bounds__(256) k_assemble_faces(Dims d, PhysDev p, const double* __restrict__ E,
                                                       const double* __restrict__ nHI,
                                                       const double* __restrict__ eta, Op<double> op,
                                                       Op<float> op32, double* sc, FaceList fl, int zb0,
                                                       int kch) {
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    bool bad = false;
    const bool screen = p.limiter == 0;
    __shared__ unsigned s_cnt;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    // the block's index in the whole grid's decomposition (its face list)
    const long long bid = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * (zb0 + blockIdx.z));
    if (tid == 0) s_cnt = 0u;
    __syncthreads();
    unsigned* seg = fl.entries ? fl.entries + bid * fl.cap : nullptr;
    COL_BEGIN_ZB(d, zb0, kch)
        const double Ec = E[c], nc = nHI[c];
        bad |= !valid_bits(Ec) || !valid_bits(nc) || !valid_bits(eta[c]);
        const double kc = nc * p.sigma;
        const double m = fma(p.mdtcs, nc, p.one_dta);
        bool okc = true;
        const float kL32 = f32_trunc(nc, okc) * p.sigmaL32;
        double w[3];
        float w32[3];
        const int ijk[3] = {i, j, k};
        const int nn[3] = {d.nx, d.ny, d.nz};
        const int per[3] = {d.px, d.py, d.pz};
        const long long st[3] = {1, sy, sz};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            long long lo;
            if (ijk[a] > 0) lo = c - st[a];
            else if (per[a]) lo = c + (long long)(nn[a] - 1) * st[a];
            else { w[a] = 0.0; w32[a] = 0.0f; continue; }
            const double El = E[lo], nl = nHI[lo];
            bool ok = okc;
            float el32, e32;
            pair32(El, Ec, el32, e32, ok);
            const float kLl = f32_trunc(nl, ok) * p.sigmaL32;
            if (screen && ok && capped32(el32, e32, kLl, kL32, p.twoL_h32[a], p.thr32)) {
                w[a] = p.wmax[a];
                w32[a] = p.wmax32[a];
                continue;
            }
            // queue the face for the compacted FP64 pass; compute it here
            // only if this block's list is full
            if (seg) {
                const unsigned pos = atomicAdd(&s_cnt, 1u);
                if (pos < (unsigned)fl.cap) {
                    seg[pos] = ((unsigned)c << 2) | (unsigned)a;
                    w[a] = 0.0;
                    w32[a] = 0.0f;
                    continue;
                }
            }
            const double D = face_D(El, Ec, nl * p.sigma, kc, p.h[a], p);
            w[a] = p.dt_h2[a] * D;
            w32[a] = (float)w[a];
        }
        op.m[c] = m;
        op.wx[c] = w[0];
        op.wy[c] = w[1];
        op.wz[c] = w[2];
        if (op32.m) {
            op32.m[c] = (float)m;
            op32.wx[c] = w32[0];
            op32.wy[c] = w32[1];
            op32.wz[c] = w32[2];
        }
    }
    if (bad) sc[S_BAD] = 1.0;
    __syncthreads();
    if (tid == 0 && seg) fl.counts[bid] = s_cnt < (unsigned)fl.cap ? s_cnt : (unsigned)fl.cap;
}

// The faces the screen left: FP64 limiter with whole warps busy.  Entry
// = (cell << 2) | axis; the face couples the cell with its lower
// neighbour along the axis (wrapping on a periodic axis; zero-gradient
// boundary faces are never listed).
__global__ void __launch_bounds__(256) k_assemble_fix(Dims d, PhysDev p, const double* __restrict__ E,
                                                     const double* __restrict__ nHI, Op<double> op,
                                                     Op<float> op32, FaceList fl) {
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
        const double D = face_D(E[lo], E[c], nHI[lo] * p.sigma, nHI[c] * p.sigma, p.h[a], p);
        const double w = p.dt_h2[a] * D;
        double* W = a == 0 ? op.wx : (a == 1 ? op.wy : op.wz);
        W[c] = w;
        if (op32.m) {
            float* W32 = a == 0 ? op32.wx : (a == 1 ? op32.wy : op32.wz);
            W32[c] = (float)w;
        }
    }
}

// Right-hand side and inverse diagonal.  In mixed mode the FP32 diagonal
// comes from the FP32 weights, so no FP64 division is needed.  BE: theta = 1
// (no rescaling of the flux); DIR: the grid has Dirichlet faces (the
// variant without them carries none of their code or registers).
template <bool BE, bool DIR>
__global__ void __launch_bounds__(RED_THREADS) k_assemble_rhs(Dims d, PhysDev p, const double* __restrict__ E,
                                                             const double* __restrict__ nHI,
                                                             const double* __restrict__ eta, Op<double> op,
                                                             Op<float> op32, double* __restrict__ b,
                                                             double* __restrict__ diag64, Bnd bnd, RedArgs ra,
                                                             int zb0, int kch) {
    const long long sy = d.nx, sz = (long long)d.nx * d.ny;
    double acc[2] = {0.0, 0.0};
    COL_BEGIN_ZB(d, zb0, kch)
        const double Ec = E[c];
        double flux = 0.0, wsum = 0.0;
        float wsum32 = 0.0f;
        // flux = sum_f w_f (E_nbr - E) = sum_f w_f E_nbr - W E, W = sum_f w_f
        // (W is the diagonal's weight sum as well)
        double swe = 0.0;
#define FACE(WARR, W32ARR, wi, nb)                                 \
        {                                                          \
            const double w_ = op.WARR[wi];                         \
            swe = fma(w_, E[nb], swe);                             \
            wsum += w_;                                            \
            if (op32.invd) wsum32 += op32.W32ARR[wi];              \
        }
        if (i > 0) FACE(wx, wx, c, c - 1) else if (d.px) FACE(wx, wx, c, c + d.nx - 1)
        if (i < d.nx - 1) FACE(wx, wx, c + 1, c + 1) else if (d.px) FACE(wx, wx, c - (d.nx - 1), c - (d.nx - 1))
        if (j > 0) FACE(wy, wy, c, c - sy) else if (d.py) FACE(wy, wy, c, c + (long long)(d.ny - 1) * sy)
        if (j < d.ny - 1) FACE(wy, wy, c + sy, c + sy) else if (d.py) FACE(wy, wy, c - (long long)(d.ny - 1) * sy, c - (long long)(d.ny - 1) * sy)
        if (k > 0) FACE(wz, wz, c, c - sz) else if (d.pz) FACE(wz, wz, c, c + (long long)(d.nz - 1) * sz)
        if (k < d.nz - 1) FACE(wz, wz, c + sz, c + sz) else if (d.pz) FACE(wz, wz, c - (long long)(d.nz - 1) * sz, c - (long long)(d.nz - 1) * sz)
#undef FACE
        if (!(BE && !DIR)) flux = fma(-wsum, Ec, swe);
        double m = op.m[c];
        float m32 = op32.invd ? op32.m[c] : 0.0f;
        if (DIR) {
            // Dirichlet faces of the box touching this cell
            const int ijk[3] = {i, j, k};
            const int nn[3] = {d.nx, d.ny, d.nz};
            const double kc = nHI[c] * p.sigma;
            double wb_sum = 0.0;
#pragma unroll
            for (int sd = 0; sd < 6; sd++) {
                const int a = sd >> 1;
                if (!((p.dmask >> sd) & 1) || ijk[a] != ((sd & 1) ? nn[a] - 1 : 0)) continue;
                const double Eb = p.ebc[sd];
                const double wb = 2.0 * p.dt_h2[a] * face_D(Eb, Ec, kc, kc, 0.5 * p.h[a], p);
                const long long f = a == 0 ? j + (long long)d.ny * k
                                           : (a == 1 ? i + (long long)d.nx * k : i + (long long)d.nx * j);
                bnd.w[bnd_offset(d, sd) + f] = wb;
                wb_sum += wb;
                flux = fma(wb, Eb - Ec, flux);
            }
            if (wb_sum != 0.0) {
                m += wb_sum;
                op.m[c] = m;
                if (op32.m) {
                    m32 = (float)m;
                    op32.m[c] = m32;
                }
            }
        }
        double bc;
        if (BE && !DIR) {
            // b = dt eta + sum_f w_f E_nbr - (W + dt (c kappa + adot/a)) E
            const double sc = fma(p.dtcs, nHI[c], p.dta);
            bc = fma(-(wsum + sc), Ec, fma(p.dt, eta[c], swe));
        } else {
            // the right-hand side takes the full weights, the operator theta times them
            if (!BE) flux *= p.inv_theta;
            const double sink = fma(p.dtcs, nHI[c], p.dta) * Ec;
            bc = fma(p.dt, eta[c], -sink) + flux;
        }
        b[c] = bc;
        acc[0] = fma(bc, bc, acc[0]);
        acc[1] = fmax(acc[1], fabs(bc));
        if (op.invd) op.invd[c] = 1.0 / (m + wsum);
        if (diag64) diag64[c] = m + wsum;
        if (op32.invd) op32.invd[c] = 1.0f / (m32 + wsum32);
    }
    const bool ismax[2] = {false, true};
    grid_reduce<2>(acc, ismax, ra);
}

AsmShape asm_shape(const Dims& d) {
    AsmShape a;
    // many blocks pay from 256^3 on; below, fewer keep the reductions short
    a.sh = col_shape(d, 256, d.n >= (1LL << 24) ? 152 * 64 : 152 * 8);
    a.kch = (d.nz + (int)a.sh.grid.z - 1) / (int)a.sh.grid.z;
    a.nzb = (d.nz + a.kch - 1) / a.kch;
    return a;
}

// z-blocks [zb0, zb0 + nzb) of the decomposition (nzb < 0: all of them)
static dim3 zb_grid(const AsmShape& a, int zb0, int& nzb) {
    if (nzb < 0 || zb0 + nzb > a.nzb) nzb = a.nzb - zb0;
    return dim3(a.sh.grid.x, a.sh.grid.y, (unsigned)nzb);
}

void launch_assemble_faces(const Dims& d, const PhysDev& p, const double* E, const double* nHI,
                           const double* eta, Op<double> op, Op<float> op32, double* sc,
                           FaceList fl, cudaStream_t s, int zb0, int nzb) {
    const AsmShape a = asm_shape(d);
    const dim3 g = zb_grid(a, zb0, nzb);
    if (nzb <= 0) return;
    k_assemble_faces<<<g, a.sh.block, 0, s>>>(d, p, E, nHI, eta, op, op32, sc, fl, zb0, a.kch);
}

void launch_assemble_fix(const Dims& d, const PhysDev& p, const double* E, const double* nHI,
                         Op<double> op, Op<float> op32, FaceList fl, cudaStream_t s, int zb0, int nzb) {
    if (!fl.entries) return;
    const AsmShape a = asm_shape(d);
    zb_grid(a, zb0, nzb);
    if (nzb <= 0) return;
    const long long per_zb = (long long)a.sh.grid.x * a.sh.grid.y;
    FaceList f = fl;
    f.entries = fl.entries + per_zb * zb0 * fl.cap;
    f.counts = fl.counts + per_zb * zb0;
    k_assemble_fix<<<(unsigned)(per_zb * nzb), 256, 0, s>>>(d, p, E, nHI, op, op32, f);
}

void face_list_shape(const Dims& d, int limiter, long long* blocks, int* cap) {
    const AsmShape a = asm_shape(d);
    *blocks = (long long)a.sh.grid.x * a.sh.grid.y * a.nzb;
    const long long cells = (long long)a.sh.block.x * a.sh.block.y * a.kch;
    // 40% of the block's faces; a fuller block computes the rest in place
    *cap = (limiter == 0 && d.n <= (1LL << 30)) ? (int)((3 * cells * 2 + 4) / 5) : 0;
}

void launch_assemble_rhs(const Dims& d, const PhysDev& p, const double* E, const double* nHI,
                         const double* eta, Op<double> op, Op<float> op32, double* b, double* diag64,
                         Bnd bnd, const RedArgs& ra, cudaStream_t s, int zb0, int nzb) {
    const AsmShape a = asm_shape(d);
    const dim3 g = zb_grid(a, zb0, nzb);
    if (nzb <= 0) return;
    const bool be = p.theta == 1.0, dir = p.dmask != 0;
    if (be && !dir)
        k_assemble_rhs<true, false><<<g, a.sh.block, 0, s>>>(d, p, E, nHI, eta, op, op32, b, diag64, bnd, ra, zb0, a.kch);
    else if (be)
        k_assemble_rhs<true, true><<<g, a.sh.block, 0, s>>>(d, p, E, nHI, eta, op, op32, b, diag64, bnd, ra, zb0, a.kch);
    else if (!dir)
        k_assemble_rhs<false, false><<<g, a.sh.block, 0, s>>>(d, p, E, nHI, eta, op, op32, b, diag64, bnd, ra, zb0, a.kch);
    else
        k_assemble_rhs<false, true><<<g, a.sh.block, 0, s>>>(d, p, E, nHI, eta, op, op32, b, diag64, bnd, ra, zb0, a.kch);
}

// Photons through the Dirichlet faces of side sd (sum, and sum of absolute
// values per face): with the theta-method the
// face flux is w_b [theta (E^{n+1} - E_b) + (1 - theta)(E^n - E_b)] / theta
// per unit volume, i.e. w_b (inv_theta (E^n - E_b) + dE) with the stored
// (theta-scaled) w_b.
__global__ void __launch_bounds__(RED_THREADS) k_bnd_outflow(Dims d, PhysDev p, int sd, Bnd bnd,
                                                            const double* __restrict__ E,
                                                            const double* __restrict__ dE, RedArgs ra) {
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
        const double fl = bnd.w[off + f] * fma(p.inv_theta, E[c] - Eb, dE[c]);
        acc[0] += fl;
        acc[1] += fabs(fl);
    }
    const bool mx[2] = {false, false};
    grid_reduce<2>(acc, mx, ra);
}

void launch_bnd_outflow(const Dims& d, const PhysDev& p, int sd, Bnd bnd, const double* E,
                        const double* dE, const RedArgs& ra, cudaStream_t st) {
    k_bnd_outflow<<<red_blocks(bnd_side_size(d, sd)), RED_THREADS, 0, st>>>(d, p, sd, bnd, E, dE, ra);
}

__global__ void k_opacity_update(long long n, const double* __restrict__ E, const double* __restrict__ nH,
                                 const double* nHI, double* out, double dt, double c, double sigma,
                                 double hnu, double alpha_B) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double h = nH[i];
        const double x = h > 0.0 ? nHI[i] / h : 0.0;
        const double gam = c * sigma * E[i] / hnu;
        const double ion = 1.0 - x;
        double xn = (x + dt * alpha_B * h * ion * ion) / (1.0 + dt * gam);
        xn = fmin(fmax(xn, 1e-12), 1.0);
        out[i] = xn * h;
    }
}

void launch_opacity_update(long long n, const double* E, const double* nH, const double* nHI,
                           double* out, double dt, double c, double sigma, double hnu,
                           double alpha_B, cudaStream_t s) {
    k_opacity_update<<<grid_blocks(n, 256), 256, 0, s>>>(n, E, nH, nHI, out, dt, c, sigma, hnu,
                                                         alpha_B);
}

}  // namespace fld
