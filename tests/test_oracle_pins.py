"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the
mathematics (limits of the flux limiter, closed forms, brute-force dense
solves, conservation and positivity), so that the oracle can be trusted as
the reference of the GPU parity tests.  CPU only."""
import math

import numpy as np
import pytest

from paper_1306_0645_gb300 import synth

C = synth.C_LIGHT


def phys(**kw):
    p = synth.Params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


# ------------------------------------------------------------- flux limiter

def test_limiter_thick_limit_paper_and_lp(oracle):
    # R -> R_min (uniform E): D = c / (3 kappa) when that is below D_max
    for lim in (synth.LIMITER_PAPER, synth.LIMITER_LP):
        p = phys(limiter=lim)
        kap = 1e-18
        D = oracle.face_D(1e-20, 1e-20, kap, kap, 1e20, p)
        assert D == pytest.approx(C / (3 * kap), rel=1e-15)


def test_limiter_harmonic_face_opacity(oracle):
    # kappa_f = 2 k1 k2 / (k1 + k2) = 1.5e-18 for 1e-18 and 3e-18 (Sec. 2)
    p = phys(limiter=synth.LIMITER_PAPER)
    D = oracle.face_D(1.0, 1.0, 1e-18, 3e-18, 1e20, p)
    assert D == pytest.approx(C / (3 * 1.5e-18), rel=1e-15)
    # either side transparent: face opacity 0 -> free-streaming limit
    h = 1.0
    D0 = oracle.face_D(1.0, 3.0, 0.0, 3e-18, h, p)
    assert D0 == pytest.approx(C * h / math.hypot(1.0, 3 * 0.0), rel=1e-15)


def test_limiter_streaming_limit_arithmetic_face_energy(oracle):
    # kappa = 0: D = c / R with R = |E2 - E1| / (h (E1 + E2)/2); E = 1, 3
    # gives R = 1/h, so D = c h (well below D_max for h = 1 cm).
    for lim in (synth.LIMITER_PAPER, synth.LIMITER_LP):
        p = phys(limiter=lim)
        for h in (1.0, 7.5):
            D = oracle.face_D(1.0, 3.0, 0.0, 0.0, h, p)
            assert D == pytest.approx(C * h, rel=1e-15)
            # order of the two cells does not matter
            assert oracle.face_D(3.0, 1.0, 0.0, 0.0, h, p) == D


def test_limiter_dmax_and_rmin(oracle):
    p = phys(limiter=synth.LIMITER_PAPER)
    Dmax = 0.006 * C * p.L_unit
    # transparent, uniform: R = R_min, c / R_min >> D_max -> D = D_max
    assert oracle.face_D(1.0, 1.0, 0.0, 0.0, 1e20, p) == Dmax
    assert oracle.face_D(0.0, 0.0, 0.0, 0.0, 1e20, p) == Dmax
    # neutral gas of the workloads: c / (3 kappa) = 6.25e30 > D_max
    kap = 1e-3 * synth.SIGMA_HI
    assert C / (3 * kap) > Dmax
    assert oracle.face_D(1e-30, 1e-30, kap, kap, 1e20, p) == Dmax
    # a larger L_unit raises the cap proportionally
    p2 = phys(limiter=synth.LIMITER_PAPER, L_unit=10 * p.L_unit)
    assert oracle.face_D(1.0, 1.0, 0.0, 0.0, 1e20, p2) == pytest.approx(10 * Dmax, rel=1e-15)


def test_limiter_paper_intermediate(oracle):
    # R = 4 kappa: D = c / sqrt(9 k^2 + 16 k^2) = c / (5 k)
    p = phys(limiter=synth.LIMITER_PAPER)
    kap = 1e-18
    h = 1e17
    # mean face energy 1 and difference R h = 0.4: R = 4 kappa
    R = 4 * kap
    d = R * h
    E1, E2 = 1.0 - d / 2, 1.0 + d / 2
    Rgot = abs(E2 - E1) / (h * 0.5 * (E1 + E2))
    D = oracle.face_D(E1, E2, kap, kap, h, p)
    assert D == pytest.approx(C / math.sqrt(9 * kap ** 2 + Rgot ** 2), rel=1e-14)
    assert D == pytest.approx(C / (5 * kap), rel=1e-10)


def test_lp_lambda_values(oracle):
    # lambda(x) = (coth x - 1/x) / x; lambda(0) = 1/3
    assert oracle.lp_lambda(0.0) == pytest.approx(1.0 / 3.0, rel=1e-16)
    assert oracle.lp_lambda(1e-3) == pytest.approx(1 / 3 - 1e-6 / 45, rel=1e-15)
    assert oracle.lp_lambda(1.0) == pytest.approx(1.0 / math.tanh(1.0) - 1.0, rel=1e-14)
    assert oracle.lp_lambda(2.0) == pytest.approx(0.26865736036377405, rel=1e-13)
    # continuity where the series hands over to the closed form
    lo = oracle.lp_lambda(np.nextafter(1e-2, 0))
    hi = oracle.lp_lambda(1e-2)
    assert abs(lo - hi) < 1e-11
    # large x: lambda ~ (1 - 1/x) / x
    x = 1e6
    assert oracle.lp_lambda(x) == pytest.approx((1 - 1 / x) / x, rel=1e-12)


def test_lp_limiter_forms(oracle):
    p = phys(limiter=synth.LIMITER_LP)
    kap = 1e-18
    h = 1e17
    R = 3 * kap
    d = R * h
    E1, E2 = 1.0 - d / 2, 1.0 + d / 2
    Rgot = abs(E2 - E1) / (h * 0.5 * (E1 + E2))
    x = Rgot / kap
    D = oracle.face_D(E1, E2, kap, kap, h, p)
    lam = (1.0 / math.tanh(x) - 1.0 / x) / x
    assert D == pytest.approx(C * lam / kap, rel=1e-12)
    # LP is below the square-root-sum form here and both lie in (c/(5k), c/(3k))
    Dp = oracle.face_D(E1, E2, kap, kap, h, phys(limiter=synth.LIMITER_PAPER))
    assert C / (5 * kap) < D < Dp < C / (3 * kap)


# ------------------------------------------------------------------ assembly

CASES = [
    ((4, 3, 5), (False, False, False), synth.LIMITER_PAPER),
    ((4, 6, 2), (True, True, True), synth.LIMITER_LP),
    ((5, 4, 3), (True, False, True), synth.LIMITER_PAPER),
    ((1, 1, 1), (False, False, False), synth.LIMITER_LP),
    ((2, 2, 2), (True, True, True), synth.LIMITER_PAPER),
    ((8, 8, 8), (False, False, False), synth.LIMITER_LP),
    ((7, 7, 7), (True, True, True), synth.LIMITER_PAPER),
]


@pytest.mark.parametrize("n,per,lim", CASES)
def test_matrix_symmetric_dominant_rowsum(oracle, n, per, lim):
    case = synth.random_case(n, seed=sum(n), periodic=per, limiter=lim, zero_frac=0.1)
    case.params.adot_over_a = 3e-18
    op = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    A = oracle.dense_matrix(case.grid, op)
    assert np.array_equal(A, A.T)                           # bitwise symmetric
    mass = 1.0 + case.params.dt * (C * case.nHI.ravel() * case.params.sigma + case.params.adot_over_a)
    np.testing.assert_allclose(A.sum(axis=1), mass, rtol=1e-12)
    off = np.abs(A).sum(axis=1) - np.abs(np.diag(A))
    assert np.all(np.diag(A) > off)                         # strict dominance
    assert np.all(A - np.diag(np.diag(A)) <= 0.0)           # M-matrix sign pattern
    np.linalg.cholesky(A)                                    # SPD


def test_boundary_faces(oracle):
    case = synth.random_case((6, 4, 4), seed=3, periodic=(True, False, False))
    op = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    assert np.all(op["wx"][:, :, 0] > 0)      # periodic wrap face
    assert np.all(op["wy"][:, 0, :] == 0)     # zero-gradient boundary: no flux
    assert np.all(op["wz"][0, :, :] == 0)


def test_rhs_uniform_E_and_flux_telescoping(oracle):
    for per in ((False,) * 3, (True,) * 3):
        case = synth.random_case((6, 5, 4), seed=11, periodic=per)
        p = case.params
        p.adot_over_a = 1e-17
        Eu = np.full(case.grid.shape, 3e-20)
        op = oracle.assemble(case.grid, p, Eu, case.nHI, case.eta)
        sink = p.dt * (C * case.nHI * p.sigma + p.adot_over_a)
        np.testing.assert_allclose(op["b"], p.dt * case.eta - sink * Eu, rtol=1e-14, atol=0)
        # random E: the flux terms cancel in the sum over cells
        op = oracle.assemble(case.grid, p, case.E, case.nHI, case.eta)
        total = p.dt * case.eta.sum() - (sink * case.E).sum()
        scale = np.abs(op["b"]).sum()
        assert abs(op["b"].sum() - total) <= 1e-13 * scale


def test_gradient_is_face_normal_only(oracle):
    # E varies along x only: y and z faces see R = R_min -> thick/capped D
    g = synth.Grid((4, 3, 3), (1e20, 2e20, 3e20))
    p = phys(limiter=synth.LIMITER_PAPER)
    kap = 1e-18
    x = np.arange(4)
    E = np.broadcast_to(10.0 ** (-20 + x), g.shape).copy()
    nHI = np.full(g.shape, kap / p.sigma)
    op = oracle.assemble(g, p, E, nHI, np.zeros(g.shape))
    Dyz = min(C / (3 * kap), 0.006 * C * p.L_unit)
    np.testing.assert_allclose(op["wy"][:, 1:, :], p.dt * Dyz / 2e20 ** 2, rtol=1e-15)
    np.testing.assert_allclose(op["wz"][1:, :, :], p.dt * Dyz / 3e20 ** 2, rtol=1e-15)
    # x faces: R = |E2 - E1| / (h (E1+E2)/2) = (9/5.5) / h
    R = 9.0 / 5.5 / 1e20
    Dx = C / math.sqrt(9 * kap ** 2 + R ** 2)
    np.testing.assert_allclose(op["wx"][:, :, 1:], p.dt * Dx / 1e40, rtol=1e-14)


# ---------------------------------------------------------------- linear solve

def test_dense_cholesky_against_lapack(oracle):
    case = synth.random_case((5, 4, 3), seed=5, periodic=(True, False, True))
    op = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    A = oracle.dense_matrix(case.grid, op)
    x = oracle.dense_solve(case.grid, op, op["b"])
    ref = np.linalg.solve(A, op["b"].ravel())
    np.testing.assert_allclose(x.ravel(), ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("n,per,lim", CASES)
@pytest.mark.parametrize("smoother", [synth.SMOOTH_RBGS, synth.SMOOTH_JACOBI])
def test_mg_pcg_matches_dense(oracle, n, per, lim, smoother):
    case = synth.random_case(n, seed=7 + sum(n), periodic=per, limiter=lim, zero_frac=0.05)
    op = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    x_dense = oracle.dense_solve(case.grid, op, op["b"])
    s = {"rtol": 1e-14, "max_iter": 200, "smoother": smoother, "coarse_cap": 64}
    if np.prod(n) > 64 and len(oracle.num_levels(n)) == 1:
        s["coarse_cap"] = 1024
    x, iters, rel, hist = oracle.pcg(case.grid, op, op["b"], s)
    assert rel <= 1e-13
    scale = np.abs(x_dense).max()
    np.testing.assert_allclose(x, x_dense, rtol=0, atol=1e-12 * scale)


def test_mg_pcg_rediscretised_hierarchy_on_16(oracle):
    # 16^3 has levels 16, 8, 4: the solve goes through two coarsenings
    case = synth.random_case((16, 16, 16), seed=21, periodic=(False, True, False))
    op = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    assert [l[0] for l in oracle.num_levels((16, 16, 16))] == [16, 8, 4]
    x, iters, rel, hist = oracle.pcg(case.grid, op, op["b"], {"rtol": 1e-13, "max_iter": 100})
    A = oracle.dense_matrix(case.grid, op)
    ref = np.linalg.solve(A, op["b"].ravel())
    np.testing.assert_allclose(x.ravel(), ref, rtol=0, atol=1e-11 * np.abs(ref).max())
    assert iters < 30


def test_single_cell_closed_form(oracle):
    g = synth.Grid((1, 1, 1), (1e20,) * 3)
    p = phys(adot_over_a=2e-17)
    E, nHI, eta = np.full((1, 1, 1), 2e-20), np.full((1, 1, 1), 1e-3), np.full((1, 1, 1), 5e-25)
    E1, info = oracle.step(g, p, {}, E, nHI, eta)
    s = C * 1e-3 * p.sigma + p.adot_over_a
    dE = p.dt * (5e-25 - s * 2e-20) / (1 + p.dt * s)
    assert E1[0, 0, 0] - 2e-20 == pytest.approx(dE, rel=1e-14)
    assert info["iters"] == 1


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("kap", [1.6e-21, 1e-18])
def test_manufactured_cosine_mode(oracle, periodic, kap):
    n = (16, 8, 12)
    g = synth.Grid(n, (2e20, 3e20, 2.5e20), (periodic,) * 3)
    p = phys(limiter=synth.LIMITER_PAPER, adot_over_a=1e-17)
    kd = (3, 1, 2)
    E0, eta0, eps = 1e-18, 4e-24, 1e-24
    idx = [np.arange(v) for v in n]
    if periodic:
        modes = [np.cos(2 * np.pi * k * i / N) for k, i, N in zip(kd, idx, n)]
        lam = [4 * np.sin(np.pi * k / N) ** 2 for k, N in zip(kd, n)]
    else:
        modes = [np.cos(np.pi * k * (i + 0.5) / N) for k, i, N in zip(kd, idx, n)]
        lam = [4 * np.sin(np.pi * k / (2 * N)) ** 2 for k, N in zip(kd, n)]
    mode = modes[2][:, None, None] * modes[1][None, :, None] * modes[0][None, None, :]
    E = np.full(g.shape, E0)
    nHI = np.full(g.shape, kap / p.sigma)
    eta = eta0 + eps * mode
    D = min(C / (3 * kap), 0.006 * C * p.L_unit)
    w = [p.dt * D / h ** 2 for h in g.h]
    m = 1 + p.dt * (C * kap + p.adot_over_a)
    exact = p.dt * (eta0 - (C * kap + p.adot_over_a) * E0) / m \
        + p.dt * eps * mode / (m + sum(wd * ld for wd, ld in zip(w, lam)))
    E1, info = oracle.step(g, p, {"rtol": 1e-14, "max_iter": 200}, E, nHI, eta)
    np.testing.assert_allclose(E1 - E0, exact, rtol=0, atol=1e-12 * np.abs(exact).max())


# ------------------------------------------------------- balance, positivity

@pytest.mark.parametrize("per", [(False,) * 3, (True,) * 3])
def test_photon_balance_and_positivity(oracle, per):
    case = synth.random_case((8, 8, 8), seed=31, periodic=per, zero_frac=0.1)
    p = case.params
    s = {"rtol": 1e-8}
    E1, info = oracle.step(case.grid, p, s, case.E, case.nHI, case.eta)
    # the floor keeps E^{n+1} >= 0 and adds no more than the tolerance allows
    assert E1.min() >= 0.0
    assert info["floor_added"] <= 1e-6 * info["emitted"]
    # |imbalance| <= V sqrt(N) ||r|| / h nu, with ||r|| = rel_res ||b||
    op = oracle.assemble(case.grid, p, case.E, case.nHI, case.eta)
    bnorm = np.linalg.norm(op["b"])
    bound = case.grid.volume * math.sqrt(case.grid.cells) * info["rel_res"] * bnorm / p.hnu
    assert abs(info["balance_abs"]) <= 1.01 * bound + 1e-9 * info["emitted"]
    # exact solve: E^{n+1} = A^{-1} (E^n + dt eta) >= 0 (M-matrix)
    dE = oracle.dense_solve(case.grid, op, op["b"])
    Ex = case.E + dE
    assert Ex.min() >= -1e-12 * Ex.max()
    # and the tight MG-PCG solve balances photons to rounding
    E2, info2 = oracle.step(case.grid, p, {"rtol": 1e-14, "max_iter": 200}, case.E, case.nHI, case.eta)
    assert info2["balance_rel"] < 1e-9


def test_zero_rhs_gives_zero_iterations(oracle):
    g = synth.Grid.cube(8)
    p = phys()
    E = np.zeros(g.shape)
    E1, info = oracle.step(g, p, {}, E, np.full(g.shape, 1e-3), np.zeros(g.shape))
    assert info["iters"] == 0 and np.all(E1 == 0)


def test_invalid_inputs_rejected(oracle):
    g = synth.Grid.cube(4)
    p = phys()
    E = np.full(g.shape, 1e-20)
    bad = E.copy()
    bad[0, 0, 0] = -1.0
    with pytest.raises(oracle.OracleError):
        oracle.assemble(g, p, bad, np.ones(g.shape), np.zeros(g.shape))
    bad[0, 0, 0] = np.nan
    with pytest.raises(oracle.OracleError):
        oracle.assemble(g, p, E, bad, np.zeros(g.shape))


# -------------------------------------------------------------- multigrid

def test_level_shapes(oracle):
    assert [l[0] for l in oracle.num_levels((32, 32, 32))] == [32, 16, 8, 4]
    assert [l[0] for l in oracle.num_levels((48, 48, 48))] == [48, 24, 12, 6, 3]
    assert [l[0] for l in oracle.num_levels((512,) * 3)] == [512, 256, 128, 64, 32, 16, 8, 4]
    assert oracle.num_levels((5, 5, 5)) == [(5, 5, 5)]
    assert oracle.num_levels((128, 64, 64))[-1] == (8, 4, 4)


@pytest.mark.parametrize("per", [(False,) * 3, (True,) * 3])
def test_prolongation_reproduces_constants_and_linears(oracle, per):
    nf = (12, 8, 16)
    nc = tuple(v // 2 for v in nf)
    ones = np.ones((nc[2], nc[1], nc[0]))
    z = oracle.prolong_add(nf, per, ones, np.zeros((nf[2], nf[1], nf[0])))
    np.testing.assert_allclose(z, 1.0, rtol=1e-15)
    # linear in x (coarse centre X = 2I + 1/2 in fine units): exact away from
    # the boundaries and the periodic seam
    Xc = 2 * np.arange(nc[0]) + 0.5
    ec = np.broadcast_to(Xc, (nc[2], nc[1], nc[0])).copy()
    z = oracle.prolong_add(nf, per, ec, np.zeros((nf[2], nf[1], nf[0])))
    xf = np.arange(nf[0]).astype(float)
    np.testing.assert_allclose(z[:, :, 1:-1], np.broadcast_to(xf[1:-1], z[:, :, 1:-1].shape), rtol=1e-14)


@pytest.mark.parametrize("per", [(False,) * 3, (True, False, True)])
def test_restriction_is_scaled_transpose(oracle, per):
    nf = (8, 12, 6)
    nc = tuple(v // 2 for v in nf)
    rng = np.random.default_rng(0)
    u = rng.standard_normal((nf[2], nf[1], nf[0]))
    v = rng.standard_normal((nc[2], nc[1], nc[0]))
    Ru = oracle.restrict(nf, per, u)
    Pv = oracle.prolong_add(nf, per, v, np.zeros_like(u))
    assert (Ru * v).sum() == pytest.approx((u * Pv).sum() / 8, rel=1e-12)
    # R 1 = 1 (averaging)
    np.testing.assert_allclose(oracle.restrict(nf, per, np.ones_like(u)), 1.0, rtol=1e-15)


def test_coarse_operator_rediscretises_constant_coefficients(oracle):
    p = phys(limiter=synth.LIMITER_PAPER, adot_over_a=1e-17)
    kap = 1e-18
    gf = synth.Grid((16, 8, 12), (1e20, 2e20, 3e20))
    gc = synth.Grid((8, 4, 6), (2e20, 4e20, 6e20))
    f = {k: oracle.assemble(g, p, np.full(g.shape, 1e-20), np.full(g.shape, kap / p.sigma),
                            np.zeros(g.shape)) for k, g in (("f", gf), ("c", gc))}
    c = oracle.coarsen(gf.n, (False,) * 3, f["f"])
    for k in ("m", "wx", "wy", "wz"):
        np.testing.assert_allclose(c[k], f["c"][k], rtol=1e-14)


def test_vcycle_contracts_on_uniform_32(oracle):
    case = synth.config1(32)
    op = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    b = op["b"]
    x = np.zeros_like(b)
    norms = []
    for it in range(4):
        r = b - oracle.apply(case.grid, op, x)
        norms.append(np.linalg.norm(r))
        x = x + oracle.vcycle(case.grid, op, r)
    rates = [norms[i + 1] / norms[i] for i in range(3)]
    assert max(rates) < 0.5


def test_vcycle_is_symmetric(oracle):
    case = synth.random_case((16, 16, 16), seed=4, periodic=(True, False, True))
    op = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(case.grid.shape)
    v = rng.standard_normal(case.grid.shape)
    Bu = oracle.vcycle(case.grid, op, u)
    Bv = oracle.vcycle(case.grid, op, v)
    assert (Bu * v).sum() == pytest.approx((u * Bv).sum(), rel=1e-12)
    assert (Bu * u).sum() > 0


@pytest.mark.parametrize("paper_order", [0, 1])
def test_vcycle_two_levels_by_dense_matrices(oracle, paper_order):
    # Table 1's cycle on 8^3 (two levels) written out with dense matrices: the
    # pre-sweep red then black from z = 0, each colour c as
    # z <- z + P_c D^-1 (r - A z) (cells of one colour do not couple), the
    # residual restricted by R, the coarse system solved exactly, P of the
    # correction added, then the post-sweep black then red (symmetric cycle)
    # or red then black (paper_order, the paper's "nonsymmetric" relaxation)
    case = synth.random_case((8, 8, 8), seed=6)
    g = case.grid
    op = oracle.assemble(g, case.params, case.E, case.nHI, case.eta)
    A = oracle.dense_matrix(g, op)
    n = A.shape[0]
    d = np.diag(A)
    idx = np.arange(n)
    red = (idx % 8 + (idx // 8) % 8 + idx // 64) % 2 == 0

    def sweep(z, r, colour):
        z = z.copy()
        z[colour] += ((r - A @ z) / d)[colour]
        return z

    # the transfer operators as matrices, from the pinned restriction and
    # prolongation; the coarse operator from the pinned coarsening
    R = np.stack([oracle.restrict(g.n, g.periodic, e.reshape(g.shape)).ravel() for e in np.eye(n)], axis=1)
    P = np.stack([oracle.prolong_add(g.n, g.periodic, e.reshape((4, 4, 4)), np.zeros(g.shape)).ravel()
                  for e in np.eye(64)], axis=1)
    gc = synth.Grid((4, 4, 4), tuple(2 * h for h in g.h), g.periodic)
    Ac = oracle.dense_matrix(gc, oracle.coarsen(g.n, g.periodic, op))
    r = np.random.default_rng(2).standard_normal(n)
    z = sweep(sweep(np.zeros(n), r, red), r, ~red)
    z = z + P @ np.linalg.solve(Ac, R @ (r - A @ z))
    for colour in ((red, ~red) if paper_order else (~red, red)):
        z = sweep(z, r, colour)
    zo = oracle.vcycle(g, op, r.reshape(g.shape), {"paper_order": paper_order}).ravel()
    np.testing.assert_allclose(zo, z, rtol=0, atol=1e-12 * np.abs(z).max())


def test_paper_order_cycle_is_nonsymmetric_and_pcg_converges(oracle):
    # red then black in both sweeps makes the cycle nonsymmetric; CG
    # preconditioned by it still reaches the dense solution
    case = synth.random_case((16, 16, 16), seed=4, periodic=(True, False, True))
    op = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(case.grid.shape)
    v = rng.standard_normal(case.grid.shape)
    s = {"paper_order": 1}
    Bu, Bv = oracle.vcycle(case.grid, op, u, s), oracle.vcycle(case.grid, op, v, s)
    assert abs((Bu * v).sum() - (u * Bv).sum()) > 1e-6 * abs((Bu * v).sum())
    small = synth.random_case((6, 6, 6), seed=8, periodic=(False, True, False))
    ops = oracle.assemble(small.grid, small.params, small.E, small.nHI, small.eta)
    x, it, rel, _ = oracle.pcg(small.grid, ops, ops["b"], {"paper_order": 1, "rtol": 1e-14, "max_iter": 100})
    xd = oracle.dense_solve(small.grid, ops, ops["b"])
    np.testing.assert_allclose(x, xd, rtol=0, atol=1e-12 * np.abs(xd).max())


def test_pcg_iteration_counts_config1(oracle):
    case = synth.config1(32)
    E1, info = oracle.step(case.grid, case.params, {}, case.E, case.nHI, case.eta)
    assert info["status"] == 0 and info["rel_res"] <= 1.01e-8
    assert info["iters"] <= 20


def test_noconv_reported(oracle):
    case = synth.config1(16)
    with pytest.raises(oracle.OracleError) as e:
        oracle.step(case.grid, case.params, {"max_iter": 1, "rtol": 1e-14}, case.E, case.nHI, case.eta)
    assert e.value.code == oracle.ENOCONV


# ------------------------------------------------------- opacity update

def test_opacity_update_equilibrium_and_dark(oracle):
    nH = np.full(5, 1e-3)
    x = np.array([0.5, 0.1, 0.9, 1e-3, 0.3])
    # photoionisation equilibrium Gamma x = alpha n_H (1 - x)^2 is a fixed point
    gam = synth.ALPHA_B * nH * (1 - x) ** 2 / x
    E = gam * synth.HNU_HI / (C * synth.SIGMA_HI)
    out = oracle.opacity_update(E, nH, x * nH, synth.DT, C, synth.SIGMA_HI, synth.HNU_HI, synth.ALPHA_B)
    np.testing.assert_allclose(out, x * nH, rtol=1e-13)
    # no radiation: pure recombination, clamped at fully neutral
    out = oracle.opacity_update(np.zeros(5), nH, x * nH, 1e3, C, synth.SIGMA_HI, synth.HNU_HI, synth.ALPHA_B)
    np.testing.assert_allclose(out, np.minimum(x + 1e3 * synth.ALPHA_B * 1e-3 * (1 - x) ** 2, 1.0) * nH, rtol=1e-14)


# ------------------------------------------------ radiation subcycling (Sec. 3.3)

def test_advance_reaches_t_span_and_adapts(oracle):
    case = synth.config1(16)
    p = case.params
    span = 20 * p.dt
    E, info = oracle.advance(case.grid, p, {}, case.E, case.nHI, case.eta, span, dt_first=0.01 * p.dt,
                             tau_tol=1e-2, dt_min=1e-6 * p.dt)
    assert info["status"] == 0 and info["t_done"] == span
    assert info["retries"] == 0 and info["substeps"] >= 3
    # time steps grew from the small first one
    assert info["dt_next"] > 0.01 * p.dt


def test_advance_retries_failed_substeps_at_a_tenth(oracle):
    # a solver allowed 2 CG iterations fails on the first large substep,
    # converges on the 0.1 dt retry
    case = synth.config1(16)
    p = case.params
    s = {"max_iter": 2, "rtol": 1e-8}
    E2, info = oracle.advance(case.grid, p, s, case.E, case.nHI, case.eta, p.dt, dt_first=p.dt,
                              tau_tol=1e3, dt_min=1e-8 * p.dt, allow_fail=True)
    assert info["retries"] >= 1
    # and when every retry fails the status says so
    E3, info3 = oracle.advance(case.grid, p, {"max_iter": 1, "rtol": 1e-14}, case.E, case.nHI, case.eta,
                               p.dt, dt_first=p.dt, tau_tol=1e3, dt_min=1e-3 * p.dt, allow_fail=True)
    assert info3["status"] == oracle.ENOCONV and info3["t_done"] < p.dt


def test_advance_converges_to_small_fixed_steps(oracle):
    # backward Euler is first order: the subcycled result approaches the
    # result of many small fixed steps as tau_tol shrinks
    case = synth.random_case((8, 8, 8), seed=3)
    p = case.params
    span = 2 * p.dt
    ref = case.E.copy()
    for _ in range(400):
        p.dt = span / 400
        ref, _ = oracle.step(case.grid, p, {"rtol": 1e-12, "max_iter": 100}, ref, case.nHI, case.eta)
    p.dt = span
    errs = []
    for tol in (1e-1, 1e-2):
        E, info = oracle.advance(case.grid, p, {"rtol": 1e-12, "max_iter": 100}, case.E, case.nHI, case.eta,
                                 span, dt_first=span / 100, tau_tol=tol, dt_min=1e-9 * span, growth=2.0)
        errs.append(np.linalg.norm(E - ref) / np.linalg.norm(ref))
    assert errs[1] < errs[0]
