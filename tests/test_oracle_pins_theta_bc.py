"""Pins of the oracle's theta-method (Sec. 3.2: backward Euler and the
trapezoidal rule) and of its per-face boundary conditions (reflecting,
Dirichlet and outflow faces, as in the tests of Sec. 4.1) against closed
forms, brute-force dense solves and conservation.  CPU only."""
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


def cosine_modes(n, kd, periodic):
    idx = [np.arange(v) for v in n]
    if periodic:
        modes = [np.cos(2 * np.pi * k * i / N) for k, i, N in zip(kd, idx, n)]
        lam = [4 * np.sin(np.pi * k / N) ** 2 for k, N in zip(kd, n)]
    else:
        modes = [np.cos(np.pi * k * (i + 0.5) / N) for k, i, N in zip(kd, idx, n)]
        lam = [4 * np.sin(np.pi * k / (2 * N)) ** 2 for k, N in zip(kd, n)]
    mode = modes[2][:, None, None] * modes[1][None, :, None] * modes[0][None, None, :]
    return mode, lam


# ------------------------------------------------------------- theta-method

@pytest.mark.parametrize("theta", [0.5, 0.75, 1.0])
@pytest.mark.parametrize("periodic", [False, True])
def test_theta_manufactured_source_mode(oracle, theta, periodic):
    # uniform E and kappa, eta = eta0 + eps * (discrete Laplacian eigenmode):
    # (I + theta dt (s - L)) dE = dt (eta - s E0), so each mode of dE is the
    # source mode over 1 + theta (dt s + sum_d w_d lambda_d)
    n = (16, 8, 12)
    g = synth.Grid(n, (2e20, 3e20, 2.5e20), (periodic,) * 3)
    kap = 1e-18
    p = phys(adot_over_a=1e-17, theta=theta)
    mode, lam = cosine_modes(n, (3, 1, 2), periodic)
    E0, eta0, eps = 1e-18, 4e-24, 1e-24
    E = np.full(g.shape, E0)
    nHI = np.full(g.shape, kap / p.sigma)
    eta = eta0 + eps * mode
    D = min(C / (3 * kap), 0.006 * C * p.L_unit)
    w = [p.dt * D / h ** 2 for h in g.h]
    s = C * kap + p.adot_over_a
    exact = p.dt * (eta0 - s * E0) / (1 + theta * p.dt * s) \
        + p.dt * eps * mode / (1 + theta * (p.dt * s + sum(wd * ld for wd, ld in zip(w, lam))))
    E1, info = oracle.step(g, p, {"rtol": 1e-14, "max_iter": 200}, E, nHI, eta)
    np.testing.assert_allclose(E1 - E0, exact, rtol=0, atol=1e-12 * np.abs(exact).max())


def capped_mode_setup(n, amp=1e-3):
    """E = E0 (1 + amp * mode) in a reflecting box with an opacity so low that
    every face is capped at D_max: the step is then linear diffusion with a
    constant coefficient, whose modes decay independently."""
    g = synth.Grid(n, (synth.BOX / n[0], synth.BOX / n[1], synth.BOX / n[2]))
    kap = 1e-21          # c / (3 kappa) > D_max = 0.006 c L for L = 6.6 kpc
    mode, lam = cosine_modes(n, (1, 1, 0), False)
    E0 = 1e-20
    E = E0 * (1 + amp * mode)
    nHI = np.full(g.shape, kap / synth.SIGMA_HI)
    Dmax = 0.006 * C * synth.BOX
    mu0 = C * kap
    mu1 = mu0 + sum(Dmax / h ** 2 * l for h, l in zip(g.h, lam))
    return g, E, nHI, E0, amp * E0 * mode, mu0, mu1


def amplification(theta, mu, dt):
    return (1 - (1 - theta) * mu * dt) / (1 + theta * mu * dt)


@pytest.mark.parametrize("theta", [0.5, 1.0])
def test_theta_one_step_map_of_a_diffusing_mode(oracle, theta):
    # the right-hand side must be dt F(E^n) with the full flux and the
    # operator I - theta dt L: each mode is multiplied by
    # (1 - (1 - theta) mu dt) / (1 + theta mu dt)
    n = (16, 8, 4)
    g, E, nHI, E0, pert, mu0, mu1 = capped_mode_setup(n)
    dt = 2.0 / mu1
    p = phys(dt=dt, theta=theta)
    E1, info = oracle.step(g, p, {"rtol": 1e-14, "max_iter": 200}, E, nHI, np.zeros(g.shape))
    exact = E0 * amplification(theta, mu0, dt) + pert * amplification(theta, mu1, dt)
    np.testing.assert_allclose(E1, exact, rtol=1e-11)


def test_trapezoidal_rule_is_second_order(oracle):
    # error of the decaying mode after a fixed time against exp(-mu t):
    # halving dt divides it by 4 for theta = 1/2 and by 2 for theta = 1
    n = (8, 8, 4)
    g, E, nHI, E0, pert, mu0, mu1 = capped_mode_setup(n)
    T = 2.0 / mu1
    amp0 = np.abs(pert).max()
    errs = {}
    for theta in (0.5, 1.0):
        errs[theta] = []
        for steps in (4, 8, 16):
            p = phys(dt=T / steps, theta=theta)
            Ek = E.copy()
            for _ in range(steps):
                Ek, _ = oracle.step(g, p, {"rtol": 1e-14, "max_iter": 200}, Ek, nHI, np.zeros(g.shape))
            # the perturbation's amplitude after removing the uniform part
            uni = E0 * amplification(theta, mu0, T / steps) ** steps
            got = np.abs(Ek - uni).max() / amp0
            errs[theta].append(abs(got - math.exp(-mu1 * T)))
    r_tr = [errs[0.5][i] / errs[0.5][i + 1] for i in range(2)]
    r_be = [errs[1.0][i] / errs[1.0][i + 1] for i in range(2)]
    assert all(3.6 < r < 4.4 for r in r_tr), r_tr
    assert all(1.7 < r < 2.3 for r in r_be), r_be


# --------------------------------------------------------- boundary faces

def test_dirichlet_faces_give_the_linear_steady_profile(oracle):
    # no opacity, no source, E held at Ea (x = 0) and Eb (x = L), reflecting
    # in y and z, D capped everywhere: after a step long enough to reach the
    # steady state E is linear in x between the face values, at the cell
    # centres x_i = (i + 1/2) h -- which fixes the half-cell distance of the
    # Dirichlet face
    n = (16, 4, 4)
    L = synth.BOX
    g = synth.Grid(n, (L / n[0], L / n[1], L / n[2]),
                   dirichlet=(True, True, False, False, False, False), ebc=(1.0e-20, 2.0e-20, 0, 0, 0, 0))
    p = phys(dt=1e25)
    E = np.full(g.shape, 1.5e-20)
    E1, info = oracle.step(g, p, {"rtol": 1e-14, "max_iter": 200}, E, np.zeros(g.shape), np.zeros(g.shape))
    x = (np.arange(n[0]) + 0.5) / n[0]
    expect = 1.0e-20 + 1.0e-20 * x
    np.testing.assert_allclose(E1, np.broadcast_to(expect, g.shape), rtol=1e-9)
    # the photons that left through x = 0 and entered at x = L balance
    assert abs(info["balance_rel"]) < 1e-9


def test_outflow_face_streams_at_c_times_face_energy(oracle):
    # one optically thin cell with an outflow (E_b = 0) face at x = 0: the
    # limiter's streaming limit D = c / R with R = E / ((h/2)(E/2)) gives the
    # flux c E_face = c E / 2 through the face, so over a short step
    # dE = -dt c E / (2 h)
    h = 1e20
    g = synth.Grid((1, 1, 1), (h, h, h), dirichlet=(True, False, False, False, False, False))
    p = phys(dt=h / C * 1e-7, L_unit=1e3 * h)
    E = np.full((1, 1, 1), 3e-20)
    E1, info = oracle.step(g, p, {"rtol": 1e-14}, E, np.zeros_like(E), np.zeros_like(E))
    rate = (E1[0, 0, 0] - 3e-20) / p.dt
    assert rate == pytest.approx(-C * 3e-20 / (2 * h), rel=1e-6)
    # and the outflow is reported as the photons that left
    lost = -(E1[0, 0, 0] - 3e-20) * g.volume / p.hnu
    assert info["outflow"] == pytest.approx(lost, rel=1e-7)   # lost has E1 - E cancellation


def test_outflow_of_a_thick_cell_is_diffusive(oracle):
    # optically thick cell with an outflow face at x = L: the limiter tends
    # to the diffusion coefficient c / (3 kappa), so over a short step the
    # loss rate is absorption c kappa E plus the diffusive face flux
    # (c / (3 kappa)) E / (h/2) over the cell width h
    h = 1e20
    kap = 1e-17
    g = synth.Grid((1, 1, 1), (h, h, h), dirichlet=(False, True, False, False, False, False))
    p = phys(dt=1e-3, L_unit=1e3 * h)
    E = np.full((1, 1, 1), 3e-20)
    nHI = np.full_like(E, kap / p.sigma)
    E1, _ = oracle.step(g, p, {"rtol": 1e-14}, E, nHI, np.zeros_like(E))
    rate = (E1[0, 0, 0] - 3e-20) / p.dt
    expect = -(C * kap * 3e-20 + C / (3 * kap) * 3e-20 / (0.5 * h) / h)
    assert rate == pytest.approx(expect, rel=1e-5)


BC_CASES = [
    ((6, 4, 8), (True, False, False, True, False, False), (2e-19, 0, 0, 0, 0, 0)),
    ((4, 4, 4), (True,) * 6, (1e-19, 2e-19, 0, 3e-19, 5e-20, 0)),
    ((5, 7, 3), (False, True) * 3, (0,) * 6),
    ((8, 8, 8), (True, True, False, False, True, False), (1e-19, 0, 0, 0, 2e-19, 0)),
]


@pytest.mark.parametrize("n,dirichlet,ebc", BC_CASES)
@pytest.mark.parametrize("theta", [0.5, 1.0])
def test_boundary_operator_symmetric_dominant_and_solved_exactly(oracle, n, dirichlet, ebc, theta):
    case = synth.random_case(n, seed=sum(n), periodic=(False, False, False))
    g = synth.Grid(case.grid.n, case.grid.h, dirichlet=dirichlet, ebc=ebc)
    p = case.params
    p.theta = theta
    op = oracle.assemble(g, p, case.E, case.nHI, case.eta)
    A = oracle.dense_matrix(g, op)
    assert np.array_equal(A, A.T)
    off = np.abs(A).sum(axis=1) - np.abs(np.diag(A))
    assert np.all(np.diag(A) > off)
    # the boundary weights sit on the diagonal of the boundary cells
    assert op["bnd"] is not None and op["bnd"].max() > 0
    mass = 1 + theta * p.dt * (C * case.nHI * p.sigma + p.adot_over_a)
    extra = (op["m"] - mass).ravel()
    assert extra.min() > -1e-12 * op["m"].max()
    assert extra.sum() == pytest.approx(op["bnd"].sum(), rel=1e-10)
    # MG-PCG with the coarsened boundary weights against the dense solve
    x_dense = oracle.dense_solve(g, op, op["b"])
    x, iters, rel, _ = oracle.pcg(g, op, op["b"], {"rtol": 1e-13, "max_iter": 200})
    np.testing.assert_allclose(x, x_dense, rtol=0, atol=1e-11 * np.abs(x_dense).max())


def test_boundary_weights_coarsen_by_rediscretisation(oracle):
    # uniform fields with E = E_b on every Dirichlet face: every face, interior
    # or boundary, takes the same D, so the coarsened operator equals the one
    # assembled on the grid of twice the spacing
    kap = 1e-18
    Eu = 1e-20
    dirichlet = (True, False, False, True, True, True)
    ebc = tuple(Eu if d else 0.0 for d in dirichlet)
    p = phys(adot_over_a=1e-17, theta=0.5)
    gf = synth.Grid((16, 8, 12), (1e20, 2e20, 3e20), dirichlet=dirichlet, ebc=ebc)
    gc = synth.Grid((8, 4, 6), (2e20, 4e20, 6e20), dirichlet=dirichlet, ebc=ebc)
    ops = {k: oracle.assemble(g, p, np.full(g.shape, Eu), np.full(g.shape, kap / p.sigma), np.zeros(g.shape))
           for k, g in (("f", gf), ("c", gc))}
    c = oracle.coarsen(gf.n, (False,) * 3, ops["f"], dirichlet=dirichlet)
    for k in ("m", "wx", "wy", "wz", "bnd"):
        np.testing.assert_allclose(c[k], ops["c"][k], rtol=1e-14)


@pytest.mark.parametrize("theta", [0.5, 1.0])
def test_vcycle_with_boundary_faces_is_symmetric(oracle, theta):
    case = synth.random_case((16, 16, 16), seed=9, periodic=(False, False, True))
    g = synth.Grid(case.grid.n, case.grid.h, periodic=(False, False, True),
                   dirichlet=(True, True, False, True, False, False), ebc=(1e-19, 0, 0, 2e-19, 0, 0))
    p = case.params
    p.theta = theta
    op = oracle.assemble(g, p, case.E, case.nHI, case.eta)
    rng = np.random.default_rng(2)
    u = rng.standard_normal(g.shape)
    v = rng.standard_normal(g.shape)
    Bu = oracle.vcycle(g, op, u)
    Bv = oracle.vcycle(g, op, v)
    assert (Bu * v).sum() == pytest.approx((u * Bv).sum(), rel=1e-12)
    assert (Bu * u).sum() > 0


@pytest.mark.parametrize("theta", [0.5, 1.0])
def test_photon_balance_with_outflow_faces(oracle, theta):
    # Sec. 4.1 boundary set: reflecting at x, y, z = 0, outflow at the others;
    # the tight solve balances emission, absorption at E^n + theta dE and
    # the photons that left through the outflow faces
    case = synth.random_case((12, 8, 10), seed=17, periodic=(False,) * 3)
    g = synth.Grid(case.grid.n, case.grid.h).outflow_upper()
    p = case.params
    p.theta = theta
    E1, info = oracle.step(g, p, {"rtol": 1e-14, "max_iter": 200}, case.E, case.nHI, case.eta)
    assert info["outflow"] > 0
    assert info["balance_rel"] < 1e-9
    # at rtol 1e-8 the imbalance stays within V sqrt(N) ||r|| / h nu
    E2, info2 = oracle.step(g, p, {"rtol": 1e-8}, case.E, case.nHI, case.eta)
    op = oracle.assemble(g, p, case.E, case.nHI, case.eta)
    bound = g.volume * math.sqrt(g.cells) * info2["rel_res"] * np.linalg.norm(op["b"]) / p.hnu
    assert abs(info2["balance_abs"]) <= 1.01 * bound + 1e-9 * info2["emitted"]


def test_invalid_boundary_and_theta_rejected(oracle):
    g = synth.Grid((4, 4, 4), (1e20,) * 3, periodic=(True, False, False),
                   dirichlet=(True, False, False, False, False, False))
    E = np.full(g.shape, 1e-20)
    with pytest.raises(oracle.OracleError):
        oracle.step(g, phys(), {}, E, E * 0, E * 0)         # Dirichlet face on a periodic axis
    g2 = synth.Grid((4, 4, 4), (1e20,) * 3, dirichlet=(True,) + (False,) * 5, ebc=(-1.0,) + (0.0,) * 5)
    with pytest.raises(oracle.OracleError):
        oracle.step(g2, phys(), {}, E, E * 0, E * 0)        # negative E_b
    with pytest.raises(oracle.OracleError):
        oracle.step(synth.Grid.cube(4), phys(theta=0.0), {}, E, E * 0, E * 0)


# ------------------------------------------------- comoving coordinates

@pytest.mark.parametrize("theta", [0.5, 1.0])
def test_comoving_widths_act_as_proper_widths(oracle, theta):
    # a grid of comoving widths h at scale factor a is the grid of proper
    # widths a h: same operator and right-hand side (the gradients of the
    # equation are proper), whatever the limiter regime of each face
    case = synth.random_case((12, 10, 8), seed=21, periodic=(True, False, False))
    a = 0.2
    p = case.params
    p.theta, p.adot_over_a = theta, 3e-17
    g_c = synth.Grid(case.grid.n, case.grid.h, case.grid.periodic,
                     dirichlet=(False, False, True, False, False, True), ebc=(0, 0, 1e-19, 0, 0, 0))
    g_p = synth.Grid(case.grid.n, tuple(a * h for h in case.grid.h), case.grid.periodic,
                     dirichlet=g_c.dirichlet, ebc=g_c.ebc)
    p.scale_factor = a
    op_c = oracle.assemble(g_c, p, case.E, case.nHI, case.eta)
    p.scale_factor = 1.0
    op_p = oracle.assemble(g_p, p, case.E, case.nHI, case.eta)
    for k in ("m", "wx", "wy", "wz", "b", "bnd"):
        np.testing.assert_allclose(op_c[k], op_p[k], rtol=1e-14, atol=0)


def test_comoving_mode_decays_with_proper_wavenumber(oracle):
    # uniform medium, eta = eta0 + eps * mode: the mode's response carries
    # the diffusion rate D lambda / (a h)^2 of the proper wavenumber
    n = (16, 8, 12)
    a = 0.25
    kap = 1e-18
    g = synth.Grid(n, (2e20, 3e20, 2.5e20))
    p = phys(adot_over_a=1e-17, scale_factor=a, theta=0.5)
    mode, lam = cosine_modes(n, (3, 1, 2), False)
    E0, eta0, eps = 1e-18, 4e-24, 1e-24
    D = min(C / (3 * kap), 0.006 * C * p.L_unit)
    w = [p.dt * D / (a * h) ** 2 for h in g.h]
    s = C * kap + p.adot_over_a
    exact = p.dt * (eta0 - s * E0) / (1 + 0.5 * p.dt * s) \
        + p.dt * eps * mode / (1 + 0.5 * (p.dt * s + sum(wd * ld for wd, ld in zip(w, lam))))
    E1, _ = oracle.step(g, p, {"rtol": 1e-14, "max_iter": 200}, np.full(g.shape, E0),
                        np.full(g.shape, kap / p.sigma), eta0 + eps * mode)
    np.testing.assert_allclose(E1 - E0, exact, rtol=0, atol=1e-12 * np.abs(exact).max())
