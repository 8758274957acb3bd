"""Isothermal ionisation of a static neutral hydrogen region (the paper's
Sec. 4.1.1 verification test, after Iliev et al. Test 1): the FLD radiation
step coupled with the hydrogen-only photoionisation/recombination update
(loosely coupled, one linearly implicit step per radiation step).

The ionisation front follows r(t) = r_s (1 - exp(-t/t_rec))^(1/3) with
r_s = (3 N_dot / (4 pi alpha_B n_H^2))^(1/3) and t_rec = 1/(alpha_B n_H).
Parameters of the test: N_dot = 5e48 photons/s, n_H = 1e-3 cm^-3,
alpha_B = 2.59e-13 cm^3/s (1e4 K, the reading of the garbled unit), box
6.6 kpc, source in the corner cell with reflecting (zero-gradient) walls so
the box is one octant of the sphere and receives N_dot / 8, initial
E = 1e-45 erg/cm^3 and ionised fraction 0.0012.

The front radius is taken from the ionised volume, r = (3 * 8 V_ion / 4 pi)^(1/3).
The oracle run pins the coupled method to the closed form on the CPU; the
GPU runs are checked against the closed form and against the oracle."""
import math
import os

import numpy as np
import pytest

from paper_1306_0645_gb300 import synth

MYR = 1e6 * synth.YEAR
N_H = 1e-3
ALPHA = synth.ALPHA_B
R_S = (3 * synth.NDOT / (4 * math.pi * ALPHA * N_H ** 2)) ** (1 / 3)
T_REC = 1 / (ALPHA * N_H)


def r_analytic(t):
    return R_S * (1 - math.exp(-t / T_REC)) ** (1 / 3)


def setup(n):
    g = synth.Grid.cube(n)
    nH = np.full(g.shape, N_H)
    nHI = (1 - 0.0012) * nH
    E = np.full(g.shape, 1e-45)
    eta = np.zeros(g.shape)
    eta[0, 0, 0] = synth.NDOT / 8 * synth.HNU_HI / g.volume
    return g, nH, nHI, E, eta


def front_radius(g, nH, nHI):
    v_ion = float(((1 - nHI / nH) * g.volume).sum())
    return (3 * 8 * v_ion / (4 * math.pi)) ** (1 / 3)


def test_stromgren_front_oracle(oracle):
    n, dt, steps = 24, 1 * MYR, 300
    g, nH, nHI, E, eta = setup(n)
    p = synth.Params(limiter=synth.LIMITER_PAPER, dt=dt)
    checks = {}
    for k in range(1, steps + 1):
        E, _ = oracle.step(g, p, {}, E, nHI, eta)
        nHI = oracle.opacity_update(E, nH, nHI, dt, p.c, p.sigma, p.hnu, ALPHA)
        if k in (100, 200, 300):
            checks[k] = front_radius(g, nH, nHI) / r_analytic(k * dt)
    assert abs(checks[100] - 1) < 0.07, checks
    assert abs(checks[200] - 1) < 0.03, checks
    assert abs(checks[300] - 1) < 0.03, checks


def gpu_run(fld, torch, n, dt, steps, precision, marks, outflow=False, theta=1.0):
    g, nH, nHI, E, eta = setup(n)
    if outflow:
        g = g.outflow_upper()
    p = synth.Params(limiter=synth.LIMITER_PAPER, dt=dt, precision=precision, theta=theta)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()
    ctx = fld.fld_create(g, p)
    Eg, nHIg, nHg, etag = dev(E), dev(nHI), dev(nH), dev(eta)
    out = {}
    for k in range(1, steps + 1):
        fld.fld_step(ctx, Eg, nHIg, etag)
        fld.fld_opacity_update(Eg, nHg, nHIg, nHIg, dt, p.c, p.sigma, p.hnu, ALPHA)
        if k in marks:
            out[k] = (Eg.cpu().numpy().reshape(g.shape), nHIg.cpu().numpy().reshape(g.shape))
    ctx.close()
    return g, nH, out


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [synth.PREC_FP64, synth.PREC_MIXED])
def test_stromgren_front_gpu(precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_0645_gb300 import fld
    dt = 0.5 * MYR
    marks = (200, 400, 800)
    g, nH, out = gpu_run(fld, torch, 64, dt, 800, precision, marks)
    ratio = {k: front_radius(g, nH, out[k][1]) / r_analytic(k * dt) for k in marks}
    assert abs(ratio[200] - 1) < 0.06, ratio      # 100 Myr
    assert abs(ratio[400] - 1) < 0.03, ratio      # 200 Myr
    assert abs(ratio[800] - 1) < 0.03, ratio      # 400 Myr


@pytest.mark.gpu
@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_stromgren_front_gpu_paper_boundaries(theta):
    # the boundary set of the test: reflecting at x, y, z = 0 (the source's
    # corner), outflow at the three far faces; backward Euler and the
    # trapezoidal rule
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_0645_gb300 import fld
    dt = 0.5 * MYR
    marks = (200, 400, 800)
    g, nH, out = gpu_run(fld, torch, 64, dt, 800, synth.PREC_MIXED, marks, outflow=True, theta=theta)
    ratio = {k: front_radius(g, nH, out[k][1]) / r_analytic(k * dt) for k in marks}
    assert abs(ratio[200] - 1) < 0.06, ratio
    assert abs(ratio[400] - 1) < 0.03, ratio
    assert abs(ratio[800] - 1) < 0.03, ratio


@pytest.mark.gpu
def test_stromgren_gpu_matches_oracle(oracle):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_0645_gb300 import fld
    n, dt, steps = 24, 2 * MYR, 60
    g, nH, out = gpu_run(fld, torch, n, dt, steps, synth.PREC_FP64, (steps,))
    _, _, nHI, E, eta = setup(n)
    p = synth.Params(limiter=synth.LIMITER_PAPER, dt=dt)
    for _ in range(steps):
        E, _ = oracle.step(g, p, {}, E, nHI, eta)
        nHI = oracle.opacity_update(E, nH, nHI, dt, p.c, p.sigma, p.hnu, ALPHA)
    Eg, nHIg = out[steps]
    # both sides run the same algorithm at rtol 1e-8 for 60 coupled steps
    assert abs(front_radius(g, nH, nHIg) / front_radius(g, nH, nHI) - 1) < 1e-6
    assert np.linalg.norm(Eg - E) / np.linalg.norm(E) < 1e-6


# --------------------------------------------- cosmological I-front (Sec. 4.1.2)
#
# The same source in an expanding Einstein-de Sitter universe (q0 = 1/2,
# H0 = 50 km/s/Mpc), from z = 4, in a comoving box of 80 kpc with the
# initial proper density 1.175e-28 g/cm^3 of hydrogen.  E and eta are per
# comoving volume, the cell widths comoving (scale factor a through
# fld_set_expansion), n_H proper and falling as a^-3; the photoionisation
# rate takes the proper E / a^3.  The luminosity is 5e46 photons/s (the
# test's 5e48 /s front leaves this box within 100 Myr, before the expansion
# matters), so the front stays inside for 2 Gyr while a doubles.
#
# Closed form: photon counting for the comoving ionised volume V of the
# octant, n_c dV/dt = N_dot/8 - alpha_B n_c^2 V / a^3 with n_c = n_H a^3
# constant (the sharp-front model behind the Shapiro-Giroux solution),
# integrated numerically.  The ionised volume of the run counts each cell's
# ionisation beyond that of gas no photon reached (the 0.0012 initial
# ionisation recombines meanwhile).

H0_EDS = 50e5 / (1e3 * synth.KPC)
A0 = 0.2
NH_Z4 = 1.175e-28 / 1.6726e-24
NDOT_COSMO = 5e46
L_COSMO = 80 * synth.KPC


def eds_a(t):
    return (1.5 * H0_EDS * t) ** (2.0 / 3.0)


def eds_t(a):
    return 2.0 / (3.0 * H0_EDS) * a ** 1.5


def cosmo_front_closed_form(t_end, expanding=True):
    from scipy.integrate import solve_ivp
    nc = NH_Z4 * A0 ** 3
    t0 = eds_t(A0)

    def rhs(t, V):
        a = eds_a(t) if expanding else A0
        return [NDOT_COSMO / (8 * nc) - ALPHA * nc * V[0] / a ** 3]

    sol = solve_ivp(rhs, (t0, t0 + t_end), [0.0], rtol=1e-10, atol=1e30)
    return (3 * 8 * sol.y[0][-1] / (4 * math.pi)) ** (1 / 3)


def cosmo_setup(n):
    g = synth.Grid.cube(n, box=L_COSMO).outflow_upper()
    E = np.full(g.shape, 1e-45 * A0 ** 3)
    eta = np.zeros(g.shape)
    eta[0, 0, 0] = NDOT_COSMO / 8 * synth.HNU_HI / g.volume
    return g, E, eta


def cosmo_radius(g, x, x_dark):
    v = float((np.maximum(x_dark - x, 0.0) * g.volume).sum())
    return (3 * 8 * v / (4 * math.pi)) ** (1 / 3)


def shapiro_giroux_radius(a_rel, q0=0.5, z0=4.0):
    """The paper's closed form (Sec. 4.1.2) for the front, with a normalised
    to 1 at z0 and the integrand's (1 - z0) read as (1 + z0): r = r_s0
    (lambda e^-tau(a) int_1^a e^tau (1 - 2 q0 + 2 q0 (1 + z0) / s)^(-1/2)
    ds)^(1/3), tau(a) = lambda (F(a) - F(1)) / (6 q0^2 (1 + z0)^2),
    F(a) = (2 - 4 q0 - 2 q0 (1 + z0) / a) (1 - 2 q0 + 2 q0 (1 + z0) / a)^(1/2)."""
    from scipy.integrate import quad
    lam = ALPHA * NH_Z4 / H0_EDS / (1 + z0)
    r_s0 = (3 * NDOT_COSMO / (4 * math.pi * ALPHA * NH_Z4 ** 2)) ** (1 / 3)
    F = lambda a: (2 - 4 * q0 - 2 * q0 * (1 + z0) / a) * (1 - 2 * q0 + 2 * q0 * (1 + z0) / a) ** 0.5
    tau = lambda a: lam * (F(a) - F(1.0)) / (6 * q0 ** 2 * (1 + z0) ** 2)
    g = lambda s: math.exp(tau(s) - tau(a_rel)) * (1 - 2 * q0 + 2 * q0 * (1 + z0) / s) ** -0.5
    integral, _ = quad(g, 1.0, a_rel, epsabs=0.0, epsrel=1e-12, limit=200)
    return r_s0 * (lam * integral) ** (1 / 3)


def test_cosmological_closed_forms_agree():
    # the photon-counting reference the fronts are compared with equals the
    # paper's closed form (its r is the comoving radius times a0); the
    # golden file holds the printed parameters this test is built on
    here = os.path.dirname(os.path.abspath(__file__))
    gold = {}
    with open(os.path.join(here, "golden", "test2_cosmological.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (t.strip() for t in line.split("=", 1))
                gold[k] = float(v)
    z0 = gold["z_start"]
    assert A0 == pytest.approx(1 / (1 + z0), rel=1e-15)
    assert H0_EDS == pytest.approx(gold["H0_over_100km_s_Mpc"] * 100e5 / (1e3 * synth.KPC), rel=1e-15)
    assert NH_Z4 == pytest.approx(gold["rho_initial_g_cm3"] / 1.6726e-24, rel=1e-15)
    assert L_COSMO == pytest.approx(gold["box_comoving_kpc"] * synth.KPC, rel=1e-15)
    for t_myr in COSMO_MARKS_MYR:
        t = t_myr * MYR
        a_rel = eds_a(eds_t(A0) + t) / A0
        r_sg = shapiro_giroux_radius(a_rel, gold["q0"], z0)
        r_ode = cosmo_front_closed_form(t)
        assert r_sg / A0 == pytest.approx(r_ode, rel=1e-6), (t_myr, r_sg / A0, r_ode)


COSMO_MARKS_MYR = (200, 1000, 2000)


def test_cosmological_front_oracle(oracle):
    n, dt = 24, 5 * MYR
    g, E, eta = cosmo_setup(n)
    p = synth.Params(limiter=synth.LIMITER_PAPER, dt=dt, L_unit=L_COSMO)
    x = np.full(g.shape, 1 - 0.0012)
    xd = np.full(1, 1 - 0.0012)
    t0 = eds_t(A0)
    t = t0
    got = {}
    for k in range(1, int(COSMO_MARKS_MYR[-1] * MYR / dt) + 1):
        a = eds_a(t + 0.5 * dt)
        p.scale_factor, p.adot_over_a = a, H0_EDS * a ** -1.5
        nHp = NH_Z4 * (A0 / a) ** 3
        E, _ = oracle.step(g, p, {}, E, x * nHp, eta)
        ae = eds_a(t + dt)
        nHe = NH_Z4 * (A0 / ae) ** 3
        cp = synth.C_LIGHT / ae ** 3          # proper E = comoving E / a^3
        x = oracle.opacity_update(E, np.full(g.shape, nHe), x * nHe, dt, cp, p.sigma, p.hnu, ALPHA) / nHe
        xd = oracle.opacity_update(np.zeros(1), np.full(1, nHe), xd * nHe, dt, cp, p.sigma, p.hnu, ALPHA) / nHe
        t += dt
        tm = round((t - t0) / MYR)
        if tm in COSMO_MARKS_MYR:
            got[tm] = cosmo_radius(g, x, xd[0]) / cosmo_front_closed_form(t - t0)
    assert all(abs(r - 1) < 0.04 for r in got.values()), got
    # the expansion matters: a static universe's front is 13% behind by 2 Gyr
    T = COSMO_MARKS_MYR[-1] * MYR
    assert cosmo_front_closed_form(T, expanding=False) < 0.9 * cosmo_front_closed_form(T)


@pytest.mark.gpu
@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_cosmological_front_gpu(theta):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_0645_gb300 import fld
    n, dt = 64, 2.5 * MYR
    g, E0, eta0 = cosmo_setup(n)
    p = synth.Params(limiter=synth.LIMITER_PAPER, dt=dt, L_unit=L_COSMO, precision=synth.PREC_MIXED,
                     theta=theta)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()
    ctx = fld.fld_create(g, p)
    E, eta = dev(E0), dev(eta0)
    x = torch.full((g.cells,), 1 - 0.0012, dtype=torch.float64, device="cuda")
    xd = torch.full((1,), 1 - 0.0012, dtype=torch.float64, device="cuda")
    zero1 = torch.zeros(1, dtype=torch.float64, device="cuda")
    t0 = eds_t(A0)
    t = t0
    got = {}
    for k in range(1, int(COSMO_MARKS_MYR[-1] * MYR / dt) + 1):
        a = eds_a(t + 0.5 * dt)
        fld.fld_set_expansion(ctx, a, H0_EDS * a ** -1.5)
        nHp = NH_Z4 * (A0 / a) ** 3
        fld.fld_step(ctx, E, x * nHp, eta)
        ae = eds_a(t + dt)
        nHe = NH_Z4 * (A0 / ae) ** 3
        cp = synth.C_LIGHT / ae ** 3
        nH = torch.full_like(x, nHe)
        nHI = x * nHe
        fld.fld_opacity_update(E, nH, nHI, nHI, dt, cp, p.sigma, p.hnu, ALPHA)
        x = nHI / nHe
        nHd = xd * nHe
        fld.fld_opacity_update(zero1, torch.full_like(xd, nHe), nHd, nHd, dt, cp, p.sigma, p.hnu, ALPHA)
        xd = nHd / nHe
        t += dt
        tm = round((t - t0) / MYR)
        if tm in COSMO_MARKS_MYR:
            xh = x.cpu().numpy().reshape(g.shape)
            got[tm] = cosmo_radius(g, xh, float(xd[0])) / cosmo_front_closed_form(t - t0)
    ctx.close()
    assert all(abs(r - 1) < 0.04 for r in got.values()), got
