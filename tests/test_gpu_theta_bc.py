"""GPU parity of the theta-method (Sec. 3.2, trapezoidal rule) and of the
per-face boundary conditions (reflecting, Dirichlet and outflow faces of the
tests of Sec. 4.1), through the C ABI, against the FP64 CPU oracle.

Tolerances as in the other parity tests: assembly to rounding (1e-13 of the
largest entry), one V-cycle 1e-12, FP64 steps solved to 1e-13 agree to
1e-10, mixed-precision steps at the paper's 1e-8 to 1e-6 (L2 and max)."""
import math

import numpy as np
import pytest

from paper_1306_0645_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fld():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_0645_gb300 import fld as f
    f.lib()
    return f


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t, shape):
    return t.cpu().numpy().reshape(shape)


def rel_max(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


def with_faces(case, dirichlet, ebc=(0.0,) * 6, theta=1.0):
    g = case.grid
    case.grid = synth.Grid(g.n, g.h, g.periodic, dirichlet=dirichlet, ebc=ebc)
    case.params.theta = theta
    return case


CASES = [
    # (name, builder)
    ("outflow_upper_be", lambda: with_faces(synth.random_case((16, 12, 20), seed=1), (False, True) * 3)),
    ("outflow_upper_tr", lambda: with_faces(synth.random_case((16, 12, 20), seed=1), (False, True) * 3,
                                            theta=0.5)),
    ("dirichlet_mixed", lambda: with_faces(synth.random_case((24, 16, 8), seed=2, periodic=(False, False, True)),
                                           (True, False, True, True, False, False),
                                           (1e-19, 0.0, 3e-20, 0.0, 0.0, 0.0), theta=0.75)),
    ("all_dirichlet_odd", lambda: with_faces(synth.random_case((5, 7, 9), seed=3), (True,) * 6,
                                             (1e-21, 2e-20, 0.0, 5e-19, 1e-22, 0.0))),
    ("trapezoidal_periodic", lambda: with_faces(synth.random_case((32, 32, 32), seed=4, periodic=(True,) * 3),
                                                (False,) * 6, theta=0.5)),
    ("one_cell_outflow", lambda: with_faces(synth.random_case((1, 1, 1), seed=5), (True, False) * 3, theta=0.5)),
]


@pytest.mark.parametrize("name,make", CASES)
def test_assembly_parity(fld, oracle, name, make):
    case = make()
    case.params.adot_over_a = 2e-17
    ref = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    ctx = fld.fld_create(case.grid, case.params)
    fld.fld_assemble(ctx, dev(case.E), dev(case.nHI), dev(case.eta))
    out = {k: torch.empty(case.grid.cells, dtype=torch.float64, device="cuda") for k in ("m", "wx", "wy", "wz", "b")}
    fld.fld_get_system(ctx, **out)
    sh = case.grid.shape
    for k in ("m", "wx", "wy", "wz"):
        np.testing.assert_allclose(host(out[k], sh), ref[k], rtol=1e-13, atol=0)
    assert rel_max(host(out["b"], sh), ref["b"]) < 1e-13
    ctx.close()


@pytest.mark.parametrize("name,make", CASES[:5])
def test_vcycle_parity(fld, oracle, name, make):
    case = make()
    op = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    ctx = fld.fld_create(case.grid, case.params)
    fld.fld_assemble(ctx, dev(case.E), dev(case.nHI), dev(case.eta))
    x = np.random.default_rng(6).standard_normal(case.grid.shape)
    z = torch.empty(case.grid.cells, dtype=torch.float64, device="cuda")
    fld.fld_vcycle(ctx, dev(x), z)
    assert rel_max(host(z, x.shape), oracle.vcycle(case.grid, op, x)) < 1e-12
    ctx.close()


@pytest.mark.parametrize("name,make", CASES)
def test_fp64_step_parity_tight(fld, oracle, name, make):
    case = make()
    p = case.params
    p.rtol, p.max_iter = 1e-13, 200
    ctx = fld.fld_create(case.grid, p)
    E = dev(case.E)
    info = fld.fld_step(ctx, E, dev(case.nHI), dev(case.eta))
    ctx.close()
    Eref, iref = oracle.step(case.grid, p, {"rtol": 1e-13, "max_iter": 200}, case.E, case.nHI, case.eta)
    E = host(E, case.grid.shape)
    assert info["rel_res"] <= 1e-13
    assert rel_max(E - case.E, Eref - case.E) < 1e-10
    np.testing.assert_allclose(E, Eref, rtol=1e-10, atol=1e-10 * np.abs(Eref).max())
    # photon accounting of the step, face fluxes included
    for k in ("emitted", "absorbed", "outflow"):
        assert info[k] == pytest.approx(iref[k], rel=1e-8, abs=1e-8 * iref["emitted"]), k
    assert info["balance_rel"] < 1e-9


@pytest.mark.parametrize("name,make", CASES[:5])
def test_mixed_step_parity_at_paper_tolerance(fld, oracle, name, make):
    case = make()
    p = case.params
    p.precision = synth.PREC_MIXED
    ctx = fld.fld_create(case.grid, p)
    E = dev(case.E)
    info = fld.fld_step(ctx, E, dev(case.nHI), dev(case.eta))
    ctx.close()
    assert info["rel_res"] <= 1e-8
    Eref, _ = oracle.step(case.grid, p, {"rtol": 1e-13, "max_iter": 200}, case.E, case.nHI, case.eta)
    E = host(E, case.grid.shape)
    el2 = np.linalg.norm(E - Eref) / np.linalg.norm(Eref)
    einf = np.abs(E - Eref).max() / np.abs(Eref).max()
    assert el2 < 1e-6 and einf < 1e-6, (el2, einf)


@pytest.mark.parametrize("precision", [synth.PREC_FP64, synth.PREC_MIXED])
@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_two_sources_anisotropic_grid(fld, oracle, precision, theta):
    # 128 x 64 x 64 cells, outflow on every face, several steps in a row
    case = synth.config_two_sources(128, theta=theta, precision=precision)
    p = case.params
    ctx = fld.fld_create(case.grid, p)
    E = dev(case.E)
    nHI, eta = dev(case.nHI), dev(case.eta)
    Eref = case.E.copy()
    for step in range(3):
        info = fld.fld_step(ctx, E, nHI, eta)
        Eref, iref = oracle.step(case.grid, p, {"rtol": 1e-13, "max_iter": 200}, Eref, case.nHI, case.eta)
        assert info["rel_res"] <= 1e-8 and info["balance_rel"] < 1e-6
        # the fronts are far from the faces: the outflow is within the
        # solver's noise on the faint background there
        assert abs(info["outflow"]) <= 1e-6 * info["emitted"]
    ctx.close()
    Eg = host(E, case.grid.shape)
    el2 = np.linalg.norm(Eg - Eref) / np.linalg.norm(Eref)
    einf = np.abs(Eg - Eref).max() / np.abs(Eref).max()
    assert el2 < 1e-6 and einf < 1e-6, (el2, einf)
    # the two sources' fronts are mirror images about the box centre (to the
    # solver tolerance relative to the peak)
    mid = Eg[32, 32, :]
    np.testing.assert_allclose(mid[38 - 10:38 + 11], mid[89 + 10:89 - 11:-1], rtol=1e-5,
                               atol=1e-7 * mid.max())


def test_theta_validation(fld):
    g = synth.Grid.cube(8)
    with pytest.raises(fld.FldError):
        fld.fld_create(g, synth.Params(theta=0.4))
    g2 = synth.Grid((8, 8, 8), (1e20,) * 3, periodic=(True, False, False),
                    dirichlet=(True,) + (False,) * 5)
    with pytest.raises(fld.FldError):
        fld.fld_create(g2, synth.Params())
    g3 = synth.Grid((8, 8, 8), (1e20,) * 3, dirichlet=(True,) + (False,) * 5, ebc=(math.inf,) + (0.0,) * 5)
    with pytest.raises(fld.FldError):
        fld.fld_create(g3, synth.Params())


def test_comoving_scale_factor_parity(fld, oracle):
    # comoving widths at scale factor a, changed between steps through
    # fld_set_expansion; FP64 steps solved tightly against the oracle
    case = with_faces(synth.random_case((24, 16, 20), seed=31), (False, True) * 3, theta=0.5)
    p = case.params
    p.rtol, p.max_iter = 1e-13, 200
    p.scale_factor, p.adot_over_a = 0.25, 4e-17
    ctx = fld.fld_create(case.grid, p)
    fld.fld_assemble(ctx, dev(case.E), dev(case.nHI), dev(case.eta))
    out = {k: torch.empty(case.grid.cells, dtype=torch.float64, device="cuda") for k in ("m", "wx", "wy", "wz", "b")}
    fld.fld_get_system(ctx, **out)
    ref = oracle.assemble(case.grid, p, case.E, case.nHI, case.eta)
    sh = case.grid.shape
    for k in ("m", "wx", "wy", "wz"):
        np.testing.assert_allclose(host(out[k], sh), ref[k], rtol=1e-13, atol=0)
    E = dev(case.E)
    Eref = case.E.copy()
    for a, h in ((0.25, 4e-17), (0.3, 3e-17), (0.5, 1e-17)):
        fld.fld_set_expansion(ctx, a, h)
        p.scale_factor, p.adot_over_a = a, h
        info = fld.fld_step(ctx, E, dev(case.nHI), dev(case.eta))
        Eref, _ = oracle.step(case.grid, p, {"rtol": 1e-13, "max_iter": 200}, Eref, case.nHI, case.eta)
        assert info["rel_res"] <= 1e-13
    with pytest.raises(fld.FldError):
        fld.fld_set_expansion(ctx, 0.0, 1e-17)
    ctx.close()
    np.testing.assert_allclose(host(E, sh), Eref, rtol=1e-10, atol=1e-10 * np.abs(Eref).max())
