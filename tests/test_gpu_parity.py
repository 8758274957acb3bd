"""GPU parity: the CUDA path, called through the C ABI, against the FP64 CPU
oracle on the same seeded inputs.

Tolerances: FP64 path 1e-10 relative in E^{n+1} (both solved to 1e-13, or
both run the same iterations); assembly, one V-cycle and the operator
application agree to rounding (1e-12 relative to the largest entry); mixed
precision 1e-6 relative in E^{n+1} (max over cells with E > 1e-6 max E, and
L2 over all cells)."""
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


def host(t):
    return t.cpu().numpy()


def rel_max(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


def e_errors(E_gpu, E_ref):
    mask = E_ref > 1e-6 * E_ref.max()
    emax = (np.abs(E_gpu - E_ref)[mask] / E_ref[mask]).max()
    el2 = np.linalg.norm(E_gpu - E_ref) / np.linalg.norm(E_ref)
    return emax, el2


SMALL = [
    ((8, 8, 8), (False,) * 3, synth.LIMITER_PAPER),
    ((16, 12, 20), (True, False, True), synth.LIMITER_LP),
    ((5, 5, 5), (True,) * 3, synth.LIMITER_PAPER),
    ((7, 6, 9), (False, True, False), synth.LIMITER_LP),
    ((32, 32, 32), (True,) * 3, synth.LIMITER_PAPER),
    ((24, 16, 40), (False,) * 3, synth.LIMITER_PAPER),
    ((1, 1, 1), (False,) * 3, synth.LIMITER_PAPER),
    ((2, 3, 1), (True,) * 3, synth.LIMITER_LP),
]


@pytest.mark.parametrize("n,per,lim", SMALL)
def test_assembly_parity(fld, oracle, n, per, lim):
    case = synth.random_case(n, seed=100 + sum(n), periodic=per, limiter=lim, zero_frac=0.05)
    case.params.adot_over_a = 2e-17
    ref = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    ctx = fld.fld_create(case.grid, case.params)
    E, nHI, eta = dev(case.E), dev(case.nHI), dev(case.eta)
    fld.fld_assemble(ctx, E, nHI, eta)
    out = {k: torch.empty_like(E) for k in ("m", "wx", "wy", "wz", "b")}
    fld.fld_get_system(ctx, **out)
    for k in ("m", "wx", "wy", "wz"):
        np.testing.assert_allclose(host(out[k]).reshape(ref[k].shape), ref[k], rtol=1e-13, atol=0)
    assert rel_max(host(out["b"]).reshape(ref["b"].shape), ref["b"]) < 1e-13
    ctx.close()


def test_assembly_paper_limiter_regimes(fld, oracle):
    # gradients spanning the capped, thick and streaming regimes of the limiter
    g = synth.Grid((64, 4, 4), (1e19, 2e20, 2e20))
    p = synth.Params(limiter=synth.LIMITER_PAPER)
    x = np.arange(64)
    E = np.broadcast_to(10.0 ** (-30 + 0.3 * np.maximum(x - 32, 0)), g.shape).copy()
    nHI = np.broadcast_to(10.0 ** (-8 + 0.15 * x), g.shape).copy()
    eta = np.zeros(g.shape)
    ref = oracle.assemble(g, p, E, nHI, eta)
    ctx = fld.fld_create(g, p)
    fld.fld_assemble(ctx, dev(E), dev(nHI), dev(eta))
    wx = torch.empty(g.cells, dtype=torch.float64, device="cuda")
    fld.fld_get_system(ctx, wx=wx)
    np.testing.assert_allclose(host(wx).reshape(g.shape), ref["wx"], rtol=1e-13, atol=0)
    D = ref["wx"][0, 0, 1:] / (p.dt / g.h[0] ** 2)
    Dmax = 0.006 * p.c * p.L_unit
    assert np.isclose(D, Dmax, rtol=1e-12).any() and (D < 0.5 * Dmax).any()


@pytest.mark.parametrize("n,per,lim", SMALL)
def test_mixed_assembly_parity(fld, oracle, n, per, lim):
    """The mixed solver's double-float operator (an FP32 high part plus a low
    part, both returned as FP64 by fld_get_system) and its FP64 right-hand
    side, assembled on the FP32 pipe, against the oracle's FP64 assembly."""
    case = synth.random_case(n, seed=100 + sum(n), periodic=per, limiter=lim, zero_frac=0.05)
    case.params.adot_over_a = 2e-17
    case.params.precision = synth.PREC_MIXED
    ref = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    ctx = fld.fld_create(case.grid, case.params)
    E, nHI, eta = dev(case.E), dev(case.nHI), dev(case.eta)
    fld.fld_assemble(ctx, E, nHI, eta)
    out = {k: torch.empty_like(E) for k in ("m", "wx", "wy", "wz", "b")}
    fld.fld_get_system(ctx, **out)
    for k in ("m", "wx", "wy", "wz"):
        np.testing.assert_allclose(host(out[k]).reshape(ref[k].shape), ref[k], rtol=1e-12, atol=0)
    assert rel_max(host(out["b"]).reshape(ref["b"].shape), ref["b"]) < 1e-12
    ctx.close()


@pytest.mark.parametrize("prec", [synth.PREC_FP64, synth.PREC_MIXED])
def test_mixed_limiter_regimes(fld, oracle, prec):
    """Capped, thick and streaming faces along one axis, with face energies
    over 43 decades: the FP64 and the double-float limiter against the
    oracle's."""
    g = synth.Grid((64, 4, 4), (1e19, 2e20, 2e20))
    p = synth.Params(limiter=synth.LIMITER_PAPER, precision=prec)
    x = np.arange(64)
    E = np.broadcast_to(10.0 ** (-30 + 1.4 * np.maximum(x - 32, 0)), g.shape).copy()
    nHI = np.broadcast_to(10.0 ** (-8 + 0.15 * x), g.shape).copy()
    eta = np.zeros(g.shape)
    ref = oracle.assemble(g, p, E, nHI, eta)
    ctx = fld.fld_create(g, p)
    fld.fld_assemble(ctx, dev(E), dev(nHI), dev(eta))
    wx = torch.empty(g.cells, dtype=torch.float64, device="cuda")
    fld.fld_get_system(ctx, wx=wx)
    np.testing.assert_allclose(host(wx).reshape(g.shape), ref["wx"], rtol=1e-12, atol=0)
    ctx.close()


@pytest.mark.parametrize("n,per,lim", SMALL[:6])
def test_apply_and_vcycle_parity(fld, oracle, n, per, lim):
    case = synth.random_case(n, seed=200 + sum(n), periodic=per, limiter=lim)
    op = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    ctx = fld.fld_create(case.grid, case.params)
    fld.fld_assemble(ctx, dev(case.E), dev(case.nHI), dev(case.eta))
    rng = np.random.default_rng(3)
    x = rng.standard_normal(case.grid.shape)
    y = torch.empty(case.grid.cells, dtype=torch.float64, device="cuda")
    fld.fld_apply(ctx, dev(x), y)
    assert rel_max(host(y).reshape(x.shape), oracle.apply(case.grid, op, x)) < 1e-13
    z = torch.empty_like(y)
    fld.fld_vcycle(ctx, dev(x), z)
    zref = oracle.vcycle(case.grid, op, x)
    assert rel_max(host(z).reshape(x.shape), zref) < 1e-12
    ctx.close()


@pytest.mark.parametrize("smoother", [synth.SMOOTH_RBGS, synth.SMOOTH_JACOBI])
@pytest.mark.parametrize("prepost", [(1, 1), (2, 2), (0, 1)])
def test_vcycle_smoother_variants(fld, oracle, smoother, prepost):
    case = synth.random_case((32, 16, 24), seed=7, periodic=(True, False, False))
    op = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    p = case.params
    p.smoother, p.pre, p.post = smoother, prepost[0], prepost[1]
    ctx = fld.fld_create(case.grid, p)
    fld.fld_assemble(ctx, dev(case.E), dev(case.nHI), dev(case.eta))
    x = np.random.default_rng(5).standard_normal(case.grid.shape)
    z = torch.empty(case.grid.cells, dtype=torch.float64, device="cuda")
    fld.fld_vcycle(ctx, dev(x), z)
    zref = oracle.vcycle(case.grid, op, x, {"smoother": smoother, "pre": prepost[0], "post": prepost[1]})
    assert rel_max(host(z).reshape(x.shape), zref) < 1e-12
    ctx.close()


@pytest.mark.parametrize("n,per,tail", [((64, 32, 48), (False, False, False), 32768),
                                        ((128, 64, 32), (True, False, True), 32768),
                                        ((96, 96, 64), (False, True, False), 32768),
                                        # nx = 4 mod 8: the zero-guess residual in the full layout
                                        ((100, 24, 24), (False, False, False), 32768),
                                        ((100, 24, 24), (True, True, False), 32768),
                                        # no persistent tail: four-cell kernels on the coarse levels too
                                        ((128, 96, 64), (False, False, True), 0)])
@pytest.mark.parametrize("pre", [1, 2])
def test_mixed_vcycle_parity(fld, oracle, n, per, tail, pre):
    # the FP32 cycle of a mixed context against the oracle's FP64 cycle.  With
    # one pre-sweep the residual takes the zero-guess form (the weighted sum
    # of the black neighbours at red cells, 0 at black cells), which equals
    # r - A z in exact arithmetic; with two pre-sweeps it is r - A z itself.
    # Both agree with the oracle to FP32 rounding of the cycle (the FP32
    # coefficients: precond_bf16 = 0; the bfloat16 ones in test_gpu_bf16.py).
    case = synth.random_case(n, seed=400 + sum(n), periodic=per, E_decades=(-20, -14))
    op = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    p = case.params
    p.precision, p.pre, p.post, p.tail_cells = synth.PREC_MIXED, pre, 1, tail
    p.precond_bf16 = 0
    ctx = fld.fld_create(case.grid, p)
    fld.fld_assemble(ctx, dev(case.E), dev(case.nHI), dev(case.eta))
    x = np.random.default_rng(11).standard_normal(case.grid.shape)
    z = torch.empty(case.grid.cells, dtype=torch.float64, device="cuda")
    fld.fld_vcycle(ctx, dev(x), z)
    ctx.close()
    zg = host(z).reshape(x.shape)
    zref = oracle.vcycle(case.grid, op, x, {"pre": pre, "post": 1})
    el2 = np.linalg.norm(zg - zref) / np.linalg.norm(zref)
    einf = np.abs(zg - zref).max() / np.abs(zref).max()
    assert el2 < 1e-5 and einf < 1e-5, (el2, einf)


def fp64_step_pair(fld, oracle, case, rtol=1e-13, max_iter=200):
    p = case.params
    p.rtol, p.max_iter = rtol, max_iter
    ctx = fld.fld_create(case.grid, p)
    E = dev(case.E)
    info = fld.fld_step(ctx, E, dev(case.nHI), dev(case.eta))
    Eref, iref = oracle.step(case.grid, p, {"rtol": rtol, "max_iter": max_iter, "smoother": p.smoother},
                             case.E, case.nHI, case.eta)
    ctx.close()
    return host(E).reshape(case.grid.shape), Eref, info, iref


STEP_CASES = [
    lambda: synth.config1(32),
    lambda: synth.config2(32),
    lambda: synth.random_case((5, 5, 5), seed=1, periodic=(True,) * 3),
    lambda: synth.random_case((24, 16, 8), seed=2, periodic=(False, True, False), limiter=synth.LIMITER_LP),
    lambda: synth.config_uniform(48, sources=8, seed=9),
    lambda: synth.random_case((1, 1, 1), seed=4),
]


@pytest.mark.parametrize("make", STEP_CASES)
def test_fp64_step_parity_tight(fld, oracle, make):
    case = make()
    E, Eref, info, iref = fp64_step_pair(fld, oracle, case)
    assert info["rel_res"] <= 1e-13
    assert rel_max(E - case.E, Eref - case.E) < 1e-10
    np.testing.assert_allclose(E, Eref, rtol=1e-10, atol=1e-10 * np.abs(Eref).max())


@pytest.mark.parametrize("make", STEP_CASES[:2])
def test_fp64_step_same_iterations_at_paper_tolerance(fld, oracle, make):
    # both sides run the same algorithm, so at rtol 1e-8 they take the same
    # number of iterations and agree to rounding
    case = make()
    E, Eref, info, iref = fp64_step_pair(fld, oracle, case, rtol=1e-8, max_iter=50)
    assert info["iters"] == iref["iters"]
    assert info["rel_res"] <= 1e-8
    assert rel_max(E - case.E, Eref - case.E) < 1e-10


def test_fp64_jacobi_step(fld, oracle):
    case = synth.config2(32)
    case.params.smoother = synth.SMOOTH_JACOBI
    E, Eref, info, iref = fp64_step_pair(fld, oracle, case)
    assert rel_max(E - case.E, Eref - case.E) < 1e-10


MIXED_CASES = [lambda: synth.config3(64, sources=64), lambda: synth.config2(64),
               lambda: synth.config4(64, sources=512),
               lambda: synth.random_case((96, 48, 40), seed=12, periodic=(True, False, True)),
               lambda: synth.random_case((16, 24, 20), seed=13, periodic=(False, True, False))]


def mixed_step(fld, case, rtol):
    p = case.params
    p.precision = synth.PREC_MIXED
    p.rtol = rtol
    ctx = fld.fld_create(case.grid, p)
    E = dev(case.E)
    info = fld.fld_step(ctx, E, dev(case.nHI), dev(case.eta))
    ctx.close()
    return host(E).reshape(case.grid.shape), info


@pytest.mark.parametrize("make", MIXED_CASES)
def test_mixed_step_parity_at_paper_tolerance(fld, oracle, make):
    # at ||r||/||b|| <= 1e-8 the result is as accurate as the tolerance allows:
    # 1e-6 in the L2 and max norms relative to the field
    case = make()
    E, info = mixed_step(fld, case, 1e-8)
    assert info["rel_res"] <= 1e-8 and info["outer_iters"] >= 1
    Eref, _ = oracle.step(case.grid, case.params, {"rtol": 1e-13, "max_iter": 200}, case.E, case.nHI, case.eta)
    el2 = np.linalg.norm(E - Eref) / np.linalg.norm(Eref)
    einf = np.abs(E - Eref).max() / np.abs(Eref).max()
    assert el2 < 1e-6 and einf < 1e-6, (el2, einf)


@pytest.mark.parametrize("make", MIXED_CASES)
def test_mixed_step_converges_pointwise_to_fp64(fld, oracle, make):
    # FP32 V-cycles inside FP64 refinement reach the FP64 answer cell by cell
    # (relative error in every cell with E > 1e-6 max E) when asked to
    case = make()
    E, info = mixed_step(fld, case, 1e-12)
    assert info["rel_res"] <= 1e-12
    Eref, _ = oracle.step(case.grid, case.params, {"rtol": 1e-13, "max_iter": 200}, case.E, case.nHI, case.eta)
    emax, el2 = e_errors(E, Eref)
    assert emax < 1e-6 and el2 < 1e-9, (emax, el2)


def test_step_balance_and_positivity_128(fld, oracle):
    case = synth.config2(128)
    ctx = fld.fld_create(case.grid, case.params)
    E = dev(case.E)
    info = fld.fld_step(ctx, E, dev(case.nHI), dev(case.eta))
    op = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    bnorm = np.linalg.norm(op["b"])
    bound = case.grid.volume * math.sqrt(case.grid.cells) * info["rel_res"] * bnorm / case.params.hnu
    assert abs(info["balance_abs"]) <= 1.01 * bound + 1e-9 * info["emitted"]
    En = host(E)
    assert En.min() >= 0.0
    assert info["floor_added"] <= 1e-6 * info["emitted"]
    # the residual of the GPU solution, recomputed by the oracle's operator
    fld.fld_assemble(ctx, dev(case.E), dev(case.nHI), dev(case.eta))
    dE = torch.empty_like(E)
    fld.fld_solve(ctx, dE)
    r = op["b"] - oracle.apply(case.grid, op, host(dE).reshape(case.grid.shape))
    assert np.linalg.norm(r) / bnorm <= 1.01e-8
    ctx.close()


def test_zero_rhs_and_single_cell(fld):
    g = synth.Grid.cube(16)
    ctx = fld.fld_create(g, synth.Params())
    E = torch.zeros(g.cells, dtype=torch.float64, device="cuda")
    info = fld.fld_step(ctx, E, torch.full_like(E, 1e-3), torch.zeros_like(E))
    assert info["iters"] == 0 and float(E.abs().max()) == 0.0
    ctx.close()


def test_noconv_leaves_E_unchanged(fld):
    case = synth.config1(32)
    ctx = fld.fld_create(case.grid, case.params, max_iter=1, rtol=1e-14)
    E = dev(case.E)
    info = fld.fld_step(ctx, E, dev(case.nHI), dev(case.eta), check=False)
    assert info["status"] == fld.FLD_ENOCONV
    assert np.array_equal(host(E).reshape(case.grid.shape), case.E)
    ctx.close()


def test_invalid_inputs_rejected(fld):
    g = synth.Grid.cube(8)
    ctx = fld.fld_create(g, synth.Params())
    E = torch.full((g.cells,), 1e-20, dtype=torch.float64, device="cuda")
    nHI = torch.full_like(E, 1e-3)
    eta = torch.zeros_like(E)
    E[3] = -1.0
    with pytest.raises(fld.FldError) as e:
        fld.fld_step(ctx, E, nHI, eta)
    assert e.value.status == fld.FLD_EINVAL
    E[3] = float("nan")
    with pytest.raises(fld.FldError):
        fld.fld_step(ctx, E, nHI, eta)
    ctx.close()
    with pytest.raises(fld.FldError) as e:
        fld.fld_create(synth.Grid.cube(101), synth.Params())
    assert e.value.status == fld.FLD_EINVAL


def test_host_buffer_step_matches_device_step(fld):
    case = synth.config1(32)
    ctx = fld.fld_create(case.grid, case.params)
    E = dev(case.E)
    fld.fld_step(ctx, E, dev(case.nHI), dev(case.eta))
    Eh = case.E.copy()
    fld.fld_step_host(ctx, Eh, case.nHI, case.eta)
    assert np.array_equal(Eh.ravel(), host(E).ravel())
    ctx.close()


@pytest.mark.parametrize("n,per,prec,outflow", [((128, 128, 128), (False, False, False), synth.PREC_MIXED, False),
                                                ((160, 128, 144), (True, True, False), synth.PREC_MIXED, False),
                                                ((128, 128, 160), (False, False, False), synth.PREC_FP64, False),
                                                ((128, 128, 128), (False, False, True), synth.PREC_MIXED, False),
                                                ((128, 128, 128), (False, False, False), synth.PREC_MIXED, True)])
def test_overlapped_host_step_matches_device_step(fld, n, per, prec, outflow):
    # from 128^3 cells on a non-periodic z axis the host-buffer step moves
    # its inputs in plane chunks and assembles each chunk as it arrives, the
    # right-hand side's reductions summed per chunk; the per-cell arithmetic
    # is that of the device-buffer step, so E agrees bit for bit whenever the
    # iteration counts do (a periodic z axis takes the plain transfer)
    case = synth.config4(128, sources=256)
    g = synth.Grid(n, tuple(case.grid.h[a] for a in range(3)), per)
    if outflow:   # Dirichlet faces: the chunked right-hand side also writes their weights
        g = g.outflow_upper()
    rng = np.random.default_rng(17)
    E0 = 10.0 ** rng.uniform(-20, -14, g.shape)
    nHI = 10.0 ** rng.uniform(-5, -2, g.shape)
    eta = np.zeros(g.shape)
    eta.ravel()[rng.choice(g.cells, 64, replace=False)] = 1e-21
    p = case.params
    p.precision = prec
    ctx = fld.fld_create(g, p)
    E = dev(E0)
    i_dev = fld.fld_step(ctx, E, dev(nHI), dev(eta))
    Eh = E0.copy()
    i_host = fld.fld_step_host(ctx, Eh, nHI, eta)
    ctx.close()
    assert (i_host["iters"], i_host["outer_iters"]) == (i_dev["iters"], i_dev["outer_iters"])
    assert np.array_equal(Eh.ravel(), host(E).ravel())
    assert abs(i_host["rel_res"] - i_dev["rel_res"]) <= 1e-12 * i_dev["rel_res"]


def test_opacity_update_parity(fld, oracle):
    rng = np.random.default_rng(8)
    n = 10000
    E = 10 ** rng.uniform(-25, -12, n)
    nH = 10 ** rng.uniform(-4, -2, n)
    nHI = nH * rng.uniform(0, 1, n)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    fld.fld_opacity_update(dev(E), dev(nH), dev(nHI), out, synth.DT, synth.C_LIGHT, synth.SIGMA_HI,
                           synth.HNU_HI, synth.ALPHA_B)
    torch.cuda.synchronize()
    ref = oracle.opacity_update(E, nH, nHI, synth.DT, synth.C_LIGHT, synth.SIGMA_HI, synth.HNU_HI,
                                synth.ALPHA_B)
    np.testing.assert_allclose(host(out), ref, rtol=1e-14)


@pytest.mark.parametrize("precision", [synth.PREC_FP64, synth.PREC_MIXED])
def test_graph_replay_equals_direct_launches(fld, precision):
    # one CUDA graph per CG iteration replays exactly the launches it holds
    case = synth.config3(48, sources=16)
    case.params.precision = precision
    out = []
    s = torch.cuda.Stream()
    for graphs in (0, 1):
        case.params.graphs = graphs
        with torch.cuda.stream(s):
            ctx = fld.fld_create(case.grid, case.params, s)
            E = dev(case.E)
            infos = [fld.fld_step(ctx, E, dev(case.nHI), dev(case.eta)) for _ in range(3)]
            s.synchronize()
            out.append((host(E), [i["iters"] for i in infos]))
            ctx.close()
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0])


def test_advance_parity_with_oracle(fld, oracle):
    # radiation subcycling (Sec. 3.3): same substep sequence and result
    case = synth.config1(32)
    p = case.params
    p.rtol, p.max_iter = 1e-12, 200
    span = 5 * p.dt
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fld.fld_create(case.grid, p, s)
        E = dev(case.E)
        info = fld.fld_advance(ctx, E, dev(case.nHI), dev(case.eta), span, 0.05 * p.dt, tau_tol=1e-2,
                               dt_min=1e-6 * p.dt)
        s.synchronize()
        ctx.close()
    Eref, iref = oracle.advance(case.grid, p, {"rtol": 1e-12, "max_iter": 200}, case.E, case.nHI, case.eta,
                                span, 0.05 * p.dt, tau_tol=1e-2, dt_min=1e-6 * p.dt)
    assert info["substeps"] == iref["substeps"] and info["retries"] == iref["retries"] == 0
    assert info["t_done"] == span
    assert rel_max(host(E).reshape(case.grid.shape), Eref) < 1e-9


def test_advance_retries_on_failure(fld):
    case = synth.config1(16)
    p = case.params
    p.max_iter = 2
    ctx = fld.fld_create(case.grid, p)
    E = dev(case.E)
    info = fld.fld_advance(ctx, E, dev(case.nHI), dev(case.eta), p.dt, p.dt, tau_tol=1e3,
                           dt_min=1e-8 * p.dt, check=False)
    assert info["retries"] >= 1
    p.max_iter, p.rtol = 1, 1e-14
    ctx2 = fld.fld_create(case.grid, p)
    E2 = dev(case.E)
    info2 = fld.fld_advance(ctx2, E2, dev(case.nHI), dev(case.eta), p.dt, p.dt, tau_tol=1e3,
                            dt_min=1e-3 * p.dt, check=False)
    assert info2["status"] == fld.FLD_ENOCONV and info2["t_done"] < p.dt
    ctx.close()
    ctx2.close()


@pytest.mark.parametrize("make", [lambda: synth.config4(128, sources=1024), lambda: synth.config2(128),
                                  lambda: synth.random_case((128, 40, 24), seed=12, periodic=(True, False, True)),
                                  lambda: synth.random_case((160, 32, 24), seed=13, periodic=(False, True, False)),
                                  lambda: synth.random_case((96, 48, 40), seed=14, periodic=(True, False, True))])
def test_fused_post_sweep_equals_colour_sweeps(fld, make):
    # the fused black+red post-sweep does the arithmetic of the two colour
    # sweeps, so the whole mixed step is bit-identical (rows of 128 cells
    # and more take the fused kernel: periodic and reflecting axes, a
    # partial last block of lanes, rows that are not a multiple of PBY); the
    # fused kernel reads FP32 coefficients, so the colour sweeps do too
    case = make()
    case.params.precision = synth.PREC_MIXED
    case.params.precond_bf16 = 0
    out = []
    for fused in (0, 1):
        case.params.fused_post = fused
        ctx = fld.fld_create(case.grid, case.params)
        E = dev(case.E)
        infos = [fld.fld_step(ctx, E, dev(case.nHI), dev(case.eta)) for _ in range(2)]
        out.append((host(E), [(i["iters"], i["outer_iters"]) for i in infos]))
        ctx.close()
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0])


def test_autotune_cache_roundtrip_and_parity(fld, oracle, tmp_path):
    case = synth.config4(64, sources=512)
    case.params.precision = synth.PREC_MIXED
    cache = str(tmp_path / "tune.json")
    res = []
    for _ in range(2):   # tuned, then loaded from the cache
        ctx = fld.fld_create(case.grid, case.params)
        table = fld.autotune(ctx, cache_path=cache)
        assert len(table) == fld.fld_tuning_size(ctx) and fld.fld_get_tuning(ctx) == table
        E = dev(case.E)
        fld.fld_step(ctx, E, dev(case.nHI), dev(case.eta))
        res.append((table, host(E).reshape(case.grid.shape)))
        ctx.close()
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])
    # records are (threads, blocks, prefetch distance); a bad record is refused
    ctx = fld.fld_create(case.grid, case.params)
    n = fld.fld_tuning_size(ctx)
    assert n == len(res[0][0]) and n % 3 == 0
    for bad in ((96, 608, 1), (256, 0, 1), (256, 608, -1), (256, 608, 9)):
        with pytest.raises(fld.FldError):
            fld.fld_set_tuning(ctx, list(bad) * (n // 3))
    with pytest.raises(fld.FldError):
        fld.fld_set_tuning(ctx, [256, 608] * (n // 3))
    assert fld.fld_get_tuning(ctx) == [256, 152 * 8, 1] * (n // 3)
    ctx.close()
    Eref, _ = oracle.step(case.grid, case.params, {"rtol": 1e-13, "max_iter": 200}, case.E, case.nHI, case.eta)
    E = res[0][1]
    assert np.linalg.norm(E - Eref) / np.linalg.norm(Eref) < 1e-6


TAIL_CASES = [
    ((32, 32, 32), (False,) * 3),
    ((64, 48, 32), (True, False, True)),
    ((24, 16, 40), (False, True, False)),
    ((128, 64, 64), (False,) * 3),
]


@pytest.mark.parametrize("n,per", TAIL_CASES)
def test_persistent_tail_vcycle(fld, oracle, n, per):
    # the coarse levels as one cluster kernel: the FP64 V-cycle matches the
    # per-level kernels and the oracle to rounding (the FP32 tail is covered
    # by the mixed steps below)
    case = synth.random_case(n, seed=300 + sum(n), periodic=per)
    x = np.random.default_rng(8).standard_normal(case.grid.shape)
    out = {}
    for tail in (32768, 0):
        p = synth.Params(tail_cells=tail)
        ctx = fld.fld_create(case.grid, p)
        fld.fld_assemble(ctx, dev(case.E), dev(case.nHI), dev(case.eta))
        z = torch.empty(case.grid.cells, dtype=torch.float64, device="cuda")
        fld.fld_vcycle(ctx, dev(x), z)
        out[tail] = host(z).reshape(x.shape)
        ctx.close()
    op = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    zref = oracle.vcycle(case.grid, op, x)
    errs = (rel_max(out[32768], zref), rel_max(out[0], zref), rel_max(out[32768], out[0]))
    assert max(errs) < 1e-12, errs


@pytest.mark.parametrize("n", [32, 64])
@pytest.mark.parametrize("prec", [synth.PREC_FP64, synth.PREC_MIXED])
def test_persistent_tail_step(fld, oracle, prec, n):
    # whole steps with and without the tail, and against the oracle (at 32^3
    # the whole V-cycle is the tail)
    case = synth.config3(n, sources=64)
    case.params.precision = prec
    Es = {}
    for tail in (32768, 0):
        case.params.tail_cells = tail
        ctx = fld.fld_create(case.grid, case.params)
        E = dev(case.E)
        info = fld.fld_step(ctx, E, dev(case.nHI), dev(case.eta))
        ctx.close()
        assert info["rel_res"] <= 1e-8
        Es[tail] = host(E).reshape(case.grid.shape)
    Eref, _ = oracle.step(case.grid, case.params, {"rtol": 1e-13, "max_iter": 200}, case.E, case.nHI, case.eta)
    for E in Es.values():
        el2 = np.linalg.norm(E - Eref) / np.linalg.norm(Eref)
        einf = np.abs(E - Eref).max() / np.abs(Eref).max()
        assert el2 < 1e-6 and einf < 1e-6, (el2, einf)
    if prec == synth.PREC_FP64:
        assert rel_max(Es[32768] - case.E, Es[0] - case.E) < 1e-10


def test_results_do_not_depend_on_launch_shapes(fld):
    # race check without a sanitizer: the FP32 sweeps must give the same
    # values whatever the tile order of their launch shapes.  One V-cycle
    # (no reductions) is bit-identical under two tuning tables far apart
    # (128-thread blocks with the fewest blocks and no prefetch, 256-thread
    # blocks with the most and the longest prefetch distance); whole steps
    # agree to the rounding of the CG reductions, whose block order does
    # follow the shape.
    case = synth.config4(128, sources=1024)
    case.params.precision = synth.PREC_MIXED
    x = np.random.default_rng(9).standard_normal(case.grid.cells)
    zs, steps = [], []
    for threads, blocks, pf in ((128, 152 * 4, 0), (256, 152 * 64, 8)):
        ctx = fld.fld_create(case.grid, case.params)
        fld.fld_set_tuning(ctx, [threads, blocks, pf] * (fld.fld_tuning_size(ctx) // 3))
        fld.fld_assemble(ctx, dev(case.E), dev(case.nHI), dev(case.eta))
        z = torch.empty(case.grid.cells, dtype=torch.float64, device="cuda")
        fld.fld_vcycle(ctx, dev(x), z)
        zs.append(host(z))
        E = dev(case.E)
        info = fld.fld_step(ctx, E, dev(case.nHI), dev(case.eta))
        steps.append((host(E), info["iters"], info["outer_iters"]))
        ctx.close()
    assert np.array_equal(zs[0], zs[1])
    assert steps[0][1:] == steps[1][1:]
    e0 = case.E.ravel()
    assert rel_max(steps[0][0].ravel() - e0, steps[1][0].ravel() - e0) < 1e-6


@pytest.mark.parametrize("n", [32, 128])
def test_host_step_failure_then_success(fld, n):
    # an invalid input through the host-buffer step (plain transfer at 32^3,
    # overlapped at 128^3) fails with EINVAL and leaves E as it was; the same
    # context then steps correctly
    case = synth.config1(n)
    ctx = fld.fld_create(case.grid, case.params)
    Eh = case.E.copy()
    Eh.ravel()[5] = -1.0
    before = Eh.copy()
    with pytest.raises(fld.FldError) as e:
        fld.fld_step_host(ctx, Eh, case.nHI, case.eta)
    assert e.value.status == fld.FLD_EINVAL
    assert np.array_equal(Eh, before)
    Eh = case.E.copy()
    fld.fld_step_host(ctx, Eh, case.nHI, case.eta)
    E = dev(case.E)
    fld.fld_step(ctx, E, dev(case.nHI), dev(case.eta))
    ctx.close()
    assert np.array_equal(Eh.ravel(), host(E).ravel())


# ------------------------------------------------------------------
# Table 1's "nonsymmetric" red/black relaxation (paper_order): post-sweeps
# red then black like the pre-sweeps

@pytest.mark.parametrize("tail", [32768, 0])
@pytest.mark.parametrize("prec", [synth.PREC_FP64, synth.PREC_MIXED])
def test_paper_order_vcycle_parity(fld, oracle, prec, tail):
    case = synth.random_case((64, 32, 48), seed=77, periodic=(True, False, False), E_decades=(-20, -14))
    op = oracle.assemble(case.grid, case.params, case.E, case.nHI, case.eta)
    p = case.params
    p.precision, p.tail_cells, p.paper_order, p.precond_bf16 = prec, tail, 1, 0
    ctx = fld.fld_create(case.grid, p)
    fld.fld_assemble(ctx, dev(case.E), dev(case.nHI), dev(case.eta))
    x = np.random.default_rng(12).standard_normal(case.grid.shape)
    z = torch.empty(case.grid.cells, dtype=torch.float64, device="cuda")
    fld.fld_vcycle(ctx, dev(x), z)
    ctx.close()
    zg = host(z).reshape(x.shape)
    zref = oracle.vcycle(case.grid, op, x, {"paper_order": 1})
    tol = 1e-12 if prec == synth.PREC_FP64 else 1e-5
    assert rel_max(zg, zref) < tol
    # the symmetric cycle is measurably different
    zsym = oracle.vcycle(case.grid, op, x)
    assert rel_max(zsym, zref) > 1e-3


def test_paper_order_steps(fld, oracle):
    # FP64 to 1e-13 against the oracle with the same relaxation, and mixed at
    # the paper's 1e-8
    case = synth.config2(32)
    case.params.paper_order = 1
    E, Eref, info, iref = fp64_step_pair(fld, oracle, case)
    Eref, _ = oracle.step(case.grid, case.params, {"rtol": 1e-13, "max_iter": 200, "paper_order": 1},
                          case.E, case.nHI, case.eta)
    assert info["rel_res"] <= 1e-13
    assert rel_max(E - case.E, Eref - case.E) < 1e-10
    m = synth.config4(64, sources=512)
    m.params.paper_order = 1
    Em, im = mixed_step(fld, m, 1e-8)
    Emref, _ = oracle.step(m.grid, m.params, {"rtol": 1e-12, "max_iter": 200, "paper_order": 1}, m.E, m.nHI, m.eta)
    assert im["rel_res"] <= 1e-8
    assert np.linalg.norm(Em - Emref) / np.linalg.norm(Emref) < 1e-6
    assert np.abs(Em - Emref).max() / np.abs(Emref).max() < 1e-6
