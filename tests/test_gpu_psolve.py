"""Persistent inner solves (fld_params.persistent_cells): one thread-block
cluster runs a request's whole FP32 MG-PCG solve (Table 1's solver: the
V-cycle over all levels, then the CG vector operations) inside the mixed
FP32/FP64 refinement, and one launch drains a work list of requests of any
grid sizes.

Checked here: parity with the FP64 oracle at the mixed-precision bar (1e-6
relative in E^{n+1}, L2 and max, at the paper's 1e-8; cell by cell at
1e-12), the same stopping rule as the launch-per-kernel path (within one
iteration of it), and the same result bit for bit alone and inside a batch
of uneven grids longer than the clusters the device holds at once."""
import numpy as np
import pytest

from paper_1306_0645_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PS_ALL = 1 << 22


@pytest.fixture(scope="module")
def fld():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_0645_gb300 import fld as f
    f.lib()
    return f


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


CASES = [
    lambda: synth.config3(32, sources=16),                                    # levels 32..4, tail-only sizes
    lambda: synth.config4(48, sources=64),                                    # 48 -> 3, odd coarse levels
    lambda: synth.random_case((64, 32, 48), seed=21, periodic=(True, False, True)),
    lambda: synth.random_case((16, 24, 20), seed=13, periodic=(False, True, False)),
    lambda: synth.config_uniform(16, sources=3, seed=1, centre=False, precision=synth.PREC_MIXED),
]


def ps_step(fld, case, rtol, persistent, stream=None):
    p = case.params
    p.precision = synth.PREC_MIXED
    p.rtol = rtol
    p.persistent_cells = persistent
    s = stream or torch.cuda.Stream()
    ctx = fld.fld_create(case.grid, p, s)
    fld.fld_profile(ctx, 0)
    E = dev(case.E)
    with torch.cuda.stream(s):
        info = fld.fld_step(ctx, E, dev(case.nHI), dev(case.eta), check=False)
    s.synchronize()
    prof = {k["name"]: k["launches"] for k in fld.fld_profile_read(ctx)}
    ctx.close()
    return E.cpu().numpy().reshape(case.grid.shape), info, prof


@pytest.mark.parametrize("make", CASES)
def test_persistent_step_parity_at_paper_tolerance(fld, oracle, make):
    case = make()
    E, info, prof = ps_step(fld, case, 1e-8, PS_ALL)
    assert info["status"] == 0 and info["rel_res"] <= 1e-8
    # the inner solves ran as persistent launches, one per refinement, and
    # no per-level kernel or coarse-tail launch of the V-cycle took place
    assert prof["psolve"] == info["outer_iters"] >= 1
    assert prof["vtail"] == 0 and prof["rb_colour"] == 0 and prof["cg_p_matvec"] == 0
    Eref, _ = oracle.step(case.grid, case.params, {"rtol": 1e-13, "max_iter": 200}, case.E, case.nHI, case.eta)
    el2 = np.linalg.norm(E - Eref) / np.linalg.norm(Eref)
    einf = np.abs(E - Eref).max() / np.abs(Eref).max()
    assert el2 < 1e-6 and einf < 1e-6, (el2, einf)


@pytest.mark.parametrize("make", CASES[:3])
def test_persistent_step_converges_pointwise_to_fp64(fld, oracle, make):
    case = make()
    E, info, _ = ps_step(fld, case, 1e-12, PS_ALL)
    assert info["status"] == 0 and info["rel_res"] <= 1e-12
    Eref, _ = oracle.step(case.grid, case.params, {"rtol": 1e-13, "max_iter": 200}, case.E, case.nHI, case.eta)
    mask = Eref > 1e-6 * Eref.max()
    emax = (np.abs(E - Eref)[mask] / Eref[mask]).max()
    assert emax < 1e-6, emax


@pytest.mark.parametrize("make", CASES[:3])
def test_persistent_solve_takes_the_iterations_of_the_launch_path(fld, make):
    # the same preconditioner, CG recurrences and stopping rule: the FP32
    # rounding differs (other summation orders), so the iteration counts may
    # differ by one
    a = ps_step(fld, make(), 1e-8, PS_ALL)[1]
    b = ps_step(fld, make(), 1e-8, 0)[1]
    assert a["outer_iters"] == b["outer_iters"]
    assert abs(a["iters"] - b["iters"]) <= a["outer_iters"], (a, b)


def with_faces(case, dirichlet, ebc=(0.0,) * 6, theta=1.0):
    g = case.grid
    case.grid = synth.Grid(g.n, g.h, g.periodic, dirichlet=dirichlet, ebc=ebc)
    case.params.theta = theta
    return case


def solver_variant(case, **kw):
    for k, v in kw.items():
        setattr(case.params, k, v)
    return case


VARIANTS = [
    # Table 1's red-then-black post-sweeps, both modes
    ("paper_order_cta", lambda: solver_variant(synth.config3(16, sources=4), paper_order=1)),
    ("paper_order_cluster", lambda: solver_variant(synth.config3(32, sources=16), paper_order=1)),
    # two pre- and post-sweeps (the colour sweeps after the zero-guess one)
    ("pre2_post2_cta", lambda: solver_variant(synth.random_case((16, 16, 16), seed=31), pre=2, post=2)),
    ("pre2_post2_cluster", lambda: solver_variant(
        synth.random_case((32, 24, 16), seed=32, periodic=(True, False, True)), pre=2, post=2)),
    # Sec. 4.1 faces (outflow above) with the trapezoidal rule, and Dirichlet
    # faces on a grid with a periodic axis
    ("outflow_trapezoidal", lambda: with_faces(synth.random_case((16, 12, 20), seed=33), (False, True) * 3,
                                               theta=0.5)),
    ("dirichlet_mixed", lambda: with_faces(synth.random_case((24, 16, 8), seed=34, periodic=(False, False, True)),
                                           (True, False, True, True, False, False),
                                           (1e-19, 0.0, 3e-20, 0.0, 0.0, 0.0), theta=0.75)),
]


@pytest.mark.parametrize("name,make", VARIANTS, ids=[v[0] for v in VARIANTS])
def test_persistent_solver_variants_match_oracle(fld, oracle, name, make):
    # the same V-cycle options and face types as the launch-per-kernel path,
    # against the oracle's step solved to 1e-13
    case = make()
    E, info, prof = ps_step(fld, case, 1e-8, PS_ALL)
    assert info["status"] == 0 and info["rel_res"] <= 1e-8
    assert prof["psolve"] == info["outer_iters"] >= 1
    Eref, _ = oracle.step(case.grid, case.params, {"rtol": 1e-13, "max_iter": 200}, case.E, case.nHI, case.eta)
    el2 = np.linalg.norm(E - Eref) / np.linalg.norm(Eref)
    einf = np.abs(E - Eref).max() / np.abs(Eref).max()
    assert el2 < 1e-6 and einf < 1e-6, (el2, einf)


def test_persistent_noconv_leaves_E_unchanged(fld):
    case = synth.config3(32, sources=16)
    case.params.max_iter = 2
    E, info, _ = ps_step(fld, case, 1e-8, PS_ALL)
    assert info["status"] == fld.FLD_ENOCONV
    assert np.array_equal(E, case.E)


def test_persistent_batch_equals_single_steps(fld):
    """More requests than resident clusters, of uneven sizes, in one
    fld_step_batched: every inner solve of the round is one launch over the
    work list; each result equals the context's own fld_step bit for bit."""
    shapes = [(16, 16, 16), (24, 16, 32), (32, 32, 32), (48, 48, 48), (64, 32, 48), (16, 24, 20)]
    cases = []
    for q in range(48):
        n = shapes[q % len(shapes)]
        c = synth.random_case(n, seed=500 + q, periodic=(q % 2 == 0, False, q % 3 == 0))
        c.params.precision = synth.PREC_MIXED
        c.params.persistent_cells = PS_ALL
        cases.append(c)
    # one large context that keeps the launch-per-kernel solve in the batch
    big = synth.config4(96, sources=64)
    big.params.precision = synth.PREC_MIXED
    big.params.persistent_cells = 65536
    cases.append(big)

    def make():
        streams = [torch.cuda.Stream() for _ in cases]
        return streams, [fld.fld_create(c.grid, c.params, s) for c, s in zip(cases, streams)]

    streams, ctxs = make()
    single = []
    for c, ctx, s in zip(cases, ctxs, streams):
        E = dev(c.E)
        with torch.cuda.stream(s):
            info = fld.fld_step(ctx, E, dev(c.nHI), dev(c.eta), check=False)
        s.synchronize()
        single.append((E.cpu().numpy(), info))
    for ctx in ctxs:
        ctx.close()
    for rep in range(2):
        streams, ctxs = make()
        for ctx in ctxs:
            fld.fld_profile(ctx, 0)
        Es = [dev(c.E) for c in cases]
        st, infos = fld.fld_step_batched(ctxs, Es, [dev(c.nHI) for c in cases], [dev(c.eta) for c in cases],
                                         check=False)
        torch.cuda.synchronize()
        assert st == 0
        launches = sum(k["launches"] for ctx in ctxs for k in fld.fld_profile_read(ctx) if k["name"] == "psolve")
        # one launch per refinement round for all 48 small contexts together
        outer = max(i["outer_iters"] for i in infos[:48])
        assert launches <= outer + 1, (launches, outer)
        for (Es_, info_s), E, info_b in zip(single, Es, infos):
            assert info_b["status"] == info_s["status"] == 0
            assert info_b["iters"] == info_s["iters"] and info_b["outer_iters"] == info_s["outer_iters"]
            assert np.array_equal(E.cpu().numpy(), Es_)
        for ctx in ctxs:
            ctx.close()
