"""GPU parity of the spectral model (Sec. 2): the grey and multigroup
spectral integrals, the group opacity/emissivity fields, the
photoionisation and photoheating rates, and a multigroup FLD step (each
group one FLD system, the groups stepped together by the batched driver),
all through the C ABI against the CPU oracle.

Tolerances: integrals 1e-10 relative (GPU Simpson's rule against adaptive
quadrature); per-cell fields and rates 1e-14; FP64 group steps solved to
1e-13 agree to 1e-10, mixed steps at 1e-8 to 1e-6."""
import numpy as np
import pytest

from oracle import sed as osed
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
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


NU1 = osed.NU_HI
EDGES = {
    "grey": [NU1, 1e3 * NU1],
    "groups6": [NU1, 1.5 * NU1, osed.NU_HEI, 3.0 * NU1, osed.NU_HEII, 10 * NU1, 1e3 * NU1],
}
SEDS = [
    ("bb3e4", {"kind": osed.BLACKBODY, "T": 3e4}),
    ("bb1e5", {"kind": osed.BLACKBODY, "T": 1e5}),
    ("bb3e5", {"kind": osed.BLACKBODY, "T": 3e5}),
    ("pl1.5", {"kind": osed.POWERLAW, "alpha": 1.5}),
    ("pl3", {"kind": osed.POWERLAW, "alpha": 3.0}),
    ("mono", {"kind": osed.MONO, "nu": 1.3 * osed.NU_HEI}),
]


def lib_sed(fld, d):
    kw = {"kind": d["kind"]}
    if d["kind"] == osed.BLACKBODY:
        kw["T"] = d["T"]
    elif d["kind"] == osed.POWERLAW:
        kw["alpha"] = d["alpha"]
    else:
        kw["nu_mono"] = d["nu"]
    s = fld.fld_sed_default(**kw)
    # the library's default cross sections are the oracle's
    for i, sp in enumerate(osed.SPECIES):
        x = s.species[i]
        assert (x.nu_threshold, x.sigma0, x.beta, x.s) == pytest.approx(osed.CROSS_SECTIONS[sp], rel=1e-15)
    return s


@pytest.mark.parametrize("edges_name", list(EDGES))
@pytest.mark.parametrize("name,d", SEDS)
def test_spectral_integrals_parity(fld, name, d, edges_name):
    edges = EDGES[edges_name]
    got = fld.fld_sed_integrals(lib_sed(fld, d), edges)
    ref = osed.group_integrals(d, edges)
    scale = np.abs(ref).max(axis=0)
    scale[scale == 0] = 1.0
    assert np.all(np.abs(got - ref) <= 1e-10 * scale), (got, ref)


def test_group_fields_and_rates_parity(fld):
    d = {"kind": osed.BLACKBODY, "T": 1e5}
    edges = EDGES["groups6"]
    coef = fld.fld_sed_integrals(lib_sed(fld, d), edges)
    G = coef.shape[0]
    rng = np.random.default_rng(3)
    n = 100_003
    nHI, nHeI, nHeII, eta = (10.0 ** rng.uniform(-6, -2, n) for _ in range(4))
    kap = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(G)]
    etas = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(G)]
    fld.fld_group_fields(coef, dev(nHI), kap, dev(nHeI), dev(nHeII), dev(eta), etas)
    rk, re = osed.group_fields(coef, nHI, nHeI, nHeII, eta)
    for g in range(G):
        np.testing.assert_allclose(kap[g].cpu().numpy(), rk[g], rtol=1e-14)
        np.testing.assert_allclose(etas[g].cpu().numpy(), re[g], rtol=1e-15)
    E = [10.0 ** rng.uniform(-20, -14, n) for _ in range(G)]
    rho = 10.0 ** rng.uniform(-28, -24, n)
    outs = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(4)]
    fld.fld_photo_rates(coef, [dev(e) for e in E], dev(nHI), dev(nHeI), dev(nHeII), dev(rho),
                        gamma_HI=outs[0], gamma_HeI=outs[1], gamma_HeII=outs[2], heating=outs[3])
    gam, heat = osed.photo_rates(coef, E, nHI, nHeI, nHeII, rho)
    for i in range(3):
        np.testing.assert_allclose(outs[i].cpu().numpy(), gam[i], rtol=1e-13)
    np.testing.assert_allclose(outs[3].cpu().numpy(), heat, rtol=1e-13)


def multigroup_case(n, seed):
    rng = np.random.default_rng(seed)
    g = synth.Grid.cube(n)
    nH = np.full(g.shape, 1e-3)
    xHI = np.clip(10.0 ** rng.uniform(-4, 0, g.shape), 0, 1)
    nHI = xHI * 0.92 * nH
    nHeI = 0.08 * nH * np.clip(xHI * 1.1, 0, 1)
    nHeII = 0.08 * nH - nHeI
    ns = 8
    pick = rng.choice(g.cells, size=ns, replace=False)
    cells = np.stack([pick % n, (pick // n) % n, pick // (n * n)], axis=1)
    eta = synth.point_source_eta(g, cells, 5e48)
    return g, nHI, nHeI, nHeII, eta


@pytest.mark.parametrize("precision", [synth.PREC_FP64, synth.PREC_MIXED])
def test_multigroup_step_parity(fld, oracle, precision):
    # three groups of a 1e5 K blackbody, each its own FLD system with the
    # group opacity (passed as n_HI with sigma = 1) and the group's share of
    # the emissivity; the groups stepped together by fld_step_batched
    g, nHI, nHeI, nHeII, eta = multigroup_case(32, 5)
    d = {"kind": osed.BLACKBODY, "T": 1e5}
    edges = [NU1, osed.NU_HEI, osed.NU_HEII, 1e3 * NU1]
    coef = fld.fld_sed_integrals(lib_sed(fld, d), edges)
    G = coef.shape[0]
    n = g.cells
    kap = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(G)]
    etas = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(G)]
    fld.fld_group_fields(coef, dev(nHI), kap, dev(nHeI), dev(nHeII), dev(eta), etas)
    rtol = 1e-13 if precision == synth.PREC_FP64 else 1e-8
    p = synth.Params(sigma=1.0, precision=precision, rtol=rtol, max_iter=200)
    streams = [torch.cuda.Stream() for _ in range(G)]
    ctxs = [fld.fld_create(g, p, s) for s in streams]
    E0 = [np.full(g.shape, synth.E0 * coef[k, 9]) for k in range(G)]
    Es = [dev(e) for e in E0]
    torch.cuda.synchronize()
    st, infos = fld.fld_step_batched(ctxs, Es, kap, etas)
    torch.cuda.synchronize()
    assert st == fld.FLD_OK
    for c in ctxs:
        c.close()
    rk, re = osed.group_fields(coef, nHI, nHeI, nHeII, eta)
    for k in range(G):
        Eref, iref = oracle.step(g, p, {"rtol": 1e-13, "max_iter": 200}, E0[k], rk[k].reshape(g.shape),
                                 re[k].reshape(g.shape))
        Eg = Es[k].cpu().numpy().reshape(g.shape)
        if precision == synth.PREC_FP64:
            np.testing.assert_allclose(Eg, Eref, rtol=1e-10, atol=1e-10 * np.abs(Eref).max())
        else:
            el2 = np.linalg.norm(Eg - Eref) / np.linalg.norm(Eref)
            einf = np.abs(Eg - Eref).max() / np.abs(Eref).max()
            assert el2 < 1e-6 and einf < 1e-6, (k, el2, einf)
        assert infos[k]["rel_res"] <= rtol


def test_one_grey_group_is_the_grey_step(fld):
    # a single group [nu_1, nu_max] with HI only: kappa = K_HI n_HI, so the
    # group step equals the plain step with sigma = K_HI, bit for bit in the
    # right-hand side and to rounding in the operator
    case = synth.config_uniform(32, sources=4, seed=2, centre=False, limiter=synth.LIMITER_PAPER)
    coef = fld.fld_sed_integrals(lib_sed(fld, {"kind": osed.BLACKBODY, "T": 1e5}), EDGES["grey"])
    kap = torch.empty(case.grid.cells, dtype=torch.float64, device="cuda")
    fld.fld_group_fields(coef, dev(case.nHI), [kap])
    assert coef[0, 9] == pytest.approx(1.0, rel=1e-15)
    p1 = synth.Params(sigma=1.0, rtol=1e-13, max_iter=200)
    p2 = synth.Params(sigma=float(coef[0, 0]), rtol=1e-13, max_iter=200)
    E1, E2 = dev(case.E), dev(case.E)
    c1, c2 = fld.fld_create(case.grid, p1), fld.fld_create(case.grid, p2)
    fld.fld_step(c1, E1, kap, dev(case.eta))
    fld.fld_step(c2, E2, dev(case.nHI), dev(case.eta))
    c1.close()
    c2.close()
    a, b = E1.cpu().numpy(), E2.cpu().numpy()
    np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-10 * np.abs(b).max())


def test_spectral_validation(fld):
    s = fld.fld_sed_default(kind=fld.FLD_SED_BLACKBODY, T=-1.0)
    with pytest.raises(fld.FldError):
        fld.fld_sed_integrals(s, EDGES["grey"])
    with pytest.raises(fld.FldError):
        fld.fld_sed_integrals(fld.fld_sed_default(), [NU1, NU1])        # edges must increase
    with pytest.raises(fld.FldError):
        fld.fld_sed_integrals(fld.fld_sed_default(), np.linspace(NU1, 1e3 * NU1, 18))   # 17 groups
