"""fld_residual_noalloc: the FP64 residual and its norms with no device
allocation, for callers that cannot call cudaMalloc (their device memory is
owned by another allocator, or they run in a loop where an allocation's
device synchronisation would stall them).

Its result must equal what the library's ordinary entry points give for the
same system: b - fld_apply(x) from an assembled context.  Two calls in a row
check that the shared fixed scratch is reset between calls; a grid with
outflow faces takes its operator (boundary weights in m) from fld_get_system;
the norms-only form (r = None) and a call on a second stream after the first
call reuse the per-device scratch address.  This file is collected last so
that a failure here leaves every other test already run."""
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


def _outflow_case():
    c = synth.random_case((20, 12, 16), seed=5)
    c.grid = c.grid.outflow_upper()
    return c


@pytest.mark.parametrize("make", [lambda: synth.config2(32),
                                  lambda: synth.random_case((24, 16, 40), seed=3, periodic=(False, True, False)),
                                  _outflow_case])
def test_noalloc_residual_matches_apply_twice(fld, make):
    case = make()
    n = case.grid.cells
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()
    ctx = fld.fld_create(case.grid, case.params)
    fld.fld_assemble(ctx, dev(case.E), dev(case.nHI), dev(case.eta))
    sys_ = {k: torch.empty(n, dtype=torch.float64, device="cuda") for k in ("m", "wx", "wy", "wz", "b")}
    fld.fld_get_system(ctx, **sys_)
    rng = np.random.default_rng(4)
    for call in range(2):
        x = dev(rng.standard_normal(n) * 1e-20)
        y = torch.empty_like(x)
        fld.fld_apply(ctx, x, y)
        want = sys_["b"] - y
        r = torch.empty_like(x)
        norms = torch.zeros(2, dtype=torch.float64, device="cuda")
        fld.fld_residual_noalloc(case.grid, sys_["m"], sys_["wx"], sys_["wy"], sys_["wz"], sys_["b"], x, r, norms)
        torch.cuda.synchronize()
        scale = float(want.abs().max())
        assert float((r - want).abs().max()) <= 1e-13 * scale, call
        nr = norms.cpu().numpy()
        assert nr[0] == pytest.approx(float((want * want).sum()), rel=1e-12)
        assert nr[1] == pytest.approx(float(want.abs().max()), rel=1e-13)
        # norms only (r = None), on a stream of its own after the first call
        side = torch.cuda.Stream()
        norms2 = torch.zeros(2, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        fld.fld_residual_noalloc(case.grid, sys_["m"], sys_["wx"], sys_["wy"], sys_["wz"], sys_["b"], x, None,
                                 norms2, stream=side)
        side.synchronize()
        assert np.array_equal(norms2.cpu().numpy(), nr), call
    ctx.close()


def test_noalloc_rejects_oversized_grid(fld):
    # a grid whose x-y plane needs more thread blocks than the fixed scratch
    # holds is refused before any device pointer is read
    import ctypes
    g = fld.make_grid(synth.Grid((2, 1 << 23, 1), (1.0, 1.0, 1.0)))
    t = torch.zeros(2, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(t.data_ptr())
    st = fld.lib().fld_residual_noalloc(ctypes.byref(g), p, p, p, p, p, p, None, p,
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == fld.FLD_EINVAL
    assert "too large" in fld.fld_last_error()
