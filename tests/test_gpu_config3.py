"""Config 3: mixed precision on a 256^3 uniform grid with 4096 sources, 20
successive steps with the hydrogen opacity update between them; the error of
E^{n+1} against the FP64 oracle is stated for every step.

Both sides advance on their own (the oracle never sees a GPU value): the
CUDA path at the paper's tolerance 1e-8 in mixed precision, the oracle in FP64
solved to 1e-12.  Each step's error is asserted at 1e-6 in the L2 norm and in
the max norm relative to max E (the accuracy a 1e-8 residual controls), and
the per-step table is written to $FLD_REPORT_DIR/config3_errors.json when
that variable is set.  A 1e-8 residual does not control the relative error
of each cell; so after the 20 steps one more step, from the oracle's state on
both sides, runs the CUDA path to 1e-11 (the oracle to 1e-13) and holds it
to 1e-6 relative in every cell with E > 1e-6 max E.  After 20 steps E is
large and nearly steady, the face fluxes are some 10^3 times |b|, and no
solver reaches 1e-12 here: the plain FP64 residual stalls near 2e-12, the
double-float one of the mixed solver near 6e-12 (both measured on this
state); 1e-11 lies above both."""
import dataclasses
import json
import os

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


def test_config3_twenty_steps(fld, oracle):
    n, sources, steps = 256, 4096, 20
    case = synth.config3(n, sources)
    p = case.params
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()
    ctx = fld.fld_create(case.grid, p)
    Eg, nHIg, etag, nHg = dev(case.E), dev(case.nHI), dev(case.eta), dev(case.nH)
    Eo, nHIo = case.E.copy(), case.nHI.copy()
    rows = []
    for s in range(steps):
        info = fld.fld_step(ctx, Eg, nHIg, etag)
        fld.fld_opacity_update(Eg, nHg, nHIg, nHIg, p.dt, p.c, p.sigma, p.hnu, synth.ALPHA_B)
        Eo, io = oracle.step(case.grid, p, {"rtol": 1e-12, "max_iter": 200}, Eo, nHIo, case.eta)
        nHIo = oracle.opacity_update(Eo, case.nH, nHIo, p.dt, p.c, p.sigma, p.hnu, synth.ALPHA_B)
        E = Eg.cpu().numpy().reshape(case.grid.shape)
        el2 = float(np.linalg.norm(E - Eo) / np.linalg.norm(Eo))
        einf = float(np.abs(E - Eo).max() / np.abs(Eo).max())
        mask = Eo > 1e-6 * Eo.max()
        ecell = float((np.abs(E - Eo)[mask] / Eo[mask]).max())
        nHI = nHIg.cpu().numpy().reshape(case.grid.shape)
        exhi = float(np.abs(nHI - nHIo).max() / np.abs(nHIo).max())
        rows.append({"step": s + 1, "inner_iters": info["iters"], "outer_iters": info["outer_iters"],
                     "rel_res": info["rel_res"], "oracle_iters": io["iters"], "err_l2": el2,
                     "err_max_rel_to_max": einf, "err_cellwise_E_gt_1e-6max": ecell,
                     "nHI_err_max_rel": exhi, "balance_rel": info["balance_rel"],
                     "floor_added_photons": info["floor_added"]})
    # the cell-wise check at a tolerance that controls it, from the oracle's state
    p12 = dataclasses.replace(p, rtol=1e-11, max_iter=200)
    ctx12 = fld.fld_create(case.grid, p12)
    Eg = dev(Eo)
    info12 = fld.fld_step(ctx12, Eg, dev(nHIo), etag)
    Eo12, _ = oracle.step(case.grid, p, {"rtol": 1e-13, "max_iter": 200}, Eo, nHIo, case.eta)
    E12 = Eg.cpu().numpy().reshape(case.grid.shape)
    mask = Eo12 > 1e-6 * Eo12.max()
    cell12 = float((np.abs(E12 - Eo12)[mask] / Eo12[mask]).max())
    rows.append({"step": "21 (from the oracle's state, CUDA path to 1e-11)", "rel_res": info12["rel_res"],
                 "err_cellwise_E_gt_1e-6max": cell12})
    ctx12.close()
    ctx.close()
    out = os.environ.get("FLD_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, "config3_errors.json"), "w") as f:
            json.dump(rows, f, indent=1)
    for r in rows[:-1]:
        assert r["rel_res"] <= 1e-8
        assert r["err_l2"] < 1e-6 and r["err_max_rel_to_max"] < 1e-6, r
    assert info12["rel_res"] <= 1e-11 and cell12 < 1e-6, rows[-1]
