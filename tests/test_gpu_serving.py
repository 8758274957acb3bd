"""Serving: continuous batching of independent FLD steps on one GPU.

A request's result is the same bit for bit alone and in the mix; results
match the FP64 oracle; admission by HBM budget rejects what can never fit
and holds back what does not fit yet, counting every context it keeps
resident."""
import numpy as np
import pytest

from paper_1306_0645_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def serving():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_0645_gb300 import serving as s
    return s


def small_stream(count, seed):
    return synth.request_stream(count=count, rate=2000.0, seed=seed, sizes=(16, 32, 48, 64))


def test_alone_equals_in_the_mix(serving):
    reqs = small_stream(24, seed=11)
    alone = serving.Server(workers=1, keep_results=True)
    ra = alone.run(reqs, realtime=False)
    alone.close()
    mix = serving.Server(workers=6, keep_results=True)
    extra = [synth.Request(1000 + r.rid, r.arrival, r.n, r.seed + 1, r.sources) for r in small_stream(24, 12)]
    rm = mix.run(reqs + extra, realtime=False)
    mix.close()
    for a, b in zip(ra, rm[: len(reqs)]):
        assert a.status == 0 and b.status == 0
        assert a.iters == b.iters and a.outer_iters == b.outer_iters
        assert np.array_equal(a.E, b.E)


def test_served_results_match_oracle(serving, oracle):
    reqs = small_stream(4, seed=21)
    srv = serving.Server(workers=2, keep_results=True)
    res = srv.run(reqs, realtime=False)
    srv.close()
    for r, out in zip(reqs, res):
        case = synth.request_case(r)
        Eref, _ = oracle.step(case.grid, case.params, {"rtol": 1e-12, "max_iter": 200},
                              case.E, case.nHI, case.eta)
        E = out.E.reshape(case.grid.shape)
        assert np.linalg.norm(E - Eref) / np.linalg.norm(Eref) < 1e-6
        assert np.abs(E - Eref).max() / np.abs(Eref).max() < 1e-6


def test_admission_by_budget(serving):
    reqs = small_stream(12, seed=31)
    probe = serving.Server(workers=1)
    need = max(probe.footprint(r.n) for r in reqs)
    probe.close()
    # a budget that holds one resident context at a time still serves every
    # request (idle contexts are evicted to make room), and the bytes charged
    # for resident contexts never exceed it
    srv = serving.Server(budget_bytes=1.2 * need, workers=4)
    res = srv.run(reqs, realtime=False)
    assert srv.peak_bytes <= srv.budget and srv.resident_bytes() <= srv.budget
    assert 0 < srv.resident_bytes()
    srv.close()
    assert all(r.status == 0 for r in res)
    # with room for all, contexts stay resident: a second run of the same
    # requests on the same worker charges nothing new
    srv = serving.Server(budget_bytes=1e12, workers=1)
    srv.run(reqs, realtime=False)
    held = srv.resident_bytes()
    srv.run(reqs, realtime=False)
    assert srv.resident_bytes() == held and srv.peak_bytes == held
    srv.close()
    # a request larger than the whole budget is rejected, the others served
    big = synth.Request(999, 0.0, 128, 5, 8)
    srv = serving.Server(budget_bytes=0.5 * serving.Server.footprint(srv, 128), workers=2)
    res = srv.run([big] + reqs[:3], realtime=False)
    srv.close()
    assert res[0].status != 0
    assert all(r.status == 0 for r in res[1:])


def test_poisson_stream_latency_report(serving):
    reqs = synth.request_stream(count=200, rate=500.0, seed=5)
    srv = serving.Server(workers=8)
    res = srv.run(reqs, realtime=True)
    srv.close()
    s = serving.summarize(res)
    assert s["ok"] == 200 and s["p99_ms"] >= s["p50_ms"] > 0


def test_step_batched_uneven_grids_equal_single_steps():
    """fld_step_batched: uneven grids in lockstep, every CG iteration of all
    of them one batch-graph launch; each result is bit-identical to a single
    fld_step of the same context, and a failing item leaves the others."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_0645_gb300 import fld
    cases = [synth.config_uniform(16, sources=3, seed=1, centre=False, precision=synth.PREC_MIXED),
             synth.random_case((24, 16, 32), seed=2, periodic=(True, False, False)),
             synth.config_uniform(48, sources=9, seed=3, centre=False, precision=synth.PREC_MIXED),
             synth.config4(64, sources=64),
             synth.config2(32),
             synth.config_uniform(32, sources=2, seed=4, centre=False, precision=synth.PREC_MIXED)]
    cases[1].params.precision = synth.PREC_MIXED
    cases[3].params.precision = synth.PREC_MIXED
    cases[4].params.precision = synth.PREC_FP64
    cases[5].params.max_iter = 1                      # fails: FLD_ENOCONV
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()

    def make():
        streams = [torch.cuda.Stream() for _ in cases]
        ctxs = [fld.fld_create(c.grid, c.params, s) for c, s in zip(cases, streams)]
        return streams, ctxs

    # single steps
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
    # the batch, twice in a row (graphs are reused the second time)
    for rep in range(2):
        streams, ctxs = make()
        Es = [dev(c.E) for c in cases]
        st, infos = fld.fld_step_batched(ctxs, Es, [dev(c.nHI) for c in cases], [dev(c.eta) for c in cases],
                                         check=False)
        torch.cuda.synchronize()
        assert st == fld.FLD_ENOCONV
        for (Es_, info_s), E, info_b, c in zip(single, Es, infos, cases):
            assert info_b["status"] == info_s["status"]
            assert info_b["iters"] == info_s["iters"] and info_b["outer_iters"] == info_s["outer_iters"]
            assert np.array_equal(E.cpu().numpy(), Es_)
        assert infos[5]["status"] == fld.FLD_ENOCONV
        assert np.array_equal(Es[5].cpu().numpy(), cases[5].E.ravel())   # unchanged on failure
        for ctx in ctxs:
            ctx.close()


def test_batched_serving_equals_alone(serving):
    # workers that step every arrived request together (fld_step_batched)
    reqs = small_stream(24, seed=41)
    alone = serving.Server(workers=1, keep_results=True)
    ra = alone.run(reqs, realtime=False)
    alone.close()
    srv = serving.Server(workers=2, keep_results=True, batch=8)
    rb = srv.run(reqs, realtime=False)
    srv.close()
    for a, b in zip(ra, rb):
        assert a.status == 0 and b.status == 0
        assert np.array_equal(a.E, b.E)


def test_cancellation_before_a_worker_takes_the_request(serving):
    # requests cancelled before they are taken come back CANCELLED, never
    # stepped; the others are served as usual, and the summary counts both
    reqs = synth.request_stream(count=40, rate=200.0, seed=51, sizes=(16, 32))
    srv = serving.Server(workers=2, keep_results=True)
    drop = {r.rid for r in reqs[::3]}
    for rid in drop:
        srv.cancel(rid)
    res = srv.run(reqs, realtime=True)
    srv.close()
    for r in res:
        if r.rid in drop:
            assert r.status == serving.CANCELLED and r.E is None and r.iters == 0
        else:
            assert r.status == 0 and r.E is not None
    s = serving.summarize(res)
    assert s["cancelled"] == len(drop) and s["ok"] == len(reqs) - len(drop) and s["failed"] == 0


@pytest.mark.parametrize("batch", [1, 3])
def test_warm_builds_every_resident_context(serving, batch):
    # warm(): one step per worker and size, so no request pays for a context
    # or graph build; a warmed server gives the same results as a cold one
    sizes = (16, 32, 48)
    reqs = small_stream(12, seed=21)
    cold = serving.Server(workers=2, keep_results=True)
    rc = cold.run(reqs, realtime=False)
    cold.close()
    srv = serving.Server(workers=2, keep_results=True, batch=batch)
    warm = srv.warm(sizes)
    assert len(warm) == 2 * len(sizes) * (2 if batch > 1 else 1)
    assert all(r.status == 0 and r.iters > 0 for r in warm)
    for w in range(2):
        assert srv.resident_sizes(w) == list(sizes)
        if batch > 1:
            assert srv.resident_sizes(w, batch=True) == list(sizes)
    rw = srv.run(reqs, realtime=False)
    srv.close()
    for a, b in zip(rc, rw):
        assert a.status == 0 and b.status == 0
        assert np.array_equal(a.E, b.E)
