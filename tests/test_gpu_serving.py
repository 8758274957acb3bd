"""Serving: continuous batching of independent FLD steps on one GPU.

A request's result is the same bit for bit alone and in the mix; results
match the FP64 oracle; admission by HBM budget rejects what can never fit
and holds back what does not fit yet."""
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
    # a budget that holds one request at a time still serves every request
    srv = serving.Server(budget_bytes=1.2 * need, workers=4)
    res = srv.run(reqs, realtime=False)
    srv.close()
    assert all(r.status == 0 for r in res)
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
