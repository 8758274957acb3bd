"""Host-side logic without a GPU: input generators, request stream, serving
statistics, and the multi-rank timing reduction of bench.py (gloo, 2 ranks)."""
import os
import socket
import sys

import numpy as np
import pytest

from paper_1306_0645_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_generators_are_seeded_and_reproducible():
    a = synth.config2(32)
    b = synth.config2(32)
    for k in ("E", "nHI", "eta"):
        assert np.array_equal(getattr(a, k), getattr(b, k))
    c4 = synth.config4(32, sources=64)
    rho = c4.nHI
    assert rho.min() >= 1e-3 * 1e-3 * 0.999 and rho.max() <= 1e3 * 1e-3 * 1.001
    assert c4.sources.shape == (64, 3)
    # every source lands in its own cell with N_dot h nu / V
    V = c4.grid.volume
    assert np.isclose(c4.eta.sum(), 64 * synth.NDOT * synth.HNU_HI / V, rtol=1e-12)


def test_config1_source_in_centre_cell():
    c = synth.config1(32)
    k, j, i = np.unravel_index(np.argmax(c.eta), c.eta.shape)
    assert (i, j, k) == (16, 16, 16)
    assert np.count_nonzero(c.eta) == 1


def test_gaussian_field_spectrum_slope():
    d = synth.gaussian_field(64, seed=3)
    assert abs(d.mean()) < 1e-12 and abs(d.std() - 1) < 1e-5
    f = np.abs(np.fft.rfftn(d)) ** 2
    kx = np.fft.rfftfreq(64)
    ky = np.fft.fftfreq(64)
    k = np.sqrt(kx[None, None, :] ** 2 + ky[None, :, None] ** 2 + ky[:, None, None] ** 2)
    lo = f[(k > 0.05) & (k < 0.07)].mean()
    hi = f[(k > 0.2) & (k < 0.28)].mean()
    slope = np.log(hi / lo) / np.log(0.24 / 0.06)
    assert -2.4 < slope < -1.6


def test_request_stream_statistics():
    reqs = synth.request_stream(count=2000, rate=500.0, seed=5)
    gaps = np.diff([r.arrival for r in reqs])
    assert abs(gaps.mean() - 1 / 500.0) < 0.1 / 500.0
    sizes = np.array([r.n for r in reqs])
    assert set(sizes) == {16, 32, 48, 64, 96, 128}
    counts = np.bincount(np.searchsorted([16, 32, 48, 64, 96, 128], sizes))
    assert counts.min() > 250
    src = np.array([r.sources for r in reqs])
    assert src.min() >= 1 and src.max() <= 64
    r = reqs[7]
    cells, rates = synth.request_sources(r)
    assert np.array_equal(cells, synth.request_case(r).sources)


def test_summarize_percentiles():
    from paper_1306_0645_gb300.serving import Result, summarize
    res = [Result(i, 32, 0.0, 0.0, (i + 1) * 1e-3, 0) for i in range(100)]
    s = summarize(res)
    assert s["ok"] == 100 and abs(s["p50_ms"] - 50.5) < 1e-9
    assert abs(s["p99_ms"] - 99.01) < 1e-6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 * (rank + 1), dist, device="cpu")
    out.put((rank, ms))
    dist.destroy_process_group()


def test_bench_max_over_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert got == [(0, 20.0), (1, 20.0)]
