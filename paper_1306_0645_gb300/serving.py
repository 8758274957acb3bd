"""Continuous-batching request loop for FLD steps on one GPU.

Independent requests (grids of different sizes, each with its own sources)
arrive over time.  Worker threads each own a CUDA stream and a set of
resident contexts (multigrid hierarchies and work buffers, one per grid size
they have served), so a request's step runs through the C ABI on that
worker's stream while other requests run on the others: work from requests
that arrived while others were on the GPU overlaps on the device.
Admission is by HBM budget over everything the server keeps on the device:
each resident context (its footprint from fld_footprint_bytes, plus its
field buffers) is charged from its creation until it is evicted.  A request
whose worker already holds a context of its size runs at no new charge;
otherwise the context is created once the charged bytes plus its footprint
fit the budget, evicting least recently used idle contexts to make room and
waiting for running ones to finish when that is not enough.  A request
that can never fit is rejected.

Every kernel launch shape depends only on the grid size and parameters and
every reduction adds in a fixed order, so a request's result is the same,
bit for bit, whether it runs alone or in the mix.

A request can be cancelled (``Server.cancel``) until a worker takes it: it
is then returned with status ``CANCELLED`` and never stepped.  A step in
progress is not interrupted.
"""
from __future__ import annotations

import dataclasses
import queue
import threading
import time
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import fld, synth

CANCELLED = -1   # Result.status of a request cancelled before it was stepped
_MAX_SOURCES = 64  # sources a request may carry
PERSISTENT_CELLS = 8192   # grids up to this size solve in one persistent CTA each


@dataclasses.dataclass
class _Resident:
    """A context kept on the device with its field buffers (E, n_HI, eta),
    the bytes charged for it, and whether a step is using it."""

    nbytes: float
    ctx: Optional[object] = None
    buf: Optional[tuple] = None
    busy: bool = True
    last: float = 0.0


@dataclasses.dataclass
class Result:
    """Outcome of one request: times on the stream clock, status, iteration
    counts, relative residual and (when kept) E^{n+1}."""

    rid: int
    n: int
    arrival: float          # s, stream time
    start: float            # s, when a worker began it
    finish: float           # s, when its E was back on the host
    status: int
    iters: int = 0
    outer_iters: int = 0
    rel_res: float = 0.0
    E: Optional[np.ndarray] = None

    @property
    def latency_ms(self) -> float:
        """Arrival to E^{n+1} on the host, ms."""
        return (self.finish - self.arrival) * 1e3

    @property
    def wait_ms(self) -> float:
        """Arrival to the start of its step (queueing), ms."""
        return (self.start - self.arrival) * 1e3


class Server:
    """A pool of worker threads stepping requests under an HBM budget."""

    def __init__(self, budget_bytes: float = 40e9, workers: int = 8, keep_results: bool = False,
                 params: Optional[synth.Params] = None, device: int = 0, batch: int = 1,
                 batch_max_n: int = 64):
        import torch
        self.torch = torch
        self.device = device
        self.budget = float(budget_bytes)
        self.workers = workers
        self.keep = keep_results
        # batch > 1: a free worker takes every request of at most
        # batch_max_n^3 cells that has arrived (up to batch) and steps them
        # together through fld_step_batched (their inner solves one
        # persistent launch over a work list, or device-side CG loops on
        # private streams); larger requests are stepped alone, so a batch
        # never waits for a large grid
        self.batch = max(1, int(batch))
        self.batch_max_n = int(batch_max_n)
        # default: mixed precision, and the inner solves of grids up to 16^3
        # as single-CTA persistent kernels (all their vectors in shared memory)
        self.params = params or synth.Params(limiter=synth.LIMITER_PAPER, precision=synth.PREC_MIXED,
                                             persistent_cells=PERSISTENT_CELLS)
        self._used = 0.0          # bytes charged for resident contexts
        self.peak_bytes = 0.0     # the most ever charged (never above the budget)
        self._cv = threading.Condition()
        self._streams = [torch.cuda.Stream(device=device) for _ in range(workers)]
        # resident contexts with their device fields, keyed (worker, kind,
        # size, index): kind "s" one per worker and size, kind "b" the k-th
        # context of a batch group; no request allocates device memory of its
        # own while its context stays resident
        self._res: Dict[tuple, _Resident] = {}
        self._pinned: List[Dict[int, object]] = [dict() for _ in range(workers)]
        self._fp_cache: Dict[int, int] = {}
        self._staging: List[Optional[object]] = [None] * workers
        self._init = None
        self._cancelled = set()
        self._cancel_lock = threading.Lock()

    def cancel(self, rid: int) -> None:
        """Cancel request rid if no worker has taken it yet."""
        with self._cancel_lock:
            self._cancelled.add(rid)

    def _take(self, r: synth.Request) -> bool:
        """True if r may be stepped (it was not cancelled); marks it taken."""
        with self._cancel_lock:
            if r.rid in self._cancelled:
                return False
            self._cancelled.discard(r.rid)
            return True

    # ---------------------------------------------------------- admission
    def footprint(self, n: int) -> int:
        """Device bytes a request of grid size n holds while it runs: the
        context (fld_footprint_bytes) and its three fields."""
        if n not in self._fp_cache:
            fp = fld.fld_footprint_bytes(synth.Grid.cube(n), self.params)
            self._fp_cache[n] = fp + 3 * n ** 3 * 8 if fp else 0
        return self._fp_cache[n]

    def resident_bytes(self) -> float:
        """Bytes charged for the contexts the server keeps on the device."""
        with self._cv:
            return self._used

    def resident_sizes(self, w: int, batch: bool = False) -> List[int]:
        """Grid sizes of worker w's resident contexts (of its batch groups
        when batch), sorted, with repeats for several contexts of one size."""
        kind = "b" if batch else "s"
        with self._cv:
            return sorted(k[2] for k in self._res if k[0] == w and k[1] == kind)

    def _evict_idle(self, need: float, keep) -> None:
        """Free least recently used idle contexts (not in keep) until need
        more bytes fit the budget or none is left; under the lock."""
        while self._used + need > self.budget:
            idle = [(e.last, k) for k, e in self._res.items() if not e.busy and k not in keep]
            if not idle:
                return
            _, k = min(idle)
            e = self._res.pop(k)
            if e.ctx is not None:
                e.ctx.close()
            e.buf = None
            self._used -= e.nbytes

    def _acquire(self, wanted) -> Optional[List[_Resident]]:
        """Mark the resident contexts of wanted [(key, n), ...] busy, charging
        the budget for those not yet resident, all at once: evicts idle
        contexts to make room and waits for busy ones when that is not
        enough.  None if the new ones together can never fit."""
        keys = {k for k, _ in wanted}
        new_bytes = sum(self.footprint(n) for k, n in wanted if k not in self._res)
        if any(self.footprint(n) <= 0 for _, n in wanted) or new_bytes > self.budget:
            return None
        with self._cv:
            while True:
                if any(k in self._res and self._res[k].busy for k in keys):
                    self._cv.wait()
                    continue
                need = sum(self.footprint(n) for k, n in wanted if k not in self._res)
                if self._used + need > self.budget:
                    self._evict_idle(need, keys)
                if self._used + need <= self.budget:
                    break
                self._cv.wait()
            out = []
            for k, n in wanted:
                e = self._res.get(k)
                if e is None:
                    e = _Resident(self.footprint(n))
                    self._res[k] = e
                    self._used += e.nbytes
                e.busy = True
                out.append(e)
            self.peak_bytes = max(self.peak_bytes, self._used)
            return out

    def _release(self, entries, failed=()):
        """Mark entries idle; drop (and uncharge) the keys in failed."""
        with self._cv:
            now = time.perf_counter()
            for e in entries:
                e.busy = False
                e.last = now
            for k in failed:
                e = self._res.pop(k, None)
                if e is not None:
                    if e.ctx is not None:
                        e.ctx.close()
                    self._used -= e.nbytes
            self._cv.notify_all()

    def _build(self, e: _Resident, w: int, n: int) -> None:
        """Create a resident entry's context (on worker w's stream) and field
        buffers (first use): E, n_HI and eta as rows of one (3, n^3)
        tensor."""
        torch = self.torch
        if e.ctx is None:
            e.ctx = fld.fld_create(synth.Grid.cube(n), self.params, self._streams[w])
        if e.buf is None:
            e.buf = torch.empty((3, n ** 3), dtype=torch.float64, device="cuda")

    # ----------------------------------------------------------- one step
    def _stage(self, w: int, slots: int):
        """Worker w's pinned staging words for `slots` requests' sources
        (reused once the worker's stream has been synchronised)."""
        torch = self.torch
        st = self._staging[w]
        if st is None or st.shape[0] < slots:
            st = torch.empty((slots, 2 * _MAX_SOURCES), dtype=torch.int64, pin_memory=True)
            self._staging[w] = st
        return st

    def _fields(self, r: synth.Request, out=None, stage=None):
        """E, n_HI and eta of a request on the current stream, built from its
        payload (distinct source cells and rates): one broadcast fill of the
        three rows of out (a (3, n^3) tensor, allocated when None), one copy
        of the payload from the pinned row stage (when given) and one
        scatter."""
        torch = self.torch
        n = r.n
        cells, rates = synth.request_sources(r)
        ns = len(cells)
        g = synth.Grid.cube(n)
        if out is None:
            out = torch.empty((3, n ** 3), dtype=torch.float64, device="cuda")
        if self._init is None:
            self._init = torch.tensor([synth.E0, 1e-3, 0.0], dtype=torch.float64, device="cuda").view(3, 1)
        out.copy_(self._init.expand(3, n ** 3))
        if stage is None:
            stage = torch.empty(2 * max(ns, 1), dtype=torch.int64, pin_memory=True)
        stage[:ns] = torch.from_numpy(cells[:, 0] + n * (cells[:, 1] + n * cells[:, 2]))
        stage[ns:2 * ns] = torch.from_numpy(rates * synth.HNU_HI / g.volume).view(torch.int64)
        dv = stage[:2 * ns].to("cuda", non_blocking=True)
        out[2].index_put_((dv[:ns],), dv[ns:].view(torch.float64))
        return out[0], out[1], out[2]

    def step_one(self, w: int, r: synth.Request, t0: float) -> Result:
        """Step one request on worker w (admission, fields, fld_step, E back to
        pinned host memory)."""
        torch = self.torch
        start = time.perf_counter() - t0
        key = (w, "s", r.n, 0)
        got = self._acquire([(key, r.n)])
        if got is None:
            return Result(r.rid, r.n, r.arrival, start, time.perf_counter() - t0, fld.FLD_ENOMEM)
        e = got[0]
        failed = ()
        try:
            with torch.cuda.stream(self._streams[w]):
                self._build(e, w, r.n)
                E, nHI, eta = self._fields(r, e.buf, self._stage(w, 1)[0])
                info = fld.fld_step(e.ctx, E, nHI, eta, check=False)
                host = self._pinned[w].get(r.n)
                if host is None:
                    host = torch.empty(r.n ** 3, dtype=torch.float64, pin_memory=True)
                    self._pinned[w][r.n] = host
                host.copy_(E, non_blocking=True)
                self._streams[w].synchronize()
                out = host.numpy().copy() if self.keep else None
        except Exception:
            failed = (key,)
            raise
        finally:
            self._release(got, failed)
        return Result(r.rid, r.n, r.arrival, start, time.perf_counter() - t0, info["status"],
                      info["iters"], info["outer_iters"], info["rel_res"], out)

    def step_batch(self, w: int, reqs: Sequence[synth.Request], t0: float) -> List[Result]:
        """Step several arrived requests together on worker w."""
        torch = self.torch
        start = time.perf_counter() - t0
        out: List[Result] = []
        admitted = []
        for r in reqs:
            nb = self.footprint(r.n)
            if nb <= 0 or nb > self.budget:
                out.append(Result(r.rid, r.n, r.arrival, start, time.perf_counter() - t0, fld.FLD_ENOMEM))
            else:
                admitted.append(r)
        if not admitted:
            return out
        # the group's contexts are acquired as a whole, so a worker never
        # holds part of the budget while waiting for the rest
        used: Dict[int, int] = {}
        wanted = []
        for r in admitted:
            k = used.get(r.n, 0)
            used[r.n] = k + 1
            wanted.append(((w, "b", r.n, k), r.n))
        got = self._acquire(wanted)
        if got is None:
            now = time.perf_counter() - t0
            return out + [Result(r.rid, r.n, r.arrival, start, now, fld.FLD_ENOMEM) for r in admitted]
        failed = ()
        try:
            with torch.cuda.stream(self._streams[w]):
                ctxs, fields = [], []
                stage = self._stage(w, len(admitted))
                for q, (r, e) in enumerate(zip(admitted, got)):
                    self._build(e, w, r.n)
                    ctxs.append(e.ctx)
                    fields.append(self._fields(r, e.buf, stage[q]))
                # the contexts overlap on private streams forked from and
                # joined to the worker's
                st, infos = fld.fld_step_batched(ctxs, [f[0] for f in fields], [f[1] for f in fields],
                                                 [f[2] for f in fields], check=False)
                # E^{n+1} of every request back to pinned host memory, as a
                # single step does
                hosts = []
                for r, f, e in zip(admitted, fields, got):
                    h = self._pinned[w].get(("b", r.n, len(hosts)))
                    if h is None:
                        h = torch.empty(r.n ** 3, dtype=torch.float64, pin_memory=True)
                        self._pinned[w][("b", r.n, len(hosts))] = h
                    h.copy_(f[0], non_blocking=True)
                    hosts.append(h)
                self._streams[w].synchronize()
                now = time.perf_counter() - t0
                for r, info, h in zip(admitted, infos, hosts):
                    out.append(Result(r.rid, r.n, r.arrival, start, now, info["status"], info["iters"],
                                      info["outer_iters"], info["rel_res"],
                                      h.numpy().copy() if self.keep else None))
        except Exception:
            failed = tuple(k for k, _ in wanted)
            raise
        finally:
            self._release(got, failed)
        return out

    # ------------------------------------------------------------ the loop
    def warm(self, sizes: Sequence[int], sources: int = 4) -> List[Result]:
        """Build every worker's resident context for each grid size (and, when
        batching, the first context of its batch pool) and step it once, so
        that allocations and the captured CUDA graphs of the solve exist before
        requests arrive; returns the warm-up results."""
        self.torch.cuda.set_device(self.device)
        t0 = time.perf_counter()
        out: List[Result] = []
        for w in range(self.workers):
            for i, n in enumerate(sizes):
                r = synth.Request(-1 - i, 0.0, int(n), seed=1000 * w + i, sources=sources)
                if self.footprint(r.n) <= 0 or self.footprint(r.n) > self.budget:
                    continue
                out.append(self.step_one(w, r, t0))
                if self.batch > 1 and r.n <= self.batch_max_n:
                    out.extend(self.step_batch(w, [r], t0))
        return out

    def run(self, requests: Sequence[synth.Request], realtime: bool = True) -> List[Result]:
        """Serve requests as they arrive (arrival times in s from now when
        realtime, else all at once); returns results in request order."""
        self.torch.cuda.set_device(self.device)
        q: "queue.Queue" = queue.Queue()
        results: Dict[int, Result] = {}
        lock = threading.Lock()
        # the stop markers go in only once every request has its result, so
        # requests put back into the queue (large grids a batching worker
        # left for the next free worker) never sit behind them
        all_done = threading.Event()
        total = len({r.rid for r in requests})
        if total == 0:
            all_done.set()
        t0 = time.perf_counter()

        def record(res):
            with lock:
                for r in res:
                    results[r.rid] = r
                if len(results) >= total:
                    all_done.set()

        def worker(w):
            """Worker thread: take requests (or groups of them) until the stop
            marker and record their results."""
            self.torch.cuda.set_device(self.device)
            while True:
                item = q.get()
                if item is None:
                    return
                group = [item]
                try:
                    res = serve(w, item, group)
                except Exception:
                    # a failed call (recorded, so run() still finishes)
                    now = time.perf_counter() - t0
                    res = [Result(r.rid, r.n, r.arrival, now, now, fld.FLD_ECUDA) for r in group]
                record(res)

        def serve(w, item, group):
            """Step item (alone, or with the other small arrived requests it
            collects into group) on worker w; returns their results."""
            if not self._take(item):
                now = time.perf_counter() - t0
                return [Result(item.rid, item.n, item.arrival, now, now, CANCELLED)]
            if self.batch == 1 or item.n > self.batch_max_n:
                return [self.step_one(w, item, t0)]
            stop, later = False, []
            used = self.footprint(item.n)
            while len(group) < self.batch:
                try:
                    nxt = q.get_nowait()
                except queue.Empty:
                    break
                if nxt is None:
                    stop = True
                    break
                if nxt.n > self.batch_max_n:
                    later.append(nxt)    # stepped alone, by the next free worker
                    continue
                fp = self.footprint(nxt.n)
                if not self._take(nxt):
                    now = time.perf_counter() - t0
                    record([Result(nxt.rid, nxt.n, nxt.arrival, now, now, CANCELLED)])
                    continue
                if used + fp > self.budget:
                    later.append(nxt)    # waits for a later group
                    break
                group.append(nxt)
                used += fp
            for r in later:
                q.put(r)
            if stop:
                q.put(None)
            return self.step_batch(w, group, t0)

        threads = [threading.Thread(target=worker, args=(w,), daemon=True) for w in range(self.workers)]
        for t in threads:
            t.start()
        order = sorted(requests, key=lambda r: r.arrival)
        for r in order:
            if realtime:
                delay = r.arrival - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
            else:
                r = dataclasses.replace(r, arrival=time.perf_counter() - t0)
            q.put(r)
        all_done.wait()
        for _ in threads:
            q.put(None)
        for t in threads:
            t.join()
        return [results[r.rid] for r in requests]

    def close(self):
        """Free every resident context and field buffer."""
        with self._cv:
            for e in self._res.values():
                if e.ctx is not None:
                    e.ctx.close()
                e.buf = None
            self._res.clear()
            self._used = 0.0


def summarize(results: Sequence[Result]) -> dict:
    """Counts, latency and waiting percentiles and throughput of a run."""
    ok = [r for r in results if r.status == fld.FLD_OK]
    cancelled = sum(1 for r in results if r.status == CANCELLED)
    lat = np.array([r.latency_ms for r in ok]) if ok else np.zeros(1)
    wait = np.array([r.wait_ms for r in ok]) if ok else np.zeros(1)
    span = (max(r.finish for r in results) - min(r.arrival for r in results)) if results else 0.0
    cells = sum(r.n ** 3 for r in ok)
    return {"requests": len(results), "ok": len(ok),
            "failed": len(results) - len(ok) - cancelled, "cancelled": cancelled,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "wait_p50_ms": float(np.percentile(wait, 50)), "wait_p99_ms": float(np.percentile(wait, 99)),
            "solves_per_s": len(ok) / span if span > 0 else None,
            "cell_solves_per_s": cells / span if span > 0 else None,
            "span_s": span}
