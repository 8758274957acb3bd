#!/usr/bin/env python
"""Benchmark of the implicit grey FLD radiation step on GB300.

Default workload: a 512^3 zero-gradient grid, log-normal density
(sigma_ln = 1.5, mean n_H = 1e-3 cm^-3, clamped to [1e-3, 1e3] x mean, i.e.
opacity contrast up to 1e6), fully neutral, 65536 sources of 5e48 photons/s
at the densest peaks; one step = assembly + MG-preconditioned CG to
||r||/||b|| <= 1e-8 + finalise, in mixed precision (FP32 V-cycles and inner
CG inside FP64 iterative refinement).  The plain FP64 GPU multigrid runs on
the same input beside it.  Inputs are synthetic (seeded generators), every
field is 1 GiB (larger than L2), and successive steps advance E in time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank steps its own
replica of the workload (no collective on the data path; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-solves/s to 1e-8 rel. residual, mixed vs FP64 MG on 1 GB300; p50/p99 latency"
UNIT = "cell-solves/s"

# DRAM traffic over algorithmic bytes of the finest-level launch of each
# kernel class, from one ncu capture per kernel of the 320^3 log-normal case
# (dram__bytes_read.sum + dram__bytes_write.sum of the launch divided by the
# bytes the kernel must stream).
# Traffic grows with the cells of a launch, so a launch's traffic is this
# ratio times its algorithmic bytes.  A class whose kernel changed since
# the capture is left out (its traffic is then reported as null).
# Compulsory bytes per cell of a mixed step under the fused-schedule model
# (FP32 inner vectors and operator, FP64 outer): assembly reads E, n_HI, eta
# and writes m, three face weights and b in FP64 plus the FP32 operator;
# one preconditioned CG iteration streams 36 FP32 words (pre-smooth fused
# with residual and restriction 12, prolongation with post-smoothing 7,
# coarse levels about 2.7, p/q/<p,q> 8, x/r update 6); one outer refinement
# reads x, b and the FP64 operator and writes the FP32 residual; finalize
# reads E and dE and writes E.
MODEL_ASM, MODEL_ITER, MODEL_IR, MODEL_FIN = 80.0, 144.0, 52.0, 24.0

TRAFFIC_OVER_ALGORITHMIC = {
    "rb_colour": 19.9 / 18.0,
    "cg_p_matvec": 40.5 / 40.0,
    "smooth_zero": 16.1 / 16.0,
    "residual": 12.0 / 12.0,
    "restrict": 2.1 / 2.5,
    "prolong_add": 6.7 / 8.5,
    "cg_update": 10.5 / 12.0,
}


def parse():
    """Command-line options of the benchmark."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--n", type=int, default=512, help="grid cells per axis")
    ap.add_argument("--sources", type=int, default=65536)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--fp32-coef-steps", type=int, default=3,
                    help="steps of the same mixed step with FP32 smoothing coefficients (precond_bf16 = 0)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--one-core-n", type=int, default=128,
                    help="grid of the one-core oracle sample of the CPU baseline (0 skips it)")
    ap.add_argument("--ref-n", type=int, default=256, help="grid of the reference arm's per-step sample")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle step at the benchmark size (CPU baseline and oracle error)")
    ap.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving leg (Poisson stream, 0 = skip)")
    ap.add_argument("--serve-rate", type=float, default=500.0)
    ap.add_argument("--variant-steps", type=int, default=3,
                    help="timed steps of each method variant (trapezoidal rule, outflow faces, "
                         "comoving units) on the same workload; 0 skips them")
    ap.add_argument("--serve-workers", type=int, default=8)
    ap.add_argument("--serve-batch", type=int, default=8,
                    help="requests a worker of the batched serving leg steps together")
    ap.add_argument("--graphs", type=int, default=-1, choices=[-1, 0, 1],
                    help="fld_params.graphs of the measured contexts (0: every launch eager, e.g. for a "
                         "profiler's launch list)")
    return ap.parse_args()


def dist_env():
    """(world size, rank, local rank) from the torchrun environment."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(n, sources, device):
    """The benchmark input at n^3 (sources scaled with the cell count below 512^3)."""
    from paper_1306_0645_gb300 import synth
    sources = max(1, min(sources, (sources * n ** 3) // 512 ** 3 if n != 512 else sources))
    return synth.config4(n=n, sources=sources, device=device)


def workload_desc(n, sources):
    """One-line description of the benchmark workload for the JSON line."""
    return (f"{n}^3 zero-gradient, log-normal density sigma_ln 1.5 mean n_H 1e-3 clamped to "
            f"[1e-3,1e3]x mean (opacity contrast 1e6), neutral, {sources} sources of 5e48 /s at the "
            f"densest peaks, dt 1e5 yr, box 6.6 kpc, paper limiter; MG-PCG to 1e-8")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        """Start sampling nvidia-smi clocks in the background."""
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        """Stop sampling; returns the median SM clock of the samples, the
        maximum clock and the throttle reasons seen active."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no clock samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def max_over_ranks(ms, dist, device="cuda"):
    """Max of a per-rank time over all ranks (the job is as slow as its
    slowest rank)."""
    import torch
    if dist is None:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_hbm_peak():
    """HBM copy bandwidth (GB/s) of MEASURED_PEAKS.json, else the fallback figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def time_steps(fld, torch, ctx, E, nHI, eta, steps):
    """K steps on the context's stream; returns (total_ms, per-step ms, infos)."""
    s = ctx.stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    infos = []
    torch.cuda.synchronize()
    ev[0].record(s)
    for k in range(steps):
        infos.append(fld.fld_step(ctx, E, nHI, eta))
        ev[k + 1].record(s)
    torch.cuda.synchronize()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    return ev[0].elapsed_time(ev[steps]), per, infos


def oracle_errors(E, Eo):
    """Error of a CUDA-path E^{n+1} against the oracle's: L2 and max norm
    relative to the field, and the largest relative error of the cells with
    E > 1e-6 max E (not controlled by a 1e-8 residual; stated only)."""
    mask = Eo > 1e-6 * Eo.max()
    return {"l2": float(np.linalg.norm(E - Eo) / np.linalg.norm(Eo)),
            "max_rel_to_max": float(np.abs(E - Eo).max() / np.abs(Eo).max()),
            "cellwise_E_gt_1e-6max": float((np.abs(E - Eo)[mask] / Eo[mask]).max())}


def oracle_sample(n):
    """One oracle step of the benchmark recipe at n^3 on this process's cores;
    prints its throughput as JSON (run by one_core_baseline in a child process
    limited to one OpenMP thread)."""
    import oracle
    from paper_1306_0645_gb300 import synth
    src = max(1, 65536 * n ** 3 // 512 ** 3)
    case = synth.config4(n=n, sources=src)
    oracle.build()
    t0 = time.perf_counter()
    _, info = oracle.step(case.grid, case.params, {}, case.E, case.nHI, case.eta)
    dt = time.perf_counter() - t0
    print(json.dumps({"value": case.grid.cells / dt, "s": dt, "cores": oracle.num_threads(),
                      "iters": info["iters"], "n": n, "sources": src}), flush=True)


def one_core_baseline(n):
    """The oracle on one host core: one step of the recipe at n^3 in a child
    process with OMP_NUM_THREADS=1."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", str(n)], env=env,
                       capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else "failed"}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["value"], "unit": UNIT, "cores": d["cores"],
            "sample": f"1 oracle step at {n}^3 with {d['sources']} sources ({d['s']:.1f} s, {d['iters']} iters)"}


def run_reference(args):
    """The reference arm: the FP64 oracle on a bounded sample of the workload,
    printed as the benchmark's JSON line (rank 0 only)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1306_0645_gb300 import synth
    oracle.build()
    n = args.ref_n
    src = max(1, args.sources * n ** 3 // 512 ** 3)
    case = synth.config4(n=n, sources=src)
    cfg_n = args.n
    cfg_src = args.sources if cfg_n == 512 else max(1, args.sources * cfg_n ** 3 // 512 ** 3)
    E = case.E.copy()
    for _ in range(args.warmup):
        E, _ = oracle.step(case.grid, case.params, {}, E, case.nHI, case.eta)
    t0 = time.perf_counter()
    per = []
    for _ in range(args.steps):
        t1 = time.perf_counter()
        E, info = oracle.step(case.grid, case.params, {}, E, case.nHI, case.eta)
        per.append((time.perf_counter() - t1) * 1e3)
    total = time.perf_counter() - t0
    value = case.grid.cells * args.steps / total
    cores = oracle.num_threads()
    sample = (f"each step: one FP64 oracle step (plain C + OpenMP, {cores} threads, MG-PCG to 1e-8) of the "
              f"workload's recipe at {n}^3 with {src} sources, a bounded sample of the {cfg_n}^3 workload "
              f"(cell-solves/s is per cell, so the sample's rate stands for the workload's)")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": total * 1e3 / args.steps,
           "p50_ms": float(np.percentile(per, 50)), "p99_ms": float(np.percentile(per, 99)),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": workload_desc(cfg_n, cfg_src), "n": cfg_n,
                                           "sources": cfg_src, "sample_n": n, "sample_sources": src},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    """The measured run: mixed step, FP64 multigrid, variants, e2e, serving and
    CPU baseline, printed as one JSON line on rank 0."""
    args = parse()
    if args.oracle_sample:
        oracle_sample(args.oracle_sample)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1306_0645_gb300 import fld, synth

    n = args.n
    sources = args.sources if n == 512 else max(1, args.sources * n ** 3 // 512 ** 3)
    case = synth.config4(n=n, sources=sources, device="cuda")
    cells = case.grid.cells
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()
    E0, nHI, eta = dev(case.E), dev(case.nHI), dev(case.eta)
    # a stream of its own (the legacy default stream cannot hold the CUDA
    # graphs of the solve); torch work below is ordered on it as well
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    torch.cuda.set_stream(stream)

    # ---- mixed precision (the measured path)
    pm = case.params
    pm.precision = synth.PREC_MIXED
    pm.graphs = args.graphs
    ctx = fld.fld_create(case.grid, pm, stream)
    tuning = fld.autotune(ctx)
    kinds = ["smooth_zero", "rb_colour", "residual", "restrict", "prolong", "cg_p_matvec", "post_smooth"]
    tuned = {k: tuning[3 * q: 3 * q + 3] for q, k in enumerate(kinds)}   # threads, blocks, prefetch
    E = E0.clone()
    for _ in range(args.warmup):
        fld.fld_step(ctx, E, nHI, eta)
    # one untimed step with every kernel class timed picks the dominant kernel
    fld.fld_profile(ctx, (1 << 62) - 1)
    Ecal = E.clone()
    fld.fld_step(ctx, Ecal, nHI, eta)
    stats = fld.fld_profile_read(ctx)
    dom = max(stats, key=lambda k: k["ms"])
    breakdown = {k["name"]: {"ms": round(k["ms"], 3), "launches": k["launches"],
                             "GBps": round(k["timed_bytes"] / (k["ms"] * 1e-3) / 1e9, 1) if k["ms"] > 0 else None}
                 for k in stats if k["launches"] > 0}
    del Ecal
    # the timed steps run the production launch path: no event timing, so
    # the CG solve runs as CUDA graphs (the whole inner loop one device-side
    # graph launch); fld_profile resets the launch and byte counts
    fld.fld_profile(ctx, 0)

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    if dist:
        dist.barrier()
    clocks.start()
    total_ms, per, infos = time_steps(fld, torch, ctx, E, nHI, eta, args.steps)
    clk = clocks.stop()
    stats = fld.fld_profile_read(ctx)
    launches = int(sum(k["launches"] for k in stats))
    # calibration of the dominant kernel: the same number of steps from a copy
    # of E with that class timed launch by launch (CUDA events on the
    # context's stream; the launches go eagerly then)
    fld.fld_profile(ctx, 1 << dom["cls"])
    Ecal = E.clone()
    cal_ms, _, _ = time_steps(fld, torch, ctx, Ecal, nHI, eta, args.steps)
    cstats = fld.fld_profile_read(ctx)
    fld.fld_profile(ctx, 0)
    del Ecal
    d = next(k for k in cstats if k["cls"] == dom["cls"])
    total_ms = max_over_ranks(total_ms, dist)
    value = cells * args.steps * world / (total_ms * 1e-3)

    peak, peak_kind = measured_hbm_peak()
    avg_ms = d["ms"] / max(d["timed"], 1)
    bytes_per = d["timed_bytes"] / max(d["timed"], 1)
    achieved = bytes_per / (avg_ms * 1e-3) / 1e9
    ratio = TRAFFIC_OVER_ALGORITHMIC.get(d["name"])
    traffic = ratio * bytes_per if ratio else None
    roofline = {"kernel": d["name"], "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                # the DRAM bytes the launch moves (ncu ratio x algorithmic) over its time: a colour
                # sweep changes half of z but writes every 16-byte group of it back
                "traffic_frac": (traffic / (avg_ms * 1e-3) / 1e9 / peak) if traffic else None,
                "launches_timed": d["timed"], "avg_launch_ms": avg_ms, "bytes_per_launch": bytes_per,
                "share_of_step": d["ms"] / cal_ms,
                "timing": "CUDA events around each launch of the class on the context's stream, over "
                          f"{args.steps} calibration steps run eagerly after the timed (graph) steps "
                          f"({cal_ms / args.steps:.2f} ms per eager step)"}
    # whole-step algorithmic bytes over step time (all kernels)
    step_bytes = sum(k["bytes"] for k in stats) / args.steps
    step_frac = step_bytes / (total_ms / args.steps * 1e-3) / (peak * 1e9)
    # the same fraction under the compulsory-traffic model of a fully fused
    # schedule (bytes per cell: assembly 80, per inner iteration 144, per
    # outer refinement 52, finalize 24, with the measured iteration counts)
    model_cell = np.mean([MODEL_ASM + i["iters"] * MODEL_ITER + i["outer_iters"] * MODEL_IR + MODEL_FIN
                          for i in infos])
    step_model = {"bytes_per_cell": float(model_cell),
                  "frac": float(model_cell * cells / (total_ms / args.steps * 1e-3) / (peak * 1e9)),
                  "own_bytes_per_cell": float(step_bytes / cells)}

    # ---- the headline step against the FP64 oracle at full size: one more
    # mixed step from the current E^n, the same step by the FP64 GPU
    # multigrid below and by the oracle on the host cores (which is also the
    # CPU baseline of this workload)
    E_n = E.clone()
    E_mx = E_n.clone()
    info_mx = fld.fld_step(ctx, E_mx, nHI, eta)
    torch.cuda.synchronize()
    E_mx_h = E_mx.cpu().numpy()
    del E_mx

    # ---- the same mixed step with the V-cycle's smoothing coefficients read
    # as FP32 (precond_bf16 = 0), with the timed context's launch shapes
    fp32_coef = None
    if args.fp32_coef_steps > 0:
        import dataclasses
        pc = dataclasses.replace(pm, precond_bf16=0)
        ctxc = fld.fld_create(case.grid, pc, stream)
        fld.fld_set_tuning(ctxc, fld.fld_get_tuning(ctx))
        Ec = E0.clone()
        fld.fld_step(ctxc, Ec, nHI, eta)
        msc, _, infc = time_steps(fld, torch, ctxc, Ec, nHI, eta, args.fp32_coef_steps)
        fp32_coef = {"value": cells * args.fp32_coef_steps / (msc * 1e-3), "unit": UNIT,
                     "ms_per_step": msc / args.fp32_coef_steps, "iters": [i["iters"] for i in infc],
                     "outer_iters": [i["outer_iters"] for i in infc], "rel_res": [i["rel_res"] for i in infc],
                     "what": "the same mixed step with the V-cycle's smoothing coefficients read as FP32 "
                             "(precond_bf16 = 0), the timed context's launch shapes"}
        ctxc.close()
        del Ec

    # ---- plain FP64 multigrid on the same input
    fp64 = None
    E_64_h = None
    if args.fp64_steps > 0:
        import dataclasses
        p64 = dataclasses.replace(pm, precision=synth.PREC_FP64)
        ctx64 = fld.fld_create(case.grid, p64, stream)
        E64 = E0.clone()
        for _ in range(min(args.warmup, 1)):
            fld.fld_step(ctx64, E64, nHI, eta)
        ms64, per64, inf64 = time_steps(fld, torch, ctx64, E64, nHI, eta, args.fp64_steps)
        fp64 = {"value": cells * args.fp64_steps / (ms64 * 1e-3), "unit": UNIT,
                "ms_per_step": ms64 / args.fp64_steps, "iters": [i["iters"] for i in inf64],
                "rel_res": [i["rel_res"] for i in inf64]}
        # its own algorithmic bytes over step time, and the per-class times
        # of one step (every class timed; eager)
        fld.fld_profile(ctx64, (1 << 62) - 1)
        E64c = E64.clone()
        fld.fld_step(ctx64, E64c, nHI, eta)
        s64 = fld.fld_profile_read(ctx64)
        fld.fld_profile(ctx64, 0)
        del E64c
        b64 = sum(k["bytes"] for k in s64)
        fp64["step_roofline_frac"] = b64 / (ms64 / args.fp64_steps * 1e-3) / (peak * 1e9)
        fp64["own_bytes_per_cell"] = b64 / cells
        fp64["kernel_breakdown_one_step"] = {
            k["name"]: {"ms": round(k["ms"], 3), "launches": k["launches"],
                        "GBps": round(k["timed_bytes"] / (k["ms"] * 1e-3) / 1e9, 1) if k["ms"] > 0 else None}
            for k in s64 if k["launches"] > 0}
        E64.copy_(E_n)
        fld.fld_step(ctx64, E64, nHI, eta)
        torch.cuda.synchronize()
        E_64_h = E64.cpu().numpy()
        ctx64.close()
        del E64

    # ---- method variants on the same workload and tuned launch shapes
    variants = None
    if args.variant_steps > 0:
        import dataclasses
        table = fld.fld_get_tuning(ctx)
        grid_out = case.grid.outflow_upper()
        variants = {}
        for name, grid_v, changes in (
                ("trapezoidal", case.grid, {"theta": 0.5}),
                ("outflow_faces", grid_out, {}),
                ("comoving_a0.5", case.grid, {"scale_factor": 0.5, "adot_over_a": 1.0e-17})):
            pv = dataclasses.replace(pm, **changes)
            ctxv = fld.fld_create(grid_v, pv, stream)
            fld.fld_set_tuning(ctxv, table)
            Ev = E0.clone()
            fld.fld_step(ctxv, Ev, nHI, eta)
            msv, perv, infv = time_steps(fld, torch, ctxv, Ev, nHI, eta, args.variant_steps)
            variants[name] = {"value": cells * args.variant_steps / (msv * 1e-3), "unit": UNIT,
                              "ms_per_step": msv / args.variant_steps,
                              "iters": [i["iters"] for i in infv], "outer_iters": [i["outer_iters"] for i in infv],
                              "rel_res": [i["rel_res"] for i in infv],
                              "balance_rel": [i["balance_rel"] for i in infv],
                              "what": {"trapezoidal": "theta = 1/2 (Sec. 3.2)",
                                       "outflow_faces": "reflecting at x, y, z = 0, outflow at the upper faces "
                                                        "(Sec. 4.1 boundary set)",
                                       "comoving_a0.5": "comoving widths at scale factor 0.5, adot/a 1e-17 /s"}[name]}
            ctxv.close()
            del Ev
        # multigroup: four groups of a 1e5 K blackbody (edges at the HI,
        # HeI, HeII thresholds, 100 nu_HI and 1000 nu_HI), each an FLD system
        # with its group opacity and share of the emissivity; a step is the
        # group fields plus all groups through the batched driver
        G = 4
        hnu_hi = synth.HNU_HI
        h_pl = 6.62607015e-27
        nu1 = hnu_hi / h_pl
        edges = [nu1, 24.6 / 13.6 * nu1, 54.4 / 13.6 * nu1, 100 * nu1, 1000 * nu1]
        coef = fld.fld_sed_integrals(fld.fld_sed_default(kind=fld.FLD_SED_BLACKBODY, T=1e5), edges)
        pg = dataclasses.replace(pm, sigma=1.0)
        gstreams = [torch.cuda.Stream() for _ in range(G)]
        gctx = [fld.fld_create(case.grid, pg, st) for st in gstreams]
        for c_ in gctx:
            fld.fld_set_tuning(c_, table)
        kap = [torch.empty_like(E0) for _ in range(G)]
        etg = [torch.empty_like(E0) for _ in range(G)]
        Eg = [E0 * float(coef[k, 9]) for k in range(G)]

        def mg_step():
            """One multigroup step: group fields, then all groups batched."""
            fld.fld_group_fields(coef, nHI, kap, eta=eta, etas=etg)
            torch.cuda.synchronize()
            return fld.fld_step_batched(gctx, Eg, kap, etg)

        mg_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        minf = []
        for _ in range(args.variant_steps):
            minf.append(mg_step()[1])
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        variants["multigroup4"] = {
            "value": cells * G * args.variant_steps / el, "unit": "cell-group-solves/s",
            "ms_per_step": el * 1e3 / args.variant_steps,
            "iters": [[i["iters"] for i in st_] for st_ in minf],
            "what": "4 groups of a 1e5 K blackbody (edges nu_HI, nu_HeI, nu_HeII, 100, 1000 nu_HI), "
                    "group opacities and emissivities by fld_group_fields, groups stepped together by "
                    "fld_step_batched; wall time of whole steps (host clock)"}
        for c_ in gctx:
            c_.close()
        del kap, etg, Eg

    # ---- end to end through the host-buffer entry point
    e2e = None
    if args.e2e_steps > 0:
        Eh = torch.empty(cells, dtype=torch.float64, pin_memory=True)
        Eh.copy_(E0.cpu())
        nh = torch.empty(cells, dtype=torch.float64, pin_memory=True)
        nh.copy_(nHI.cpu())
        eh = torch.empty(cells, dtype=torch.float64, pin_memory=True)
        eh.copy_(eta.cpu())
        Ehn, nhn, ehn = Eh.numpy(), nh.numpy(), eh.numpy()
        fld.fld_step_host(ctx, Ehn, nhn, ehn)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            fld.fld_step_host(ctx, Ehn, nhn, ehn)
        el = time.perf_counter() - t0
        e2e = {"value": cells * args.e2e_steps / el, "unit": UNIT, "h2d_bytes_per_step": 3 * cells * 8,
               "d2h_bytes_per_step": cells * 8}

    # ---- serving: a Poisson stream of independent grids, continuous batching
    serving_out = None
    if args.serve_requests > 0:
        from paper_1306_0645_gb300 import serving
        reqs = synth.request_stream(count=args.serve_requests, rate=args.serve_rate, seed=5 + rank)
        sizes = [16, 32, 48, 64, 96, 128]

        def serve_leg(batch):
            """Realtime latency and saturation throughput of one serving mode."""
            srv = serving.Server(budget_bytes=40e9, workers=args.serve_workers, batch=batch)
            # every worker's resident contexts and solve graphs for every size
            srv.warm(sizes)
            res = srv.run(reqs, realtime=True)
            # saturation: the same requests all arriving at once
            sat = serving.summarize(srv.run(reqs, realtime=False))
            srv.close()
            out = serving.summarize(res)
            out["mode"] = ("threads: one request per worker" if batch == 1 else
                           f"a free worker steps up to {batch} arrived requests of at most {srv.batch_max_n}^3 "
                           f"cells in one fld_step_batched (persistent inner solves over a work list); larger "
                           f"ones alone")
            out["saturation"] = {"solves_per_s": sat["solves_per_s"],
                                 "cell_solves_per_s": sat["cell_solves_per_s"], "span_s": sat["span_s"],
                                 "what": "the same requests all arriving at time 0 (the server's throughput "
                                         "limit; latencies then measure the queue)"}
            return out

        serving_out = serve_leg(1)
        serving_out.update({"rate_per_s": args.serve_rate, "workers": args.serve_workers,
                            "budget_GB": 40, "sizes": sizes,
                            "precision": "mixed", "latency": "arrival to E^{n+1} on the host"})
        serving_out["batched"] = serve_leg(args.serve_batch)

    cpu = None
    oracle_err = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        E_in = E_n.cpu().numpy().reshape(case.grid.shape)
        t0 = time.perf_counter()
        Eo, io = oracle.step(case.grid, case.params, {}, E_in, case.nHI, case.eta)
        t_or = time.perf_counter() - t0
        cpu = {"value": cells / t_or, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"1 FP64 oracle step (plain C + OpenMP, MG-PCG to 1e-8) of the benchmark workload "
                         f"itself, {n}^3 with {sources} sources, from the E^n of the timed steps "
                         f"({t_or:.1f} s, {io['iters']} iters)"}
        if args.one_core_n > 0:
            cpu["one_core"] = one_core_baseline(args.one_core_n)
        oracle_err = {"reference": f"FP64 oracle step to ||r||/||b|| <= 1e-8 from the same E^n "
                                   f"({io['iters']} iterations)",
                      "mixed": dict(oracle_errors(E_mx_h.reshape(case.grid.shape), Eo),
                                    rel_res=info_mx["rel_res"], iters=info_mx["iters"],
                                    outer_iters=info_mx["outer_iters"])}
        if E_64_h is not None:
            oracle_err["fp64_mg"] = oracle_errors(E_64_h.reshape(case.grid.shape), Eo)
        del Eo, E_in

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "p50_ms": float(np.percentile(per, 50)), "p99_ms": float(np.percentile(per, 99)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 inner / f64 outer (mixed)", "data": "synthetic (seeded generators, no dataset)",
            "config": {"workload": workload_desc(n, sources), "n": n, "sources": sources,
                       "precision": "mixed", "l2": "inputs larger than L2 (each field 1 GiB at 512^3)",
                       "parallelism": f"{world} independent replica(s)",
                       "tuned_finest_level": {k: {"threads": v[0], "blocks": v[1]} for k, v in tuned.items()}},
            "iters": [i["iters"] for i in infos], "outer_iters": [i["outer_iters"] for i in infos],
            "rel_res": [i["rel_res"] for i in infos],
            "fp64_mg": fp64,
            "mixed_over_fp64": (value / world) / fp64["value"] if fp64 else None,
            "mixed_fp32_coefficients": fp32_coef,
            "roofline": roofline, "step_roofline_frac": step_frac, "step_roofline_model": step_model,
            "kernel_breakdown_one_step": breakdown,
            "oracle_err": oracle_err,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "serving": serving_out, "variants": variants,
        }
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
