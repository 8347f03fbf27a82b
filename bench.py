#!/usr/bin/env python
"""Benchmark of the MRCM Darcy solve on one GB300 (or N replicas).

One step = the whole hot path (factor_local, build_basis, solve_interface,
reconstruct) on the 256x64 channelised workload (binary K, contrast 1e6,
16x16 subdomains, cubic interface spaces: 8 unknowns per interface), replayed
from a CUDA graph with inputs resident in HBM.  The workload (0.4 MB) fits in
L2, so L2 is flushed (a 256 MB write) before every timed step; only the step
itself is inside the CUDA events.  Prints one JSON line.

The same line carries, under "batched", the batched workload: 32 lognormal
realisations of 1024 x 1024 cells (16 x 16-cell subdomains in the first 16,
32 x 32 in the rest, 2 to 8 unknowns per interface), timed the same way
(whole solve as one CUDA graph, inputs in HBM; its 2.4 GB of inputs and
outputs exceed L2), with its own FP64 path, roofline, e2e and CPU baseline,
checked against the oracle on sampled outputs.

A value is reported only when the accuracy check passed: relative L2 error
<= 1e-8 in p and u against the oracle (headline), sampled pressures and
continuity defects <= 1e-10 and global balance <= 1e-8 (batched).

--impl reference times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

METRIC = "fine cells/s of MRCM Darcy solve, mixed vs FP64 GPU, at rel L2 err ≤1e-8"
WORKLOAD = "channels-256x64 binary K 1e3/1e-3, 16x16 subdomains (64), m=8 per interface (864 unknowns)"
BATCH_WORKLOAD = ("lognormal-32x1024x1024 sigma^2=3, 16x16 subdomains (r<16) and 32x32 (r>=16), "
                  "m in {2,4,6,8} per interface")
ACC_TOL = 1e-8            # relative L2 in p and u against the oracle (the metric's bound)
SAMPLE_P_TOL = 1e-10      # batched: sampled subdomain pressures (relative)
SAMPLE_DEFECT_TOL = 1e-10 # batched: sampled interface continuity defects (relative)
BALANCE_TOL = 1e-8        # batched: global mass balance


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(x: float, ws: int, device) -> float:
    """The largest x over the ranks of the default process group (x itself
    on one rank).  Every rank must call it at the same point."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_value(units_per_rank_step: float, steps: int, ws: int, t_max: float) -> float:
    """Whole-job throughput: the units all ranks processed (each rank owns
    its own problems, weak scaling) over the slowest rank's time."""
    return units_per_rank_step * steps * ws / t_max


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = Path(os.environ.get("TMPDIR", "/tmp")) / f"mrcm_clocks_{os.getpid()}.csv"

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = [l.split(",") for l in self.path.read_text().splitlines() if l.strip()]
        try:
            self.path.unlink()
        except Exception:
            pass
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------- peaks
def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        try:
            return json.loads(p.read_text()), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ----------------------------------------------------------------- CPU arm
def _oracle_worker(seconds: float, max_solves: int):
    """Times the oracle as it stands on the workload; one thread."""
    from oracle import mrcm_oracle as O
    from paper_2104_04653_gb300 import workloads as W
    prob = W.config2()
    cells = prob.cells()
    times = []
    t_end = time.perf_counter() + seconds
    while len(times) < max_solves and (not times or time.perf_counter() < t_end):
        t0 = time.perf_counter()
        O.mrcm_solve(prob)
        times.append(time.perf_counter() - t0)
    return {"cells": cells, "times": times}


def cpu_baseline(seconds: float = 12.0, max_solves: int = 50):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench._oracle_worker(%f, %d)))" % (str(ROOT), seconds, max_solves))
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         cwd=str(ROOT), timeout=600)
    if res.returncode != 0:
        return {"value": None, "unit": "cells/s", "cores": 1, "kind": "oracle",
                "sample": "failed: " + res.stderr.strip().splitlines()[-1][:200]}
    d = json.loads(res.stdout.strip().splitlines()[-1])
    t = statistics.median(d["times"])
    return {"value": d["cells"] / t, "unit": "cells/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(d['times'])} full solves of the workload (median {t * 1e3:.1f} ms), "
                      f"numpy/scipy FP64, 1 thread"}


def _host_cores() -> int:
    """Cores this process may run on: the CPU affinity set, capped by a
    cgroup (v2) CPU quota when one is set."""
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    try:
        quota, period = open("/sys/fs/cgroup/cpu.max").read().split()[:2]
        if quota != "max":
            n = min(n, max(1, int(int(quota) // int(period))))
    except (OSError, ValueError):
        pass
    return max(1, n)


def cpu_baseline_all_cores(seconds: float = 12.0, max_solves: int = 50):
    """The same single-threaded oracle run as one process per host core,
    all at once (each solves the whole workload; the realisations of a job
    are independent, so this is the host's job throughput)."""
    n = _host_cores()
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench._oracle_worker(%f, %d)))" % (str(ROOT), seconds, max_solves))
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, env=env, cwd=str(ROOT))
             for _ in range(n)]
    total, solves = 0.0, 0
    for p in procs:
        try:
            out, err = p.communicate(timeout=600)
        except subprocess.TimeoutExpired:
            p.kill()
            out, err = p.communicate()
        if p.returncode != 0:
            return {"value": None, "unit": "cells/s", "cores": n, "kind": "oracle",
                    "sample": "failed: " + (err.strip().splitlines() or [""])[-1][:200]}
        d = json.loads(out.strip().splitlines()[-1])
        total += d["cells"] / statistics.median(d["times"])     # as cpu_baseline
        solves += len(d["times"])
    return {"value": total, "unit": "cells/s", "cores": n, "kind": "oracle",
            "sample": f"{n} concurrent single-threaded processes, {solves} full solves of the "
                      f"workload in all"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import mrcm_oracle as O
    from paper_2104_04653_gb300 import workloads as W
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    prob = W.config2()
    cells = prob.cells()
    for _ in range(args.warmup):
        O.mrcm_solve(prob)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.mrcm_solve(prob)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    val = cells * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "cells/s",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "impl": "FP64 CPU oracle (numpy/scipy)"},
            "cpu_baseline": {"value": val, "unit": "cells/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full solves of the workload"},
            "e2e": {"value": val, "unit": "cells/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU arm
def _packed(tensors, torch):
    """Copies of the given FP64 CUDA tensors as views of ONE contiguous
    device buffer (so that a host<->device transfer of all of them is one
    copy); returns (buffer, views)."""
    n = sum(t.numel() for t in tensors)
    buf = torch.empty(n, dtype=torch.float64, device="cuda")
    views, o = [], 0
    for t in tensors:
        v = buf[o:o + t.numel()].view(t.shape)
        v.copy_(t)
        views.append(v)
        o += t.numel()
    return buf, views


def _capture(solver, K, L, Q, out, torch):
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        solver.L.mrcm_set_stream(solver.ctx, side.cuda_stream)
        for _ in range(2):
            solver.solve(K, L, Q, out=out)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        solver.L.mrcm_set_stream(solver.ctx, torch.cuda.current_stream().cuda_stream)
        solver.solve(K, L, Q, out=out)
    solver.L.mrcm_set_stream(solver.ctx, torch.cuda.current_stream().cuda_stream)
    return g


def _time_graph(g, steps, flush, torch):
    st = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for a, b in ev:
        flush.zero_()
        a.record(st)
        g.replay()
        b.record(st)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) * 1e-3 for a, b in ev]


def _time_calls(solver, K, L, Q, out, steps, flush, torch):
    """Per-ABI-call device time (eager launches, L2 flushed before each step)."""
    st = torch.cuda.current_stream()
    names = ["factor_local", "build_basis", "solve_interface", "reconstruct"]
    recs = []
    for _ in range(steps):
        flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        e[0].record(st)
        solver.mrcm_factor_local(K, L)
        e[1].record(st)
        solver.mrcm_build_basis(Q)
        e[2].record(st)
        solver.mrcm_solve_interface()
        e[3].record(st)
        solver.mrcm_reconstruct(*out)
        e[4].record(st)
        recs.append(e)
    torch.cuda.synchronize()
    res = {}
    for i, n in enumerate(names):
        res[n] = statistics.median(r[i].elapsed_time(r[i + 1]) * 1e-3 for r in recs)
    res["_steps"] = [r[0].elapsed_time(r[4]) * 1e-3 for r in recs]
    return res


def _e2e(inbuf, outbuf, graph, steps, warmup, flush, torch):
    """Mean time of a step that copies the inputs in from pinned host memory,
    replays the solve and copies p, ux, uy back (one copy each way: the
    buffers are contiguous), all inside CUDA events; warm-up steps first."""
    hin = inbuf.cpu().pin_memory()
    hout = torch.empty(outbuf.shape, dtype=outbuf.dtype).pin_memory()
    st = torch.cuda.current_stream()

    def step():
        inbuf.copy_(hin, non_blocking=True)
        graph.replay()
        hout.copy_(outbuf, non_blocking=True)

    for _ in range(warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    evs = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        step()
        b.record(st)
        evs.append((a, b))
    torch.cuda.synchronize()
    t = statistics.mean(a.elapsed_time(b) * 1e-3 for a, b in evs)
    return t, hin.numel() * hin.element_size(), hout.numel() * hout.element_size()


def _survey_roofline(prob, solver, step_s, peaks, src, clocks):
    """The whole step against the scope table's own counts (perfmodel.
    survey_work): 40 B per cell of HBM traffic over the step time against the
    HBM peak, and the banded factor + solve flops over the step time against
    the FP32 SIMT peak."""
    from paper_2104_04653_gb300 import perfmodel
    w = perfmodel.survey_work(prob, solver)
    sm_mhz = (clocks or {}).get("sm_mhz") or 1900.0
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    simt = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    gbs = w["path_bytes"] / step_s / 1e9
    tfl = w["flops"] / step_s / 1e12
    return {"path_hbm": {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "bytes_per_step": w["path_bytes"], "peak_source": f"{src} HBM copy"},
            "path_flops": {"achieved": tfl, "peak": simt, "unit": "TFLOP/s", "frac": tfl / simt,
                           "flops_per_step": w["flops"], "local_sweeps": w["sweeps"],
                           "peak_source": f"FP32 SIMT at the sampled {sm_mhz:.0f} MHz"},
            "per_unit": w["per_unit"]}


def _batch_sample_problems():
    """The batched workload's CPU sample: the lower-left 384 x 384 window of
    realisation 0 (16 x 16-cell subdomains) and of realisation 16 (32 x 32)."""
    import numpy as np
    from paper_2104_04653_gb300 import workloads as W
    out = []
    for r in (0, 16):
        K, s, m = W.config3_realisation(r, 32, 1024, 3.0)
        t, v = W.bc_left_right(1024, 1024)
        one = W.Problem(nx=1024, ny=1024, ly=1.0, sub_size=[s], K=K[None], lam=np.ones((1,) + K.shape),
                        q=np.zeros((1,) + K.shape), bc_type=t, bc_val=v,
                        iface_nU=[(m // 2).astype(np.int32)], iface_nP=[(m // 2).astype(np.int32)],
                        name=f"lognormal-1024x1024 r={r}")
        out.append(W.window(one, 0, 384))
    return out


def _oracle_batch_worker(reps: int):
    """Times the oracle as it stands on the batched workload's sample."""
    from oracle import mrcm_oracle as O
    probs = _batch_sample_problems()
    cells, secs = 0, 0.0
    for _ in range(reps):
        for p in probs:
            t0 = time.perf_counter()
            O.mrcm_solve(p)
            secs += time.perf_counter() - t0
            cells += p.cells()
    return {"cells": cells, "secs": secs}


def cpu_baseline_batch(all_cores: bool):
    n = _host_cores() if all_cores else 1
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench._oracle_batch_worker(1)))" % str(ROOT))
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, env=env, cwd=str(ROOT))
             for _ in range(n)]
    total = 0.0
    for p in procs:
        try:
            out, err = p.communicate(timeout=900)
        except subprocess.TimeoutExpired:
            p.kill()
            out, err = p.communicate()
        if p.returncode != 0:
            return {"value": None, "unit": "cells/s", "cores": n, "kind": "oracle",
                    "sample": "failed: " + (err.strip().splitlines() or [""])[-1][:200]}
        d = json.loads(out.strip().splitlines()[-1])
        total += d["cells"] / d["secs"]
    what = ("one process" if n == 1 else f"{n} concurrent single-threaded processes, each")
    return {"value": total, "unit": "cells/s", "cores": n, "kind": "oracle",
            "sample": f"{what} solving the 384x384 lower-left windows of realisations 0 "
                      f"(16x16 subdomains) and 16 (32x32) of the batch, numpy/scipy FP64, "
                      f"1 thread each"}


def run_batched(args, flush, torch, ws, rank, local):
    """The batched workload: mixed path timed as CUDA-graph replays, FP64
    path by per-call events (its graph replay matches the eager sum within
    0.1%), e2e through pinned host buffers (3 warm-up steps, then as many
    timed steps as the graph timing), accuracy on sampled outputs."""
    import numpy as np
    from paper_2104_04653_gb300 import mrcm, workloads as W
    from oracle import sampled as S
    t_gen = time.time()
    prob = W.config3(workers=min(16, _host_cores()))
    gen_s = time.time() - t_gen
    cells = prob.cells()
    inbuf, (K, L, Q) = _packed(mrcm.device_inputs(prob), torch)
    opts = mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR, iface_tol=1e-11)
    s = mrcm.Mrcm(prob, opts)
    widths = s.mrcm_autotune(K, L, Q, reps=2)
    outbuf, out = _packed(s.alloc_outputs(), torch)
    s.solve(K, L, Q, out=out)
    info = s.mrcm_get_info(check=False)
    g = _capture(s, K, L, Q, out, torch)
    for _ in range(3):
        flush.zero_()
        g.replay()
    torch.cuda.synchronize()
    nb = max(3, args.steps // 40)
    clock = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clock.start()
    time.sleep(0.3)
    t_mixed = _time_graph(g, nb, flush, torch)
    torch.cuda.synchronize()
    clocks = clock.stop()
    if ws > 1:
        torch.distributed.barrier()
    tot = _max_over_ranks(sum(t_mixed), ws, "cuda")
    value = _job_value(cells, nb, ws, tot)
    ms = 1e3 * tot / nb
    calls = _time_calls(s, K, L, Q, out, 3, flush, torch)
    calls.pop("_steps")
    launches = s.launch_count()
    e2e_t, h2d, d2h = _e2e(inbuf, outbuf, g, nb, 3, flush, torch)
    e2e_t = _max_over_ranks(e2e_t, ws, "cuda")
    # accuracy on sampled outputs (oracle building blocks, FP64)
    p, ux, uy = (t_.cpu().numpy() for t_ in out)
    x = s.interface_solution().cpu().numpy()
    rng = np.random.default_rng(2024)
    wp, wd = S.sampled_checks(prob, p, x, rng, n_sub=6, n_if=6, reals=[0, 16])
    bal = S.global_balance(prob, ux, uy)
    ok = (wp <= SAMPLE_P_TOL and wd <= SAMPLE_DEFECT_TOL and bal <= BALANCE_TOL
          and info["flags"] == 0 and info["iface_resid"] <= 1e-10)
    peaks, src = measured_peaks()
    dom = max(calls, key=calls.get)
    roof = roofline_entry(dom, calls[dom], prob, s, peaks, src, clocks)
    roof.pop("algorithmic", None)
    survey = _survey_roofline(prob, s, ms * 1e-3, peaks, src, clocks)
    path = s.interface_path()
    del g
    s.close()
    del out, outbuf
    torch.cuda.empty_cache()
    # FP64 path on the same inputs: one warm-up solve, then two timed steps
    s64 = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP64, iface_tol=1e-11))
    s64.mrcm_set_basis_width(widths[0], min(widths[1], 8))   # FP64: s = 32 width 4 or 8
    out64 = s64.alloc_outputs()
    s64.solve(K, L, Q, out=out64)
    info64 = s64.mrcm_get_info(check=False)
    c64 = _time_calls(s64, K, L, Q, out64, 2, flush, torch)
    fp64_ms = 1e3 * _max_over_ranks(statistics.mean(c64.pop("_steps")), ws, "cuda")
    p64 = out64[0].cpu().numpy()
    x64 = s64.interface_solution().cpu().numpy()
    wp64, wd64 = S.sampled_checks(prob, p64, x64, np.random.default_rng(2024), n_sub=6, n_if=6,
                                  reals=[0, 16])
    s64.close()
    del out64, K, L, Q, inbuf
    torch.cuda.empty_cache()
    res = {
        "workload": BATCH_WORKLOAD, "cells_per_step": cells, "value": value if ok else None,
        "unit": "cells/s", "steps": nb, "warmup": 3, "ms_per_step": ms,
        "interface_path": path, "interface_unknowns": int(sum(
            int(np.sum(prob.iface_nU[r] + prob.iface_nP[r])) for r in range(prob.n_real))),
        "basis_width_autotuned": {"s16": widths[0], "s32": widths[1]},
        "l2": "inputs and outputs (2.4 GB) larger than L2; flushed (256 MB write) as well",
        "fp64_path": {"value": cells * ws / (fp64_ms * 1e-3), "ms_per_step": fp64_ms,
                      "calls_ms": {k: v * 1e3 for k, v in c64.items()},
                      "timing": "per-call CUDA events, eager launches, 2 steps after 1 warm-up",
                      "accuracy": {"sampled_p": wp64, "sampled_defect": wd64}},
        "speedup_vs_fp64": fp64_ms / ms,
        "speedup_per_call": {k: c64[k] / calls[k] for k in calls},
        "calls_ms": {k: v * 1e3 for k, v in calls.items()},
        "accuracy": {"valid": bool(ok), "sampled_p": wp, "sampled_defect": wd,
                     "global_balance": bal, "iface_resid": info["iface_resid"],
                     "local_resid_max": info["local_resid_max"], "flags": info["flags"],
                     "fp64_iface_resid": info64["iface_resid"],
                     "how": "realisations 0 and 16: 6 subdomains re-solved by the oracle from the "
                            "GPU's interface solution, 6 interfaces' continuity defects; global "
                            "balance over all 32"},
        "roofline": roof, "survey_roofline": survey,
        "e2e": {"value": cells * ws / e2e_t, "unit": "cells/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches * nb,
        "clocks": clocks, "generation_s": gen_s,
    }
    if ws == 1 and rank == 0 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline_batch(False)
        res["cpu_baseline"]["all_cores"] = cpu_baseline_batch(True)
    return res


def run_gpu(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2104_04653_gb300 import build, mrcm, workloads as W
    build.build()
    prob = W.config2()
    cells = prob.cells()
    # K, lambda, q (and below each solver's p, ux, uy) as views of one
    # contiguous buffer, so the end-to-end run moves each direction in one copy
    inbuf, (K, L, Q) = _packed(mrcm.device_inputs(prob), torch)
    # fp32_ir: the headline (one-launch cluster interface kernel); fp64: the
    # plain FP64 path (its slab tiles do not fit one cluster, so it runs the
    # multi-kernel reduction); fp32_ir_slab: the mixed path forced onto that
    # same multi-kernel reduction, so that fp64 / fp32_ir_slab compares
    # precision alone
    opts = {"fp32_ir": (mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR), False),
            "fp64": (mrcm.SolverOptions(prec=mrcm.PREC_FP64), False),
            "fp32_ir_slab": (mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR), True)}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    results = {}
    widths = {}
    for name, (o, no_cluster) in opts.items():
        prev = os.environ.pop("MRCM_NO_CLUSTER", None)
        if no_cluster:
            os.environ["MRCM_NO_CLUSTER"] = "1"
        s = mrcm.Mrcm(prob, o)
        os.environ.pop("MRCM_NO_CLUSTER", None)
        if prev is not None:
            os.environ["MRCM_NO_CLUSTER"] = prev
        if args.basis_width:
            w16, w32 = (int(v) for v in args.basis_width.split(","))
            s.mrcm_set_basis_width(w16, w32)
            widths[name] = (w16, w32)
        else:
            widths[name] = s.mrcm_autotune(K, L, Q, reps=5)
        outbuf, out = _packed(s.alloc_outputs(), torch)
        s.solve(K, L, Q, out=out)
        info = s.mrcm_get_info()
        g = _capture(s, K, L, Q, out, torch)
        for _ in range(args.warmup):
            flush.zero_()
            g.replay()
        torch.cuda.synchronize()
        results[name] = dict(solver=s, graph=g, out=out, outbuf=outbuf, info=info,
                             launches=s.launch_count(), path=s.interface_path())
    # accuracy against the oracle (computed once on the host)
    acc = {}
    acc_ok = True
    if rank == 0 and not args.no_accuracy:
        from oracle import mrcm_oracle as O
        ref = O.mrcm_solve(prob)
        for name, r in results.items():
            p, ux, uy = (t.cpu().numpy() for t in r["out"])
            ep, eu = O.errors(dict(p=p, ux=ux, uy=uy), ref)
            acc[name] = {"p": ep, "u": eu}
            acc_ok = acc_ok and ep <= ACC_TOL and eu <= ACC_TOL
    # timed region: mixed path (the headline), clocks sampled meanwhile
    clock = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clock.start()
    time.sleep(0.3)
    t_mixed = _time_graph(results["fp32_ir"]["graph"], args.steps, flush, torch)
    torch.cuda.synchronize()
    clocks = clock.stop()
    t_fp64 = _time_graph(results["fp64"]["graph"], max(args.steps // 4, 3), flush, torch)
    t_slab = _time_graph(results["fp32_ir_slab"]["graph"], max(args.steps // 4, 3), flush, torch)
    if ws > 1:
        torch.distributed.barrier()
    tot = _max_over_ranks(sum(t_mixed), ws, "cuda")
    value = _job_value(cells, args.steps, ws, tot)
    ms = 1e3 * tot / args.steps
    fp64_ms = 1e3 * _max_over_ranks(statistics.mean(t_fp64), ws, "cuda")
    slab_ms = 1e3 * _max_over_ranks(statistics.mean(t_slab), ws, "cuda")
    # per-call breakdown (eager) and the dominant kernel's roofline
    s = results["fp32_ir"]["solver"]
    calls = _time_calls(s, K, L, Q, results["fp32_ir"]["out"], 30, flush, torch)
    calls64 = _time_calls(results["fp64"]["solver"], K, L, Q, results["fp64"]["out"], 10, flush,
                          torch)
    calls_slab = _time_calls(results["fp32_ir_slab"]["solver"], K, L, Q,
                             results["fp32_ir_slab"]["out"], 10, flush, torch)
    for c in (calls, calls64, calls_slab):
        c.pop("_steps")
    e2e_t, h2d, d2h = _e2e(inbuf, results["fp32_ir"]["outbuf"], results["fp32_ir"]["graph"],
                           max(args.steps // 4, 3), args.warmup, flush, torch)
    e2e_t = _max_over_ranks(e2e_t, ws, "cuda")
    peaks, src = measured_peaks()
    dom = max(calls, key=calls.get)
    roof = roofline_entry(dom, calls[dom], prob, s, peaks, src, clocks)
    all_roofs = {c: roofline_entry(c, calls[c], prob, s, peaks, src, clocks) for c in calls}
    for v in all_roofs.values():
        v.pop("algorithmic", None)
    survey = _survey_roofline(prob, s, ms * 1e-3, peaks, src, clocks)
    launches = results["fp32_ir"]["launches"]
    infos = {k: r["info"] for k, r in results.items()}
    paths = {k: r["path"] for k, r in results.items()}
    for r in results.values():
        del r["graph"]
        r["solver"].close()
    del results, inbuf, K, L, Q
    torch.cuda.empty_cache()
    batched = None
    if not args.no_batch:
        batched = run_batched(args, flush, torch, ws, rank, local)
    if rank != 0:
        return
    valid = acc_ok and not args.no_accuracy
    line = {
        "metric": METRIC, "value": value if valid else None, "unit": "cells/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64-refine", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "FP32 factors/solves, FP64 refinement",
                   "parallelism": f"replicas x{ws}", "l2": "flushed (256 MB write) before each step",
                   "graph": "CUDA graph replay",
                   "basis_width": {k: {"s16": v[0], "s32": v[1]} for k, v in widths.items()},
                   "basis_width_autotuned": not args.basis_width},
        "fp64_path": {"value": cells * ws / (fp64_ms * 1e-3), "ms_per_step": fp64_ms,
                      "interface_path": paths["fp64"],
                      "calls_ms": {k: v * 1e3 for k, v in calls64.items()}},
        "speedup_vs_fp64": fp64_ms / ms,
        "speedup_per_call": {k: calls64[k] / calls[k] for k in calls},
        "mixed_same_kernels_as_fp64": {
            "ms_per_step": slab_ms, "interface_path": paths["fp32_ir_slab"],
            "calls_ms": {k: v * 1e3 for k, v in calls_slab.items()},
            "speedup_vs_fp64": fp64_ms / slab_ms,
            "note": "the mixed path on the FP64 path's multi-kernel interface reduction: "
                    "the speedup from precision alone"},
        "interface_path": paths["fp32_ir"],
        "rel_err_vs_oracle": acc,
        "accuracy": {"valid": bool(valid), "tol": ACC_TOL,
                     "checked": not args.no_accuracy},
        "calls_ms": {k: v * 1e3 for k, v in calls.items()},
        "solver_info": infos,
        "roofline": roof,
        "calls_roofline": all_roofs,
        "survey_roofline": survey,
        "e2e": {"value": cells * ws / e2e_t, "unit": "cells/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
    }
    if batched is not None:
        line["batched"] = batched
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
        line["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores()
    print(json.dumps(line), flush=True)
    if not valid:
        sys.exit(1 if not args.no_accuracy else 0)


# DRAM traffic per launch from the committed ncu capture (profiles/
# k_iface_cluster_channels-256x64.md), valid only while the kernel sources are
# the ones that were profiled.
TRAFFIC = {"k_iface_cluster": {"bytes": 1281792.0, "sha": "209df39d077bf46b",
                               "sources": ["csrc/iface_cluster.cu", "csrc/iface_common.cuh"]},
           "k_basis": {"bytes": 1145600.0, "sha": "59bb576505df3741", "sources": ["csrc/local.cu"]},
           "k_factor": {"bytes": 325120.0, "sha": "59bb576505df3741", "sources": ["csrc/local.cu"]}}


def _traffic(kernel):
    import hashlib
    e = TRAFFIC.get(kernel)
    if not e or not e["sha"]:
        return None
    h = hashlib.sha256()
    for rel in e["sources"]:
        h.update((ROOT / "paper_2104_04653_gb300" / rel).read_bytes())
    return e["bytes"] if h.hexdigest()[:16] == e["sha"] else None


def roofline_entry(call, seconds, prob, solver, peaks, src, clocks):
    """Algorithmic work of the dominant call per launch, over its device
    time; the bound and the per-unit figures come from perfmodel.call_work."""
    from paper_2104_04653_gb300 import perfmodel
    w = perfmodel.call_work(call, prob, solver)
    sm_mhz = (clocks or {}).get("sm_mhz") or 1900.0
    if w["bound"] == "hbm":
        peak = float(peaks.get("hbm_gbs", 6800.0))
        ach = w["bytes"] / seconds / 1e9
        unit = "GB/s"
        note = f"{src} HBM copy bandwidth"
    elif w["bound"] == "tensor":
        # composite: the time each part of the call takes at its own unit's
        # peak.  Products (FP32-equivalent, 3 TF32 products each) at the
        # measured sustained bf16 rate x the nominal TF32/bf16 ratio
        # (1.1/2.25) / 3; inverses and solves at the FP32 SIMT rate; the FP64
        # residual terms at 1.67 FP64 FMA per clock per SM (measured on this
        # part); peak = all the call's flops / that time
        simt = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        bf16 = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0)))
        tc = bf16 * (1.1 / 2.25) / 3.0
        f64 = 152 * 1.67 * 2 * sm_mhz * 1e6 / 1e12
        t_min = (w["flops_products"] / tc + (w["flops_inverse"] + w["flops_solve"]) / simt +
                 w["flops_fp64"] / f64) / 1e12
        peak = w["flops"] / t_min / 1e12
        ach = w["flops"] / seconds / 1e12
        unit = "TFLOP/s"
        note = (f"composite at the sampled {sm_mhz:.0f} MHz: products at {tc:.0f} TFLOP/s "
                f"({src} sustained bf16 {bf16:.0f} x 1.1/2.25 / 3 TF32 products), inverses and "
                f"solves at FP32 SIMT {simt:.1f}, FP64 residual terms at {f64:.2f}")
    else:
        # FP32 SIMT issue rate: 152 SMs x 128 FP32 lanes x 2 flop x clock
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        ach = w["flops"] / seconds / 1e12
        unit = "TFLOP/s"
        note = f"FP32 SIMT peak at the sampled {sm_mhz:.0f} MHz (152 SMs x 128 lanes x 2)"
    return {"kernel": w["kernel"], "bound": w["bound"], "achieved": ach, "peak": peak,
            "unit": unit, "frac": ach / peak, "traffic": _traffic(w["kernel"]), "peak_source": note,
            "call_ms": seconds * 1e3, "algorithmic": w}


# --------------------------------------------------------- workload suite
def _global_balance(prob, p, ux, uy):
    """max over realisations |sum q h^2 - boundary outflow| / sum |q h^2|,
    or over the boundary flux when there are no sources."""
    h = prob.h
    worst = 0.0
    for r in range(prob.n_real):
        src = float(prob.q[r].sum()) * h * h
        out = (ux[r][:, -1].sum() - ux[r][:, 0].sum() + uy[r][-1, :].sum() - uy[r][0, :].sum()) * h
        scale = max(abs(src), float(np.abs(ux[r][:, 0]).sum() * h), 1e-300)
        worst = max(worst, abs(src - out) / scale)
    return worst


def _suite_resolve10(precs, flush, torch, np, mrcm, W):
    """The re-factor workload as a time-stepping loop: ten solves k = 1..10
    of the 512x512 Buckley-Leverett front case on ONE context, lambda_k
    copied into the context's input buffer before each step (outside the
    timed region), every call inside CUDA events, L2 flushed before each
    step.  Per step: device time, the solver's FP64 residuals and the
    global mass balance."""
    probs = [W.config5(k, n=512) for k in range(1, 11)]
    st = torch.cuda.current_stream()
    for prec in precs:
        opts = mrcm.SolverOptions(prec=prec, iface_tol=1e-11)
        s = mrcm.Mrcm(probs[0], opts)
        K, L, Q = mrcm.device_inputs(probs[0])
        lams = [torch.from_numpy(np.ascontiguousarray(p.lam)).to("cuda") for p in probs]
        tuned = s.mrcm_autotune(K, L, Q, reps=2)
        out = s.alloc_outputs()
        for lam in lams:                       # warm-up pass over the ten steps
            L.copy_(lam)
            s.solve(K, L, Q, out=out)
        torch.cuda.synchronize()
        steps = []
        for k, lam in enumerate(lams):
            L.copy_(lam)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            s.mrcm_factor_local(K, L)
            s.mrcm_build_basis(Q)
            inf = s.mrcm_solve_interface(info=True)
            s.mrcm_reconstruct(*out)
            e1.record(st)
            torch.cuda.synchronize()
            p, ux, uy = (t.cpu().numpy() for t in out)
            steps.append({"ms": e0.elapsed_time(e1), "iface_resid": inf["iface_resid"],
                          "local_resid_max": inf["local_resid_max"], "flags": inf["flags"],
                          "global_balance": _global_balance(probs[k], p, ux, uy)})
        tot = sum(x["ms"] for x in steps) * 1e-3
        line = {"suite": "bl-front-512x512-s16-m4, steps 1..10 on one context (re-factor each)",
                "prec": "fp32_ir" if prec else "fp64", "cells": probs[0].cells(),
                "interface_solver": "gmres" if s.uses_gmres() else "direct",
                "ms_total_10_steps": tot * 1e3, "ms_per_step": [round(x["ms"], 4) for x in steps],
                "cells_per_s": 10 * probs[0].cells() / tot,
                "iface_resid_max": max(x["iface_resid"] for x in steps),
                "local_resid_max": max(x["local_resid_max"] for x in steps),
                "flags": sorted({x["flags"] for x in steps}),
                "global_balance_max": max(x["global_balance"] for x in steps),
                "basis_width_autotuned": {"s16": tuned[0], "s32": tuned[1]}}
        s.close()
        print(json.dumps(line), flush=True)
        del K, L, Q, out, lams
        torch.cuda.empty_cache()


def _suite_learned(args, flush, torch, np, mrcm, LP, W):
    """The learned preconditioner at the channel workload's scale: train on
    seeded 512x512 channel windows (seeds 5000.., 32x32-cell subdomains,
    m = 4, channel density of the 2048x2048 case), then solve the
    2048x2048 system by GMRES to 1e-8 with no preconditioner, block-Jacobi
    and the network's blocks: steps, interface time (CUDA events, L2
    flushed), the network's inference time, and the solution's error
    against the direct path."""
    ntrain = args.suite_train
    st = torch.cuda.current_stream()
    t0 = time.time()
    train_p = [W.config4(n=512, s=32, n_ch=16, seed=5000 + k) for k in range(ntrain)]
    x, t = LP.make_dataset(train_p, 4)
    net = LP.LearnedPrecond(32, 4, max_batch=1024, seed=0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    rep = LP.train(net, x, t, steps=args.suite_train_steps, batch=256, lr=1e-3)
    e1.record(st)
    torch.cuda.synchronize()
    train_s = e0.elapsed_time(e1) * 1e-3
    prep_s = time.time() - t0 - train_s
    del x, t
    prob = W.config4(n=2048, s=32, n_ch=64)
    K, L, Q = mrcm.device_inputs(prob)
    # reference interface solution: the direct path
    sd = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR, iface_tol=1e-12))
    ref = [t_.clone() for t_ in sd.solve(K, L, Q)]
    sd.close()
    xv, tv = LP.make_dataset([prob], 4)
    w = 1.0 / tv.double().var(dim=0).clamp_min(1e-8)
    val, _ = net.gradient(xv[:1024].contiguous(), tv[:1024].contiguous())
    zero = float(((tv[:1024].double() ** 2) * w).mean())
    del xv, tv
    res = {}
    for name, pc in (("none", mrcm.PRECOND_NONE), ("block_jacobi", mrcm.PRECOND_BLOCK_JACOBI),
                     ("learned", mrcm.PRECOND_USER),
                     ("neighbourhood", mrcm.PRECOND_NEIGHBOURHOOD)):
        s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR,
                                               iface_solver=mrcm.IFACE_GMRES, precond=pc,
                                               gmres_tol=1e-8, gmres_max=20000))
        out = s.alloc_outputs()
        s.mrcm_factor_local(K, L)
        s.mrcm_build_basis(Q)
        torch.cuda.synchronize()
        flush.zero_()
        a0, a1, a2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a0.record(st)
        if pc == mrcm.PRECOND_USER:
            LP.apply(s, net, K, L)
        a1.record(st)
        status = "MRCM_OK"
        try:
            s.mrcm_solve_interface()
        except mrcm.MrcmError as ex:          # no convergence within gmres_max: reported
            status = str(ex).split(":")[0]
        a2.record(st)
        inf = s.mrcm_get_info(check=False)
        s.mrcm_reconstruct(*out)
        torch.cuda.synchronize()
        errs = [float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
                for a, b in zip(out, ref)]
        nunk = s.num_interface_unknowns()
        res[name] = {"converged": bool(inf["iface_resid"] <= 1e-8),
                     "fell_back_to_block_jacobi": bool(inf["flags"] & mrcm.FLAG_PRECOND_FALLBACK),
                     "status": status, "gmres_iters": inf["gmres_iters"],
                     "iface_ms": a1.elapsed_time(a2),
                     "apply_ms": a0.elapsed_time(a1), "iface_resid": inf["iface_resid"],
                     "flags": inf["flags"], "rel_err_vs_direct": {"p": errs[0], "ux": errs[1],
                                                                  "uy": errs[2]}}
        s.close()
    line = {"suite": "learned preconditioner: channels-2048x2048-s32-m4, GMRES to 1e-8",
            "train": {"systems": ntrain, "grid": "512x512", "samples": rep.samples,
                      "adam_steps": rep.steps, "train_s": train_s, "dataset_s": prep_s,
                      "loss_first": rep.loss_first, "loss_last": rep.loss_last},
            "eval_loss": {"network": val, "zero_block_jacobi": zero, "samples": 1024},
            "interface_unknowns": nunk, "results": res}
    net.close()
    print(json.dumps(line), flush=True)


def _suite_transport(flush, torch, np, mrcm, W):
    """Sequential implicit and sequential fully implicit time stepping on the
    512 x 512 lognormal field (variance 2, 16 x 16 subdomains, m = 4, M = 5):
    from the Buckley-Leverett front of step 1, ten SI steps (mrcm_si_step:
    the five Darcy calls then the transport step) and two SFI steps
    (mrcm_sfi_step, outer tolerance 1e-4), each inside CUDA events; per step
    the Darcy and transport device times, Newton iterations and the water
    balance of the transport step."""
    from paper_2104_04653_gb300 import transport as TP
    from oracle import transport as T
    prob = W.config5(1, n=512)
    M = 5.0
    n = prob.nx
    h = prob.h
    st = torch.cuda.current_stream()
    ctx = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR, iface_tol=1e-11))
    tp = TP.Transport(n, n, 1, prob.ly, TP.TransportOptions(M=M))
    K, L, Q = mrcm.device_inputs(prob)
    s0 = torch.as_tensor(np.asarray(prob.meta["saturation"])[None], device="cuda").contiguous()
    lam = (s0 * s0 + (1 - s0) ** 2 / M).contiguous()
    p, ux, uy = ctx.alloc_outputs()
    sa, sb = s0.clone(), torch.empty_like(s0)
    dt = 0.01
    # warm-up: one SI step from s0 (not counted)
    TP.mrcm_si_step(ctx, tp, dt, K, lam.clone(), Q, s0, sb, p, ux, uy)
    tp.mrcm_transport_get_info()
    lam = (s0 * s0 + (1 - s0) ** 2 / M).contiguous()
    steps = []
    for k in range(10):
        flush.zero_()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(st)
        ctx.solve(K, lam, Q, out=(p, ux, uy))
        e1.record(st)
        tp.mrcm_transport_step(dt, ux, uy, sa, sb, lam)
        e2.record(st)
        inf = tp.mrcm_transport_get_info()
        s_old, s_new = sa.cpu().numpy()[0], sb.cpu().numpy()[0]
        uxn, uyn = ux.cpu().numpy()[0], uy.cpu().numpy()[0]
        dv = float(np.sum(s_new - s_old)) * h * h
        out = T.boundary_outflow(s_new, uxn, uyn, h, M)
        steps.append({"darcy_ms": e0.elapsed_time(e1), "transport_ms": e1.elapsed_time(e2),
                      "newton": inf["newton_iters"][0], "linear_max": inf["linear_iters_max"],
                      "water_balance_rel": abs(dv + dt * out) / max(dt * abs(out), 1e-300)})
        sa, sb = sb, sa
    tot = sum(x["darcy_ms"] + x["transport_ms"] for x in steps) * 1e-3
    # SFI steps from the state reached, at this dt and at a quarter of it;
    # an outer loop that does not reach the tolerance is reported as such
    sfi = []
    sw = torch.empty_like(sa)
    for dts in (dt, 0.25 * dt):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            outer = TP.mrcm_sfi_step(ctx, tp, dts, 1e-4, 20, K, lam, Q, sa, sb, sw, p, ux, uy)
            ok = True
        except mrcm.MrcmError as ex:
            outer, ok = 20, False
        torch.cuda.synchronize()
        inf = tp.mrcm_transport_get_info(check=False)
        sfi.append({"dt": dts, "outer": outer, "converged": ok,
                    "last_change": inf["change_max"], "wall_ms": 1e3 * (time.perf_counter() - t0)})
    line = {"suite": "si/sfi: bl-front-512x512-s16-m4, M=5, dt=0.01 (10 SI steps; SFI at dt and dt/4)",
            "cells": prob.cells(), "si_ms_per_step": 1e3 * tot / len(steps),
            "si_cells_per_s": len(steps) * prob.cells() / tot, "si_steps": steps,
            "sfi_steps": sfi}
    tp.close()
    ctx.close()
    print(json.dumps(line), flush=True)


def _suite_quadtree(flush, torch, np, mrcm, W):
    """Lognormal fields (variance 2) on 32 x 32 blocks with 30% of them split
    into 16 x 16 subdomains, m = 4, mixed precision, GMRES(64) to 1e-10:
    512 x 512 with block-Jacobi and with the shared neighbourhood
    preconditioner, 1024 x 1024 with block-Jacobi, each next to the same
    field on uniform 32 x 32 subdomains: per-call device times, GMRES steps,
    cells/s.  (The shared form wins on channel fields and loses on these
    lognormal ones: the oracle's own GMRES on the uniform 512^2 system takes
    2,359 steps with it against 357 with block-Jacobi.)"""
    cases = []
    for n in (512, 1024):
        K = np.exp(W.grf_exponential(n, n, 1.0 / n, 2.0, 0.1, np.random.default_rng(3000)))
        ref = W.random_refinement(n, n, 32, 0.3, np.random.default_rng(3001))
        qt = W.quadtree_problem(n, n, 32, K, [ref])
        uni = W.make_problem(n, n, 32, K, bc=W.bc_left_right(n, n), n_u=2, n_p=2)
        nsub = int(np.sum(1 + 3 * ref.astype(np.int64)))
        pcs = [mrcm.PRECOND_BLOCK_JACOBI] + ([mrcm.PRECOND_NEIGHBOURHOOD_SHARED] if n == 512 else [])
        for pc in pcs:
            pname = "block-Jacobi" if pc == mrcm.PRECOND_BLOCK_JACOBI else "shared neighbourhood"
            cases.append((f"{n}x{n}, quadtree 30% split, {pname}", qt, pc, nsub))
            cases.append((f"{n}x{n}, uniform 32x32, {pname}", uni, pc, (n // 32) ** 2))
    for name, prob, pc, nsub in cases:
        s = mrcm.Mrcm(prob, mrcm.SolverOptions(prec=mrcm.PREC_FP32_IR, iface_solver=mrcm.IFACE_GMRES,
                                               precond=pc, gmres_tol=1e-10, gmres_max=20000,
                                               gmres_restart=64))
        Kd, Ld, Qd = mrcm.device_inputs(prob)
        out = s.alloc_outputs()
        s.solve(Kd, Ld, Qd, out=out)
        info = s.mrcm_get_info(check=False)
        calls = _time_calls(s, Kd, Ld, Qd, out, 2, flush, torch)
        calls.pop("_steps")
        tot = sum(calls.values())
        line = {"suite": f"quadtree: lognormal {name}, m=4, GMRES(64) to 1e-10",
                "cells": prob.cells(), "subdomains": nsub,
                "interface_unknowns": s.num_interface_unknowns(), "ms_per_step": tot * 1e3,
                "cells_per_s": prob.cells() / tot,
                "calls_ms": {k: v * 1e3 for k, v in calls.items()},
                "gmres_iters": info["gmres_iters"], "iface_resid": info["iface_resid"],
                "status": info["status"]}
        s.close()
        print(json.dumps(line), flush=True)


def run_suite(args):
    """The large workloads at full size (one line each): per-call device
    times, interface solver, GMRES steps, the solver's own FP64 residuals and
    the global mass balance.  Not the headline line."""
    import torch
    from paper_2104_04653_gb300 import build, learned as LP, mrcm, workloads as W
    build.build()
    global np
    import numpy as np
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    cases = []
    if "resolve" in args.suite.split(","):
        cases.append(("bl-front-512x512-s16-m4 (step 5)", W.config5(5, n=512), {}))
    if "channels" in args.suite.split(","):
        cases.append(("channels-2048x2048-s32-m4", W.config4(n=2048, s=32, n_ch=64), {}))
    if "batch" in args.suite.split(","):
        cases.append(("lognormal-32x1024x1024-s16/32-m2..8", W.config3(), {}))
    # profiling-size cases of the same generators
    if "batch4" in args.suite.split(","):
        cases.append(("lognormal-4x1024x1024-s16/32-m2..8", W.config3(n_real=4), {}))
    if "channels1024" in args.suite.split(","):
        cases.append(("channels-1024x1024-s32-m4", W.config4(n=1024, s=32, n_ch=32), {}))
    precs = {"both": (mrcm.PREC_FP32_IR, mrcm.PREC_FP64), "fp32_ir": (mrcm.PREC_FP32_IR,),
             "fp64": (mrcm.PREC_FP64,)}[args.suite_prec]
    if "resolve10" in args.suite.split(","):
        _suite_resolve10(precs, flush, torch, np, mrcm, W)
    if "learned" in args.suite.split(","):
        _suite_learned(args, flush, torch, np, mrcm, LP, W)
    if "transport" in args.suite.split(","):
        _suite_transport(flush, torch, np, mrcm, W)
    if "quadtree" in args.suite.split(","):
        _suite_quadtree(flush, torch, np, mrcm, W)
    if "batch2" in args.suite.split(","):
        cases.append(("lognormal-2x1024x1024-s16/32-m2..8", W.config3(n_real=2), {}))
    for name, prob, extra in cases:
        for prec in precs:
            opts = mrcm.SolverOptions(prec=prec, iface_tol=1e-11, gmres_tol=1e-11, gmres_max=6000,
                                      **extra)
            s = mrcm.Mrcm(prob, opts)
            K, L, Q = mrcm.device_inputs(prob)
            if args.basis_width:
                tuned = tuple(int(v) for v in args.basis_width.split(","))
                s.mrcm_set_basis_width(*tuned)
            else:
                tuned = s.mrcm_autotune(K, L, Q, reps=2)
            out = s.alloc_outputs()
            s.solve(K, L, Q, out=out)
            info = s.mrcm_get_info(check=False)
            calls = _time_calls(s, K, L, Q, out, args.suite_steps, flush, torch)
            calls.pop("_steps")
            tot = sum(calls.values())
            g = _capture(s, K, L, Q, out, torch)          # the whole solve as one CUDA graph
            for _ in range(2):
                g.replay()
            graph_ms = statistics.median(_time_graph(g, args.suite_steps, flush, torch)) * 1e3
            del g
            p, ux, uy = (t.cpu().numpy() for t in out)
            line = {"suite": name, "prec": "fp32_ir" if prec else "fp64",
                    "cells": prob.cells(), "interface_solver": "gmres" if s.uses_gmres() else "direct",
                    "ms_per_step": tot * 1e3, "cells_per_s": prob.cells() / tot,
                    "graph_ms_per_step": graph_ms, "graph_cells_per_s": prob.cells() / (graph_ms * 1e-3),
                    "calls_ms": {k: v * 1e3 for k, v in calls.items()},
                    "gmres_iters": info["gmres_iters"], "iface_resid": info["iface_resid"],
                    "local_resid_max": info["local_resid_max"], "status": info["status"],
                    "global_balance": _global_balance(prob, p, ux, uy),
                    "interface_unknowns": s.num_interface_unknowns(),
                    "basis_width_autotuned": {"s16": tuned[0], "s32": tuned[1]}}
            s.close()
            print(json.dumps(line), flush=True)
            del K, L, Q, out
            torch.cuda.empty_cache()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="mrcm", choices=["mrcm", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the accuracy check (the line then carries no value)")
    ap.add_argument("--no-batch", action="store_true",
                    help="leave out the batched 32 x 1024^2 workload")
    ap.add_argument("--basis-width", default="",
                    help="N16,N32: basis-kernel RHS columns per CTA instead of autotuning "
                         "(profiling runs that must launch only the timed configuration)")
    ap.add_argument("--suite", default="", help="comma list of resolve,resolve10,channels,batch,"
                    "batch2,learned,transport,quadtree: the large workloads at full size instead "
                    "of the headline line")
    ap.add_argument("--suite-steps", type=int, default=3)
    ap.add_argument("--suite-train", type=int, default=500,
                    help="training systems (512x512 channel windows) for --suite learned")
    ap.add_argument("--suite-train-steps", type=int, default=2000)
    ap.add_argument("--suite-prec", default="both", choices=["both", "fp32_ir", "fp64"])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws_env = os.environ.get("WORLD_SIZE")
    if ws_env is None and args.gpus > 1:
        # one process per GPU: run this same command under torch.distributed.run
        import socket
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
               f"--nproc-per-node={args.gpus}", "--master-addr", "127.0.0.1",
               "--master-port", str(port), str(Path(__file__).resolve()), *sys.argv[1:]]
        sys.exit(subprocess.call(cmd))
    if ws_env is not None and int(ws_env) != args.gpus:
        print(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={ws_env}; launch one process per GPU "
              f"with --nproc-per-node equal to --gpus", file=sys.stderr)
        sys.exit(2)
    if args.suite:
        run_suite(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
