#!/usr/bin/env python3
"""Benchmark of the LOD diffusion-decay-source step (Eq. 1) on GB300.

Default workload: the 200^3 x 2 tumour problem in FP64 (oxygen with a
Dirichlet shell plus a secreted factor, 250 000 cells in a central sphere;
see paper_2110_13368_gb300.inputs).  One bench step is one full LOD step
(Dirichlet prologue, x, y, z sweeps, cell sources) over the whole grid.

Timing: W untimed warm-up steps, then K timed steps.  Before every timed
step a 512 MB buffer is written to flush the 135 MB L2; each step is timed
with CUDA events on the library's stream, and the per-kernel device times
come from the library's own event brackets (option 5).  value = voxel-
substrate updates per second over the K steps (max over ranks; for N > 1
each rank runs an independent replica: the single grid does not shard).

Prints one JSON line.  --impl reference times the CPU oracle (the plain FP64
reference) on the host cores instead, on the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0
DFMA_PER_CLK_PER_SM = 2       # nominal FP64 FMA lanes per clock per SM of a GB300
SM_MAX_MHZ_FALLBACK = 2070.0
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tumour_200",
                    choices=["tumour_200", "tumour_200_fp32", "plain_50"])
    ap.add_argument("--variant", type=int, default=None, help="FP64 sweep form: 0 plain, 1 rescaled")
    ap.add_argument("--one-launch", type=int, default=None, choices=[0, 1, 2],
                    help="library option 8: 0 per-axis launches, 1 automatic, 2 one launch per step")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--skip-extras", action="store_true",
                    help="timed steps only: no e2e, continuous run or CPU baseline (profiling runs)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP32 / batched / adjoint form measurements")
    ap.add_argument("--form-steps", type=int, default=10)
    ap.add_argument("--form", default=None,
                    choices=["fp32", "batched", "batched_fp32", "batched_phases", "adjoint",
                             "two_d", "nodes", "slabs"],
                    help="time one form of the step on its own (for profiling runs): "
                         "--warmup untimed and --steps timed steps, one JSON line")
    return ap.parse_args()


def make_problem(name):
    from paper_2110_13368_gb300 import inputs
    if name == "tumour_200":
        return inputs.tumour_200(steps=1000, precision=64)
    if name == "tumour_200_fp32":
        return inputs.tumour_200(steps=1000, precision=32)
    if name == "plain_50":
        return inputs.plain_50()
    raise ValueError(name)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def sm_max_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except Exception:
        return SM_MAX_MHZ_FALLBACK


def fp64_pipe_peak(n_sm, stream):
    """The FP64 FMA rate of this GPU, measured live: independent FMA chains
    on every SM (bfvm_fp64_fma_rate) for a few warp and chain counts, the
    best of them, as TFLOP/s (2 flop per FMA); beside it the nominal rate
    from the unit count (SMs x 2 FMA lanes per clock x maximum SM clock)."""
    from paper_2110_13368_gb300 import bfvm
    runs = []
    for warps in (4, 8, 16):
        for chains in (1, 2, 4):
            iters = max(1, int(1.2e10 / (n_sm * 32 * warps * 8 * chains)))
            rate, ms = bfvm.bfvm_fp64_fma_rate(warps, chains, iters, stream)
            runs.append({"warps_per_sm": warps, "chains": chains, "tflops": 2 * rate / 1e12,
                         "ms": ms})
    best = max(runs, key=lambda r: r["tflops"])
    nominal = n_sm * DFMA_PER_CLK_PER_SM * 2 * sm_max_mhz() * 1e6 / 1e12
    return {"measured_tflops": best["tflops"], "best": {k: best[k] for k in ("warps_per_sm", "chains")},
            "nominal_tflops": nominal, "sms": n_sm,
            "nominal_source": f"{n_sm} SMs x {DFMA_PER_CLK_PER_SM} FMA/clk x 2 flop x "
                              f"{sm_max_mhz():.0f} MHz",
            "runs": runs}


def sweep_traffic(workload):
    """DRAM bytes per sweep launch from the committed ncu summary, if it was
    taken on the current sweep source; else None."""
    h = hashlib.sha256()
    for f in ("sweeps.cu", "sweep_persistent.cuh", "sweep_pair.cuh", "sweep_step.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2110_13368_gb300", "csrc", f), "rb").read())
    digest = h.hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.txt")  # e.g. tumour_200_fp64
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#") or ":" not in line:
            continue
        k, v = line.split(":", 1)
        vals[k.strip()] = v.strip()
    if vals.get("sweeps_sha256_16") != digest:
        return None
    out = {}
    for k in ("x", "y", "z", "sources", "xyz"):
        if k in vals:
            out[k] = float(vals[k])
    return out


class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is None:
            return
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def host_link_rates(host_in, host_out, stream, reps=3):
    """Best-of-reps GB/s of pinned host -> device and device -> host copies of
    host_in's size on `stream` (CUDA events)."""
    import torch
    dev_buf = torch.empty(host_in.shape, dtype=host_in.dtype, device="cuda")
    nbytes = host_in.numel() * host_in.element_size()
    best = [0.0, 0.0]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for _ in range(reps):
            for k, (dst, src) in enumerate(((dev_buf, host_in), (host_out, dev_buf))):
                torch.cuda.synchronize()
                e0.record(stream)
                dst.copy_(src, non_blocking=True)
                e1.record(stream)
                torch.cuda.synchronize()
                best[k] = max(best[k], nbytes / (e0.elapsed_time(e1) / 1e3) / 1e9)
    del dev_buf
    return best[0], best[1]


def max_over_ranks(value, world, device=None):
    """The job's time from each rank's own: the maximum over the ranks of
    the initialised process group (the value itself on one rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units every rank processed over the job's
    time (each rank runs its own replica of the workload)."""
    return units_per_rank * world / seconds


def cpu_baseline(p, seconds):
    """The oracle as it stands, on this host's cores, on a bounded sample of
    the workload: whole steps of the full grid until `seconds` have passed."""
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    rho = p.rho0
    steps = 0
    t0 = time.perf_counter()
    while True:
        rho = oracle.run(p, rho0=rho, n_steps=1, n_threads=threads)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds or steps >= 50:
            break
    ups = p.updates_per_step * steps / el
    # and on one core: whole steps until a fifth of the budget has passed
    rho = p.rho0
    steps1 = 0
    t0 = time.perf_counter()
    while True:
        rho = oracle.run(p, rho0=rho, n_steps=1, n_threads=1)
        steps1 += 1
        el1 = time.perf_counter() - t0
        if el1 >= seconds / 5 or steps1 >= 10:
            break
    return {"value": ups, "unit": "voxel-substrate updates/s", "cores": threads,
            "kind": "oracle",
            "sample": f"{steps} full step(s) of the {p.nx}x{p.ny}x{p.nz}x{p.n_sub} workload "
                      f"from its initial field, {el:.1f} s, {threads} OpenMP threads",
            "single_core": {"value": p.updates_per_step * steps1 / el1, "cores": 1,
                            "sample": f"{steps1} full step(s), {el1:.1f} s, 1 thread"}}


def accuracy(got, ref):
    """Per substrate: max|got - ref| / max|ref| and ||got - ref||_2 / ||ref||_2."""
    import numpy as np
    mx, l2 = [], []
    for s in range(ref.shape[0]):
        d = got[s] - ref[s]
        mx.append(float(np.abs(d).max() / max(np.abs(ref[s]).max(), 1e-300)))
        l2.append(float(np.linalg.norm(d) / max(np.linalg.norm(ref[s]), 1e-300)))
    return {"max_rel_err_per_substrate": mx, "l2_rel_err_per_substrate": l2}


def timed_steps(step_fn, k, stream, flush):
    """Sum of CUDA-event times of k calls of step_fn, L2 flushed before each."""
    import torch
    st = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
    torch.cuda.synchronize()
    for i in range(k):
        flush.fill_(float(i))
        st[i].record(stream)
        step_fn()
        en[i].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in zip(st, en))


def measure_forms(args, plain_ups, dev, stream, flush):
    """The FP32, batched and adjoint forms against the plain FP64 form."""
    import numpy as np
    import torch
    from paper_2110_13368_gb300 import bfvm, inputs
    K = args.form_steps
    out = {}
    # FP32 form of the tumour workload; its error against the FP64 GPU path
    p64 = inputs.tumour_200(steps=K)
    s32 = bfvm.Sim.from_problem(p64, precision=32)
    s32.step(3)
    s32.set_density(torch.as_tensor(p64.rho0, dtype=torch.float32, device=dev))
    ms = timed_steps(lambda: s32.step(1), K, stream, flush)
    ups32 = p64.updates_per_step * K / (ms / 1e3)
    s64 = bfvm.Sim.from_problem(p64)
    s64.step(K)
    a = s32.get_density().double()
    b = s64.get_density()
    err = [float((a[s] - b[s]).abs().max() / b[s].abs().max()) for s in range(p64.n_sub)]
    out["fp32"] = {"value": ups32, "speedup_vs_fp64": ups32 / plain_ups, "steps": K,
                   "max_rel_err_vs_fp64_gpu_per_substrate": err,
                   "accuracy_gate": "<= 1e-5 vs the FP64 oracle (parity tests)"}
    s32.close()
    s64.close()
    # the FP32 form of the 50^3 workload over its 100 steps, against the FP64
    # GPU path here and against the FP64 oracle in the cpu_baseline leg
    p50 = inputs.plain_50()
    fields = {}
    for prec in (32, 64):
        sm = bfvm.Sim.from_problem(p50, precision=prec)
        sm.step(p50.steps)
        fields[prec] = sm.get_density().double().cpu().numpy()
        sm.close()
    out["fp32"]["plain_50_100_steps"] = {
        "vs_fp64_gpu": accuracy(fields[32], fields[64])}
    out["_plain_50_fp32_field"] = fields[32]
    # batched: 256 uneven members, one launch per phase, against the same
    # members stepped one context at a time
    for prec in (64, 32):
        probs = inputs.batch_256(seed=0, precision=prec)
        sims = [bfvm.Sim.from_problem(q) for q in probs]
        batch = bfvm.Batch(sims)
        n_upd = sum(q.updates_per_step for q in probs)
        batch.step(3)
        msb = timed_steps(lambda: batch.step(1), K, stream, flush)
        info = batch.info()
        batch.close()
        for q, sm in zip(probs, sims):
            sm.set_density(torch.as_tensor(q.rho0, dtype=sm.dtype, device=dev))

        def one_by_one():
            for sm in sims:
                sm.step(1)
        one_by_one()
        mss = timed_steps(one_by_one, max(2, K // 2), stream, flush) * K / max(2, K // 2)
        for sm in sims:
            sm.close()
        out[f"batched_fp{prec}"] = {
            "value": n_upd * K / (msb / 1e3), "members": len(probs),
            "updates_per_step": n_upd, "launches_per_step": info["launches"] // max(3 + K, 1),
            "one_by_one_value": n_upd * K / (mss / 1e3),
            "speedup_vs_one_by_one": mss / msb,
            "speedup_vs_plain_fp64_tumour": (n_upd * K / (msb / 1e3)) / plain_ups,
            "steps": K}
    # 2-D variant: a 1000 x 1000 x 1 x 2 grid, oxygen Dirichlet + a
    # zero-flux factor, 20k cells (2000 lines of 1000 voxels per axis: the
    # split line solve, 16-voxel segments joined through their end values)
    p2 = inputs.make_problem(1000, 1000, 1, n_sub=2, D=[1e5, 1e3], lam=[0.1, 0.01],
                             bc_kind=[1, 0], bc_value=[38.0, 0.0], field_mode="zero",
                             n_cells=20_000, U=[10.0, 0.0], S=[0.0, 10.0],
                             rho_star=[1.0, 1.0], steps=K, seed=0, dims=2)
    s2 = bfvm.Sim.from_problem(p2)
    s2.step(3)
    ms2 = timed_steps(lambda: s2.step(1), K, stream, flush)
    s2.close()
    ups2 = p2.updates_per_step * K / (ms2 / 1e3)
    out["two_d"] = {"value": ups2, "grid": [p2.nx, p2.ny, 1], "n_sub": 2, "steps": K,
                    "form": "plain Thomas, x and y sweeps, split line solve", "ratio_vs_plain_fp64_3d": ups2 / plain_ups,
                    "hbm_frac_32B_per_update": ups2 * 4 * 8 / 1e9 / peaks()[0]}
    # Dirichlet nodes: the 200^3 x 2 workload with 40 vessel columns of
    # oxygen nodes (FP64: a node-fill launch plus the one-launch step)
    pt = inputs.tumour_200(steps=K)
    rng = np.random.default_rng(5)
    vox, sub, val = [], [], []
    for _ in range(40):
        x, y = rng.integers(10, 190, size=2)
        v, sb, vl = inputs.vessel_nodes(pt.nx, pt.ny, pt.nz, substrate=0, value=38.0, x=int(x), y=int(y))
        vox.append(v); sub.append(sb); val.append(vl)
    pn = pt.with_(nodes=(np.concatenate(vox), np.concatenate(sub), np.concatenate(val)))
    sn = bfvm.Sim.from_problem(pn)
    sn.step(3)
    msn = timed_steps(lambda: sn.step(1), K, stream, flush)
    sn.close()
    upsn = pn.updates_per_step * K / (msn / 1e3)
    out["dirichlet_nodes"] = {"value": upsn, "nodes": int(len(pn.nodes[0])), "steps": K,
                              "ratio_vs_plain_fp64_no_nodes": upsn / plain_ups}
    # moving cells: re-binning the 250k tumour cells on the device
    # (bfvm_update_cells) against bfvm_set_cells, and a run that moves the
    # cells every 10 steps
    sc_ = bfvm.Sim.from_problem(pt)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    arrs = [t(pt.pos), t(pt.vol), t(pt.S), t(pt.U), t(pt.rho_star)]
    moved = [t(np.clip(pt.pos + rng.normal(0, 5.0, pt.pos.shape), 0, 200 * pt.dx))] + arrs[1:]
    sc_.update_cells(*moved)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(5):
        sc_.update_cells(*(moved if i % 2 == 0 else arrs))
    e1.record(stream)
    torch.cuda.synchronize()
    upd_ms = e0.elapsed_time(e1) / 5
    t0 = time.perf_counter()
    for i in range(3):
        sc_.set_cells(*(moved if i % 2 == 0 else arrs))
    torch.cuda.synchronize()
    set_ms = (time.perf_counter() - t0) * 1e3 / 3
    sc_.set_cells(*arrs)
    sc_.step(10)
    torch.cuda.synchronize()
    n_cad = 10
    e0.record(stream)
    for i in range(n_cad):
        sc_.update_cells(*(moved if i % 2 == 0 else arrs))
        sc_.step(10)
    e1.record(stream)
    torch.cuda.synchronize()
    cad_ms = e0.elapsed_time(e1)
    sc_.close()
    out["moving_cells"] = {"cells": pt.n_cells, "update_cells_ms": upd_ms,
                           "set_cells_ms_host_timed": set_ms,
                           "cadence_value": pt.updates_per_step * 10 * n_cad / (cad_ms / 1e3),
                           "cadence": "cells re-binned on the device every 10 steps, 100 steps"}
    # adjoint: forward with checkpoints every 20 steps, then the backward
    p, q = inputs.adjoint_problem()
    target = None
    sa = bfvm.Sim.from_problem(q)
    sa.step(q.steps)
    target = sa.get_density()
    sa.close()
    sim = bfvm.Sim.from_problem(p)
    sim.step(p.steps)   # warm the graphs and kernels
    # and the backward's kernels (their modules load at first launch)
    sim.set_density(torch.as_tensor(p.rho0, device=dev))
    sim.record(1)
    sim.step(2)
    sim.backward(torch.zeros_like(sim.get_density()))
    torch.cuda.synchronize()
    sim.close()
    sim = bfvm.Sim.from_problem(p)
    sim.step(p.steps)
    sim.set_density(torch.as_tensor(p.rho0, device=dev))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(p.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_plain_ms = e0.elapsed_time(e1)
    sim.set_density(torch.as_tensor(p.rho0, device=dev))
    sim.record(20)
    t0 = time.perf_counter()
    sim.step(p.steps)
    fin = sim.get_density()
    torch.cuda.synchronize()
    fwd_rec_s = time.perf_counter() - t0
    g = 2.0 * (fin - target)
    t0 = time.perf_counter()
    grads = sim.backward(g)
    torch.cuda.synchronize()
    bwd_s = time.perf_counter() - t0
    sim.close()
    out["adjoint"] = {"workload": p.name, "steps": p.steps, "checkpoint_every": 20,
                      "forward_plain_ms": fwd_plain_ms, "forward_recorded_ms": fwd_rec_s * 1e3,
                      "backward_ms": bwd_s * 1e3,
                      "fwd_plus_bwd_over_2x_fwd": (fwd_rec_s + bwd_s) / (2 * fwd_plain_ms / 1e3),
                      "dD": float(grads["dD"][0]), "dlambda": float(grads["dlambda"][0]),
                      "accuracy_gate": "1e-10 vs the CPU adjoint; 1e-4 vs central differences (tests)"}
    return out


def metric_name():
    return "voxel-substrate LOD updates/s at 200^3x2 FP64 + % HBM roofline"


def run_reference(args):
    world, rank, local = dist_setup(args)
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    p = make_problem(args.workload)
    threads = oracle.max_threads()
    rho = p.rho0
    for _ in range(args.warmup):
        rho = oracle.run(p, rho0=rho, n_steps=1, n_threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rho = oracle.run(p, rho0=rho, n_steps=1, n_threads=threads)
    el = time.perf_counter() - t0
    ups = p.updates_per_step * args.steps / el
    line = {"metric": metric_name(), "value": ups, "unit": "voxel-substrate updates/s",
            "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": p.name, "grid": [p.nx, p.ny, p.nz], "n_sub": p.n_sub,
                       "cells": p.n_cells, "l2": "n/a (host)"},
            "cpu_baseline": {"value": ups, "unit": "voxel-substrate updates/s", "cores": threads,
                             "kind": "oracle",
                             "sample": f"{args.steps} timed full steps after {args.warmup} warm-up"},
            "e2e": {"value": ups, "unit": "voxel-substrate updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2110_13368_gb300 import build as pbuild
    from paper_2110_13368_gb300 import bfvm
    pbuild.build()
    p = make_problem(args.workload)
    prec = p.precision
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    sim = bfvm.Sim.from_problem(p)
    if args.variant is not None:
        sim.set_option(bfvm.OPT_VARIANT, args.variant)
    if args.one_launch is not None:
        sim.set_option(bfvm.OPT_FUSED_STEP, args.one_launch)
    sim.set_option(bfvm.OPT_TIME_KERNELS, 1)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        flush.fill_(1.0)
        sim.step(1)
    torch.cuda.synchronize()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp64 = fp64_pipe_peak(n_sm, stream) if prec == 64 else None
    torch.cuda.synchronize()
    bfvm.bfvm_kernel_times(sim.handle, reset=True)
    info0 = sim.info()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t_wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))
            starts[i].record(stream)
            sim.step(1)
            ends[i].record(stream)
        torch.cuda.synchronize()
        barrier()
        t_wall = time.perf_counter() - t_wall0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = max_over_ranks(float(sum(step_ms)), world, dev)
    kms, kn = bfvm.bfvm_kernel_times(sim.handle, reset=True)
    info1 = sim.info()
    launches = info1["launches"] - info0["launches"]

    N = p.updates_per_step
    ups = job_rate(N * args.steps, world, total_ms / 1e3)
    ms_per_step = total_ms / args.steps
    es = 8 if prec == 64 else 4
    hbm, hbm_src = peaks()

    # kinds: per-axis sweeps, sources + Dirichlet shell, and the three
    # sweeps as one launch (then one launch covers 3 sweeps' work)
    kinds = ["x", "y", "z", "sources", "xyz"]
    sweeps_per_launch = [1, 1, 1, 0, 3]
    kernels = {}
    for k, name in enumerate(kinds):
        if kn[k]:
            avg = kms[k] / kn[k]
            bytes_per_launch = 2 * es * N * sweeps_per_launch[k]
            kernels[name] = {"launches": kn[k], "avg_ms": avg, "share": kms[k] / max(sum(kms), 1e-12)}
            if bytes_per_launch:
                kernels[name]["gbs"] = bytes_per_launch / (avg / 1e3) / 1e9
    dom = max((0, 1, 2, 4), key=lambda k: kms[k])
    dom_avg = kms[dom] / max(kn[dom], 1)
    dom_sweeps = sweeps_per_launch[dom]
    traffic = sweep_traffic(f"{args.workload.replace('_fp32', '')}_fp{prec}")
    info = sim.info()
    rescaled = prec == 64 and info["variant"] == 1
    kname = "x, y and z sweeps (one launch)" if dom == 4 else f"{kinds[dom]} sweep"
    alg_bytes = 2 * es * N * dom_sweeps
    achieved_bw = alg_bytes / (dom_avg / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": kname, "achieved": achieved_bw, "peak": hbm,
            "unit": "GB/s", "frac": achieved_bw / hbm,
            "peak_source": f"{hbm_src}: MEASURED_PEAKS.json hbm_gbs (copy, burst)",
            "bytes_per_update_per_sweep": 2 * es, "sweeps_per_launch": dom_sweeps,
            "updates_per_launch": N, "algorithmic_bytes_per_launch": alg_bytes,
            "avg_launch_ms": dom_avg,
            "traffic": traffic.get(kinds[dom]) if traffic else None}
    if prec == 64:
        flops_per_elem = 4 if rescaled else 5
        achieved = flops_per_elem * N * dom_sweeps / (dom_avg / 1e3) / 1e12
        roof["fp64_pipe"] = {"achieved_tflops": achieved,
                             "measured_peak_tflops": fp64["measured_tflops"],
                             "frac_of_measured": achieved / fp64["measured_tflops"],
                             "nominal_peak_tflops": fp64["nominal_tflops"],
                             "frac_of_nominal": achieved / fp64["nominal_tflops"],
                             "flops_per_element_per_sweep": flops_per_elem,
                             "algorithmic_flops_per_launch": flops_per_elem * N * dom_sweeps,
                             "probe": fp64}

    if args.skip_extras:
        sim.close()
        if rank == 0:
            print(json.dumps({"metric": metric_name(), "value": ups, "unit": "voxel-substrate updates/s",
                              "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": ms_per_step, "roofline": roof, "kernels": kernels,
                              "gpu_launches": launches, "note": "--skip-extras"}), flush=True)
        return 0

    # end to end through the C ABI with host buffers: upload the field,
    # one step, read the field back, every step
    host_in = torch.empty(p.rho0.shape, dtype=sim.dtype).pin_memory()
    host_in.copy_(torch.as_tensor(p.rho0, dtype=sim.dtype))
    host_out = torch.empty_like(host_in).pin_memory()
    sim.set_option(bfvm.OPT_TIME_KERNELS, 0)
    h = sim.handle
    bfvm.bfvm_set_density(h, host_in)
    bfvm.bfvm_step(h, 1)
    bfvm.bfvm_get_density(h, host_out)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        bfvm.bfvm_set_density(h, host_in)
        bfvm.bfvm_step(h, 1)
        bfvm.bfvm_get_density(h, host_out)
    torch.cuda.synchronize()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    nbytes = host_in.numel() * host_in.element_size()
    e2e = {"value": job_rate(N * args.e2e_steps, world, e2e_s), "unit": "voxel-substrate updates/s",
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
           "steps": args.e2e_steps,
           "call": "bfvm_set_density(host) + bfvm_step(1) + bfvm_get_density(host)"}
    # the host link's own rates (pinned buffers of the same size, copy engine)
    # and the e2e rate they allow: both copies plus the device step
    h2d, d2h = host_link_rates(host_in, host_out, stream)
    link_ms = nbytes / h2d / 1e6 + nbytes / d2h / 1e6 + ms_per_step
    e2e["host_link"] = {"h2d_gbs": h2d, "d2h_gbs": d2h,
                        "bound_value": N / (link_ms / 1e3),
                        "frac_of_bound": e2e["value"] / world / (N / (link_ms / 1e3)),
                        "note": "pinned cudaMemcpyAsync of the field in each direction; "
                                "bound = updates per (H2D + D2H + ms_per_step)"}

    forms = None
    if not args.no_forms and world == 1:
        forms = measure_forms(args, ups, dev, stream, flush)

    # continuous run for context: 1000 steps in one call (graphs, no flush)
    sim.set_option(bfvm.OPT_TIME_KERNELS, 0)
    sim.set_density(torch.as_tensor(p.rho0, dtype=sim.dtype, device=dev))
    sim.step(info["period"] if rescaled else 16)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(p.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    cont_ms = e0.elapsed_time(e1)
    continuous = {"value": N * p.steps / (cont_ms / 1e3), "steps": p.steps,
                  "ms_per_step": cont_ms / p.steps,
                  "note": "one bfvm_step(n) call, CUDA graphs, no L2 flush between steps"}
    sim.close()

    if rank == 0:
        line = {"metric": metric_name(), "value": ups, "unit": "voxel-substrate updates/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if prec == 64 else "f32", "data": "synthetic",
                "config": {"workload": p.name, "grid": [p.nx, p.ny, p.nz], "n_sub": p.n_sub,
                           "cells": p.n_cells, "sweep": "rescaled" if rescaled else "plain",
                           "l2": "512 MB buffer written before every timed step",
                           "parallelism": "replicas" if world > 1 else "single"},
                "hbm_frac_step": ups / world * 6 * es / 1e9 / hbm,
                "roofline": roof, "kernels": kernels, "gpu_launches": launches,
                "wall_s_timed_region": t_wall, "e2e": e2e, "continuous": continuous}
        if forms is not None:
            line["forms"] = forms
        clocks = clk.summary()
        line["clocks"] = clocks
        f32 = forms.pop("_plain_50_fp32_field", None) if forms is not None else None
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(p, args.cpu_seconds)
            if f32 is not None:
                # the FP64 oracle's 100 steps of the 50^3 workload, timed here
                # too, against the FP32 GPU result
                import oracle
                from paper_2110_13368_gb300 import inputs
                p50 = inputs.plain_50()
                t0 = time.perf_counter()
                ref50 = oracle.run(p50, n_threads=oracle.max_threads())
                el = time.perf_counter() - t0
                line["forms"]["fp32"]["plain_50_100_steps"]["vs_fp64_oracle"] = accuracy(f32, ref50)
                line["cpu_baseline"]["plain_50"] = {
                    "value": p50.updates_per_step * p50.steps / el, "steps": p50.steps,
                    "cores": oracle.max_threads(), "seconds": el}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_form(args):
    """One form of the step on its own: W untimed and K timed steps (CUDA
    events, 512 MB L2 flush before each), its rate in voxel-substrate
    updates per second.  For profiling runs; the default run measures every
    form beside the headline."""
    import numpy as np
    import torch
    from paper_2110_13368_gb300 import bfvm, inputs, slabs
    from paper_2110_13368_gb300 import build as pbuild
    pbuild.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    form = args.form
    closers = []
    if form == "fp32":
        p = inputs.tumour_200(steps=1000, precision=32)
        sim = bfvm.Sim.from_problem(p)
        closers.append(sim)
        n_upd, step = p.updates_per_step, (lambda: sim.step(1))
        launches = lambda: sim.info()["launches"]
    elif form in ("batched", "batched_fp32", "batched_phases"):
        # batched_phases: the FP64 batch on its tuned per-phase launches
        probs = inputs.batch_256(seed=0, precision=32 if form == "batched_fp32" else 64)
        sims = [bfvm.Sim.from_problem(q) for q in probs]
        batch = bfvm.Batch(sims)
        if form == "batched_phases":
            batch.set_option(bfvm.BATCH_OPT_ONE_LAUNCH, 0)
        closers += [batch] + sims
        n_upd, step = sum(q.updates_per_step for q in probs), (lambda: batch.step(1))
        launches = lambda: batch.info()["launches"]
    elif form == "adjoint":
        # one timed unit = a recorded forward of the workload and its backward
        p, q = inputs.adjoint_problem()
        sim = bfvm.Sim.from_problem(p)
        closers.append(sim)
        rho0 = torch.as_tensor(p.rho0, device=dev)
        target = torch.ones_like(rho0)

        def step():
            sim.set_density(rho0)
            sim.record(20)
            sim.step(p.steps)
            sim.backward(2.0 * (sim.get_density() - target))
        n_upd = p.updates_per_step * p.steps
        launches = lambda: sim.info()["launches"]
    elif form == "two_d":
        p = inputs.make_problem(1000, 1000, 1, n_sub=2, D=[1e5, 1e3], lam=[0.1, 0.01],
                                bc_kind=[1, 0], bc_value=[38.0, 0.0], field_mode="zero",
                                n_cells=20_000, U=[10.0, 0.0], S=[0.0, 10.0],
                                rho_star=[1.0, 1.0], steps=10, seed=0, dims=2)
        sim = bfvm.Sim.from_problem(p)
        closers.append(sim)
        n_upd, step = p.updates_per_step, (lambda: sim.step(1))
        launches = lambda: sim.info()["launches"]
    elif form == "nodes":
        pt = inputs.tumour_200(steps=10)
        rng = np.random.default_rng(5)
        vox, sub, val = [], [], []
        for _ in range(40):
            x, y = rng.integers(10, 190, size=2)
            v, sb, vl = inputs.vessel_nodes(pt.nx, pt.ny, pt.nz, substrate=0, value=38.0,
                                            x=int(x), y=int(y))
            vox.append(v); sub.append(sb); val.append(vl)
        p = pt.with_(nodes=(np.concatenate(vox), np.concatenate(sub), np.concatenate(val)))
        sim = bfvm.Sim.from_problem(p)
        closers.append(sim)
        n_upd, step = p.updates_per_step, (lambda: sim.step(1))
        launches = lambda: sim.info()["launches"]
    else:   # slabs: the 200^3 x 2 tumour grid as two z-slabs on this one GPU
        p = inputs.tumour_200(steps=10)
        z = slabs.partition(p.nz, 2)
        parts = [slabs.Slab.from_problem(p, z, j) for j in range(2)]
        closers += parts
        n_upd, step = p.updates_per_step, (lambda: slabs.step_together(parts, 1))
        launches = lambda: sum(bfvm.bfvm_get_info(s.handle)["launches"] for s in parts)
    for _ in range(max(args.warmup, 1)):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    l0 = launches()
    ms = timed_steps(step, args.steps, stream, flush)
    l1 = launches()
    for o in closers:
        o.close()
    print(json.dumps({"form": form, "metric": "voxel-substrate updates/s",
                      "value": n_upd * args.steps / (ms / 1e3),
                      "ms_per_step": ms / args.steps, "steps": args.steps,
                      "launches_per_step": (l1 - l0) / args.steps,
                      "l2": "512 MB buffer written before every timed step"}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.form is not None:
        return run_form(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
