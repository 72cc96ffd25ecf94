#!/usr/bin/env python
"""Benchmark: the sheared-suspension step (lattice Boltzmann + particles) on
the 96^3 dense bulk-shear workload (bidisperse radii 4 / 5.6, phi_3 = 0.50,
N = 882, kn = 1e3, kt = 0.5 kn, mu = 1, shear rate 1e-4, FP32 storage).

One "step" is one full pass of the hot path: collide-stream with bounce-back
and Lees-Edwards planes, link momentum exchange, particle sub-steps (cell
list, contacts, repulsion, lubrication, integration), node-map update and the
stress / histogram accumulation.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the same workload instead (bounded sample per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("MLUPS and particle-steps/s vs HBM roofline; batched reduced-precision vs plain "
          "at ≤2% stress")
FALLBACK_HBM_GBS = 6800.0


def workload(seed_offset: int = 0, L: int = 96):
    from paper_1904_02929_gb300 import inputs
    return inputs.config_dst(seed=1002 + seed_offset, phi3=0.50, L=L, rate=1e-4, precision="fp32")


def max_over_ranks(x: float, dist=None) -> float:
    """Largest value of x over the ranks of the process group (x itself
    without one); the tensor lives where the backend wants it."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank: float, steps: int, t_max_ms: float) -> float:
    """Whole-job rate in millions of units per second: every rank advanced
    its own units (weak scaling), the slowest rank sets the time."""
    return world * units_per_rank * steps / (t_max_ms / 1e3) / 1e6


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBps", "hbm_copy_gbs", "hbm"):
                if k in d and isinstance(d[k], (int, float)):
                    return float(d[k]), "measured"
            for k, val in d.items():
                if "hbm" in k.lower() and isinstance(val, (int, float)):
                    return float(val), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def k1_traffic(workload_name: str, kernel: str, record: str = "k_collide_stream_dst96_traffic.txt"):
    """DRAM bytes per collide-stream launch from a committed ncu summary,
    valid only for the workload and kernel captured and while its source is
    unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", record)
    if not os.path.exists(path):
        return None
    src = open(os.path.join(ROOT, "paper_1904_02929_gb300", "csrc", "lbm.cu"), "rb").read()
    h = hashlib.sha256(src).hexdigest()[:16]
    fields = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            k, v = line.strip().split("=", 1)
            fields[k.strip()] = v.strip()
    if fields.get("lbm_cu_sha256_16") != h or fields.get("workload") != workload_name:
        return None
    if fields.get("kernel", "k_collide_stream<fp32>") != kernel:
        return None
    try:
        return float(fields["dram_bytes_per_launch"])
    except Exception:
        return None


# Collide-stream launch shape for every leg: None lets the tuner choose
# (default); --launch-shape ROWS,BLOCKS,STAGED fixes it (e.g. to profile the
# shape an unprofiled run chose, since the tuner's timings differ under ncu).
LAUNCH_SHAPE = None


def shape_for(obj) -> dict:
    """Tune the box or batch obj, or apply the fixed --launch-shape; returns
    the shape in use."""
    if LAUNCH_SHAPE is None:
        return obj.tune()
    obj.set_launch_shape(*LAUNCH_SHAPE[:3])
    obj.set_overlap(LAUNCH_SHAPE[3])
    return dict(obj.launch_shape(), us=None, fixed=True)


def lb_kernel(shape: dict, storage: str) -> str:
    """Name of the collide-stream kernel a launch shape runs."""
    return ("k_collide_stream_tma" if shape.get("staged") else "k_collide_stream") + f"<{storage}>"


STAGE_KERNELS = {
    "collide_stream": ("k_collide_stream or k_collide_stream_tma (the tuner's choice)", "hbm"),
    "particles": ("k_dem_step (all particle sub-steps and the step's finalisation, one cooperative launch)",
                  "latency: one warp per particle, a grid barrier per sub-step, ~0.5 MB of DRAM traffic"),
    "finalize": ("k_finalize (only when no particle moves)", "latency"),
    "node_map": ("k_uncover + k_cover", "latency: bounding-box scans per particle"),
    "links": ("k_links", "latency: surface-shell gather per particle"),
}


def dominant_stage(stages: dict) -> dict:
    """The stage that took the most time in the timed steps, its kernel(s)
    and what bounds it."""
    tot = sum(stages.values()) or 1.0
    name = max(stages, key=stages.get)
    kern, bound = STAGE_KERNELS[name]
    return {"stage": name, "kernel": kern, "share": stages[name] / tot, "bound": bound}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.p = None
        # the raw samples go to $SUSP_CLOCKS_DIR (default: the temp directory)
        out_dir = os.environ.get("SUSP_CLOCKS_DIR") or tempfile.gettempdir()
        self.out = os.path.join(out_dir, f"clocks_{os.getpid()}.csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            os.makedirs(os.path.dirname(self.out), exist_ok=True)
            self.f = open(self.out, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "100", "-i", str(index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        with open(self.out) as f:
            return parse_clock_lines(f)


CLOCK_REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


def parse_clock_lines(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen
    (reported as Active in any sample) from nvidia-smi CSV lines of the
    query above; None without a usable sample."""
    sm, smax, reasons = [], [], set()
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax.append(float(parts[2]))
        except ValueError:
            continue
        for nm, val in zip(CLOCK_REASONS, parts[5:9]):
            if val.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
            "samples": len(sm)}


VOIDING_REASONS = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}


def clocks_rejected(clk) -> bool:
    """True when the timed region's clock record voids its number: a
    hardware or thermal slowdown was active, or the SM clock sat well below
    its maximum with no reason given (a clock lock left behind).  A power cap
    alone is kept."""
    if not clk:
        return False
    if VOIDING_REASONS & set(clk["reasons"]):
        return True
    return not clk["reasons"] and clk["sm_mhz"] < 0.8 * clk["sm_max_mhz"]


def timed_with_retake(run, sampler, agree=lambda flag: flag):
    """Run the timed region once with clocks sampled; if the clock record
    is rejected, run it once more.  run() returns the region's result,
    sampler() a started clock sampler (or None), agree(flag) the decision all
    ranks take.  Returns (result, clocks, clocks of the rejected first try or
    None)."""
    first = None
    for attempt in range(2):
        smp = sampler()
        res = run()
        clk = smp.stop() if smp else None
        if not agree(attempt == 0 and clocks_rejected(clk)):
            return res, clk, first
        first = clk
    raise AssertionError("unreachable")


def cpu_baseline(w, budget_s: float = 15.0, keep=None):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload.
    ``keep`` (a list), if given, receives the oracle and its step count, so
    that the GPU result of the same steps can be compared with it."""
    import oracle as O
    kw = dict(w.params)
    o = O.Oracle(w.nx, w.ny, w.nz, w.radius, w.pos, **kw)
    sh = O.shear(**w.shear)
    t0 = time.perf_counter()
    o.step(1, sh)
    t1 = time.perf_counter()
    per = t1 - t0
    k = max(1, min(20, int(budget_s / max(per, 1e-3)) - 1))
    t0 = time.perf_counter()
    o.step(k, sh)
    dt = time.perf_counter() - t0
    steps = k
    if keep is not None:
        keep.extend([o, 1 + k])
    return {
        "value": w.ncell * steps / dt / 1e6,
        "unit": "MLUPS",
        "cores": 1,
        "kind": "oracle",
        "sample": f"{w.name}: {steps} FP64 oracle steps after 1 warm-up step on one host core "
                  f"({dt:.1f} s)",
        "particle_steps_per_s": w.n * steps / dt,
    }


def batched_launches(boxes) -> int:
    """Kernels per batched step for boxes given as (particles, brute-force
    pair search): the collide-stream, the cell-list build (four kernels, only
    when a box with particles is too large for the brute-force search), the
    particle kernel (which ends with the finalisation), the node map (two)
    and the links; a batch without particles runs the collide-stream and the
    finalisation only."""
    if not any(n > 0 for n, _ in boxes):
        return 2
    any_cells = any(n > 0 and not brute for n, brute in boxes)
    return 1 + (4 if any_cells else 0) + 1 + 2 + 1


def batched_leg(ws, steps: int, warmup: int):
    """The 64-box sweep (edges 48-96, phi_3 0.45-0.58, mixed constant and
    oscillatory shear): BF16 deviation storage stepped as one batch (one
    launch sequence for all boxes, replayed as a CUDA graph) against the same
    boxes in FP32 stepped one box per launch sequence (plain launches, no
    graph), in turn on one stream.
    Both run warmup + steps steps from rest with the stresses reset after the
    warm-up; the time-averaged shear stresses are compared box by box, and
    the smallest box against the FP64 oracle."""
    import numpy as np
    import torch
    from paper_1904_02929_gb300 import inputs
    from paper_1904_02929_gb300 import susp as S
    nodes = sum(w.ncell for w in ws)
    parts = sum(w.n for w in ws)

    def timed(stream, fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b)

    # batched, BF16
    bs = torch.cuda.Stream()
    boxes = [S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, stream=bs, precision="bf16", **w.params)
             for w in ws]
    batch = S.Batch(len(ws), stream=bs)
    for w, g in zip(ws, boxes):
        batch.attach(g, S.make_shear(**w.shear))
    batch.step(warmup)
    tuned = shape_for(batch)                        # collide-stream launch shape for this batch
    for g in boxes:
        g.stress_reset()
    batch.step(1)                                   # capture the step graph untimed
    torch.cuda.synchronize()
    ms_b = timed(bs, lambda: batch.step(steps))
    sb = [g.stress(S.TOTAL)[0][0, 1] for g in boxes]   # raises on any device error flag
    # stage times: as many further steps, profiled (event nodes in the graph)
    batch.profile(True)
    batch.step(1)
    torch.cuda.synchronize()
    batch.profile(True)
    batch.step(steps)
    torch.cuda.synchronize()
    stages, k1_n = S.susp_batch_profile_stages(batch.b)
    k1_ms = stages["collide_stream"]
    batch.profile(False)
    launches_b = batched_launches([(g.n, g.info().brute_force_pairs) for g in boxes])
    mem_b = sum(g.nbytes for g in boxes)
    batch.close()
    for g in boxes:
        g.close()
    del boxes
    # plain, FP32, one box per launch sequence
    ps = torch.cuda.Stream()
    plain = [S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, stream=ps, precision="fp32", **w.params)
             for w in ws]
    for g in plain:
        g.set_graphs(False)                         # plain launches, as a one-box code would issue them
    shears = [S.make_shear(**w.shear) for w in ws]
    for g, sh in zip(plain, shears):
        g.step(warmup, sh)
    for g in plain:
        g.stress_reset()
    for g, sh in zip(plain, shears):
        g.step(1, sh)                               # one extra step like the batch
    torch.cuda.synchronize()

    def run_plain():
        for _ in range(steps):
            for g, sh in zip(plain, shears):
                g.step(1, sh)
    ms_p = timed(ps, run_plain)
    sp = [g.stress(S.TOTAL)[0][0, 1] for g in plain]
    for g in plain:
        g.close()
    del plain
    dev = [abs(b - p) / abs(p) for b, p in zip(sb, sp)]
    # the smallest box against the FP64 oracle, same protocol
    import oracle as O
    k = int(np.argmin([w.ncell for w in ws]))
    w = ws[k]
    o = O.Oracle(w.nx, w.ny, w.nz, w.radius, w.pos, **w.params)
    o.step(warmup, O.shear(**w.shear))
    o.stress_reset()
    o.step(steps + 1, O.shear(**w.shear))
    so = o.stress(O.TOTAL)[0][0, 1]
    mb = nodes * steps / (ms_b / 1e3) / 1e6
    mp = nodes * steps / (ms_p / 1e3) / 1e6
    k1 = k1_ms / max(k1_n, 1)
    alg = 2 * 19 * 2 * nodes                        # BF16 populations of every lattice cell
    peak, kind = peak_hbm()
    return {
        "boxes": len(ws), "lattice_nodes": nodes, "particles": parts, "steps": steps,
        "warmup": warmup, "storage": "bf16", "compute": "f32 (positions, offsets, stress sums f64)",
        "value": mb, "unit": "MLUPS", "ms_per_step": ms_b / steps,
        "particle_steps_per_s": parts * steps / (ms_b / 1e3),
        "k_collide_stream_avg_ms": k1,
        "roofline": {"bound": "hbm", "kernel": lb_kernel(tuned, "bf16"), "achieved": alg / (k1 / 1e3) / 1e9,
                     "peak": peak, "unit": "GB/s", "frac": alg / (k1 / 1e3) / 1e9 / peak,
                     "peak_source": kind, "algorithmic_bytes_per_launch": alg, "avg_launch_ms": k1,
                     "traffic": k1_traffic("batch64-bf16", lb_kernel(tuned, "bf16"),
                                           "k_collide_stream_bf16_batch64_traffic.txt") if len(ws) == 64 else None},
        "launch_shape": tuned,
        "stage_us": {k: round(1e3 * v / max(k1_n, 1), 1) for k, v in stages.items()},
        "gpu_launches_per_step": launches_b, "workspace_bytes": mem_b,
        "l2": "not flushed: the boxes hold > 1.9 GB of populations, far above L2",
        "plain": {"storage": "fp32", "value": mp, "unit": "MLUPS", "ms_per_step": ms_p / steps,
                  "launch": "one box per launch sequence, no graph, boxes in turn on one stream"},
        "speedup_vs_plain": mb / mp,
        "stress_xy_rel_dev_vs_plain": {"max": max(dev), "median": float(np.median(dev))},
        "stress_xy_vs_oracle": {"box": w.name, "gpu_bf16": float(sb[k]), "oracle_f64": float(so),
                                "rel_err": abs(sb[k] - so) / abs(so)},
    }


def profiled_window(g, sh, steps: int, flush=None):
    """Stage times of ``steps`` further steps of box ``g`` (CUDA events
    recorded by event nodes inside the replayed step graph, on the box's
    stream), with an optional L2 flush before each step; profiling off after."""
    import torch
    from paper_1904_02929_gb300 import susp as S
    S.susp_profile(g.h, True)
    g.step(1, sh)                           # capture the profiled graph, untimed
    torch.cuda.synchronize()
    S.susp_profile(g.h, True)               # a new window
    with torch.cuda.stream(g.stream):
        for _ in range(steps):
            if flush is not None:
                flush.zero_()
            g.step(1, sh)
    torch.cuda.synchronize()
    stages, n = S.susp_profile_stages(g.h)
    S.susp_profile(g.h, False)
    return stages, n


def errors_vs_oracle(g, o, kinds=("total",)) -> dict:
    """Errors of a GPU machine against the FP64 oracle after the same steps from
    the same state: populations over the nodes fluid on both sides (max
    absolute difference over the oracle's largest value), centres (max
    absolute difference, lattice units) and the time-averaged stress (max
    component difference over the oracle's largest component, and the shear
    component alone)."""
    import numpy as np
    import oracle as O
    from paper_1904_02929_gb300 import susp as S
    fo, fg = o.populations(), g.populations()
    fl = (o.owner() < 0) & (g.owner() < 0)
    out = {"populations": float(np.abs(fg[:, fl] - fo[:, fl]).max() / np.abs(fo[:, fl]).max()),
           "node_map_agrees": bool((o.owner() == g.owner()).all())}
    if o.n:
        out["centres"] = float(np.abs(g.particles()[0] - o.particles()[0]).max())
    for name in kinds:
        so = o.stress(getattr(O, name.upper()))[0]
        sg = g.stress(getattr(S, name.upper()))[0]
        out[f"stress_{name}"] = float(np.abs(sg - so).max() / np.abs(so).max())
        out[f"stress_{name}_xy"] = float(abs(sg[0, 1] - so[0, 1]) / abs(so[0, 1]))
    return out


def precision_leg(oracle_96=None, mono_steps: int = 2):
    """Each storage's error against the FP64 oracle on the workloads whose
    rows the reduced-precision target names: the 96^3 bulk-shear box in FP32
    (the oracle of the CPU baseline, same steps), the 512 x 512 x 28 monolayer
    in FP16 (``mono_steps`` oracle steps), and the 32^3 20-sphere box in FP32,
    FP16 and BF16 (200 steps at rate 1e-3)."""
    import oracle as O
    from paper_1904_02929_gb300 import inputs
    from paper_1904_02929_gb300 import susp as S
    out = {}
    if oracle_96:
        o, k = oracle_96
        w = workload()
        g = S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, precision="fp32", **w.params)
        g.step(k, S.make_shear(**w.shear))
        out["dst96_fp32"] = dict(errors_vs_oracle(g, o, ("total", "contact", "viscous")), steps=k)
        g.close()
    w = inputs.config_monolayer(seed=1003, phi=0.70, Lz=28, gamma0=0.1, precision="fp16")
    o = O.Oracle(w.nx, w.ny, w.nz, w.radius, w.pos, **w.params)
    o.step(mono_steps, O.shear(**w.shear))
    g = S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, precision="fp16", **w.params)
    g.step(mono_steps, S.make_shear(**w.shear))
    out["monolayer_fp16"] = dict(errors_vs_oracle(g, o, ("total", "viscous")), steps=mono_steps)
    g.close()
    del o
    w = inputs.config_small()
    o = O.Oracle(w.nx, w.ny, w.nz, w.radius, w.pos, **w.params)
    sh = dict(kind=0, rate=1e-3)
    o.step(200, O.shear(**sh))
    for prec in ("fp32", "fp16", "bf16"):
        g = S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, precision=prec, **w.params)
        g.step(200, S.make_shear(**sh))
        out[f"small32_{prec}"] = dict(errors_vs_oracle(g, o, ("total",)), steps=200)
        g.close()
    out["note"] = ("max relative errors against the FP64 oracle after the same steps from the same "
                   "state; populations over nodes fluid on both sides")
    return out


def sweep_leg(steps: int, chunk: int = 500):
    """The bulk-shear sweep at 96^3 in FP32: phi_3 in {0.50, 0.54, 0.58} and
    shear rate in {1e-5, 1e-4, 1e-3}.  Each point runs up to ``steps`` lattice
    steps in chunks, reading the device status after every chunk, and
    reports the steps completed before any flag (the survival of the dense
    packing under shear), its throughput, and the time-averaged shear stress
    with the relative viscosity sigma_xy / (eta0 rate)."""
    import torch
    from paper_1904_02929_gb300 import inputs
    from paper_1904_02929_gb300 import susp as S
    rows = []
    for phi in (0.50, 0.54, 0.58):
        for rate in (1e-5, 1e-4, 1e-3):
            w = inputs.config_dst(phi3=phi, L=96, rate=rate)
            g = S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, precision="fp32", **w.params)
            sh = S.make_shear(**w.shear)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            done, status, sxy = 0, "ok", None
            ms = 0.0
            while done < steps:
                n = min(chunk, steps - done)
                torch.cuda.synchronize()
                a.record(g.stream)
                g.step(n, sh)
                b.record(g.stream)
                try:
                    st, _ = g.stress(S.TOTAL)       # synchronises; raises on a device flag
                except S.SuspError as e:
                    status = S.status_name(e.status)
                    break
                ms += a.elapsed_time(b)
                done += n
                sxy = float(st[0, 1])
            info = g.info()
            g.close()
            eta0 = w.params["rho0"] * (w.params["tau"] - 0.5) / 3.0
            rows.append({"phi3": phi, "rate": rate, "particles": w.n, "dem_substeps": info.dem_substeps,
                         "steps_completed": done, "status": status,
                         "mlups": w.ncell * done / (ms / 1e3) / 1e6 if done else None,
                         "particle_steps_per_s": w.n * done / (ms / 1e3) if done else None,
                         "sigma_xy": sxy, "eta_rel": sxy / (eta0 * rate) if sxy is not None else None})
    return {"lattice": [96, 96, 96], "storage": "fp32", "steps_per_point": steps, "chunk": chunk,
            "points": rows,
            "note": "steps_completed < steps_per_point means the named device flag ended the run"}


def monolayer_leg(steps: int, warmup: int):
    """Quasi-2D oscillatory shear at the paper's resolution: 512 x 512 x 28,
    radii 5 / 7 (L_z = 4 a_max), phi = 0.70 (N = 1580), reduced amplitude
    gamma0 = 0.1, FP16 deviation storage, FP32 compute: throughput and the
    collide-stream roofline on a working set larger than L2 (no flush).  The
    12-high variant with radii scaled to 3 / 2.14 is under-resolved (node
    claims collide within tens of steps, in the oracle too)."""
    import torch
    from paper_1904_02929_gb300 import inputs
    from paper_1904_02929_gb300 import susp as S
    w = inputs.config_monolayer(seed=1003, phi=0.70, Lz=28, gamma0=0.1, precision="fp16")
    g = S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, precision="fp16", **w.params)
    sh = S.make_shear(**w.shear)
    g.step(warmup, sh)
    tuned = shape_for(g)
    g.step(1, sh)                                   # capture the step graph, untimed
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(g.stream):
        a.record(g.stream)
        g.step(steps, sh)
        b.record(g.stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    stages, n = profiled_window(g, sh, steps)
    g.stress(S.TOTAL)                               # raises on any device error flag
    info = g.info()
    g.close()
    k1 = stages["collide_stream"] / n
    alg = 2 * 19 * 2 * w.ncell                      # FP16 populations of every lattice cell
    peak, kind = peak_hbm()
    return {"workload": w.name, "lattice": [w.nx, w.ny, w.nz], "particles": w.n, "storage": "fp16",
            "steps": steps, "value": w.ncell * steps / (ms / 1e3) / 1e6, "unit": "MLUPS",
            "ms_per_step": ms / steps, "particle_steps_per_s": w.n * steps / (ms / 1e3),
            "dem_substeps": info.dem_substeps,
            "stage_us": {k: round(1e3 * v / n, 1) for k, v in stages.items()},
            "roofline": {"bound": "hbm", "kernel": lb_kernel(tuned, "fp16"), "achieved": alg / (k1 / 1e3) / 1e9,
                         "peak": peak, "unit": "GB/s", "frac": alg / (k1 / 1e3) / 1e9 / peak,
                         "peak_source": kind, "algorithmic_bytes_per_launch": alg, "avg_launch_ms": k1,
                         "traffic": k1_traffic(w.name, lb_kernel(tuned, "fp16"),
                                               "k_collide_stream_fp16_monolayer_traffic.txt")},
            "launch_shape": tuned,
            "l2": "not flushed: 560 MB of populations per buffer, above L2"}


def variant_leg(w, what: str, steps: int, warmup: int, **over):
    """Throughput of one FP32 box built from workload ``w`` with parameter
    overrides (Ladd's collision operator, bumpy walls): tuned, L2 flushed
    between timed steps like the default leg, per-step CUDA events on the
    box's stream; MLUPS, particle-steps/s, stage times and the
    collide-stream roofline."""
    import torch
    from paper_1904_02929_gb300 import susp as S
    kw = dict(w.params)
    kw.update(over)
    g = S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, precision="fp32", **kw)
    sh = S.make_shear(**w.shear)
    g.step(warmup, sh)
    tuned = shape_for(g)
    g.step(2, sh)                                   # capture the step graph, untimed
    torch.cuda.synchronize()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    with torch.cuda.stream(g.stream):
        for a, b in ev:
            flush.zero_()
            a.record(g.stream)
            g.step(1, sh)
            b.record(g.stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    stages, n = profiled_window(g, sh, steps, flush)
    g.stress(S.TOTAL)                               # raises on any device error flag
    info = g.info()
    g.close()
    del flush
    k1 = stages["collide_stream"] / n
    alg = 2 * 19 * 4 * w.ncell
    peak, kind = peak_hbm()
    return {"workload": w.name, "variant": what, "lattice": [w.nx, w.ny, w.nz], "particles": w.n,
            "storage": "fp32", "steps": steps, "value": w.ncell * steps / (ms / 1e3) / 1e6, "unit": "MLUPS",
            "ms_per_step": ms / steps, "particle_steps_per_s": w.n * steps / (ms / 1e3),
            "dem_substeps": info.dem_substeps,
            "stage_us": {k: round(1e3 * v / n, 1) for k, v in stages.items()},
            "roofline": {"bound": "hbm", "kernel": lb_kernel(tuned, "fp32"), "achieved": alg / (k1 / 1e3) / 1e9,
                         "peak": peak, "unit": "GB/s", "frac": alg / (k1 / 1e3) / 1e9 / peak,
                         "peak_source": kind, "algorithmic_bytes_per_launch": alg, "avg_launch_ms": k1},
            "launch_shape": tuned, "l2": "flushed between timed steps (256 MB write)"}


def serving_leg(requests: int = 40, rate: float = 20.0, steps: int = 5000, budget_frac: float = 0.8):
    """A fixed horizon of Poisson-arriving requests (rate per second) drawn
    50 / 50 from quasi-2D 512 x 512 and 256 x 256 monolayers (phi
    0.70 / 0.75 / 0.80) at the paper's resolution (radii 5 / 7, L_z = 28),
    each ``steps`` lattice steps (chunks of 1000) in FP16 deviation storage,
    served by continuous batching within an HBM budget of ``budget_frac`` of
    the device's free memory; queue wait, service time and latency
    percentiles (also per 1000 steps) and aggregate MLUPS."""
    import torch
    from paper_1904_02929_gb300 import inputs, serve
    free, _ = torch.cuda.mem_get_info()
    budget = int(budget_frac * free)
    big = [inputs.config_monolayer(seed=3000 + k, phi=phi, Lz=28, precision="fp16")
           for k, phi in enumerate((0.70, 0.75, 0.80))]
    small = [inputs.config_monolayer(seed=3100 + k, phi=phi, Lx=256, Ly=256, Lz=28, precision="fp16")
             for k, phi in enumerate((0.70, 0.75, 0.80))]
    pool = big + small
    # the reduced amplitudes of the protocol: at 512 lattice units of height
    # the initial amplitude 1.0 would drive the Lees-Edwards image at 0.3 per
    # step, far outside the lattice-Boltzmann Mach range
    reqs = serve.poisson_requests(pool, rate, 0.0, steps, seed=1005, oscillatory_only=True,
                                  amplitudes=(0.01, 0.1), count=requests)
    srv = serve.Server(budget, max_boxes=64, chunk=25, precision="fp16")
    srv.run(reqs)
    rep = srv.report()
    srv.close()
    rep.update({"arrival_rate_per_s": rate, "horizon_requests": requests, "steps_per_request": steps,
                "chunks_per_request": steps // 1000, "hbm_budget_frac_of_free": budget_frac,
                "storage": "fp16",
                "pool": "monolayers 512x512x28 and 256x256x28 (radii 5 / 7) at phi 0.70 / 0.75 / 0.80, drawn 50 / 50",
                "protocol": "oscillatory, gamma0 in {0.01, 0.1}, omega 6e-4, theta in {0, pi/2}"})
    return rep


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    w = workload()
    kw = dict(w.params)
    sh = O.shear(**w.shear)
    o = O.Oracle(w.nx, w.ny, w.nz, w.radius, w.pos, **kw)
    t0 = time.perf_counter()
    o.step(1, sh)
    per = time.perf_counter() - t0
    sample = w
    if (args.steps + args.warmup) * per > 150.0:
        sample = workload(L=48)
        o = O.Oracle(sample.nx, sample.ny, sample.nz, sample.radius, sample.pos, **dict(sample.params))
    for _ in range(args.warmup):
        o.step(1, sh)
    t0 = time.perf_counter()
    o.step(args.steps, sh)
    dt = time.perf_counter() - t0
    val = sample.ncell * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "lattice": [w.nx, w.ny, w.nz], "particles": w.n,
                   "storage": "fp64", "sample": sample.name},
        "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                         "sample": f"{sample.name}, {args.steps} timed oracle steps"},
        "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "particle_steps_per_s": sample.n * args.steps / dt,
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=100)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-monolayer", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the Ladd-operator and bumpy-wall legs")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--sweep-steps", type=int, default=5000)
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--launch-shape", default=None,
                    help="ROWS,BLOCKS,STAGED[,OVERLAP]: fix the collide-stream launch shape (and whether it "
                         "runs beside the particle kernel) of every leg instead of tuning")
    ap.add_argument("--serve-requests", type=int, default=40,
                    help="requests of the serving horizon (200 for the full sweep horizon)")
    args = ap.parse_args()
    global LAUNCH_SHAPE
    if args.launch_shape:
        f = [int(x) for x in args.launch_shape.split(",")] + [0]
        LAUNCH_SHAPE = (f[0], f[1], bool(f[2]), bool(f[3]))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    from paper_1904_02929_gb300 import susp as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # independent boxes per rank (weak scaling, no data-path collective)
    w = workload(seed_offset=rank)
    g = S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, precision="fp32", **w.params)
    info = g.info()
    sh = S.make_shear(**w.shear)
    g.step(args.warmup, sh)
    tuned = shape_for(g)                        # collide-stream launch shape (untimed)
    torch.cuda.synchronize()
    nfluid = int((g.owner() < 0).sum())

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 126 MB L2
    K = args.steps
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    S.susp_profile(g.h, True)
    g.step(2, sh)                           # capture the step graphs before timing
    torch.cuda.synchronize()

    def run_timed():
        # the timed steps replay the plain step graph: the profiled graph's
        # per-step event-node updates would put host time inside the region
        S.susp_profile(g.h, False)
        barrier()
        with torch.cuda.stream(g.stream):
            for k in range(K):
                flush.zero_()               # L2 flushed between timed steps (untimed)
                ev0[k].record(g.stream)
                g.step(1, sh)
                ev1[k].record(g.stream)
        barrier()
        return sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))

    def agree(flag):
        if dist is None:
            return flag
        t = torch.tensor([1 if flag else 0], device="cuda")
        dist.broadcast(t, 0)
        return bool(t.item())

    ms, clk, clk_rejected = timed_with_retake(
        run_timed, lambda: ClockSampler(torch.cuda.current_device()) if rank == 0 else None, agree)
    # stage times: the same number of steps right after, L2 flushed the same
    # way, with CUDA events recorded by event nodes inside the replayed graph
    stages, k1_n = profiled_window(g, sh, K, flush)
    k1_ms = stages["collide_stream"]
    st = S.susp_stress(g.h, S.TOTAL, g.nbins)   # raises on any device error flag
    t_max = max_over_ranks(ms, dist)
    mlups = job_throughput(world, w.ncell, K, t_max)
    psteps = job_throughput(world, w.n, K, t_max) * 1e6

    # --- end to end through the public API: create (host arrays up), K steps,
    # every step's results (error word, stress sums and counters, histogram,
    # centres, velocities, spins) copied to pinned host memory in one
    # transfer enqueued behind the step, and decoded on the host (positions
    # and total stress) while the next step runs
    del flush
    pos_host = torch.empty(3 * w.n, dtype=torch.float64).pin_memory()
    barrier()
    t0 = time.perf_counter()
    e = S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, precision="fp32", **w.params)
    e.tune()
    bufs = [e.results_buffer(), e.results_buffer()]
    evs = [torch.cuda.Event(), torch.cuda.Event()]

    def consume(buf):
        R, _, _ = e.results_particles(buf)   # raises on any device error flag
        pos_host.numpy()[:] = R.ravel()
        return e.results_stress(buf, S.TOTAL)[0]

    for k in range(K):
        e.step(1, sh)
        e.read_results(bufs[k % 2], True)
        evs[k % 2].record(e.stream)
        if k > 0:
            evs[(k - 1) % 2].synchronize()
            consume(bufs[(k - 1) % 2])
    evs[(K - 1) % 2].synchronize()
    s_tot = consume(bufs[(K - 1) % 2])
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    d2h = bufs[0].numel()                               # one results block per step
    e.close()
    e2e_s = max_over_ranks(e2e_s, dist)
    h2d = (w.n * (8 + 24 + 24 + 24)) / K                # radii, positions, velocities, spins

    if rank == 0:
        peak, peak_kind = peak_hbm()
        alg_bytes = 2 * 19 * 4 * w.ncell                 # FP32 populations of every lattice cell
        k1_avg_s = (k1_ms / max(k1_n, 1)) / 1e3
        achieved = alg_bytes / k1_avg_s / 1e9
        traffic = k1_traffic(w.name, lb_kernel(tuned, "fp32"))
        line = {
            "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": t_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "lattice": [w.nx, w.ny, w.nz], "particles": w.n,
                       "phi3": 0.50, "storage": "fp32", "shear_rate": w.shear["rate"],
                       "dem_substeps": info.dem_substeps, "fluid_nodes": nfluid,
                       "l2": "flushed between timed steps (256 MB write)",
                       "launch_shape": tuned,
                       "parallelism": f"replicas{world}"},
            "particle_steps_per_s": psteps,
            "stage_us": {k: round(1e3 * v / max(k1_n, 1), 1) for k, v in stages.items()},
            "stage_timing": ("the timed steps replay the plain step graph; stage times and the "
                             "collide-stream launch time come from as many steps right after, L2 "
                             "flushed the same way, timed by event nodes inside the replayed graph "
                             "on the streams the kernels run on" +
                             ("; the step overlaps the collide-stream with the particle kernel: "
                              "'particles' is the particle time not hidden behind the collide-stream"
                              if tuned.get("overlap") else "")),
            "dominant_kernel": dominant_stage(stages),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": lb_kernel(tuned, "fp32"), "peak_source": peak_kind,
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "avg_launch_ms": k1_ms / max(k1_n, 1)},
            "e2e": {"value": world * w.ncell * K / e2e_s / 1e6, "unit": "MLUPS",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "readback": "create from host arrays and tune inside the timed region; every step one "
                                "results block (status, stress sums, histogram, particles) copied to pinned "
                                "host memory behind the step and decoded on the host one step later"},
            "gpu_launches": info.launches_per_step * K,
            "clocks": clk,
            "stress_xy_total": float(st[0][0, 1]),
        }
        if clk_rejected is not None:
            line["clocks_rejected_first_try"] = clk_rejected
        if world == 1 and not args.no_monolayer:
            line["monolayer"] = monolayer_leg(args.batched_steps * 2, args.warmup)
        if world == 1 and not args.no_variants:
            from paper_1904_02929_gb300 import inputs
            legs = {"ladd": lambda: variant_leg(w, "Ladd's linear collision operator, tau_bulk = 0.8",
                                                args.batched_steps * 2, args.warmup, collision="ladd",
                                                tau_bulk=0.8),
                    "walls": lambda: variant_leg(inputs.config_walls(L=96, phi3=0.30, precision="fp32"),
                                                 "bumpy walls of driven spheres, U = 0.02",
                                                 args.batched_steps * 2, args.warmup)}
            for name, leg in legs.items():
                try:
                    line[name] = leg()
                except S.SuspError as e:     # a device flag in a side leg: report it, keep the line
                    line[name] = {"error": str(e)}
        if world == 1 and not args.no_batched:
            from paper_1904_02929_gb300 import inputs
            line["batched"] = batched_leg(inputs.batch_sweep(), args.batched_steps, args.warmup)
        if world == 1 and not args.no_sweep:
            line["sweep"] = sweep_leg(args.sweep_steps)
        if world == 1 and not args.no_serve:
            line["serving"] = serving_leg(args.serve_requests)
        keep = []
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w, keep=keep)
        if world == 1 and not args.no_precision:
            line["precision"] = precision_leg(keep if keep else None)
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
