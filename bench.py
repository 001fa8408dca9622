#!/usr/bin/env python
"""Benchmark of the IPC Newton hot path on B300.

Workload: 64 randomly oriented Neo-Hookean tori (1,084,416 tets, 257,024
vertices) piled in a 1 m box, dt = 0.01 s, dhat = 1e-3 m (the synthetic stand-in
for the paper's bunny-pile scenes).  A step is one implicit time step
(yasps_step): every Newton iteration in it runs the whole hot path (contact
detection, element + barrier derivatives with projection, assembly, block-
Jacobi PCG, CCD step bound, line search).  The metric counts Newton
iterations (assembly + solve passes) per second; the SpMV inside PCG is
measured live with CUDA events for the HBM roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

With N > 1 (torchrun) every rank simulates its own replica of the scene
(independent problems, no data-path collective): value = all ranks' Newton
iterations / the slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Newton steps/s & PCG SpMV HBM GB/s at 1M tets; FP32-mixed vs FP64 plain"
# The 1M-tet workload states no Newton tolerance; the paper's own benchmark
# (Sec. "Cloths on Bunny on Cloth") stops when ||dx||_inf / dt < 1e-2 m/s and
# uses a CG relative tolerance of 1e-4.
NEWTON_VEL_TOL = 1e-2
PCG_TOL = 1e-4
WORKLOAD = ("64 Neo-Hookean tori (R 0.08 m, r 0.03 m, ~8 mm voxels; 1,084,416 tets, 257,024 verts), "
            "seeded uniform-quaternion orientations, E log-uniform [1e4,1e6] Pa, 1 m box, dt 0.01 s, dhat 1e-3 m")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


def source_sha(*files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_rate(kernel_files):
    """DRAM bytes per second of the PCG kernel from a committed ncu capture
    (dram__bytes_read.sum + dram__bytes_write.sum over gpu__time_duration.sum of
    one launch), if it was taken on the current source; else None."""
    p = os.path.join(ROOT, "profiles", "pcg_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_sha") != source_sha(*kernel_files):
        return None
    return d.get("dram_bytes") / d.get("duration_s")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        smax = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(n_gpus):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def _reduce_device():
    import torch

    return "cuda" if torch.cuda.is_available() else "cpu"


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def allreduce_max(world, v):
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(world, v):
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
def native(args):
    import torch

    import paper_2605_23088_b300 as yb
    import scenes

    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    scene = scenes.tori_scene()
    n_tets = len(scene["tets"])
    ntol = NEWTON_VEL_TOL * scene["dt"]
    G = yb.System(scene, precision=1, pcg_rel_tol=PCG_TOL, newton_tol=ntol)
    x, v = G.initial_state()
    preroll = args.preroll
    if args.load_state:
        # the state a pre-roll left (written by --save-state): skips the untimed pre-roll
        st = np.load(args.load_state)
        x.copy_(torch.as_tensor(st["x"], device=dev))
        v.copy_(torch.as_tensor(st["v"], device=dev))
        preroll = int(st["preroll"])
    else:
        # untimed pre-roll: let the pile fall until tori touch the ground and each other
        for _ in range(args.preroll):
            G.step(x, v, raise_on_error=False)
    torch.cuda.synchronize()
    x0, v0 = x.clone(), v.clone()
    # the system holds the last step's assembly: pick the PCG launch configuration on it
    tune = {}
    for prec_sys, tag in ((G, "fp32_mixed"),):
        var, us = prec_sys.autotune_pcg(30)
        tune[tag] = {"variant": var, "us_per_iter": [round(u, 2) for u in us]}
    if args.save_state and rank == 0:
        np.savez(args.save_state, x=x0.cpu().numpy(), v=v0.cpu().numpy(), preroll=preroll)
    npt, nee, npg = G.detect_pairs(x0)

    def timed(system, precision_name, steps, warmup, profile):
        xs, vs = x0.clone(), v0.clone()
        for _ in range(warmup):
            system.step(xs, vs, raise_on_error=False)
        torch.cuda.synchronize()
        barrier(world)
        if profile:
            system.profile_enable(True)
        l0 = system.kernel_launches()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        passes = 0
        newton = 0
        pcg = 0
        status = []
        with ClockSampler(local) as clk:
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push(f"timed_{precision_name}")
            e0.record(stream)
            for _ in range(steps):
                st = system.step(xs, vs, raise_on_error=False)
                newton += st["newton_iters"]
                passes += st["newton_iters"] + (1 if st["rc"] == 0 else 0)
                pcg += st["pcg_iters_total"]
                status.append(st["rc"])
            e1.record(stream)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
        ms = e0.elapsed_time(e1)
        launches = system.kernel_launches() - l0
        prof = {k: system.profile_get(i) for i, k in enumerate(yb.STAGE_NAMES)} if profile else None
        phases = system.pcg_phase_ms() if profile else None
        if profile:
            system.profile_enable(False)
        barrier(world)
        ms_max = allreduce_max(world, ms)
        passes_all = allreduce_sum(world, passes)
        return dict(ms=ms, ms_max=ms_max, passes=passes, passes_all=passes_all, newton=newton, pcg=pcg,
                    launches=launches, status=status, prof=prof, phases=phases, clocks=clk.summary(),
                    precision=precision_name)

    mixed = timed(G, "fp32-mixed", args.steps, args.warmup, True)
    # end-to-end through the C ABI with host buffers: pinned host state in, state out
    xh = x0.cpu().pin_memory()
    vh = v0.cpu().pin_memory()
    xd, vd = torch.empty_like(x0), torch.empty_like(v0)
    for _ in range(args.warmup):
        xd.copy_(xh, non_blocking=True); vd.copy_(vh, non_blocking=True)
        G.step(xd, vd, raise_on_error=False)
        xh.copy_(xd, non_blocking=True); vh.copy_(vd, non_blocking=True)
    xh = x0.cpu().pin_memory()
    vh = v0.cpu().pin_memory()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    e2e_passes = 0
    for _ in range(args.steps):
        xd.copy_(xh, non_blocking=True)
        vd.copy_(vh, non_blocking=True)
        st = G.step(xd, vd, raise_on_error=False)
        e2e_passes += st["newton_iters"] + (1 if st["rc"] == 0 else 0)
        xh.copy_(xd, non_blocking=True)
        vh.copy_(vd, non_blocking=True)
        torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3
    e2e_ms = allreduce_max(world, e2e_ms)
    e2e_passes = allreduce_sum(world, e2e_passes)
    bytes_state = 2 * x0.numel() * 8

    fp64 = None
    if not args.skip_fp64:
        G64 = yb.System(scene, precision=0, pcg_rel_tol=PCG_TOL, newton_tol=ntol)
        xs, vs = x0.clone(), v0.clone()
        G64.step(xs, vs, raise_on_error=False)  # an assembly to tune on
        var, us = G64.autotune_pcg(30)
        tune["fp64"] = {"variant": var, "us_per_iter": [round(u, 2) for u in us]}
        fp64 = timed(G64, "fp64", args.steps, args.warmup, True)
        G64.close()

    peak, peak_kind = load_peaks()
    sp = mixed["prof"]["spmv"]
    spmv_gbs = sp["bytes"] / (sp["ms"] * 1e-3) / 1e9 if sp["count"] and sp["ms"] > 0 else None
    # dominant kernel: the persistent PCG kernel (one launch per solve / refinement sweep)
    pk = mixed["prof"]["pcg_kernel"]
    pk_gbs = pk["bytes"] / (pk["ms"] * 1e-3) / 1e9 if pk["count"] and pk["ms"] > 0 else None
    launch_s = pk["ms"] * 1e-3 / max(pk["count"], 1)
    rate = traffic_rate(["paper_2605_23088_b300/csrc/solver.cu"])
    roof = {"bound": "hbm", "kernel": "k_pcg_persistent<float,float> (block-Jacobi PCG, FP32 inner solve)",
            "achieved": pk_gbs, "peak": peak, "unit": "GB/s",
            "frac": (pk_gbs / peak) if pk_gbs else None,
            "traffic": rate * launch_s if rate else None, "peak_kind": peak_kind,
            "bytes_per_launch": pk["bytes"] / max(pk["count"], 1), "launch_us": launch_s * 1e6,
            "launches": pk["count"], "iterations_per_launch": mixed["pcg"] / max(pk["count"], 1),
            "spmv_phase_gbs": spmv_gbs}

    value = mixed["passes_all"] / (mixed["ms_max"] * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "Newton iterations/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mixed["ms_max"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32-mixed (f64 positions/gradients/energies)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_tets": n_tets, "n_nodes": G.n_nodes, "preroll_steps": preroll,
                   "newton_tol": "||dx||_inf/dt < 1e-2 m/s", "pcg_rel_tol": PCG_TOL,
                   "pairs_at_start": {"pt": npt, "ee": nee, "pg": npg}, "newton_iters": mixed["newton"],
                   "pcg_iters": mixed["pcg"], "statuses": sorted(set(mixed["status"])),
                   "l2": "inputs larger than L2 (BSR + element data > 126 MB): no flush",
                   "pcg_autotune": tune,
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "spmv_gbs": spmv_gbs,
        "roofline": roof,
        "stages_ms": {k: (v["ms"], v["count"]) for k, v in mixed["prof"].items()},
        "pcg_phase_us_per_iter": {k: v * 1e3 / max(mixed["pcg"], 1) for k, v in mixed["phases"].items()},
        "e2e": {"value": e2e_passes / (e2e_ms * 1e-3), "unit": "Newton iterations/s", "h2d_bytes_per_step": bytes_state,
                "d2h_bytes_per_step": bytes_state},
        "gpu_launches": mixed["launches"],
        "clocks": mixed["clocks"],
    }
    if fp64:
        sp64 = fp64["prof"]["spmv"]
        line["fp64_plain"] = {
            "value": fp64["passes_all"] / (fp64["ms_max"] * 1e-3), "unit": "Newton iterations/s",
            "ms_per_step": fp64["ms_max"] / args.steps, "newton_iters": fp64["newton"], "pcg_iters": fp64["pcg"],
            "spmv_gbs": sp64["bytes"] / (sp64["ms"] * 1e-3) / 1e9 if sp64["count"] and sp64["ms"] > 0 else None,
            "pcg_kernel_gbs": (fp64["prof"]["pcg_kernel"]["bytes"] / (fp64["prof"]["pcg_kernel"]["ms"] * 1e-3) / 1e9
                               if fp64["prof"]["pcg_kernel"]["ms"] > 0 else None),
            "stages_ms": {k: (v["ms"], v["count"]) for k, v in fp64["prof"].items()},
            "gpu_launches": fp64["launches"], "clocks": fp64["clocks"]}
    if not args.skip_batch:
        line["batch"] = batch_bench(args, dev)
    if rank == 0 and world == 1 and not args.skip_cpu:
        line["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    G.close()


# ---------------------------------------------------------------------------
BATCH_SCENES = 256


def batch_bench(args, dev):
    """The batching form on its own workload: 256 independent two-finger soft
    grippers closing on deformable objects (sizes log-uniform in 1k-20k tets),
    all in one system, one implicit step of every scene per call.  Reported
    per precision: scene-steps/s and Newton iterations/s summed over scenes;
    and, against it, the first 16 scenes stepped one system at a time."""
    import torch

    import paper_2605_23088_b300 as yb
    import scenes

    parts = scenes.gripper_batch(BATCH_SCENES)
    b = scenes.concat_scenes(parts)
    ntol = NEWTON_VEL_TOL * b["dt"]
    out = {"workload": f"{BATCH_SCENES} soft grippers on deformable objects (1k-20k tets each, log-uniform)",
           "n_scenes": BATCH_SCENES, "n_tets": int(len(b["tets"])), "steps": args.batch_steps,
           "newton_tol": "||dx||_inf/dt < 1e-2 m/s", "pcg_rel_tol": PCG_TOL}
    stream = torch.cuda.current_stream()
    for prec, name in ((1, "fp32_mixed"), (0, "fp64")):
        G = yb.System(b, precision=prec, pcg_rel_tol=PCG_TOL, newton_tol=ntol)
        x, v = G.initial_state()
        G.step(x, v, raise_on_error=False)  # warm-up
        var, us = G.autotune_pcg(30)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        newton = 0
        rcs = []
        e0.record(stream)
        for _ in range(args.batch_steps):
            st = G.step(x, v, raise_on_error=False)
            rcs.append(st["rc"])
            newton += int(G.scene_stats()[0].sum())
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3
        out[name] = {"scene_steps_per_s": BATCH_SCENES * args.batch_steps / sec, "newton_iters_per_s": newton / sec,
                     "ms_per_step": sec * 1e3 / args.batch_steps, "statuses": sorted(set(rcs)),
                     "pcg_autotune": {"variant": var, "us_per_iter": [round(u, 2) for u in us]}}
        G.close()
    # the same kind of work without batching: 16 scenes, one system each
    seq = 0.0
    nseq = 16
    for sc in parts[:nseq]:
        G = yb.System(sc, precision=1, pcg_rel_tol=PCG_TOL, newton_tol=ntol)
        x, v = G.initial_state()
        G.step(x, v, raise_on_error=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.batch_steps):
            G.step(x, v, raise_on_error=False)
        torch.cuda.synchronize()
        seq += time.perf_counter() - t0
        G.close()
    seq_rate = nseq * args.batch_steps / seq
    out["sequential_fp32_mixed"] = {"scenes": nseq, "scene_steps_per_s": seq_rate}
    out["batched_vs_sequential"] = out["fp32_mixed"]["scene_steps_per_s"] / seq_rate
    return out


# ---------------------------------------------------------------------------
def cpu_sample():
    """The oracle on a bounded sample: one vertical column of 2 of the 64 tori
    (same generator), one implicit time step from rest.  Scaled to the full
    workload by tet count."""
    import oracle
    import scenes

    sub = scenes.tori_scene(nx=1, ny=2, nz=1)
    full_tets = 64 * len(scenes.torus_mesh()[1])
    O = oracle.OracleSystem(sub)
    x, v = O.initial_state()
    t0 = time.perf_counter()
    x1, v1, rc, st = O.step(x, v)
    dt = time.perf_counter() - t0
    passes = st["newton_iters"] + (1 if rc == 0 else 0)
    scale = len(sub["tets"]) / full_tets
    return {"value": passes / dt * scale, "unit": "Newton iterations/s", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"one time step of a 2-torus column ({len(sub['tets'])} tets, "
                                        f"{passes} Newton iterations in {dt:.1f} s), scaled by {scale:.4f}"}


def cpu_baseline(args):
    return cpu_sample()


def reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vals = []
    for _ in range(max(1, args.steps)):
        vals.append(cpu_sample())
    v = statistics.median([c["value"] for c in vals])
    c = vals[0]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Newton iterations/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v if v else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": c["sample"]},
            "cpu_baseline": {"value": v, "unit": c["unit"], "cores": c["cores"], "kind": "oracle", "sample": c["sample"]},
            "e2e": {"value": v, "unit": "Newton iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--preroll", type=int, default=14)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-batch", action="store_true", help="leave out the batching-form measurement")
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--save-state", default=None, help="write the post-pre-roll state (.npz) for --load-state")
    ap.add_argument("--load-state", default=None, help="start from a state written by --save-state")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference(args)
    else:
        native(args)


if __name__ == "__main__":
    main()
