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
# Cap on Newton iterations per step (a safeguard; the paper states none).  The
# pile's impact steps need 80-310 iterations of projected Newton at this
# tolerance, so the cap sits well above that.
NEWTON_CAP = 1000
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


def alu_counts(kernel_file):
    """Per-tet FP64 / FP32 flop counts of the tet kernel from a committed ncu
    counter capture (profiles/snh_kernel_counts.json), if it was taken on the
    current source; else None."""
    p = os.path.join(ROOT, "profiles", "snh_kernel_counts.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    return d if d.get("source_sha") == source_sha(kernel_file) else None


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
def run_steps(system, x0, v0, steps, profile, world, host_io, label):
    """K implicit steps from (x0, v0).  host_io: every step copies x, v in from
    pinned host memory and the result back out (the end-to-end path through
    the C ABI with host buffers); the step itself is bracketed by CUDA events
    on the launching stream, the whole iteration by the host clock.  The
    steps sit inside the NVTX range `label` (for ncu --nvtx-include)."""
    import torch

    import paper_2605_23088_b300 as yb

    stream = torch.cuda.current_stream()
    xs, vs = x0.clone(), v0.clone()
    if host_io:
        xh, vh = x0.cpu().pin_memory(), v0.cpu().pin_memory()
    torch.cuda.synchronize()
    barrier(world)
    if profile:
        system.profile_enable(True)
    l0 = system.kernel_launches()
    per = []
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push(label)
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            if host_io:
                xs.copy_(xh, non_blocking=True)
                vs.copy_(vh, non_blocking=True)
            e0.record(stream)
            st = system.step(xs, vs, raise_on_error=False)
            e1.record(stream)
            if host_io:
                xh.copy_(xs, non_blocking=True)
                vh.copy_(vs, non_blocking=True)
            torch.cuda.synchronize()
            wall = (time.perf_counter() - t0) * 1e3
            per.append({"rc": st["rc"], "newton": st["newton_iters"],
                        "passes": st["newton_iters"] + (1 if st["rc"] == 0 else 0), "pcg": st["pcg_iters_total"],
                        "pairs": [st["n_pt"], st["n_ee"], st["n_pg"]], "ms": e0.elapsed_time(e1), "e2e_ms": wall})
        torch.cuda.nvtx.range_pop()
    launches = system.kernel_launches() - l0
    prof = {k: system.profile_get(i) for i, k in enumerate(yb.STAGE_NAMES)} if profile else None
    phases = system.pcg_phase_ms() if profile else None
    if profile:
        system.profile_enable(False)
    barrier(world)
    if host_io:
        xs.copy_(xh)
        vs.copy_(vh)
    return dict(per=per, launches=launches, prof=prof, phases=phases, clocks=clk.summary(), x=xs, v=vs)


def summarize(run, world, n=None):
    per = run["per"][:n] if n else run["per"]
    ms = sum(p["ms"] for p in per)
    e2e = sum(p["e2e_ms"] for p in per)
    passes = sum(p["passes"] for p in per)
    return dict(ms=ms, ms_max=allreduce_max(world, ms), e2e_max=allreduce_max(world, e2e),
                passes=passes, passes_all=allreduce_sum(world, passes), newton=sum(p["newton"] for p in per),
                pcg=sum(p["pcg"] for p in per), statuses=[p["rc"] for p in per])


def native(args):
    import torch

    import paper_2605_23088_b300 as yb
    import scenes

    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    L = args.lattice
    scene = scenes.tori_scene(nx=L, ny=L, nz=L)
    n_tets = len(scene["tets"])
    workload = WORKLOAD if L == 4 else (f"{L ** 3} Neo-Hookean tori on a {L}x{L}x{L} lattice (a small case of the "
                                        f"64-tori workload for profiling; {n_tets} tets)")
    ntol = NEWTON_VEL_TOL * scene["dt"]
    common = dict(pcg_rel_tol=PCG_TOL, newton_tol=ntol, newton_max_iter=NEWTON_CAP)
    G = yb.System(scene, precision=1, **common)
    x, v = G.initial_state()
    preroll = args.preroll
    pre_rc = []
    if args.load_state:
        # the state a pre-roll left (written by --save-state): skips the untimed pre-roll
        st = np.load(args.load_state)
        x.copy_(torch.as_tensor(st["x"], device=dev))
        v.copy_(torch.as_tensor(st["v"], device=dev))
        preroll = int(st["preroll"])
    else:
        # untimed pre-roll: let the pile fall until tori touch the ground and each other
        for _ in range(args.preroll):
            pre_rc.append(G.step(x, v, raise_on_error=False)["rc"])
    # untimed warm-up steps continue the same trajectory
    for _ in range(args.warmup):
        pre_rc.append(G.step(x, v, raise_on_error=False)["rc"])
    torch.cuda.synchronize()
    x0, v0 = x.clone(), v.clone()
    # the system holds the last step's assembly: pick the PCG launch configuration on it
    tune = {}
    var, us = G.autotune_pcg(30)
    tune["fp32_mixed"] = {"variant": var, "us_per_iter": [round(u, 2) for u in us]}
    if args.save_state and rank == 0:
        np.savez(args.save_state, x=x0.cpu().numpy(), v=v0.cpu().numpy(), preroll=preroll + args.warmup)
    npt, nee, npg = G.detect_pairs(x0)

    # FP32-mixed: the timed steps, each with its host copies (value: step time
    # on the device; e2e: the whole iteration through pinned host buffers)
    mixed_run = run_steps(G, x0, v0, args.steps, True, world, host_io=True, label="timed_fp32-mixed")
    mixed = summarize(mixed_run, world)
    bytes_state = 2 * x0.numel() * 8

    fp64 = None
    n64 = min(args.steps, args.fp64_steps)
    if not args.skip_fp64 and n64 > 0:
        G64 = yb.System(scene, precision=0, **common)
        xs, vs = x0.clone(), v0.clone()
        G64.step(xs, vs, raise_on_error=False)  # an assembly to tune on
        var, us = G64.autotune_pcg(30)
        tune["fp64"] = {"variant": var, "us_per_iter": [round(u, 2) for u in us]}
        fp64_run = run_steps(G64, x0, v0, n64, True, world, host_io=False, label="timed_fp64")
        fp64 = summarize(fp64_run, world)
        fp64["prof"] = fp64_run["prof"]
        fp64["launches"] = fp64_run["launches"]
        fp64["clocks"] = fp64_run["clocks"]
        fp64["x"] = fp64_run["x"]
        G64.close()

    peak, peak_kind = load_peaks()
    prof = mixed_run["prof"]
    sp = prof["spmv"]
    spmv_gbs = sp["bytes"] / (sp["ms"] * 1e-3) / 1e9 if sp["count"] and sp["ms"] > 0 else None
    # dominant kernel: the persistent PCG kernel (one launch per solve / refinement sweep)
    pk = prof["pcg_kernel"]
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

    # secondary rooflines: the assembly (HBM; the local evaluation with its
    # scatter, fused) and the tet kernel (FP64 pipe, against the live FMA probe)
    nnzb = G.bsr_nnzb(0) + G.bsr_nnzb(1)
    pairs_mean = sum(sum(p["pairs"]) for p in mixed_run["per"]) / max(len(mixed_run["per"]), 1)
    es = 4  # FP32 Hessian blocks in the mixed form; positions, material, gradient FP64
    asm_bytes = n_tets * (16 + 96 + 96) + nnzb * 9 * es + G.n_nodes * (9 * es + 24) + pairs_mean * 12
    ev = prof["eval"]
    asm_s = ev["ms"] * 1e-3 / max(ev["count"], 1)
    secondary = {"assembly": {"bound": "hbm", "kernels": "local evaluation + scatter (tet, barrier, inertia)",
                              "bytes_per_eval": asm_bytes, "eval_us": asm_s * 1e6,
                              "achieved": asm_bytes / asm_s / 1e9 if asm_s > 0 else None, "peak": peak,
                              "unit": "GB/s", "frac": asm_bytes / asm_s / 1e9 / peak if asm_s > 0 else None}}
    cnt = alu_counts("paper_2605_23088_b300/csrc/elements.cu")
    tt = prof["tet"]
    if cnt and tt["count"] and tt["ms"] > 0:
        t_s = tt["ms"] * 1e-3 / tt["count"]
        f64_peak, f32_peak = yb.probe_fma_tflops(0), yb.probe_fma_tflops(1)
        a64 = cnt["fp64_flops_per_tet"] * n_tets / t_s / 1e12
        a32 = cnt["fp32_flops_per_tet"] * n_tets / t_s / 1e12
        secondary["k_snh<float>"] = {"bound": "alu", "pipe": "fp64", "achieved": a64, "peak": f64_peak,
                                     "unit": "TFLOP/s", "frac": a64 / f64_peak, "launch_us": t_s * 1e6,
                                     "fp32_achieved": a32, "fp32_peak": f32_peak, "fp32_frac": a32 / f32_peak,
                                     "peak_kind": "measured (FMA probe, this run)",
                                     "flops_per_tet": [cnt["fp64_flops_per_tet"], cnt["fp32_flops_per_tet"]]}

    value = mixed["passes_all"] / (mixed["ms_max"] * 1e-3)
    per_step = [{"rc": p["rc"], "newton": p["newton"], "pcg": p["pcg"], "pairs_pt_ee_pg": p["pairs"],
                 "ms": round(p["ms"], 2)} for p in mixed_run["per"]]
    line = {
        "metric": METRIC, "value": value, "unit": "Newton iterations/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mixed["ms_max"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32-mixed (f64 positions/gradients/energies)",
        "data": "synthetic",
        "config": {"workload": workload, "n_tets": n_tets, "n_nodes": G.n_nodes,
                   "preroll_steps": preroll, "timed_steps": f"{preroll + args.warmup}..{preroll + args.warmup + args.steps - 1}",
                   "newton_tol": "||dx||_inf/dt < 1e-2 m/s", "newton_max_iter": NEWTON_CAP, "pcg_rel_tol": PCG_TOL,
                   "pairs_at_start": {"pt": npt, "ee": nee, "pg": npg}, "newton_iters": mixed["newton"],
                   "pcg_iters": mixed["pcg"], "statuses": mixed["statuses"],
                   "preroll_statuses": sorted(set(pre_rc)), "per_step": per_step,
                   "l2": "inputs larger than L2 (BSR + element data > 126 MB): no flush",
                   "pcg_autotune": tune,
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "spmv_gbs": spmv_gbs,
        "roofline": roof,
        "secondary_rooflines": secondary,
        "stages_ms": {k: (v_["ms"], v_["count"]) for k, v_ in prof.items()},
        "pcg_phase_us_per_iter": {k: v_ * 1e3 / max(mixed["pcg"], 1) for k, v_ in mixed_run["phases"].items()},
        "e2e": {"value": mixed["passes_all"] / (mixed["e2e_max"] * 1e-3), "unit": "Newton iterations/s",
                "h2d_bytes_per_step": bytes_state, "d2h_bytes_per_step": bytes_state,
                "steps": "the same timed steps as value, each with its host copies"},
        "gpu_launches": mixed_run["launches"],
        "clocks": mixed_run["clocks"],
    }
    if fp64:
        sp64 = fp64["prof"]["spmv"]
        same = summarize(mixed_run, world, n64)
        dx = float((fp64["x"] - mixed_run["x"]).abs().max()) if n64 == args.steps else None
        line["fp64_plain"] = {
            "value": fp64["passes_all"] / (fp64["ms_max"] * 1e-3), "unit": "Newton iterations/s",
            "steps": n64, "statuses": fp64["statuses"],
            "ms_per_step": fp64["ms_max"] / n64, "newton_iters": fp64["newton"], "pcg_iters": fp64["pcg"],
            "fp32_mixed_same_steps": same["passes_all"] / (same["ms_max"] * 1e-3),
            "spmv_gbs": sp64["bytes"] / (sp64["ms"] * 1e-3) / 1e9 if sp64["count"] and sp64["ms"] > 0 else None,
            "pcg_kernel_gbs": (fp64["prof"]["pcg_kernel"]["bytes"] / (fp64["prof"]["pcg_kernel"]["ms"] * 1e-3) / 1e9
                               if fp64["prof"]["pcg_kernel"]["ms"] > 0 else None),
            "stages_ms": {k: (v_["ms"], v_["count"]) for k, v_ in fp64["prof"].items()},
            "gpu_launches": fp64["launches"], "clocks": fp64["clocks"]}
        if dx is not None:
            line["fp64_plain"]["max_dx_vs_fp32_mixed_m"] = dx
    if not args.skip_spmv_study:
        line["spmv_study"] = spmv_study(G)
        line["spmv_scaling"] = spmv_scaling()
        line["projection_study"] = projection_study()
    if not args.skip_batch:
        line["batch"] = batch_bench(args, dev)
    if rank == 0 and world == 1 and not args.skip_cpu:
        line["cpu_baseline"], line["accuracy"] = cpu_baseline_and_accuracy(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    G.close()
    bad = [s_ for s_ in mixed["statuses"] if s_ != 0] + ([s_ for s_ in fp64["statuses"] if s_ != 0] if fp64 else [])
    if bad:
        print(f"bench: {len(bad)} timed step(s) did not converge (statuses {sorted(set(bad))})", file=sys.stderr)
        sys.exit(3)


# ---------------------------------------------------------------------------
def spmv_layouts(row_u, col_u, vals_u, diag, perm=None):
    """The four layouts of the SpMV study from the upper blocks of a symmetric
    block matrix (host arrays), optionally after renumbering node i as
    perm[i]: (diag, {layout: (row, col, vals)}).  Upper layouts keep row <
    col (a block that the renumbering turns around is transposed), the full
    ones carry both triangles; BSR and BCOO layouts are the same sorted
    arrays, read by different kernels."""
    row_u, col_u = np.asarray(row_u, np.int64), np.asarray(col_u, np.int64)
    vals_u = np.asarray(vals_u).reshape(-1, 3, 3)
    if perm is not None:
        r, c = perm[row_u], perm[col_u]
        swap = r > c
        vals_u = vals_u.copy()
        vals_u[swap] = vals_u[swap].transpose(0, 2, 1)
        row_u, col_u = np.where(swap, c, r), np.where(swap, r, c)
        d = np.empty_like(diag)
        d[perm] = diag
        diag = d
    o = np.lexsort((col_u, row_u))
    upper = (row_u[o].astype(np.int32), col_u[o].astype(np.int32), np.ascontiguousarray(vals_u[o]))
    R = np.concatenate([row_u, col_u])
    C = np.concatenate([col_u, row_u])
    V = np.concatenate([vals_u, vals_u.transpose(0, 2, 1)])
    o2 = np.lexsort((C, R))
    full = (R[o2].astype(np.int32), C[o2].astype(np.int32), np.ascontiguousarray(V[o2]))
    return diag, {"upper_bsr": upper, "full_bsr": full, "full_bcoo": full, "upper_bcoo": upper}


def spmv_scaling(lattices=(1, 2, 3, 4), reps=10):
    """The shape of the paper's SpMV experiment (Sec. "Evaluation"): the
    elastic (stable Neo-Hookean) Hessian of N objects, vertices randomly
    renumbered, time per call of every layout as N grows; here N = 1, 8, 27,
    64 tori of the workload's generator at rest (no contact), FP32 and FP64."""
    import torch

    import paper_2605_23088_b300 as yb
    import scenes

    out = {"tori": [], "upper_blocks": [], "us": {}}
    for L in lattices:
        sc = scenes.tori_scene(nx=L, ny=L, nz=L)
        G = yb.System(sc, precision=1)
        x, _ = G.initial_state()
        G.eval_local(x, x, term_mask=yb.TERM_TET, project=True)
        st = spmv_study(G, reps=reps, orders=("permuted",))
        out["tori"].append(L ** 3)
        out["upper_blocks"].append(st["upper_blocks"])
        for k, v in st.items():
            if isinstance(v, dict):
                out["us"].setdefault(k, []).append(round(v["us"], 2))
        G.close()
        torch.cuda.synchronize()
    return out


def spmv_study(G, reps=20, orders=("natural", "permuted")):
    """Time y = A x on the system's current matrix in every layout and
    precision, natural node order and a seeded random renumbering, with L2
    flushed before every timed call; GB/s of algorithmic bytes (blocks and
    their indices, diagonal, x and y once) against the measured HBM peak."""
    import torch

    import paper_2605_23088_b300 as yb

    n = G.n_nodes
    rows, cols, vals = [], [], []
    diag = None
    for which in (0, 1):
        rp, col, blk, dg = G.export_bsr(which)
        rows.append(np.repeat(np.arange(n), np.diff(rp)))
        cols.append(col)
        vals.append(blk)
        if which == 0:
            diag = dg
    row_u, col_u, vals_u = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    peak, kind = load_peaks()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # twice the L2
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(3)
    x64 = rng.normal(size=(n, 3))
    out = {"n_nodes": n, "upper_blocks": int(len(row_u)), "peak_gbs": peak, "peak_kind": kind, "reps": reps,
           "l2": "flushed before every call (256 MB write)"}
    ref = None
    for order in orders:
        perm = None if order == "natural" else rng.permutation(n)
        d, lay = spmv_layouts(row_u, col_u, vals_u, diag, perm)
        xo = x64 if perm is None else x64[np.argsort(perm)]  # x in the new numbering: x'[perm[i]] = x[i]
        for prec, dt, nbyte in ((1, torch.float32, 4), (0, torch.float64, 8)):
            X = torch.as_tensor(xo, dtype=dt, device="cuda")
            D = torch.as_tensor(d, dtype=dt, device="cuda")
            for name in yb.SPMV_FORMATS:
                r_, c_, v_ = lay[name]
                R_ = torch.as_tensor(r_, device="cuda")
                C_ = torch.as_tensor(c_, device="cuda")
                V_ = torch.as_tensor(v_, dtype=dt, device="cuda")
                Y = torch.empty_like(X)
                flag = torch.zeros(1, dtype=torch.int32, device="cuda")
                fmt = yb.SPMV_FORMATS.index(name)
                for _ in range(3):  # untimed warm-up calls
                    yb.spmv_format(fmt, n, R_, C_, V_, D, X, Y, flag)
                ms = []
                for _ in range(reps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    yb.spmv_format(fmt, n, R_, C_, V_, D, X, Y, flag)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms.append(e0.elapsed_time(e1))
                y = Y.double().cpu().numpy()
                if perm is not None:
                    y = y[perm]  # back to the natural numbering
                if ref is None:
                    ref = y
                err = float(np.abs(y - ref).max() / np.abs(ref).max())
                nb = len(r_)
                algo = nb * (9 * nbyte + 8) + n * 9 * nbyte + 2 * 3 * nbyte * n
                t = statistics.median(ms) * 1e-3
                out[f"{order}_{'fp32' if prec else 'fp64'}_{name}"] = {
                    "us": t * 1e6, "gbs": algo / t / 1e9, "frac": algo / t / 1e9 / peak, "bytes": algo,
                    "max_rel_diff_vs_first": err, "flag": int(flag.item())}
    return out


# ---------------------------------------------------------------------------
def pp_barrier_hessians(count, dhat=1e-3, kappa=1e4, seed=5):
    """Synthetic point-point barrier Hessians (the projection study's inputs):
    pairs at distances 0.1-0.9 dhat in random directions; position-space 6 x 6
    Hessians kappa (b'' grad s grad s^T + b' hess s) of the barrier
    -(s - sh)^2 ln(s / sh), s = |p - a|^2, and their node-space images through
    the UNION Jacobians for a free and an affine vertex (15 x 15) and for two
    affine vertices (24 x 24), with body-relative offsets r of a few cm."""
    rng = np.random.default_rng(seed)
    sh = dhat * dhat
    d = dhat * rng.uniform(0.1, 0.9, count)
    u = rng.normal(size=(count, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    w = d[:, None] * u
    s_ = d * d
    L = np.log(s_ / sh)
    db = -2.0 * (s_ - sh) * L - (s_ - sh) ** 2 / s_
    d2b = -2.0 * L - 4.0 * (s_ - sh) / s_ + (s_ - sh) ** 2 / s_ ** 2
    g = np.concatenate([2 * w, -2 * w], axis=1)
    I3 = np.eye(3)
    hs = 2.0 * np.block([[I3, -I3], [-I3, I3]])
    H6 = kappa * (d2b[:, None, None] * g[:, :, None] * g[:, None, :] + db[:, None, None] * hs[None])
    def union_J(r):  # 3 x 12: [I3, r1 I3, r2 I3, r3 I3]
        return np.concatenate([I3] + [ri * I3 for ri in r], axis=1)
    r1 = rng.uniform(-0.05, 0.05, (count, 3))
    r2 = rng.uniform(-0.05, 0.05, (count, 3))
    H15 = np.empty((count, 15, 15))
    H24 = np.empty((count, 24, 24))
    for k in range(count):
        J15 = np.zeros((6, 15))
        J15[:3, :3] = I3
        J15[3:, 3:] = union_J(r1[k])
        H15[k] = J15.T @ H6[k] @ J15
        J24 = np.zeros((6, 24))
        J24[:3, :12] = union_J(r1[k])
        J24[3:, 12:] = union_J(r2[k])
        H24[k] = J24.T @ H6[k] @ J24
    # the library's PP form: the 3 x 3 in w = p - a (K = 2 H_w)
    H3 = kappa * (d2b[:, None, None] * 4 * w[:, :, None] * w[:, None, :] + db[:, None, None] * 2 * I3[None]) * 2
    return {24: H24, 15: H15, 6: H6, 3: H3}


def projection_study(count=16384, reps=5):
    """EVD micro-benchmark (Sec. "Eigendecomposition: Automatic Optimization",
    the 24 / 15 / 6 sizes): time of projecting point-point barrier Hessians
    in node space (24 x 24 between two affine vertices, 15 x 15 between a free
    and an affine one), in position space (6 x 6) and in the reduced variable
    w = p - a (3 x 3, what the library's barrier kernel does), per precision."""
    import torch

    import paper_2605_23088_b300 as yb

    mats = pp_barrier_hessians(count)
    stream = torch.cuda.current_stream()
    out = {"pairs": count, "reps": reps}
    for prec, dt in ((1, torch.float32), (0, torch.float64)):
        t = {}
        for n, H in mats.items():
            Hd = torch.as_tensor(H, dtype=dt, device="cuda")
            Od = torch.empty_like(Hd)
            yb.project_batch(Hd, Od)
            ms = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                yb.project_batch(Hd, Od)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            t[n] = statistics.median(ms) * 1e3 / count  # microseconds per pair
        name = "fp32" if prec else "fp64"
        out[name] = {"us_per_pair": {str(k): v for k, v in t.items()},
                     "speedup_24_to_6": t[24] / t[6], "speedup_15_to_6": t[15] / t[6], "speedup_6_to_3": t[6] / t[3],
                     "speedup_24_to_3": t[24] / t[3]}
    return out


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
    if not args.skip_cpu:
        out["accuracy"] = batch_accuracy(parts[:8])
    return out


def batch_accuracy(parts):
    """The batched FP32-mixed form against the FP64 oracle: a batch of the
    given scenes takes one Newton iteration (PCG to 1e-10) from the initial
    state; the smallest scene's positions are compared with one Newton
    iteration of the oracle on that scene alone."""
    import torch

    import oracle
    import paper_2605_23088_b300 as yb
    import scenes

    b = scenes.concat_scenes(parts)
    G = yb.System(b, precision=1, pcg_rel_tol=1e-10, newton_tol=0.0, newton_max_iter=1)
    x, v = G.initial_state()
    G.step(x, v, raise_on_error=False)
    xb = x.cpu().numpy()
    G.close()
    # nodes of each scene: its free (unfixed) vertices, in vertex order
    sizes = []
    for sc in parts:
        free = np.ones(len(sc["rest_pos"]), bool)
        free[np.asarray(sc["fixed"], int)] = False
        sizes.append(int(free.sum()))
    k = int(np.argmin([len(sc["tets"]) for sc in parts]))
    off = int(np.sum(sizes[:k]))
    sc = parts[k]
    O = oracle.OracleSystem(sc, pcg_tol=1e-10)
    x0, v0 = O.initial_state()
    # a step first moves the prescribed (fixed) vertices by h times their velocity
    Pf = O.fixed_positions()
    fx = np.asarray(sc["fixed"], int)
    Pf[fx] += sc["dt"] * np.asarray(sc["fixed_vel"]).reshape(-1, 3)
    O.set_fixed_positions(Pf)
    x1, _ = oracle_newton_iteration(O, x0, O.xtilde(x0, v0), 1e-10)
    err = float(np.abs(xb[off:off + sizes[k]] - x1).max())
    return {"sample": f"scene {k} of a batch of {len(parts)} ({len(parts[k]['tets'])} tets), one Newton iteration "
                      f"from the initial state, PCG to 1e-10, against the oracle on that scene alone",
            "fp32_mixed_position_err_m": err, "position_err_rel_bbox": err / parts[k]["bbox_diag"]}


# ---------------------------------------------------------------------------
def torus_impact_sample():
    """A bounded sample of the workload: one torus of the same generator
    (first orientation and modulus), its lowest vertex 0.3 mm above the ground
    and falling at 0.5 m/s, so the first Newton iterations carry contact."""
    import scenes

    s = dict(scenes.tori_scene(nx=1, ny=1, nz=1))
    P = s["rest_pos"]
    s["rest_pos"] = P - np.array([0.0, P[:, 1].min() - 3e-4, 0.0])
    s["vel0"] = np.tile([0.0, -0.5, 0.0], (len(P), 1))
    return s


def oracle_newton_iteration(O, x, xt, pcg_tol):
    """One Newton iteration of the oracle, composed from its calls in the order
    of its own step: projected assembly, PCG, CCD bound, halving line search."""
    g = O.assemble(x, xt, project=True)
    p, _, _ = O.pcg(g, tol=pcg_tol)
    alpha = O.ccd_bound(x, p)
    E0 = O.energy(x, xt)
    x1 = x
    for _ in range(30):
        x1 = x - alpha * p
        if O.energy(x1, xt) <= E0 + 1e-12 * abs(E0):
            break
        alpha *= 0.5
    return x1, p


def oracle_iterations(budget_s, max_iters):
    """The oracle's Newton iterations on the sample until budget_s has passed
    (at least one): (iterations, seconds, tets of the sample, threads)."""
    import oracle

    s = torus_impact_sample()
    O = oracle.OracleSystem(s, pcg_tol=PCG_TOL, newton_tol=NEWTON_VEL_TOL * s["dt"])
    x, v = O.initial_state()
    xt = O.xtilde(x, v)
    n, t0 = 0, time.perf_counter()
    while n < max_iters and (n == 0 or time.perf_counter() - t0 < budget_s):
        x, p = oracle_newton_iteration(O, x, xt, PCG_TOL)
        n += 1
        if np.abs(p).max() <= NEWTON_VEL_TOL * s["dt"]:
            x, v = O.initial_state()  # the sample's step converged: start it again
    return n, time.perf_counter() - t0, len(s["tets"]), oracle.num_threads()


def cpu_baseline_and_accuracy(args):
    """cpu_baseline: the oracle's Newton iterations on the one-torus sample for
    about 15 s, scaled to the workload by tet count.  accuracy: the GPU forms
    against the FP64 oracle on the same sample, teacher-forced (both start
    from the oracle's state): the Newton direction solved to 1e-10 relative
    residual, and the positions after one Newton iteration (CCD bound and line
    search included) with both solves at 1e-10."""
    import torch

    import oracle
    import paper_2605_23088_b300 as yb
    import scenes

    n, sec, tets, cores = oracle_iterations(15.0, 50)
    full_tets = 64 * len(scenes.torus_mesh()[1])
    scale = tets / full_tets
    base = {"value": n / sec * scale, "unit": "Newton iterations/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} Newton iterations of one torus striking the ground ({tets} tets) in {sec:.1f} s, "
                      f"scaled by {scale:.4f}"}
    s = torus_impact_sample()
    O = oracle.OracleSystem(s, pcg_tol=1e-10)
    x, v = O.initial_state()
    xt = O.xtilde(x, v)
    x1_ref, p_ref = oracle_newton_iteration(O, x, xt, 1e-10)
    bbox = s["bbox_diag"]
    acc = {"sample": "one torus striking the ground (16,944 tets), teacher-forced from the oracle's state",
           "tolerance_basis": "direction: PCG to 1e-10 on both sides; positions: one Newton iteration, PCG 1e-10"}
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    for prec, name in ((1, "fp32_mixed"), (0, "fp64")):
        G = yb.System(s, precision=prec, pcg_rel_tol=1e-10, newton_tol=0.0, newton_max_iter=1)
        G.detect_pairs(T(x))
        G.eval_local(T(x), T(xt))
        p, _, _ = G.pcg_solve(G.export_gradient(), rel_tol=1e-10)
        dp = float(np.abs(p.cpu().numpy() - p_ref).max() / np.abs(p_ref).max())
        xg, vg = T(x), T(v)
        G.step(xg, vg, raise_on_error=False)  # one Newton iteration (the cap), then E_NOCONV
        dx = float(np.abs(xg.cpu().numpy() - x1_ref).max())
        acc[name] = {"direction_rel_err": dp, "position_err_m": dx, "position_err_rel_bbox": dx / bbox}
        G.close()
    return base, acc


def reference(args):
    """The oracle as it stands on the host cores: every step is one Newton
    iteration of the one-torus sample (a bounded sample of the workload),
    continuing its Newton solve; value scaled to the workload by tet count."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import scenes

    steps = max(1, args.steps)
    oracle_iterations(0.0, 1)  # one untimed iteration (builds and pages in the oracle)
    n, sec, tets, cores = oracle_iterations(1e30, steps)
    scale = tets / (64 * len(scenes.torus_mesh()[1]))
    v = n / sec * scale
    sample = (f"{n} Newton iterations of one torus striking the ground ({tets} tets; the workload's generator) "
              f"in {sec:.1f} s, scaled by {scale:.4f} to the 64-torus workload")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Newton iterations/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample,
                       "ms_per_step_note": "measured per sample iteration, not scaled"},
            "cpu_baseline": {"value": v, "unit": "Newton iterations/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
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
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed FP64 steps (the first of the timed steps)")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-batch", action="store_true", help="leave out the batching-form measurement")
    ap.add_argument("--skip-spmv-study", action="store_true", help="leave out the SpMV layout study")
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--save-state", default=None, help="write the post-pre-roll state (.npz) for --load-state")
    ap.add_argument("--load-state", default=None, help="start from a state written by --save-state")
    ap.add_argument("--lattice", type=int, default=4,
                    help="tori per lattice edge (4: the 64-tori workload; smaller: a small case for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference(args)
    else:
        native(args)


if __name__ == "__main__":
    main()
