"""Benchmark of the D3Q27 colour-gradient central-moment LB step on GB300.

One "step" is one full time step of the method over the whole lattice (boundary planes,
phase field, fused collide-perturb-recolour with pull streaming).  The default workload
is the 96x96x384 liquid-liquid jet (D = 16, u = 0.05, gamma = 1.5, Re = 2000, We = 100,
1% inlet noise, convective outflow), FP32 populations; its 1.53 GB state is larger than
the 129 MB L2, so no flush is needed between steps.

Prints one JSON line.  With torchrun (N > 1 ranks) every rank advances its own replica of
the lattice (weak scaling; there is no data exchange), times are maxed over ranks.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "MLUPS & % HBM peak, FP32 vs FP16-storage at stated error; adjoint/forward ratio"
# algorithmic bytes per node update (FP32): 54 population reads + 54 writes + rho_r/rho_b
# write and read (the method's minimum; the step's two passes also write and read the 48-byte
# collision moments).  Per kernel: moment_kernel reads 54 populations and writes the 8-byte
# phase entry and the 48-byte moments; collide_kernel reads the moments and the phase
# entries of its stencil (8 B per node once cached) and writes 54 populations.
BYTES_STEP = 448
BYTES_MOMENTS = 48
BYTES_KERNEL = {"collide_kernel": 216 + 8 + BYTES_MOMENTS, "moment_kernel": 216 + 8 + BYTES_MOMENTS}
# FP16 storage: 26 half2 (4 B) + one float2 rest (8 B) = 112 B of populations per node; the
# phase entries are float4 (16 B).  moment_kernel: read 112 + own previous entry 16, write the
# entry 16 + moments 48; collide_kernel: read the moments 48 + the stencil's entries 16, write
# 112.
BYTES_STEP_FP16 = 112 + 112 + 16 + 16
BYTES_KERNEL_FP16 = {"collide_kernel": 112 + 16 + BYTES_MOMENTS, "moment_kernel": 112 + 2 * 16 + BYTES_MOMENTS}
# fitted FP16 encoding: the same bytes (the FP8 odd fit is packed into the 16-byte phase entry)
BYTES_STEP_FIT = BYTES_STEP_FP16
BYTES_KERNEL_FIT = dict(BYTES_KERNEL_FP16)
STORAGE_TEXT = {
    1: "moving populations as half-precision deviations from the reading node's rest equilibrium, "
       "rest population FP32",
    2: "moving populations as half-precision deviations from a prediction of the reading node "
       "(rho_k (1 - alpha-bar) k_q plus an FP8 least-squares odd fit of its previous gather, packed "
       "in its 16-byte phase entry), rest population FP32"}


def adjoint_leg(lb, torch, name="jet64", T=500, objective="area", args=(1e-3,), checkpoint=0):
    """Cost of lb_adjoint (T steps forward with ceil(sqrt T) checkpoints, objective, reverse
    sweep) against lb_step(T) from the same state, both timed with CUDA events."""
    cfg = workloads.CONFIGS[name]
    nx, ny, nz = cfg["grid"]
    lat = lb.Lattice((nx, ny, nz), cfg["params"], bc=cfg["bc"])
    lat.init_jet()
    lat.step(20)
    state = lat.save()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    lat.adjoint(T, objective, args, checkpoint)  # workspace allocation and warm-up
    lat.load(state)
    torch.cuda.synchronize()
    ev[0].record(lat.stream)
    lat.step(T)
    ev[1].record(lat.stream)
    torch.cuda.synchronize()
    lat.load(state)
    torch.cuda.synchronize()
    ev[2].record(lat.stream)
    J, g = lat.adjoint(T, objective, args, checkpoint)
    ev[3].record(lat.stream)
    torch.cuda.synchronize()
    fwd, adj = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    k = checkpoint if checkpoint > 0 else int(np.ceil(np.sqrt(T)))
    lat.close()
    del lat
    torch.cuda.empty_cache()
    return {"workload": cfg["text"], "T": T, "checkpoint_interval": k, "objective": objective,
            "objective_args": list(args), "J": J, "grad_norm": float(np.linalg.norm(g)),
            "forward_ms": fwd, "adjoint_ms": adj, "ratio": adj / fwd,
            "work": "T forward steps with checkpoints + T recomputed forward steps + T reverse steps",
            "precision": "FP32 kernels, FP64 parameter-gradient accumulation"}


def fp16_error(lb, cfg, steps, storage=1):
    """FP16 (either encoding) against FP32 storage on the same workload after `steps` steps:
    relative L2 error of the velocity and largest change of the order parameter."""
    import torch
    out = {}
    lats = [lb.Lattice(cfg["grid"], dict(cfg["params"], storage=s), bc=cfg["bc"]) for s in (0, storage)]
    for l in lats:
        l.init_jet() if cfg["init"]["kind"] == "jet" else l.init_droplet(cfg["init"]["R"], cfg["init"]["W"])
        l.step(steps)
    F = [l.fields(names=("phi", "ux", "uy", "uz")) for l in lats]
    du = torch.stack([F[1][k] - F[0][k] for k in ("ux", "uy", "uz")]).double()
    u32 = torch.stack([F[0][k] for k in ("ux", "uy", "uz")]).double()
    out = {"steps": steps, "rel_u_l2": float(du.norm() / u32.norm()),
           "max_abs_dphi": float((F[1]["phi"] - F[0]["phi"]).abs().max())}
    for l in lats:
        l.close()
    torch.cuda.empty_cache()
    return out


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profile_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken from the
    current kernel source (its sha256 is recorded in the summary)."""
    import hashlib
    src = os.path.join(ROOT, "paper_1804_08923_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(src)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(src, f), "rb").read())
    sha = h.hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    try:
        kv = {}
        for line in open(path):
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("source_sha256_16") != sha:
            return None
        return float(kv["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(prefix="clocks", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.out.close()

    def summary(self):
        try:
            rows = [l.split(",") for l in open(self.out.name).read().strip().splitlines() if l.strip()]
            os.unlink(self.out.name)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def cpu_baseline(cfg, seconds_target=15.0):
    """The FP64 oracle as it stands, on the host cores, over a bounded sample of the
    workload: whole oracle steps of the full lattice from the workload's initial state."""
    import oracle
    nx, ny, nz = cfg["grid"]
    lat = oracle.Lattice(oracle.make_grid(nx, ny, nz, *cfg["bc"]), oracle.make_params(cfg["params"]))
    lat.init_jet() if cfg["init"]["kind"] == "jet" else lat.init_droplet(cfg["init"]["R"], cfg["init"]["W"])
    t0 = time.perf_counter()
    lat.step(1)
    steps = 1
    el = time.perf_counter() - t0
    while el + el / steps < seconds_target:
        lat.step(1)
        steps += 1
        el = time.perf_counter() - t0
    el = time.perf_counter() - t0
    return {"value": nx * ny * nz * steps / el / 1e6, "unit": "MLUPS", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"{steps} full FP64 oracle step(s) of the {nx}x{ny}x{nz} lattice "
                                        f"({el:.1f} s)"}


def run_reference(args, cfg):
    """Reference arm: the FP64 oracle on the host cores, timed on bounded samples of the
    workload (a z-slab of the lattice with the same boundaries and parameters)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    nx, ny, nz = cfg["grid"]
    # slab depth sized so that W + K oracle steps take about two minutes
    probe = oracle.Lattice(oracle.make_grid(nx, ny, 4, *cfg["bc"]), oracle.make_params(cfg["params"]))
    probe.init_jet()
    t0 = time.perf_counter()
    probe.step(1)
    rate = nx * ny * 4 / (time.perf_counter() - t0)
    budget = 120.0 / max(1, args.steps + args.warmup)
    nzs = int(max(3, min(nz, rate * budget / (nx * ny))))
    lat = oracle.Lattice(oracle.make_grid(nx, ny, nzs, *cfg["bc"]), oracle.make_params(cfg["params"]))
    lat.init_jet()
    lat.step(args.warmup)
    t0 = time.perf_counter()
    lat.step(args.steps)
    el = time.perf_counter() - t0
    nodes = nx * ny * nzs
    v = nodes * args.steps / el / 1e6
    sample = f"{nx}x{ny}x{nzs} slab of the {nx}x{ny}x{nz} lattice, same boundaries and parameters"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_block(cfg),
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def reduce_max(v, dist, device):
    """Largest value over the ranks (the slowest rank times the job); identity without a group."""
    if dist is None or not dist.is_initialized():
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(nodes_per_rank, steps, world, ms_max):
    """Whole-job throughput: every rank advances its own lattice (replicas, weak scaling)."""
    return nodes_per_rank * steps * world / (ms_max * 1e-3) / 1e6


def config_block(cfg):
    nx, ny, nz = cfg["grid"]
    return {"workload": f"{cfg['name']}: {cfg['text']}", "lattice": [nx, ny, nz], "nodes": nx * ny * nz,
            "storage": "fp32 SoA populations [k][i][z][y][x]",
            "l2": "state 2 x 54 x 4 B x nodes > 129 MB L2; no flush between steps",
            "parallelism": "one lattice per GPU (replicas, no exchange)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="jet96")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp16", action="store_true")
    ap.add_argument("--error-steps", type=int, default=500)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-paper-workload", action="store_true")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="only the adjoint leg (lb_adjoint against lb_step on the 64x64x256 jet)")
    ap.add_argument("--adjoint-steps", type=int, default=500)
    ap.add_argument("--adjoint-checkpoint", type=int, default=0)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    cfg = workloads.CONFIGS[args.config]
    if args.impl == "reference":
        return run_reference(args, cfg)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import paper_1804_08923_gb300 as lb
    if args.adjoint_only:
        if rank == 0:
            print(json.dumps({"adjoint": adjoint_leg(lb, torch, T=args.adjoint_steps,
                                                     checkpoint=args.adjoint_checkpoint)}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    nx, ny, nz = cfg["grid"]
    nodes = nx * ny * nz
    lat = lb.Lattice(cfg["grid"], cfg["params"], bc=cfg["bc"])
    lat.init_jet() if cfg["init"]["kind"] == "jet" else lat.init_droplet(cfg["init"]["R"], cfg["init"]["W"])
    stream = lat.stream

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
            torch.cuda.synchronize()

    def max_over_ranks(v):
        return reduce_max(v, dist, "cuda")

    # ---- warm-up, then the timed region (device events on the library's stream)
    lat.step(args.warmup)
    barrier()
    l0 = lat.kernel_launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        lat.step(args.steps)
        e1.record(stream)
        barrier()
    launches = lat.kernel_launches - l0
    ms = max_over_ranks(e0.elapsed_time(e1))
    ms_step = ms / args.steps
    value = job_mlups(nodes, args.steps, world, ms)
    clocks = clk.summary()

    # ---- per-kernel durations over a second timed pass of the same length
    lat.profile_enable(args.steps)
    barrier()
    lat.step(args.steps)
    prof = lat.profile_read()
    lat.profile_enable(0)
    peak, peak_kind = measured_peaks()
    k_ms, k_n = prof["collide_kernel"]
    coll_ms = k_ms / max(k_n, 1)
    achieved = BYTES_KERNEL["collide_kernel"] * nodes / (coll_ms * 1e-3) / 1e9
    traffic = profile_traffic("collide_kernel", cfg["name"])
    kernels = {name: {"avg_ms": t / max(n, 1), "launches": n,
                      "share": t / max(sum(v[0] for v in prof.values()), 1e-30)} for name, (t, n) in prof.items() if n}
    roofline = {"bound": "hbm", "kernel": "collide_kernel", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"hbm_gbs of {peak_kind}",
                "algorithmic_bytes_per_node": BYTES_KERNEL["collide_kernel"],
                "traffic": traffic * 1.0 if traffic is not None else None}

    # ---- the same workload with the paper's free-slip side walls (Section IV.A) in place of
    #      periodic x and y: throughput only
    sw = lb.Lattice(cfg["grid"], cfg["params"], bc=tuple(cfg["bc"])[:2] + (1, 1))
    sw.init_jet() if cfg["init"]["kind"] == "jet" else sw.init_droplet(cfg["init"]["R"], cfg["init"]["W"])
    sw.step(args.warmup)
    sw_steps = min(args.steps, 500)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    s0.record(sw.stream)
    sw.step(sw_steps)
    s1.record(sw.stream)
    barrier()
    sw_ms = max_over_ranks(s0.elapsed_time(s1))
    side_walls = {"value": job_mlups(nodes, sw_steps, world, sw_ms), "unit": "MLUPS", "steps": sw_steps,
                  "ms_per_step": sw_ms / sw_steps, "boundaries": "free-slip walls at x and y (Section IV.A)"}
    sw.close()
    del sw

    # ---- the paper's own workload: UT Case 1 (240x240x1200 melt jet, free-slip side walls,
    #      gravity), whose 20 000 iterations the paper reports as about 32 hours
    paper = None
    if world == 1 and not args.no_paper_workload:
        ucfg = workloads.CONFIGS["ut1"]
        un = int(np.prod(ucfg["grid"]))
        ut = lb.Lattice(ucfg["grid"], ucfg["params"], bc=ucfg["bc"])
        ut.init_jet()
        ut.step(args.warmup)
        u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        u0.record(ut.stream)
        ut.step(200)
        u1.record(ut.stream)
        torch.cuda.synchronize()
        ums = u0.elapsed_time(u1)
        paper = {"workload": ucfg["text"], "nodes": un, "steps": 200, "value": un * 200 / (ums * 1e-3) / 1e6,
                 "unit": "MLUPS", "ms_per_step": ums / 200, "hours_for_20000_steps": ums / 200 * 20000 / 3.6e6,
                 "paper": "about 32 h for 20 000 iterations on unstated hardware: 12 MLUPS for the 69.12 M nodes "
                          "of this lattice (1.2 MLUPS for the 6.912 M nodes the text prints)"}
        ut.close()
        del ut
        torch.cuda.empty_cache()

    # ---- fragment analysis of the state the timed steps reached (lb_fragments, Section IV.B)
    fr_t0 = time.perf_counter()
    frag = lat.fragments(6)
    fr_ms = (time.perf_counter() - fr_t0) * 1e3
    fragments = {"connectivity": 6, "n_fragments": int(len(frag["roots"])),
                 "column_volume": frag["column_volume"], "mass_median_diameter": frag["mass_median_diameter"],
                 "wall_ms": fr_ms, "state": f"after {args.warmup + 2 * args.steps} steps of the workload"}

    # ---- end to end through the public API with host buffers
    rr = torch.zeros(cfg["grid"][::-1], dtype=torch.float32).pin_memory()
    rb = torch.full(cfg["grid"][::-1], cfg["params"]["rho_b0"], dtype=torch.float32).pin_memory()
    uu = torch.zeros((3,) + tuple(cfg["grid"][::-1]), dtype=torch.float32).pin_memory()
    outs = {k: torch.empty(cfg["grid"][::-1], dtype=torch.float32).pin_memory() for k in ("rho_r", "rho_b", "ux", "uy", "uz")}
    barrier()
    t0 = time.perf_counter()
    lat.init_fields(rr.numpy(), rb.numpy(), uu.numpy())
    lat.step(args.steps)
    got = lat.fields(names=tuple(outs), device=False, out={k: v.numpy() for k, v in outs.items()})
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    h2d = 5 * 4 * nodes
    d2h = 4 * nodes * len(got)
    e2e = {"value": nodes * args.steps * world / e2e_s / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "job": f"host fields -> lb_init, {args.steps} x lb_step, lb_fields -> host (pinned)"}

    # ---- FP16 storage (both encodings) on the same workload: throughput, roofline, error vs FP32
    def fp16_leg(storage, bytes_step, bytes_kernel, tag):
        h = lb.Lattice(cfg["grid"], dict(cfg["params"], storage=storage), bc=cfg["bc"])
        h.init_jet() if cfg["init"]["kind"] == "jet" else h.init_droplet(cfg["init"]["R"], cfg["init"]["W"])
        h.step(args.warmup)
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(h.stream)
        h.step(args.steps)
        f1.record(h.stream)
        barrier()
        ms16 = max_over_ranks(f0.elapsed_time(f1))
        h.profile_enable(args.steps)
        h.step(args.steps)
        p16 = h.profile_read()
        h.profile_enable(0)
        c_ms = p16["collide_kernel"][0] / max(p16["collide_kernel"][1], 1)
        h.close()
        del h
        torch.cuda.empty_cache()
        achieved = bytes_kernel["collide_kernel"] * nodes / (c_ms * 1e-3) / 1e9
        return {"value": nodes * args.steps * world / (ms16 * 1e-3) / 1e6, "unit": "MLUPS",
                "ms_per_step": ms16 / args.steps, "storage": STORAGE_TEXT[storage],
                "bytes_per_node_algorithmic": bytes_step,
                "roofline": {"bound": "hbm", "kernel": f"collide_kernel<{tag}>", "achieved": achieved,
                             "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                             "algorithmic_bytes_per_node": bytes_kernel["collide_kernel"], "traffic": None},
                "kernels": {name: {"avg_ms": t / max(n, 1), "launches": n} for name, (t, n) in p16.items() if n},
                "error_vs_fp32": fp16_error(lb, cfg, args.error_steps, storage)}

    fp16 = fit = None
    if not args.no_fp16:
        lat.close()
        del lat
        torch.cuda.empty_cache()
        fp16 = fp16_leg(1, BYTES_STEP_FP16, BYTES_KERNEL_FP16, "fp16")
        fit = fp16_leg(2, BYTES_STEP_FIT, BYTES_KERNEL_FIT, "fp16_fit")

    if rank == 0:
        base = None
        adjoint = None
        if world == 1 and not args.no_adjoint:
            adjoint = adjoint_leg(lb, torch, T=args.adjoint_steps, checkpoint=args.adjoint_checkpoint)
        if world == 1 and not args.no_cpu_baseline:
            base = cpu_baseline(cfg)
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config_block(cfg),
                "hbm_pct_of_peak": 100.0 * value * 1e6 * BYTES_STEP / (peak * 1e9) / world,
                "bytes_per_node_algorithmic": BYTES_STEP,
                "roofline": roofline, "kernels": kernels, "cpu_baseline": base, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks,
                "fp16_storage": fp16, "fp16_fit_storage": fit, "adjoint_forward_ratio": adjoint["ratio"] if adjoint else None,
                "adjoint": adjoint, "fragments": fragments, "side_walls": side_walls,
                "paper_workload": paper}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
