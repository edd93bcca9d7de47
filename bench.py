"""Benchmark of the D3Q27 colour-gradient central-moment LB step on GB300.

One "step" is one full time step of the method over the whole lattice: the boundary planes,
the gather pass (pull streaming, phase field, collision moments) and the collision pass
(gradients, central-moment collision, perturbation, recolouring).  The default workload is
the high-Re jet on 256x256x1024 (67 M nodes; D = 32, u = 0.04, gamma = 2, Re = 1e5,
We = 1000, Fr = 100 with gravity along +z, 0.5% inlet noise, convective outflow), FP32
populations as the headline, with both half-precision storages on the same lattice beside
it; the 29 GB state is far larger than the 129 MB L2, so no flush is needed between steps.

Prints one JSON line.  With torchrun (N > 1 ranks) every rank advances its own replica of
the lattice (weak scaling; there is no data exchange), times are maxed over ranks.
--impl reference times the FP64 CPU oracle on the host cores instead.
--only-main times the headline loop alone (the command the ncu summaries are taken with).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
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



STORAGE_NAMES = {0: "fp32", 1: "fp16", 2: "fp16_fit"}
BYTES = {0: (BYTES_STEP, BYTES_KERNEL), 1: (BYTES_STEP_FP16, BYTES_KERNEL_FP16), 2: (BYTES_STEP_FIT, BYTES_KERNEL_FIT)}
# the fused step kernel (both passes in one launch) needs only the method's bytes
for _s, (_b, _k) in BYTES.items():
    _k["step_kernel"] = _b


def init_state(lat, cfg):
    lat.init_jet() if cfg["init"]["kind"] == "jet" else lat.init_droplet(cfg["init"]["R"], cfg["init"]["W"])


def with_storage(params, storage):
    return dict(params, storage=storage)


def timed_steps(lat, steps, torch, barrier=None):
    """Device milliseconds of `steps` lb_step calls between CUDA events on the library's stream."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    (barrier or torch.cuda.synchronize)()
    e0.record(lat.stream)
    lat.step(steps)
    e1.record(lat.stream)
    (barrier or torch.cuda.synchronize)()
    return e0.elapsed_time(e1)


def kernel_profile(lat, steps, nodes, storage, peak, cfg_name):
    """Per-kernel device times from a second pass (events around each launch on the stream),
    with each kernel's achieved algorithmic GB/s; the roofline entry is the kernel with the
    largest share of the step."""
    lat.profile_enable(steps)
    lat.step(steps)
    prof = lat.profile_read()
    lat.profile_enable(0)
    _, bk = BYTES[storage]
    total = max(sum(v[0] for v in prof.values()), 1e-30)
    kernels = {}
    for name, (t, n) in prof.items():
        if not n:
            continue
        k = {"avg_ms": t / n, "launches": n, "share": t / total}
        if name in bk:
            k["algorithmic_bytes_per_node"] = bk[name]
            k["achieved_gbs"] = bk[name] * nodes / (t / n * 1e-3) / 1e9
        kernels[name] = k
    top = max((k for k in kernels if k in bk), key=lambda k: kernels[k]["share"])
    tag = STORAGE_NAMES[storage]
    traffic = profile_traffic(top if storage == 0 else f"{top}_{tag}", cfg_name)
    achieved = kernels[top]["achieved_gbs"]
    roofline = {"bound": "hbm", "kernel": top if storage == 0 else f"{top}<{tag}>", "achieved": achieved,
                "peak": peak[0], "unit": "GB/s", "frac": achieved / peak[0], "peak_source": f"hbm_gbs of {peak[1]}",
                "algorithmic_bytes_per_node": bk[top],
                "traffic": traffic * 1.0 if traffic is not None else None,
                "traffic_per_node": traffic / nodes if traffic is not None else None}
    # the same kernel against the instruction issue limit: thread instructions per node from the
    # committed ncu summary (same sources) over the live duration
    ipn = profile_value(top if storage == 0 else f"{top}_{tag}", cfg_name, "thread_instructions_per_node")
    if ipn is not None:
        rate = ipn * nodes / (kernels[top]["avg_ms"] * 1e-3)
        roofline["issue"] = {"thread_instructions_per_node": ipn, "achieved": rate / 1e12, "peak": ISSUE_PEAK_TINST_S / 1e12,
                             "unit": "T thread-instructions/s", "frac": rate / ISSUE_PEAK_TINST_S,
                             "peak_source": "152 SMs x 4 schedulers x 32 lanes x 2.07 GHz"}
    return kernels, roofline


def storage_leg(lb, torch, cfg, storage, steps, warmup, peak, world, max_over_ranks, barrier):
    """MLUPS, per-kernel times and the dominant kernel's roofline of one storage."""
    nodes = int(np.prod(cfg["grid"]))
    lat = lb.Lattice(cfg["grid"], with_storage(cfg["params"], storage), bc=cfg["bc"])
    init_state(lat, cfg)
    lat.step(warmup)
    ms = max_over_ranks(timed_steps(lat, steps, torch, barrier))
    kernels, roofline = kernel_profile(lat, steps, nodes, storage, peak, cfg["name"])
    lat.close()
    del lat
    torch.cuda.empty_cache()
    bs, _ = BYTES[storage]
    v = job_mlups(nodes, steps, world, ms)
    return {"value": v, "unit": "MLUPS", "ms_per_step": ms / steps, "steps": steps,
            "storage": STORAGE_TEXT.get(storage, "fp32 populations"), "bytes_per_node_algorithmic": bs,
            "hbm_pct_of_peak": 100.0 * v * 1e6 * bs / (peak[0] * 1e9) / world,
            "roofline": roofline, "kernels": kernels}


def error_vs_fp32(lb, torch, cfg, checkpoints):
    """Both half-precision storages against FP32 on the same workload, stepped in lockstep:
    relative L2 error of the velocity and the largest change of the order parameter at each
    checkpoint step."""
    lats = {s: lb.Lattice(cfg["grid"], with_storage(cfg["params"], s), bc=cfg["bc"]) for s in (0, 1, 2)}
    for l in lats.values():
        init_state(l, cfg)
    out = {STORAGE_NAMES[s]: [] for s in (1, 2)}
    done = 0
    for cp in checkpoints:
        for l in lats.values():
            l.step(cp - done)
        done = cp
        F = {s: l.fields(names=("phi", "ux", "uy", "uz")) for s, l in lats.items()}
        u32 = torch.stack([F[0][k] for k in ("ux", "uy", "uz")]).double()
        for s in (1, 2):
            du = torch.stack([F[s][k] - F[0][k] for k in ("ux", "uy", "uz")]).double()
            out[STORAGE_NAMES[s]].append({"steps": cp, "rel_u_l2": float(du.norm() / u32.norm()),
                                          "max_abs_dphi": float((F[s]["phi"] - F[0]["phi"]).abs().max())})
        del F
    for l in lats.values():
        l.close()
    torch.cuda.empty_cache()
    return out


def mass_drift_leg(lb, torch, name, steps_by_storage):
    """MLUPS and the FP64 per-colour mass change over a run, per storage, on a large jet (blue
    has neither source nor sink until the inlet's pressure wave reaches the outflow, so its
    change is the storage's drift; red grows by the inlet flux)."""
    cfg = workloads.CONFIGS[name]
    nodes = int(np.prod(cfg["grid"]))
    out = {"workload": cfg["text"], "nodes": nodes}
    for s, steps in steps_by_storage.items():
        lat = lb.Lattice(cfg["grid"], with_storage(cfg["params"], s), bc=cfg["bc"])
        init_state(lat, cfg)
        m0 = lat.mass()
        ms = timed_steps(lat, steps, torch)
        m1 = lat.mass()
        out[STORAGE_NAMES[s]] = {"steps": steps, "value": nodes * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS",
                                 "ms_per_step": ms / steps, "mass_start": m0.tolist(), "mass_end": m1.tolist(),
                                 "blue_rel_drift": float((m1[1] - m0[1]) / m0[1]),
                                 "red_gain_per_step": float((m1[0] - m0[0]) / steps),
                                 "device_gb": sum(b.numel() for b in lat._bufs) / 1e9}
        lat.close()
        del lat
        torch.cuda.empty_cache()
    p = cfg["params"]
    out["red_inflow_per_step_nominal"] = float(np.pi * (p["d_in"] / 2) ** 2 * p["u_in"] * p["rho_r0"])
    return out


def oracle_error_leg(lb, torch, checkpoints=(100,)):
    """Every storage against the FP64 oracle on the 48x48x192 jet (D = 8, the 96x96x384
    jet's lattice parameters): relative L2 error of the velocity and max |d phi| at each
    checkpoint step (all lattices stepped in lockstep)."""
    import oracle
    cfg = workloads.scaled_jet("jet96", 48, 48, 192, D=8)
    nx, ny, nz = cfg["grid"]
    ref = oracle.Lattice(oracle.make_grid(nx, ny, nz, *cfg["bc"]), oracle.make_params(cfg["params"]))
    ref.init_jet()
    lats = {s: lb.Lattice(cfg["grid"], with_storage(cfg["params"], s), bc=cfg["bc"]) for s in (0, 1, 2)}
    for lat in lats.values():
        lat.init_jet()
    out = {"workload": "jet 48x48x192, D=8, the 96x96x384 jet's lattice parameters", "oracle_cores": oracle.num_threads(),
           "oracle_seconds": 0.0, "checkpoints": []}
    done = 0
    for cp in checkpoints:
        t0 = time.perf_counter()
        ref.step(cp - done)
        out["oracle_seconds"] += time.perf_counter() - t0
        R = ref.fields()
        un = np.linalg.norm(R["u"])
        row = {"steps": cp}
        for s, lat in lats.items():
            lat.step(cp - done)
            F = lat.fields(device=False)
            du = np.stack([F[k].astype(np.float64) - R["u"][d] for d, k in enumerate(("ux", "uy", "uz"))])
            row[STORAGE_NAMES[s]] = {"rel_u_l2": float(np.linalg.norm(du) / un),
                                     "max_abs_dphi": float(np.abs(F["phi"] - R["phi"]).max())}
        out["checkpoints"].append(row)
        done = cp
    for lat in lats.values():
        lat.close()
    return out


def fragments_leg(lb, torch):
    """lb_fragments on a broken-up state: 1500 seeded random droplets (radii 1.5-4.5) on the
    96x96x384 lattice, timed with CUDA events on the library's stream (the call also
    allocates its scratch, sorts the kept fragments on the host and synchronises; its host
    wall time is reported too)."""
    cfg = workloads.CONFIGS["jet96"]
    nx, ny, nz = cfg["grid"]
    rr, rb, u = workloads.random_droplet_fields((nz, ny, nx), 1500, 1.5, 4.5, 7, 1.0, cfg["params"]["rho_b0"])
    lat = lb.Lattice(cfg["grid"], cfg["params"], bc=(0, 0))
    lat.init_fields(rr, rb, u)
    lat.fragments(6, exclude_inlet=False)  # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record(lat.stream)
    fr = lat.fragments(6, exclude_inlet=False)
    e1.record(lat.stream)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) * 1e3
    lat.close()
    return {"state": "1500 random droplets, radii 1.5-4.5, 96x96x384 periodic", "connectivity": 6,
            "n_fragments": int(len(fr["roots"])), "total_volume": fr["total_volume"],
            "mass_median_diameter": fr["mass_median_diameter"], "device_ms": e0.elapsed_time(e1), "wall_ms": wall}


def oracle_slab(cfg, seconds):
    """An oracle lattice on a z-slab of the workload's lattice, deep enough for about
    `seconds` of FP64 work per step, with the workload's boundaries and parameters."""
    import oracle
    nx, ny, nz = cfg["grid"]
    probe = oracle.Lattice(oracle.make_grid(nx, ny, 4, *cfg["bc"]), oracle.make_params(cfg["params"]))
    init_state(probe, cfg)
    t0 = time.perf_counter()
    probe.step(1)
    rate = nx * ny * 4 / (time.perf_counter() - t0)
    nzs = int(max(4, min(nz, rate * seconds / (nx * ny))))
    lat = oracle.Lattice(oracle.make_grid(nx, ny, nzs, *cfg["bc"]), oracle.make_params(cfg["params"]))
    init_state(lat, cfg)
    return lat, nzs


def cpu_baseline(cfg, seconds_target=15.0):
    """The FP64 oracle as it stands, on the host cores, over a bounded sample of the
    workload: whole oracle steps of a z-slab of the lattice (same boundaries and parameters)."""
    import oracle
    nx, ny, nz = cfg["grid"]
    lat, nzs = oracle_slab(cfg, seconds_target / 4)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds_target and steps < 1000:
        lat.step(1)
        steps += 1
    el = time.perf_counter() - t0
    return {"value": nx * ny * nzs * steps / el / 1e6, "unit": "MLUPS", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"{steps} FP64 oracle step(s) of a {nx}x{ny}x{nzs} slab of the {nx}x{ny}x{nz} "
                                        f"lattice, same boundaries and parameters ({el:.1f} s)"}


def run_reference(args, cfg):
    """Reference arm: the FP64 oracle on the host cores, timed on bounded samples of the
    workload (a z-slab of the lattice with the same boundaries and parameters)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    nx, ny, nz = cfg["grid"]
    # slab depth sized so that W + K oracle steps take about two minutes
    lat, nzs = oracle_slab(cfg, 120.0 / max(1, args.steps + args.warmup))
    lat.step(args.warmup)
    t0 = time.perf_counter()
    lat.step(args.steps)
    el = time.perf_counter() - t0
    v = nx * ny * nzs * args.steps / el / 1e6
    sample = f"{nx}x{ny}x{nzs} slab of the {nx}x{ny}x{nz} lattice, same boundaries and parameters"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_block(cfg, 0),
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# The sources a kernel is compiled from, besides the shared headers: its translation unit, and
# for the fused step kernel the host code that builds its item sequence.
KERNEL_SOURCES = {"step_kernel": ("lbcm_step.cu", "lbcm_api.cu")}


def kernel_source_sha(kernel: str, src: str = None) -> str:
    """sha256 (16 hex digits) of the sources `kernel` is built from: every header of csrc/ and
    the kernel's own translation unit(s), so that a summary stays valid while those are
    unchanged."""
    import hashlib
    src = src or os.path.join(ROOT, "paper_1804_08923_gb300", "csrc")
    units = KERNEL_SOURCES.get(kernel, ("lbcm_adjoint.cu",) if kernel.startswith("adj_") else ("lbcm_step.cu",))
    h = hashlib.sha256()
    for f in sorted(os.listdir(src)):
        if f.endswith((".cuh", ".h")) or f in units:
            h.update(open(os.path.join(src, f), "rb").read())
    return h.hexdigest()[:16]


def profile_value(kernel: str, workload: str, key: str):
    """A number from the committed ncu summary of `kernel` on `workload`, if the summary was
    taken from the current sources of the kernel (their sha256 is recorded in it)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    try:
        kv = {}
        for line in open(path):
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("source_sha256_16") != kernel_source_sha(kernel):
            return None
        return float(kv[key].split()[0])
    except Exception:
        return None


def profile_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary (None if stale or absent)."""
    return profile_value(kernel, workload, "dram_bytes_per_launch")


# Instruction issue capacity of a GB300: 152 SMs x 4 schedulers x 32 lanes x 2.07 GHz
# (one warp instruction per scheduler and clock), in thread instructions per second.
ISSUE_PEAK_TINST_S = 152 * 4 * 32 * 2.07e9


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


def run_slabs(args, cfg, lb, torch, dist, rank, world, local, barrier, max_over_ranks, peak):
    """One lattice split into `world` z-slabs, one per rank, halos over NCCL (device buffers):
    strong scaling; the throughput counts the lattice's nodes once."""
    from paper_1804_08923_gb300 import slab
    nodes = int(np.prod(cfg["grid"]))
    s = slab.SlabLattice(cfg["grid"], with_storage(cfg["params"], args.storage), cfg["bc"], rank, world, dist,
                         device=f"cuda:{local}")
    init_state(s, cfg)
    s.step(args.warmup)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record()
        s.step(args.steps)
        e1.record()
        barrier()
    ms = max_over_ranks(e0.elapsed_time(e1))
    value = nodes * args.steps / (ms * 1e-3) / 1e6
    bytes_step, _ = BYTES[args.storage]
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32" if args.storage == 0 else "f32 arithmetic, f16 population storage",
            "data": "synthetic", "config": dict(config_block(cfg, args.storage),
                                                parallelism=f"z-slabs over {world} GPUs, halos over NCCL"),
            "hbm_pct_of_peak": 100.0 * value * 1e6 * bytes_step / (peak[0] * 1e9) / world,
            "slab_planes": [list(r) for r in slab.partition(cfg["grid"][2], world)],
            "mass": s.mass().tolist(), "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist.barrier()
    dist.destroy_process_group()


def config_block(cfg, storage):
    nx, ny, nz = cfg["grid"]
    return {"workload": f"{cfg['name']}: {cfg['text']}", "lattice": [nx, ny, nz], "nodes": nx * ny * nz,
            "storage": {0: "fp32 SoA populations [i][z][y][x] of (red, blue) pairs"}.get(storage, STORAGE_TEXT.get(storage)),
            "l2": "state >> 129 MB L2 (every population is read and written once per step); no flush between steps",
            "parallelism": "one lattice per GPU (replicas, no exchange)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="jet256")
    ap.add_argument("--storage", type=int, default=0, choices=[0, 1, 2],
                    help="storage of the headline loop (0 FP32, 1 FP16, 2 FP16_FIT)")
    ap.add_argument("--only-main", action="store_true", help="the headline loop alone (ncu summaries)")
    ap.add_argument("--error-steps", default="100,500,2000")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp16", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-paper-workload", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 384x384x1536 mass-drift leg")
    ap.add_argument("--no-oracle-error", action="store_true")
    ap.add_argument("--oracle-error-steps", default="100", help="checkpoints of the FP64-oracle error leg")
    ap.add_argument("--step-kernel", type=int, default=0, choices=[0, 1],
                    help="headline loop: 0 one launch per pass (default), 1 the fused step kernel")
    ap.add_argument("--slabs", action="store_true",
                    help="with N > 1 ranks: split the one lattice into z-slabs (halo exchange over NCCL, strong "
                         "scaling) instead of one replica per rank")
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

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
            torch.cuda.synchronize()

    def max_over_ranks(v):
        return reduce_max(v, dist, "cuda")

    nx, ny, nz = cfg["grid"]
    nodes = nx * ny * nz
    peak = measured_peaks()
    st = args.storage
    if args.slabs and world > 1:
        return run_slabs(args, cfg, lb, torch, dist, rank, world, local, barrier, max_over_ranks, peak)
    lat = lb.Lattice(cfg["grid"], dict(with_storage(cfg["params"], st), step_kernel=args.step_kernel), bc=cfg["bc"])
    init_state(lat, cfg)
    stream = lat.stream

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
    bytes_step, _ = BYTES[st]
    kernels, roofline = kernel_profile(lat, args.steps, nodes, st, peak, cfg["name"])
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if st == 0 else "f32 arithmetic, f16 population storage",
            "data": "synthetic", "config": config_block(cfg, st),
            "hbm_pct_of_peak": 100.0 * value * 1e6 * bytes_step / (peak[0] * 1e9) / world,
            "bytes_per_node_algorithmic": bytes_step,
            "bytes_per_node_design": 2 * BYTES[st][1]["collide_kernel"] if st == 0 else
            BYTES[st][1]["collide_kernel"] + BYTES[st][1]["moment_kernel"],
            "roofline": roofline, "kernels": kernels, "gpu_launches": launches, "clocks": clocks}
    if args.only_main:
        lat.close()
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    # ---- end to end through the public API with host buffers: host fields -> lb_init,
    #      K x lb_step, lb_fields -> host (pinned), all inside the timed region
    shp = cfg["grid"][::-1]
    rr = torch.zeros(shp, dtype=torch.float32).pin_memory()
    rb = torch.full(shp, cfg["params"]["rho_b0"], dtype=torch.float32).pin_memory()
    uu = torch.zeros((3,) + tuple(shp), dtype=torch.float32).pin_memory()
    outs = {k: torch.empty(shp, dtype=torch.float32).pin_memory() for k in ("rho_r", "rho_b", "ux", "uy", "uz")}
    # three repeats of the whole job, the median reported (the host side of the copies varies
    # from one box to the next)
    # the box's own pinned-copy bandwidth, outside the timed region, for reading the e2e figure
    host_gbs = None
    try:
        dev = torch.empty(5 * nodes, dtype=torch.float32, device=f"cuda:{local}")
        hbuf = torch.empty(5 * nodes, dtype=torch.float32).pin_memory()
        bw = []
        for src, dst in ((hbuf, dev), (dev, hbuf)):
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            tc = time.perf_counter()
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            bw.append(round(5 * nodes * 4 / (time.perf_counter() - tc) / 1e9, 1))
        host_gbs = {"h2d": bw[0], "d2h": bw[1]}
        del dev, hbuf
        torch.cuda.empty_cache()
    except Exception:
        pass
    reps, parts = [], []
    with ClockSampler(local) as clk_e2e:
        for _ in range(3):
            barrier()
            t0 = time.perf_counter()
            lat.init_fields(rr.numpy(), rb.numpy(), uu.numpy())  # returns once the fields are copied
            t1 = time.perf_counter()
            lat.step(args.steps)
            barrier()
            t2 = time.perf_counter()
            got = lat.fields(names=tuple(outs), device=False, out={k: v.numpy() for k, v in outs.items()})
            barrier()
            t3 = time.perf_counter()
            reps.append(max_over_ranks(t3 - t0))
            parts.append([round(t1 - t0, 4), round(t2 - t1, 4), round(t3 - t2, 4)])
    e2e_s = sorted(reps)[1]
    h2d = 5 * 4 * nodes
    d2h = 4 * nodes * len(got)
    line["e2e"] = {"value": nodes * args.steps * world / e2e_s / 1e6, "unit": "MLUPS",
                   "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                   "job": f"host fields -> lb_init, {args.steps} x lb_step, lb_fields -> host (pinned); "
                          "median of 3 repeats",
                   "repeats_s": reps, "repeat_parts_s": {"init, steps, fields": parts},
                   "clocks": clk_e2e.summary(), "pinned_copy_gbs_torch": host_gbs}
    lat.close()
    del lat, rr, rb, uu, outs
    torch.cuda.empty_cache()

    # ---- the other storages on the same lattice, and their error against FP32
    if not args.no_fp16:
        for s in (0, 1, 2):
            if s != st:
                line[f"{STORAGE_NAMES[s]}_storage"] = storage_leg(lb, torch, cfg, s, args.steps, args.warmup, peak,
                                                                  world, max_over_ranks, barrier)
        cps = [int(v) for v in args.error_steps.split(",") if v.strip()]
        if cps and world == 1:  # numerics, not throughput: one GPU only
            line["error_vs_fp32"] = error_vs_fp32(lb, torch, cfg, cps)
            line["error_vs_fp32"]["note"] = ("velocity relative L2 and max |d phi| against FP32 on the same "
                                             "lattice; by step 2000 the high-Re jet is chaotic and the two "
                                             "runs diverge on their own")

    # ---- the paper's free-slip side walls (Section IV.A) in place of periodic x and y
    sw = lb.Lattice(cfg["grid"], cfg["params"], bc=tuple(cfg["bc"])[:2] + (1, 1))
    init_state(sw, cfg)
    sw.step(args.warmup)
    sw_ms = max_over_ranks(timed_steps(sw, args.steps, torch, barrier))
    line["side_walls"] = {"value": job_mlups(nodes, args.steps, world, sw_ms), "unit": "MLUPS",
                          "steps": args.steps, "ms_per_step": sw_ms / args.steps,
                          "boundaries": "free-slip walls at x and y (Section IV.A)"}
    sw.close()
    del sw
    torch.cuda.empty_cache()

    if rank == 0 and world == 1:
        # ---- the 96x96x384 jet (FP32), a smaller lattice of the same kind
        if args.config != "jet96":
            line["jet96"] = storage_leg(lb, torch, workloads.CONFIGS["jet96"], 0, max(args.steps, 100), args.warmup,
                                        peak, 1, lambda v: v, None)
        # ---- the 384x384x1536 atomisation jet: throughput and FP64 colour-mass drift
        if not args.no_large:
            line["jet384"] = mass_drift_leg(lb, torch, "jet384", {0: 300, 1: 1000, 2: 1000})
        # ---- the paper's own workload: UT Case 1 (240x240x1200 melt jet, free-slip side
        #      walls, gravity), whose 20 000 iterations the paper reports as about 32 hours
        if not args.no_paper_workload:
            ucfg = workloads.CONFIGS["ut1"]
            un = int(np.prod(ucfg["grid"]))
            ut = lb.Lattice(ucfg["grid"], ucfg["params"], bc=ucfg["bc"])
            ut.init_jet()
            ut.step(args.warmup)
            ums = timed_steps(ut, 200, torch)
            line["paper_workload"] = {
                "workload": ucfg["text"], "nodes": un, "steps": 200, "value": un * 200 / (ums * 1e-3) / 1e6,
                "unit": "MLUPS", "ms_per_step": ums / 200, "hours_for_20000_steps": ums / 200 * 20000 / 3.6e6,
                "paper": "about 32 h for 20 000 iterations on unstated hardware: 12 MLUPS for the 69.12 M nodes "
                         "of this lattice (1.2 MLUPS for the 6.912 M nodes the text prints)"}
            ut.close()
            del ut
            torch.cuda.empty_cache()
        # ---- fragment analysis (Section IV.B) of a broken-up state
        line["fragments"] = fragments_leg(lb, torch)
        # ---- adjoint against forward cost
        if not args.no_adjoint:
            adjoint = adjoint_leg(lb, torch, T=args.adjoint_steps, checkpoint=args.adjoint_checkpoint)
            line["adjoint"] = adjoint
            line["adjoint_forward_ratio"] = adjoint["ratio"]
        # ---- error of every storage against the FP64 oracle
        if not args.no_oracle_error:
            line["error_vs_oracle"] = oracle_error_leg(
                lb, torch, [int(v) for v in args.oracle_error_steps.split(",") if v.strip()])
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(cfg)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
