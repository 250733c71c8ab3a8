#!/usr/bin/env python3
"""Throughput benchmark of the D3Q19 cascaded-LBM step on GB300.

Workload: the periodic 256^3 Kolmogorov box (F_x = 1e-5 sin(2 pi z / 256),
nu = 0.01, rho = 1, seeded divergence-free u0 with max |u| = 0.02 on
wavenumbers 1..4), FP32 populations, A/B pull scheme. One bench step is one
lattice time step: one launch of the fused stream-and-collide kernel over all
16,777,216 nodes. The two population buffers (1.27 GB each) are ten times the
129 MB L2, so every step streams from HBM.

Prints one JSON line (rank 0). Under torchrun (N > 1) the ranks hold the z-slabs
of one 256 x 256 x (256 N) periodic Kolmogorov box, 256^3 nodes each (weak
scaling), and exchange the 5 populations that cross each slab face after every
step with NCCL point-to-point transfers that overlap the slab interior's update
(--decomp replicas runs N independent boxes instead; --scaling strong splits
one 512^3 box into N slabs); the timed region is bracketed by barriers and the
slowest rank's time is used.

--impl reference times the FP64 CPU oracle, as it stands, on the host cores on
a bounded slab of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3Q19 CLBM MLUPS at 256³ and % HBM roofline; adjoint/forward time ratio"
N_SIDE = 256
NU = 0.01
F0 = 1e-5
UMAX = 0.02
BYTES_PER_NODE = 152  # 19 x 4 B read + 19 x 4 B written (FP32 A/B)
NOMINAL_HBM_GBS = 7900.0  # HBM3e nominal, context beside the measured copy peak
WORKLOAD = "periodic 256^3 Kolmogorov box, F_x = 1e-5 sin(2 pi z/256), nu = 0.01, FP32 populations"


def workload_name(side, args):
    """The bench workload's name for this run's size, storage and lattice."""
    w = WORKLOAD.replace("256", str(side))
    if args.storage != "f32":
        w = w.replace("FP32 populations", f"{args.storage} populations")
    if args.lattice == 27:
        w = w.replace("Kolmogorov box", "Kolmogorov box, D3Q27")
    return w


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the FP16/BF16, adjoint and batched lines")
    ap.add_argument("--batch-steps", type=int, default=5000, help="steps per mode of the 64-domain batch")
    ap.add_argument("--only", default="", metavar="LINE",
                    help="profiling: of the variant lines run only LINE (e.g. d3q27_f32, adjoint_kernel_256)")
    ap.add_argument("--batch-only", type=int, default=0, metavar="NDOMAINS",
                    help="profiling: run only the batched sweep over the first NDOMAINS domains and print it")
    ap.add_argument("--block", default="0,0", help="step kernel block shape bx,by (0,0 = default)")
    ap.add_argument("--size", type=int, default=N_SIDE,
                    help="box side (the benchmark workload is 256; smaller sides are for profiling captures)")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16", "f16sr", "bf16sr"],
                    help="storage of the timed lattice (the benchmark line is f32; others for profiling)")
    ap.add_argument("--variant", type=int, default=0, help="step kernel form (0/1: one node per thread, 2: two)")
    ap.add_argument("--lattice", type=int, default=19, choices=[19, 27])
    ap.add_argument("--model", default="cascaded", choices=["cascaded", "srt", "mrt"],
                    help="collision of the timed lattice (the benchmark line is cascaded; others for profiling)")
    ap.add_argument("--pattern", default="ab", choices=["ab", "aa"],
                    help="storage pattern of the timed lattice (the benchmark line is ab; aa for profiling)")
    ap.add_argument("--decomp", default="slab", choices=["slab", "replicas"],
                    help="N > 1: z-slabs of one lattice with face exchange (default) or independent boxes")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="N > 1: weak (256^3 per GPU, the default) or strong (one --strong-side^3 box split into N "
                         "z-slabs)")
    ap.add_argument("--strong-side", type=int, default=512, help="side of the box of --scaling strong")
    ap.add_argument("--dist-backend", default="nccl", choices=["nccl", "gloo"],
                    help="N > 1: nccl (faces between GPUs) or gloo (faces through host memory; several ranks may "
                         "share one GPU, for testing the decomposition)")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_digest():
    h = hashlib.sha256()
    # the headers that define the FP32 step kernel (step.cu only instantiates it)
    for rel in ("paper_1801_04586_gb300/csrc/step_kernels.cuh", "paper_1801_04586_gb300/csrc/d3q19.cuh",
                "paper_1801_04586_gb300/csrc/cascaded.cuh"):
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    if the kernel sources still match the digest recorded there."""
    path = os.path.join(ROOT, "profiles", "k_step_f32_kolmogorov256.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    d = re.search(r"source_digest:\s*([0-9a-f]+)", text)
    if not m or not d or d.group(1) != kernel_source_digest():
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the run."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, t0, t1):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                rows.append((ts, float(parts[1]), float(parts[2]), parts[4:]))
            except Exception:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        inside = [r for r in rows if t0 - 1.0 <= r[0] <= t1 + 1.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in inside for k, v in enumerate(r[3][1:5]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_rate(seconds: float = 10.0, max_steps: int = 20):
    """FP64 oracle on a 256 x 256 x 16 periodic slab of the workload with all
    host cores: MLUPS over whole steps until `seconds` have elapsed."""
    import numpy as np

    import oracle
    from paper_1801_04586_gb300 import synthetic

    nz = 16
    shape = (nz, N_SIDE, N_SIDE)
    lat = oracle.Lattice.from_nu(N_SIDE, N_SIDE, nz, NU)
    F = synthetic.profile_to_field(synthetic.kolmogorov_profile(N_SIDE, F0)[:, :nz], shape)
    u0 = synthetic.divfree_velocity((N_SIDE, N_SIDE, N_SIDE), seed=1, umax=UMAX)[:, :nz]
    f = oracle.init(lat, None, np.ascontiguousarray(u0), F)
    f = oracle.step(lat, f, F, 1)  # warm
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps:
        f = oracle.step(lat, f, F, 1)
        steps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    cores = oracle.num_threads()
    # one thread on a thinner slab (the thread count is set last: it stays set)
    lat1 = oracle.Lattice.from_nu(N_SIDE, N_SIDE, 2, NU)
    F1, f1 = np.ascontiguousarray(F[:, :2]), np.ascontiguousarray(f[:, :2])
    t1 = time.perf_counter()
    oracle.step(lat1, f1, F1, 2, nthreads=1)
    dt1 = time.perf_counter() - t1
    return {"value": lat.n * steps / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{steps} steps of a 256x256x16 periodic slab of the workload ({lat.n} nodes), "
                      f"FP64, OpenMP over rows, {dt:.1f} s",
            "value_1_thread": lat1.n * 2 / dt1 / 1e6,
            "sample_1_thread": f"2 steps of a 256x256x2 slab ({lat1.n} nodes), one thread, {dt1:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    from paper_1801_04586_gb300 import synthetic

    oracle.build()
    nz = 4
    shape = (nz, N_SIDE, N_SIDE)
    lat = oracle.Lattice.from_nu(N_SIDE, N_SIDE, nz, NU)
    F = synthetic.profile_to_field(synthetic.kolmogorov_profile(N_SIDE, F0)[:, :nz], shape)
    u0 = synthetic.divfree_velocity((N_SIDE, N_SIDE, N_SIDE), seed=1, umax=UMAX)[:, :nz]
    f = oracle.init(lat, None, np.ascontiguousarray(u0), F)
    for _ in range(args.warmup):
        f = oracle.step(lat, f, F, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = oracle.step(lat, f, F, 1)
    dt = time.perf_counter() - t0
    value = lat.n * args.steps / dt / 1e6
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": "256x256x4 periodic slab per step"},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{args.steps} steps of a 256x256x4 periodic slab ({lat.n} nodes)"},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _segmented(stream, K, run, nseg=10):
    """Time K steps of a context line as up to nseg consecutive segments
    (run(m) enqueues m steps on `stream`), CUDA events between them. Returns
    (median ms per step over the segments, mean ms per step over all K): a
    one-off stall of the device inside a short run moves the mean, not the
    median. The headline keeps one bracketed region."""
    import statistics

    import torch
    nseg = max(1, min(nseg, K))
    sizes = [K // nseg + (1 if i < K % nseg else 0) for i in range(nseg)]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(nseg + 1)]
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for i, m in enumerate(sizes):
            run(m)
            ev[i + 1].record(stream)
    torch.cuda.synchronize()
    per = [ev[i].elapsed_time(ev[i + 1]) / sizes[i] for i in range(nseg)]
    return statistics.median(per), ev[0].elapsed_time(ev[nseg]) / K


def bench_storage(storage, K, warmup, dev, side, prof, u0, peak, variant=0, lattice=19, pattern="ab",
                  model="cascaded", walls=0):
    """The same workload in another storage format, step-kernel form, lattice
    (D3Q27 of Sec. II), storage pattern (in-place AA) or collision model (the
    SRT and non-orthogonal MRT comparison models)."""
    import torch

    from paper_1801_04586_gb300 import Lattice
    lat = Lattice(side, side, side, NU, storage=storage, device=dev, variant=variant, lattice=lattice,
                  pattern=pattern, model=model, walls=walls)
    info = lat.info()
    lat.set_force_profile_z(prof)
    lat.init_equilibrium(None, u0)
    lat.step(warmup)
    torch.cuda.synchronize()
    ms, mean = _segmented(lat.stream, K, lat.step)
    lat.check()
    n = lat.n
    lat.close()
    bpn = (4 if storage == "f32" else 2) * 2 * lattice
    achieved = bpn * n / (ms * 1e-3) / 1e9
    return {"value": n / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "ms_per_step_mean": mean,
            "bytes_per_node": bpn,
            "achieved_gbs": achieved, "frac": achieved / peak, "nodes_per_thread": info["nodes_per_thread"],
            "buffers": info["buffers"], "state_gb": info["buffers"] * info["state_bytes"] / 1e9}


def bench_duct(storage, K, warmup, dev, peak):
    """The mixed-precision square duct: 512 (periodic, x) x 128 x 128 with walls
    on y and z, uniform F_x = 2e-6, nu = 0.05, from rest."""
    import torch

    from paper_1801_04586_gb300 import Lattice
    lat = Lattice(512, 128, 128, 0.05, walls=6, storage=storage, device=dev)
    lat.set_force_uniform(2e-6)
    lat.init_equilibrium()
    lat.step(warmup)
    torch.cuda.synchronize()
    ms, mean = _segmented(lat.stream, K, lat.step)
    lat.check()
    n = lat.n
    lat.close()
    bpn = (4 if storage == "f32" else 2) * 2 * 19
    achieved = bpn * n / (ms * 1e-3) / 1e9
    return {"value": n / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "ms_per_step_mean": mean,
            "bytes_per_node": bpn, "achieved_gbs": achieved, "frac": achieved / peak}


def bench_slab_self(K, warmup, dev, side, prof, u0, peak, storage="f32"):
    """One side^3 z-slab that is its own neighbour on both faces (a periodic z
    axis on one GPU), stepped as faces then interior, the face exchange
    (device copies on a side stream) overlapping the interior: the per-GPU
    cost of the slab decomposition."""
    import torch

    from paper_1801_04586_gb300 import Lattice, slabs
    from paper_1801_04586_gb300._capi import SLAB_FACES, SLAB_INTERIOR
    lat = Lattice(side, side, side, NU, storage=storage, device=dev, slab=3, z0=0)
    lat.set_force_profile_z(prof)
    lat.init_equilibrium(None, u0)

    def one():  # as the ranks of a multi-GPU run: the face copies overlap the interior part
        lat.slab_step(SLAB_FACES)
        reqs = slabs.exchange_faces(lat, 0, 1, wait=False)
        lat.slab_step(SLAB_INTERIOR)
        for r in reqs:
            r.wait()

    with torch.cuda.stream(lat.stream):
        for _ in range(warmup):
            one()
    torch.cuda.synchronize()

    def run(m):
        for _ in range(m):
            one()

    ms, mean = _segmented(lat.stream, K, run)
    lat.check()
    n = lat.n
    lat.close()
    bpn = (4 if storage == "f32" else 2) * 2 * 19
    achieved = bpn * n / (ms * 1e-3) / 1e9
    return {"value": n / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "ms_per_step_mean": mean,
            "bytes_per_node": bpn, "achieved_gbs": achieved, "frac": achieved / peak}


def compact(variants):
    """The variant lines in short form for the benchmark line: [MLUPS, fraction
    of the measured copy roofline] for throughput lines, the ratios for the
    adjoint and the batch. The full figures go to stderr."""
    out = {}
    for name, v in variants.items():
        if "value" in v:
            out[name] = [round(v["value"]), round(v["frac"], 3)]
        elif name.startswith("adjoint_kernel"):
            out[name] = {"ratio": round(v["ratio"], 3), "frac": round(v["adjoint_frac"], 3)}
        elif name.startswith("adjoint_unroll"):
            out[name] = {"ratio": round(v["ratio"], 3)}
        elif name.startswith("batched"):
            out[name] = {"graph": round(v["graph_mlups"]), "per_domain": round(v["per_domain_mlups"]),
                         "frac": round(v["graph_frac"], 3)}
            if "aa_graph_mlups" in v:
                out[name]["aa_graph"] = round(v["aa_graph_mlups"])
        else:
            out[name] = v
    return out


def bench_adjoint(dev, side, K, peak):
    """Adjoint step kernel versus forward step kernel on the same lattice with a
    force field (F ~ N(0, 1e-5^2), seed 3): per-launch times."""
    import numpy as np
    import torch

    from paper_1801_04586_gb300 import Lattice, synthetic
    shape = (side, side, side)
    lat = Lattice(side, side, side, 0.02, device=dev)
    F = torch.from_numpy(synthetic.gaussian_force(shape, 1e-5, seed=3)).to(dev)
    lat.set_force_field(F)
    lat.init_equilibrium()
    lat.step(5)
    state = lat.export_state()
    lam = torch.from_numpy(synthetic.rng(4).normal(size=(19,) + shape).astype(np.float32)).to(dev) \
        if side <= 64 else torch.full((19,) + shape, 1e-3, device=dev)
    lam2 = torch.empty_like(lam)
    gF = torch.zeros((3,) + shape, device=dev)
    for _ in range(3):
        lat.adjoint_step(state, lam, lam2, gF)
    lat.step(3)
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record(lat.stream)
    lat.step(K)
    e1.record(lat.stream)
    torch.cuda.synchronize()
    ms_f = e0.elapsed_time(e1) / K
    e0.record(lat.stream)
    a, b = lam, lam2
    for _ in range(K):
        lat.adjoint_step(state, a, b, gF)
        a, b = b, a
    e1.record(lat.stream)
    torch.cuda.synchronize()
    ms_a = e0.elapsed_time(e1) / K
    n = lat.n
    lat.close()
    return {"forward_ms": ms_f, "adjoint_ms": ms_a, "ratio": ms_a / ms_f,
            "forward_gbs": 164 * n / (ms_f * 1e-3) / 1e9, "adjoint_gbs": 264 * n / (ms_a * 1e-3) / 1e9,
            "adjoint_frac": 264 * n / (ms_a * 1e-3) / 1e9 / peak}


def bench_unroll(dev, reps=3):
    """The differentiable 64^3 box: 200-step unroll with checkpoints every 20,
    full backward (recompute + adjoint) over full forward (steps + checkpoints)."""
    import torch

    from paper_1801_04586_gb300 import Lattice, synthetic
    from paper_1801_04586_gb300.autograd import final_velocity
    n = 64
    shape = (n, n, n)
    lat = Lattice(n, n, n, 0.02, device=dev)
    F = torch.from_numpy(synthetic.gaussian_force(shape, 1e-5, seed=3)).to(dev)
    ut = torch.from_numpy(synthetic.divfree_velocity(shape, seed=4, umax=1e-3)).to(dev)
    lat.init_equilibrium()
    init = lat.export_state().clone()
    fw, bw = [], []
    for _ in range(reps + 1):
        Ft = F.clone().requires_grad_(True)
        torch.cuda.synchronize()
        e0, e1 = _events()
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record()
        u = final_velocity(Ft, lat, init, 200, 20)
        e1.record()
        loss = 0.5 * ((u - ut) ** 2).sum()
        g = torch.autograd.grad(loss, [u])[0]
        e1b = torch.cuda.Event(enable_timing=True)
        e1b.record()
        u.backward(g)
        e2.record()
        torch.cuda.synchronize()
        fw.append(e0.elapsed_time(e1))
        bw.append(e1b.elapsed_time(e2))
    lat.close()
    fwm, bwm = statistics.median(fw[1:]), statistics.median(bw[1:])
    return {"forward_ms": fwm, "backward_ms": bwm, "ratio": bwm / fwm, "steps": 200, "checkpoint_every": 20,
            "note": "64^3 is L2-resident: time ratio, not a roofline figure"}


def bench_batch(dev, steps, peak, ndomains=64):
    """64 independent channels/ducts (sides U{32..128}, nu U[0.005, 0.1],
    F_x U[1e-7, 1e-5], seed 6): autotuned block, then the whole batch stepped
    with one launch per step replayed from a CUDA graph, one launch per step
    issued directly, and one launch per domain per step. A smaller ndomains
    (the first of the same draw) is for profiling captures."""
    import torch

    from paper_1801_04586_gb300 import Batch, synthetic
    doms = synthetic.batch_domains(64, seed=6)[:ndomains]
    b = Batch(doms, device=dev)
    b.init_equilibrium()
    threads = b.autotune(trial_steps=10)
    b.step(32, Batch.GRAPH)
    nodes = b.total_nodes
    out = {"domains": len(doms), "total_nodes": nodes, "steps": steps, "threads_per_block": threads}
    for name, mode in (("graph", Batch.GRAPH), ("direct", Batch.DIRECT), ("per_domain", Batch.PER_DOMAIN)):
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record(b.stream)
        b.step(steps, mode)
        e1.record(b.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name + "_mlups"] = nodes * steps / (ms * 1e-3) / 1e6
    b.check()
    b.close()
    out["graph_vs_per_domain"] = out["graph_mlups"] / out["per_domain_mlups"]
    # the same batch in place (one buffer), graph mode
    a = Batch(doms, device=dev, pattern="aa")
    a.init_equilibrium()
    a.autotune(trial_steps=10)
    a.step(32, Batch.GRAPH)
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record(a.stream)
    a.step(steps, Batch.GRAPH)
    e1.record(a.stream)
    torch.cuda.synchronize()
    a.check()
    a.close()
    out["aa_graph_mlups"] = nodes * steps / (e0.elapsed_time(e1) * 1e-3) / 1e6
    out["graph_gbs"] = BYTES_PER_NODE * out["graph_mlups"] * 1e6 / 1e9
    out["graph_frac"] = out["graph_gbs"] / peak
    return out


def run_gb300(args):
    import numpy as np
    import torch

    from paper_1801_04586_gb300 import Lattice, slabs, synthetic
    from paper_1801_04586_gb300._capi import SLAB_FACES, SLAB_INTERIOR
    from paper_1801_04586_gb300.builder import build

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        if args.dist_backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            torch.cuda.set_device(local % torch.cuda.device_count())
            dist.init_process_group("gloo")
    else:
        dist = None
        torch.cuda.set_device(0)
    if rank == 0:
        build()
    if dist is not None:
        dist.barrier()
    dev = torch.device("cuda", torch.cuda.current_device())
    bx, by = (int(v) for v in args.block.split(","))
    side = args.size
    strong = args.scaling == "strong"
    if strong and args.decomp != "slab":
        raise SystemExit("--scaling strong splits one box into z-slabs (--decomp slab)")
    gside = args.strong_side if strong else side
    if strong and gside % side:
        raise SystemExit("--strong-side must be a multiple of --size (the period of the initial field)")
    slab = ws > 1 and args.decomp == "slab"
    host_faces = slab and args.dist_backend == "gloo"
    # The box of the run: weak scaling, 256 x 256 x (256 N) (one 256^3 slab per
    # rank); strong scaling, one gside^3 box split into N z-slabs. The force
    # profile and u0 repeat every `side` nodes along each axis, so every slab
    # takes its planes of the single side^3 box's fields.
    if strong:
        nxy = gside
        z0, z1 = slabs.partition(gside, ws)[rank]
    else:
        nxy = side
        z0, z1 = (rank * side, (rank + 1) * side) if slab else (0, side)
    nzl = z1 - z0
    shape = (nzl, nxy, nxy)
    skw = dict(slab=3, z0=z0) if slab else {}
    variant = 1 if slab and args.variant == 0 else args.variant
    lat = Lattice(nxy, nxy, nzl, NU, walls=0, storage=args.storage, block=(bx, by), device=dev,
                  variant=variant, lattice=args.lattice, pattern=args.pattern, model=args.model, **skw)
    zi, xi = np.arange(z0, z1) % side, np.arange(nxy) % side
    prof = torch.from_numpy(np.ascontiguousarray(synthetic.kolmogorov_profile(side, F0)[:, zi])).to(dev)
    u_base = synthetic.divfree_velocity((side, side, side), seed=1, umax=UMAX)
    u0_np = np.ascontiguousarray(u_base[:, zi][:, :, xi][:, :, :, xi])
    u0 = torch.from_numpy(u0_np).to(dev)
    lat.set_force_profile_z(prof)
    lat.init_equilibrium(None, u0)
    stream = lat.stream
    sampler = ClockSampler(dev.index) if rank == 0 else None

    def one_step(L):
        if not slab:
            L.step(1)
            return
        # faces first; their transfer overlaps the interior planes' update
        L.slab_step(SLAB_FACES)
        reqs = slabs.exchange_faces(L, rank, ws, dist, host=host_faces, wait=False)
        L.slab_step(SLAB_INTERIOR)
        for r in reqs:
            r.wait()

    # warm-up
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step(lat)
    torch.cuda.synchronize()
    lat.check()

    K = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_host0 = time.time()
    with torch.cuda.stream(stream):
        for k in range(K):
            starts[k].record(stream)
            one_step(lat)
            ends[k].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t_host1 = time.time()
    elapsed_ms = starts[0].elapsed_time(ends[-1])
    per_launch = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    lat.check()
    if dist is not None:
        tt = torch.tensor([elapsed_ms], device=dev if args.dist_backend == "nccl" else "cpu")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed_ms = float(tt.item())
    clocks = sampler.stop(t_host0, t_host1) if sampler else None

    nodes = lat.n
    job_nodes = gside ** 3 if strong else ws * nodes
    value = job_nodes * K / (elapsed_ms * 1e-3) / 1e6
    mean_launch_s = statistics.mean(per_launch) * 1e-3
    peak, peak_kind = measured_peaks()
    bytes_per_node = (2 if args.storage != "f32" else 4) * 2 * args.lattice
    achieved = bytes_per_node * nodes / mean_launch_s / 1e9
    default_case = (args.storage, args.lattice, args.pattern, args.variant, args.model) == (
        "f32", 19, "ab", 0, "cascaded") and not slab and not strong
    traffic = profiled_traffic() if default_case and side == N_SIDE else None

    e2e = None
    if not args.no_e2e:
        rho_h = torch.ones(shape, dtype=torch.float32).pin_memory()
        u_h = torch.from_numpy(u0_np).pin_memory()
        rho_o = torch.empty(shape, dtype=torch.float32).pin_memory()
        u_o = torch.empty((3,) + shape, dtype=torch.float32).pin_memory()
        mom = torch.empty(4 * (K + 1), dtype=torch.float64).pin_memory()
        if not slab:
            lat_e = Lattice(nxy, nxy, nzl, NU, walls=0, storage="f32", block=(bx, by), device=dev)
            lat_e.set_force_profile_z(prof)
            wk = max(1, min(args.warmup, 3))
            lat_e.run_host(rho_h, u_h, wk, rho_o, u_o, mom[: 4 * (wk + 1)])
            what = ("clbm_run_host: pinned host rho,u -> init -> K steps, each step's FP64 mass/momentum "
                    "sums (formed in the step kernel) copied back, final rho,u read back")
        else:
            lat_e = Lattice(nxy, nxy, nzl, NU, walls=0, storage="f32", block=(bx, by), device=dev, variant=1,
                            **skw)
            lat_e.set_force_profile_z(prof)
            what = ("z-slabs: pinned host rho,u -> init -> K steps with face exchange, each step's FP64 "
                    "mass/momentum sums copied back, final rho,u read back")
        d_rho = torch.empty(shape, dtype=torch.float32, device=dev)
        d_u = torch.empty((3,) + shape, dtype=torch.float32, device=dev)
        d_mom = torch.empty(4 * (K + 1), dtype=torch.float64, device=dev)

        def slab_job():
            with torch.cuda.stream(lat_e.stream):
                d_rho.copy_(rho_h, non_blocking=True)
                d_u.copy_(u_h, non_blocking=True)
                lat_e.init_equilibrium(d_rho, d_u)
                for k in range(K):
                    lat_e.reduce_moments(d_mom[4 * k: 4 * k + 4])
                    one_step(lat_e)
                lat_e.reduce_moments(d_mom[4 * K:])
                lat_e.macros(d_rho, d_u)
                rho_o.copy_(d_rho, non_blocking=True)
                u_o.copy_(d_u, non_blocking=True)
                mom.copy_(d_mom, non_blocking=True)
            torch.cuda.synchronize()

        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if slab:
            slab_job()
        else:
            lat_e.run_host(rho_h, u_h, K, rho_o, u_o, mom)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if dist is not None:
            tt = torch.tensor([dt], device=dev if args.dist_backend == "nccl" else "cpu")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            dt = float(tt.item())
        h2d = (rho_h.numel() + u_h.numel()) * 4
        d2h = (rho_o.numel() + u_o.numel()) * 4 + mom.numel() * 8
        e2e = {"value": job_nodes * K / dt / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": h2d / K,
               "d2h_bytes_per_step": d2h / K, "steps": K, "what": what, "ms_total": dt * 1e3}
        del d_rho, d_u, d_mom
        lat_e.close()

    variants = None
    if not args.no_variants and not slab and not strong:
        S = lambda storage, **kw: (lambda: bench_storage(storage, K, args.warmup, dev, side, prof, u0, peak,  # noqa
                                                          **kw))
        D = lambda storage: (lambda: bench_duct(storage, K, args.warmup, dev, peak))  # noqa
        lines = {
            "f16sr": S("f16sr"),
            "bf16sr": S("bf16sr"),
            "f16": S("f16"),
            "bf16": S("bf16"),
            "duct_f32": D("f32"),
            "duct_f16sr": D("f16sr"),
            "duct_bf16sr": D("bf16sr"),
            "f16_1node": S("f16", variant=1),
            "f32_2node": S("f32", variant=2),
            "aa_f32": S("f32", pattern="aa"),
            "aa_f16": S("f16", pattern="aa"),
            "aa_f16sr": S("f16sr", pattern="aa"),
            "walls_yz_f32": S("f32", walls=6),
            "srt_f32": S("f32", model="srt"),
            "mrt_f32": S("f32", model="mrt"),
            "q27_f32": S("f32", lattice=27),
            "q27_srt_f32": S("f32", lattice=27, model="srt"),
            "q27_mrt_f32": S("f32", lattice=27, model="mrt"),
            "q27_aa_f32": S("f32", lattice=27, pattern="aa"),
            "q27_f16": S("f16", lattice=27),
            "slab_self_f32": lambda: bench_slab_self(K, args.warmup, dev, side, prof, u0, peak),
            "slab_self_f16sr": lambda: bench_slab_self(K, args.warmup, dev, side, prof, u0, peak, "f16sr"),
            "adjoint_kernel_256": lambda: bench_adjoint(dev, side, max(10, min(K, 100)), peak),
            "adjoint_unroll_64": lambda: bench_unroll(dev),
            "batched_64_domains": lambda: bench_batch(dev, args.batch_steps, peak),
        }
        if args.only and args.only not in lines:
            raise SystemExit(f"--only: unknown line {args.only!r}; one of {sorted(lines)}")
        variants = {name: fn() for name, fn in lines.items() if not args.only or name == args.only}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_oracle_rate()
        except Exception as exc:  # reported, never fatal for the GPU number
            cpu = {"error": str(exc)[:200]}

    if rank == 0:
        info = lat.info()
        if strong and ws == 1:
            parallelism = f"the whole {gside}^3 box on one GPU"
            workload = (workload_name(side, args).replace(f"periodic {side}^3", f"periodic {gside}^3")
                        + f" (force and initial field of period {side})")
        elif strong:
            parallelism = (f"{ws} z-slabs of one {gside}^3 box, {gside}x{gside}x{nzl} on rank 0, face exchange "
                           f"over {args.dist_backend} overlapped with the interior update")
            workload = (workload_name(side, args).replace(f"periodic {side}^3", f"periodic {gside}^3")
                        + f" (force and initial field of period {side})")
        elif slab:
            parallelism = (f"{ws} z-slabs of one {side}x{side}x{side * ws} box, {side}^3 each, face exchange "
                           f"over {args.dist_backend} overlapped with the interior update")
            workload = workload_name(side, args).replace(f"periodic {side}^3", f"periodic {side}x{side}x{side * ws}")
        else:
            parallelism = f"{ws} independent replica(s), one per GPU"
            workload = workload_name(side, args)
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": K, "warmup": args.warmup,
            "ms_per_step": elapsed_ms / K, "higher_is_better": True, "scaling": "strong" if strong else "weak",
            "vs_baseline": None,
            "dtype": "f32" if args.storage == "f32" else f"f32 arithmetic, {args.storage} storage",
            "data": "synthetic",
            "config": {"workload": workload,
                       "nx": nxy, "ny": nxy, "nz": gside if strong else nzl * (ws if slab else 1), "nu": NU, "F0": F0,
                       "storage": f"{args.storage} {args.pattern.upper()} "
                                  + ("staged in shared memory" if info["staged"] else "one node per thread"),
                       "block": [info["block_x"], info["block_y"]],
                       "l2": f"inputs larger than L2: {info['buffers']} population buffer(s) of "
                             f"{info['state_bytes'] / 1e9:.2f} GB vs 129 MB L2, no flush",
                       "parallelism": parallelism},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                         "algorithmic_bytes_per_launch": bytes_per_node * nodes,
                         "kernel": "k_step<Cascaded,float,1,false>" if default_case
                         else f"step kernel, {args.model} collision, {args.storage} storage, D3Q{args.lattice}, "
                              f"{args.pattern} pattern" + (", z-slab (faces + interior launches)" if slab else "")},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": K * (2 if slab else 1),
            "clocks": clocks,
            "variants": compact(variants) if variants else None,
        }
        if variants:
            print(json.dumps({"variants_full": variants}), file=sys.stderr, flush=True)
        print(json.dumps(line), flush=True)
    lat.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_batch_only(args):
    """Profiling aid: the batched sweep alone over the first --batch-only domains."""
    import torch

    from paper_1801_04586_gb300.builder import build
    build()
    torch.cuda.set_device(0)
    peak, _ = measured_peaks()
    out = bench_batch(torch.device("cuda", 0), args.batch_steps, peak, ndomains=args.batch_only)
    print(json.dumps({"batch_only": out}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.batch_only:
        return run_batch_only(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
