"""Benchmark of the implicit HGKS hot path on GB300.

One step = one pass of Algorithm 1's outer loop on the whole mesh: local time
step, residual R(U) (non-compact WENO reconstruction + BGK flux + gather),
assembly of A, 3 cycles of Jacobi-preconditioned GMRES(20), update.

Workload: inviscid flow past a unit sphere at M = 0.3, cubed-sphere O-grid with
6 patches of 32 x 32, 64 layers stretched by 1.08 to r = 10, split into
2,359,296 tetrahedra, uniform free-stream start; synthetic mesh (no dataset).
The working set (mesh data, Jacobian blocks, Krylov basis: ~15 GB) is far larger
than L2, so no flush is needed between steps.

Prints one JSON line (see the keys in `result`). `--impl reference` times the
CPU oracle on the same metric instead (a bounded sample of the workload).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "residual Mcells/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 (non-tensor) arithmetic peak of one GB300: 152 SMs x 2 DFMA per SM and clock
# (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on peak_sustained = 2/cycle) x 2
# flops x 2070 MHz = 1259 GFLOP/s, the recipe's nominal 1.25 TFLOP/s.
FP64_PEAK_GFLOPS = 1258.6
# FP64 flops per unit of work of each kernel (2 per DFMA, 1 per DADD/DMUL), from the
# ncu sass counters of the kernels on the 124,416-tet sphere (non-compact scheme,
# inviscid, Pr = 1); see DESIGN.md "Roofline". unit -> (flops per unit, units)
# DRAM bytes per unit of work from the same ncu captures (dram__bytes_read.sum +
# dram__bytes_write.sum divided by the units of the 124,416-tet launch); the
# traffic of a full launch is this times its units (traffic grows with the units).
KERNEL_TRAFFIC = {"flux": 490.1, "recon": 4265.0, "jacobi": 931.0, "spmv": 889.0}
KERNEL_FLOPS = {
    "flux": (3853.0, lambda N, F: 3 * F),        # per face Gauss point
    "recon": (4298.0, lambda N, F: 4 * N),       # per (cell, face)
    "jacobi": (229.0, lambda N, F: N),           # per cell and sweep
    "spmv": (205.0, lambda N, F: N),             # per cell
}


def workload(small=False):
    from paper_2304_09485_gb300 import inputs as I
    if small:
        m = I.sphere_mesh(12, 24, stretch=1.2)
        name = "sphere O-grid 6x12x12x24 -> 124,416 tets (scaled-down sample of the 6x32x32x64 case)"
    else:
        m = I.sphere_mesh(32, 64, stretch=1.08)
        name = "sphere O-grid 6x32x32x64, stretch 1.08 to r=10 -> 2,359,296 tets, inviscid M=0.3, WENO, GMRES(20)x3, Jacobi 2, CFL 10"
    cond = I.sphere_conditions(0.3)
    kw = dict(scheme=0, krylov_dim=20, restarts=3, jacobi_sweeps=2, cfl=10.0, **cond)
    return m, cond, kw, name


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1])); mx.append(float(r[2]))
                for k, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(k)
            except (ValueError, IndexError):
                pass
        if sm:
            out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def aggregate(local_ms, n_cells, steps, world, device="cpu"):
    """Max of the per-rank times (all ranks run their own replica) and the
    whole-job throughput in Mcells/s: world * cells * steps / max time."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, world * n_cells * steps / (ms / 1000.0) / 1e6


def measured_peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except (OSError, ValueError):
        return {}


def cpu_baseline(steps=1, max_seconds=30.0):
    """The oracle (FP64 C, OpenMP over the host cores) on a bounded sample of the
    workload: implicit steps on the scaled-down sphere of the same construction."""
    import oracle as O
    from paper_2304_09485_gb300 import inputs as I
    m, cond, kw, name = workload(small=True)
    om = O.OracleMesh(m)
    p = O.make_params(**kw)
    Q = I.state_from_conditions(m.n_tet, cond)
    om.gmres_step(p, Q)          # warm the fits (setup, not timed)
    t0 = time.perf_counter()
    done = 0
    for _ in range(steps):
        Q, _, _, _ = om.gmres_step(p, Q)
        done += 1
        if time.perf_counter() - t0 > max_seconds:
            break
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": m.n_tet * done / dt / 1e6, "unit": "Mcells/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} implicit step(s) on {m.n_tet} tets (6x12x12x24 sphere, same scheme and parameters)",
            "seconds": dt}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    steps = []
    for _ in range(args.warmup):
        pass
    cb = None
    t_all = 0.0
    vals = []
    for k in range(args.steps):
        cb = cpu_baseline(steps=1)
        vals.append(cb["value"])
        t_all += cb["seconds"]
    value = float(np.median(vals)) if vals else 0.0
    m, cond, kw, name = workload(small=True)
    res = {"metric": METRIC, "value": value, "unit": "Mcells/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1000.0 * t_all / max(1, args.steps), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": name, "sample_of": workload.__doc__ or "sphere 6x32x32x64"},
           "impl": "reference", "cpu_baseline": cb,
           "e2e": {"value": value, "unit": "Mcells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hgks", choices=["hgks", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--small", action="store_true", help="scaled-down mesh (profiling runs)")
    ap.add_argument("--launch-list", action="store_true",
                    help="warm-up then the timed steps only (no e2e, no residual-only pass): for ncu launch lists")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    import paper_2304_09485_gb300 as H
    from paper_2304_09485_gb300 import inputs as I

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    # the CPU oracle runs before any GPU work (and only on rank 0, N = 1)
    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(steps=1)
        cb.pop("seconds", None)

    m, cond, kw, name = workload(small=args.small)
    hm = H.hgks_mesh_create(m, scheme_mask=1, device=local)
    p = H.hgks_default_params(**kw)
    Q0 = I.state_from_conditions(m.n_tet, cond)
    Q = hm.to_internal(Q0, device=f"cuda:{local}")
    stream = torch.cuda.current_stream()
    nwarm = args.warmup if args.launch_list else max(3, args.warmup)
    for _ in range(nwarm):
        H.hgks_gmres_step(hm, p, Q)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    H.hgks_launch_count(reset=True)
    H.hgks_profile_begin()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        H.hgks_gmres_step(hm, p, Q)
    ev1.record(stream)
    barrier()
    prof = H.hgks_profile_end()
    launches = H.hgks_launch_count()
    clk = clocks.stop()
    ms, value = aggregate(ev0.elapsed_time(ev1), m.n_tet, args.steps, world, device=f"cuda:{local}")

    if args.launch_list:
        if rank == 0:
            print(json.dumps({"launch_list": True, "ms_per_step": ms / args.steps, "gpu_launches": int(launches),
                              "kernels_ms": {k: round(v[0], 3) for k, v in prof.items()}, "n_cells": m.n_tet}))
        return 0
    # residual alone (the R(U) kernels), same stream, for the residual throughput
    Rt = torch.empty_like(Q)
    H.hgks_residual(hm, p, Q, None, Rt)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    nres = 3
    for _ in range(nres):
        H.hgks_residual(hm, p, Q, None, Rt)
    e1.record(stream)
    torch.cuda.synchronize()
    res_ms = e0.elapsed_time(e1) / nres

    # the same step with the Krylov part in FP32 (precision = mixed), same state
    pm = H.hgks_default_params(precision=1, **kw)
    Qm = Q.clone()
    for _ in range(2):
        H.hgks_gmres_step(hm, pm, Qm)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        H.hgks_gmres_step(hm, pm, Qm)
    e1.record(stream)
    torch.cuda.synchronize()
    mixed_ms = e0.elapsed_time(e1) / args.steps
    del Qm

    # end to end through the C ABI with host buffers: copies inside the timed region
    Qh = torch.empty((5, m.n_tet), dtype=torch.float64, pin_memory=True)
    Qh.copy_(Q)
    Qh_np = Qh.numpy()
    H.hgks_gmres_step_host(hm, p, Qh_np)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        H.hgks_gmres_step_host(hm, p, Qh_np)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_val = world * m.n_tet * args.steps / e2e_s / 1e6

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    # roofline of the dominant kernel
    F = int(H.hgks_mesh_info(hm).n_faces)

    def kroof(name):
        kms, kcnt = prof[name]
        avg_s = kms / kcnt / 1000.0
        r = {"kernel": name, "bound": "alu", "unit": "GFLOP/s", "peak": FP64_PEAK_GFLOPS,
             "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (recipe nominal FP64 1.25 TFLOP/s)",
             "avg_launch_ms": avg_s * 1000.0, "launches": kcnt, "traffic": None}
        if name in KERNEL_FLOPS:
            per, units = KERNEL_FLOPS[name]
            fl = per * units(m.n_tet, F)
            r.update({"achieved": fl / avg_s / 1e9, "frac": fl / avg_s / 1e9 / FP64_PEAK_GFLOPS, "flops_per_launch": fl})
            if name in KERNEL_TRAFFIC:
                r["traffic"] = KERNEL_TRAFFIC[name] * units(m.n_tet, F)
                r["traffic_note"] = "bytes per launch: ncu dram bytes per unit on the 124,416-tet sphere x units"
        else:
            r.update({"achieved": None, "frac": None})
        return r
    kname = max(prof.items(), key=lambda kv: kv[1][0])[0] if prof else ""
    roof = kroof(kname) if kname else {}
    roof_all = {k: round(kroof(k)["frac"], 3) for k in KERNEL_FLOPS if k in prof}
    result = {
        "metric": METRIC, "value": value, "unit": "Mcells/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "n_cells": m.n_tet, "n_faces": F, "parallelism": f"replicas{world}",
                   "step": "dt + R(U) + A + 3 x GMRES(20) + update",
                   "l2": "inputs larger than L2 (mesh data + Jacobian + Krylov basis >> 129 MB)"},
        "residual_only": {"value": m.n_tet / (res_ms / 1000.0) / 1e6, "unit": "Mcells/s", "ms": res_ms},
        "mixed": {"value": world * m.n_tet / (mixed_ms / 1000.0) / 1e6, "unit": "Mcells/s", "ms_per_step": mixed_ms,
                  "note": "same step with FP32 Krylov basis, Arnoldi and Jacobi (FP64 residual and update)"},
        "e2e": {"value": e2e_val, "unit": "Mcells/s", "h2d_bytes_per_step": 5 * 8 * m.n_tet,
                "d2h_bytes_per_step": 5 * 8 * m.n_tet},
        "gpu_launches": int(launches),
        "kernels_ms": {k: round(v[0], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])},
        "roofline": roof,
        "roofline_frac_by_kernel": roof_all,
        "clocks": clk,
        "cpu_baseline": cb,
    }
    print(json.dumps(result))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
