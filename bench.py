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
import math
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
# FP64 (non-tensor) arithmetic peak of one GB300 from the unit counts: 152 SMs x 2
# DFMA per SM and clock (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on
# peak_sustained = 2/cycle) x 2 flops x 2070 MHz = 1259 GFLOP/s. The roofline uses
# the rate measured in the same run (hgks_fp64_peak: DFMA chains); this nominal
# figure is reported beside it.
FP64_NOMINAL_GFLOPS = 1258.6
# The work per unit of each FP64-bound kernel, held fixed (the roofline
# numerator): FP64 flops (2 per DFMA, 1 per DADD/DMUL) per unit, counted once by
# ncu's SASS instruction counters on the 124,416-tet sphere (non-compact scheme,
# inviscid, Pr = 1) for the kernels of the step at 190.8 ms per 2.36M-tet step,
# and frozen there as the method's work per unit: a later rewrite that needs
# fewer operations for the same result shows as a higher fraction, not a lower
# count. DRAM bytes per unit of work from the same ncu captures
# (dram__bytes_read.sum + dram__bytes_write.sum divided by the units of the
# 124,416-tet launch); the traffic of a full launch is this times its units.
# Since those captures the kernels were templated on the cell shape; their
# tetrahedral instances are the same loops with the face count as a template
# argument, compile to the same registers, stack frame and spills (-Xptxas -v)
# and take the same time per launch, so the counters still describe them.
KERNEL_TRAFFIC = {"flux": 395.6, "recon": 957.6, "jacobi": 858.0, "spmv": 935.0}
KERNEL_FLOPS = {
    "flux": (2242.5, lambda N, F: 3 * F),        # per face Gauss point
    "recon": (3000.9, lambda N, F: 4 * N),       # per (cell, face)
    # the Krylov products: "jacobi" = products D^-1 O x (120 of a C2 step's 126
    # launches are the E products of the Neumann form, 195.7 flop; 6 are the sweeps
    # of the restart vector, ~219), "spmv" = products with O plus a vector (60 of 63
    # are the final v + E z products with the fused inner product, 216.9; 3 are
    # r0 = b - A x, 195.7): launch-weighted means per cell
    "jacobi": (196.8, lambda N, F: N),
    "spmv": (215.9, lambda N, F: N),
}


def workload(small=False, sphere_n=0):
    from paper_2304_09485_gb300 import inputs as I
    if sphere_n:
        m = I.sphere_mesh(sphere_n, 2 * sphere_n, stretch=I.sphere_stretch(2 * sphere_n))
        name = f"sphere O-grid 6x{sphere_n}x{sphere_n}x{2 * sphere_n} -> {m.n_tet:,} tets (profiling size)"
    elif small:
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
    t1 = time.perf_counter()
    om.residual(p, Q)                  # the residual alone (fits already built)
    res_s = time.perf_counter() - t1
    cores = O.set_threads(0)           # the OpenMP threads the timed steps ran on (0: query only)
    # the residual of the compact cavity (3,072 tets, HWENO, viscous) on one core and on all
    mc = I.cavity_mesh(8)
    cc = I.cavity_conditions(0.15, 100.0)
    oc = O.OracleMesh(mc)
    pc = O.make_params(scheme=1, Pr=0.72, **cc)
    Qc, Gc = I.smooth_state(mc, amp=0.02, base=(1.0, 0.1, 0.0, 0.0, cc["p_inf"]))
    oc.residual(pc, Qc, Gc)                                  # fits (setup, not timed)
    cav = {}
    prev = O.set_threads(1)
    for label, nt in (("1_core", 1), (f"{prev}_cores", prev)):
        O.set_threads(nt)
        t2 = time.perf_counter()
        for _ in range(5):
            oc.residual(pc, Qc, Gc)
        cav[label] = mc.n_tet * 5 / (time.perf_counter() - t2) / 1e6
    O.set_threads(prev)
    return {"value": m.n_tet * done / dt / 1e6, "unit": "Mcells/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} implicit step(s) on {m.n_tet} tets (6x12x12x24 sphere, same scheme and parameters)",
            "residual_only": {"value": m.n_tet / res_s / 1e6, "unit": "Mcells/s"},
            "residual_cavity_3072_hweno_mcells_per_s": cav,
            "seconds": dt}


def step_config(name, n_cells, n_faces, world):
    """The `config` object of the whole-step line (both arms)."""
    return {"workload": name, "n_cells": int(n_cells), "n_faces": int(n_faces), "parallelism": f"replicas{world}",
            "step": "dt + R(U) + A + 3 x GMRES(20) + update",
            "l2": "inputs larger than L2 (mesh data + Jacobian + Krylov basis >> 129 MB)"}


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle (the paper publishes no code) on the same
    metric and workload, on a bounded sample of it: implicit steps on the
    124,416-tet sphere of the same construction, W untimed warm-up steps (the
    first builds the fits) and K timed ones. Rank 0 only."""
    if rank != 0:
        return 0
    import oracle as O
    from paper_2304_09485_gb300 import inputs as I
    m, cond, kw, _ = workload(small=True)
    om = O.OracleMesh(m)
    p = O.make_params(**kw)
    Q = I.state_from_conditions(m.n_tet, cond)
    for _ in range(max(1, args.warmup)):
        Q, _, _, _ = om.gmres_step(p, Q)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Q, _, _, _ = om.gmres_step(p, Q)
    t_all = time.perf_counter() - t0
    value = m.n_tet * args.steps / t_all / 1e6 if args.steps else 0.0
    _, _, _, name = workload(small=True)
    cores = O.set_threads(0)           # the OpenMP threads the timed steps ran on (0: query only)
    cb = {"value": value, "unit": "Mcells/s", "cores": cores, "kind": "oracle",
          "sample": f"{args.steps} implicit step(s) on {m.n_tet} tets (6x12x12x24 sphere, same scheme and "
                    f"parameters) after {max(1, args.warmup)} untimed"}
    res = {"metric": METRIC, "value": value, "unit": "Mcells/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1000.0 * t_all / max(1, args.steps), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": step_config(name, m.n_tet, om.nf, world),
           "impl": "reference", "cpu_baseline": cb,
           "e2e": {"value": value, "unit": "Mcells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res))
    return 0


def paper_timing_context(H, I, device):
    """Seconds per 100 implicit steps on the paper's efficiency case: lid-driven
    cavity, 6 x 20^3 tets with h_min = 2.5e-2 at the walls, Ma 0.15, Re 1000,
    GMRES(10) x 3, Jacobi 2, CFL 10, FP64, from rest. The paper's figures are
    30 s (non-compact) and 32 s (compact) on a Quadro RTX 8000."""
    import torch
    m = I.cavity_mesh(20, h_min=2.5e-2)
    cond = I.cavity_conditions(0.15, 1000.0)
    hm = H.hgks_mesh_create(m, scheme_mask=3, device=device)
    out = {"workload": "cavity 6x20^3 = 48,000 tets, h_min 2.5e-2, Ma 0.15, Re 1000, GMRES(10)x3, Jacobi 2, CFL 10, FP64",
           "paper_rtx8000_s_per_100_steps": {"weno": 30.0, "hweno": 32.0}}
    for name, scheme in (("weno", 0), ("hweno", 1)):
        p = H.hgks_default_params(scheme=scheme, Pr=0.72, krylov_dim=10, restarts=3, jacobi_sweeps=2, **cond)
        Q = hm.to_internal(I.state_from_conditions(m.n_tet, cond), device=f"cuda:{device}")
        G = torch.zeros((15, m.n_tet), dtype=torch.float64, device=f"cuda:{device}") if scheme else None
        for _ in range(3):
            H.hgks_gmres_step(hm, p, Q, G)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info, hist, _ = H.hgks_solve_steady(hm, p, Q, G, drop_tol=1e-300, max_steps=100)
        torch.cuda.synchronize()
        out[f"{name}_s_per_100_steps"] = (time.perf_counter() - t0) * 100.0 / max(1, info.steps)
        out[f"{name}_residual_drop_after_100"] = float(hist[-1] / hist.max())
    return out


def run_batch(args, rank, world):
    """Many independent steady problems of uneven size advanced together
    (hgks_batch_*: one launch per phase for all meshes, the step replayed from a
    CUDA graph) against the same meshes stepped one at a time through the
    single-mesh path. Prints one JSON line of its own."""
    import torch
    import paper_2304_09485_gb300 as H
    from paper_2304_09485_gb300 import inputs as I
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    t0 = time.perf_counter()
    probs = I.batch_problems(args.batch_meshes, seed=I.BASE_SEED + 400 + 1000 * rank)
    scheme = 1 if args.batch_scheme == "hweno" else 0
    prec = 1 if args.batch_precision == "mixed" else 0
    meshes, params, states = [], [], []
    for pr in probs:
        hm = H.hgks_mesh_create(pr["mesh"], scheme_mask=2 if scheme else 1, device=local)
        kw = dict(pr["cond"], scheme=scheme, precision=prec, Pr=0.72, krylov_dim=10, restarts=3, jacobi_sweeps=2)
        meshes.append(hm)
        params.append(H.hgks_default_params(**kw))
        Q = hm.to_internal(I.state_from_conditions(pr["n_cells"], pr["cond"]), device=f"cuda:{local}")
        G = torch.zeros((15, pr["n_cells"]), dtype=torch.float64, device=f"cuda:{local}") if scheme else None
        states.append((Q, G))
        pr["mesh"] = None
    setup_s = time.perf_counter() - t0
    n_cells = sum(p["n_cells"] for p in probs)
    b = H.hgks_batch_create(meshes, params)
    init_states = [(Q.clone(), None if G is None else G.clone()) for Q, G in states]
    for k, (Q, G) in enumerate(states):
        H.hgks_batch_set_state(b, k, Q, G)
    blk = H.hgks_batch_autotune(b)
    for _ in range(max(3, args.warmup)):
        H.hgks_batch_gmres_step(b)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    if args.launch_list:                  # one batched step after the warm-up (ncu launch lists)
        H.hgks_launch_count(reset=True)
        H.hgks_profile_begin()
        H.hgks_batch_gmres_step(b)
        prof = H.hgks_profile_end()
        if rank == 0:
            print(json.dumps({"launch_list": True, "gpu_launches": H.hgks_launch_count(), "n_cells": n_cells,
                              "kernels_ms": {k: round(v[0], 3) for k, v in prof.items()}}))
        return 0
    clocks = ClockSampler(local)
    clocks.start()
    # (a) batched steps replayed from the captured graph of the step
    H.hgks_batch_gmres_step(b, use_graph=True)          # capture (not timed)
    torch.cuda.synchronize()
    H.hgks_launch_count(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        H.hgks_batch_gmres_step(b, use_graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1)
    launches = H.hgks_launch_count()
    # (a') per-kernel times of one eager batched step
    H.hgks_profile_begin()
    H.hgks_batch_gmres_step(b, use_graph=False)
    prof = H.hgks_profile_end()
    # (b) batched steps, eager launches
    e0.record(stream)
    for _ in range(args.steps):
        H.hgks_batch_gmres_step(b, use_graph=False)
    e1.record(stream)
    torch.cuda.synchronize()
    eager_ms = e0.elapsed_time(e1)
    # (b') the device-side convergence loop (hgks_batch_solve_steady, graph replay):
    # steps steps, then one last residual and test per mesh
    e0.record(stream)
    infos, _, _ = H.hgks_batch_solve_steady(b, 1e-300, args.steps, use_graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    solve_ms = e0.elapsed_time(e1)
    # (c) the same meshes one after another through the single-mesh path
    for hm, p, (Q, G) in zip(meshes, params, states):
        H.hgks_gmres_step(hm, p, Q, G)
    torch.cuda.synchronize()
    e0.record(stream)
    for hm, p, (Q, G) in zip(meshes, params, states):
        for _ in range(args.steps):
            H.hgks_gmres_step(hm, p, Q, G)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    # (d) optionally: every mesh solved from its initial state to a drop, as one batch
    # (device-side convergence test, graph replay): how many converge, in how many steps
    solve = None
    if args.batch_drop > 0:
        for k, (Q0k, G0k) in enumerate(init_states):
            H.hgks_batch_set_state(b, k, Q0k, G0k)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        infos_d, hist_d, _ = H.hgks_batch_solve_steady(b, args.batch_drop, args.batch_max_steps, use_graph=True,
                                                       raise_nonfinite=False)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t1
        bad = [i for i in infos_d if not math.isfinite(i.res_final)]
        solve = {"drop": args.batch_drop, "max_steps": args.batch_max_steps, "seconds": wall,
                 "converged": sum(1 for i in infos_d if i.converged), "meshes": len(infos_d),
                 "non_finite": len(bad),
                 "steps_converged": sorted(int(i.steps) for i in infos_d if i.converged),
                 "final_drop_not_converged": sorted(float(i.res_final / i.res_ref) for i in infos_d
                                                   if not i.converged and i.res_ref > 0
                                                   and math.isfinite(i.res_final))}
    if rank != 0:
        return 0
    rate = lambda ms, steps: n_cells * steps / (ms / 1000.0) / 1e6
    res = {"metric": "batched implicit steps Mcells/s", "value": rate(graph_ms, args.steps),
           "unit": "Mcells/s", "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
           "ms_per_step": graph_ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64+f32" if prec else "f64", "data": "synthetic",
           "config": {"workload": f"{len(probs)} independent steady problems, cavity/sphere, "
                                  f"{min(p['n_cells'] for p in probs)}-{max(p['n_cells'] for p in probs)} tets "
                                  f"({n_cells} total), Mach U(0.1,0.5), Re logU(50,1000), "
                                  f"{args.batch_scheme}, {args.batch_precision}, GMRES(10)x3, Jacobi 2, CFL 10",
                      "n_cells": n_cells, "padded_cells": int(H.hgks_batch_info(b).n_cells),
                      "l2": "inputs larger than L2", "blk_recon_flux": list(blk)},
           "graph": {"value": rate(graph_ms, args.steps), "ms": graph_ms},
           "eager": {"value": rate(eager_ms, args.steps), "ms": eager_ms},
           "solve_loop": {"value": rate(solve_ms, args.steps), "ms": solve_ms,
                          "note": "hgks_batch_solve_steady (graph replay, device-side convergence test): "
                                  "steps full steps plus the final residual and test, counted as steps steps"},
           "sequential_single_mesh": {"value": rate(seq_ms, args.steps), "ms": seq_ms},
           "speedup_vs_sequential": seq_ms / graph_ms,
           "kernels_ms_one_step": {k: round(v[0], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])},
           "gpu_launches": int(launches), "setup_s": setup_s, "clocks": clk,
           "solve_to_drop": solve,
           "sizes": sorted(p["n_cells"] for p in probs)}
    print(json.dumps(res))
    return 0


def run_precision(args, rank, world):
    """The precision workload: viscous flow past a sphere (Re 118, Ma 0.2535,
    6 x 24 x 24 patches, 48 layers stretched so that the first is 3e-2 thick,
    ~995k tets, adiabatic no-slip wall), compact HWENO, CFL 20. The same steps
    in FP64 and with the FP32 Krylov part, from the free stream: density
    residual history, drag coefficient every few steps, state difference, time
    per step. With Algorithm 1's gradient update the compact solve settles into
    a two-step cycle at the separation line on these tetrahedral sphere grids,
    so C_D is reported over the last steps as the mean and the spread; with
    --grad-relax 0.5 the cycle is damped and the solve keeps converging. The
    comparison with the oracle on a scaled-down
    sphere of the same construction is a GPU test
    (tests/test_gpu_precision.py)."""
    import torch
    import paper_2304_09485_gb300 as H
    from paper_2304_09485_gb300 import inputs as I
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    cond = I.sphere_conditions(0.2535, Re=118.0)
    kw = dict(scheme=1, Pr=0.72, cfl=20.0, krylov_dim=10, restarts=3, jacobi_sweeps=2, grad_relax=args.grad_relax)
    qinf = 0.5 * cond["rho_inf"] * cond["u_inf"][0] ** 2 * math.pi * 0.25

    def cd(hm, p, Q, G):
        return float(H.hgks_wall_force(hm, p, Q, G, I.BC_NOSLIP_ADIA)[0] / qinf)

    out = {}
    # the full-size case on the GPU: FP64 against mixed
    m = I.sphere_mesh(24, 48, stretch=I.sphere_stretch(48, dr1=3e-2), wall_tag=I.BC_NOSLIP_ADIA)
    hm = H.hgks_mesh_create(m, scheme_mask=2, device=local)
    traj = {}
    every = max(1, args.steps // 20)
    for prec in (0, 1):
        p = H.hgks_default_params(precision=prec, **cond, **kw)
        Q = hm.to_internal(I.state_from_conditions(m.n_tet, cond), device=f"cuda:{local}")
        G = torch.zeros((15, m.n_tet), dtype=torch.float64, device=f"cuda:{local}")
        cds, hist, ms = [], [], 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for k in range(args.steps):
            e0.record()
            info = H.hgks_gmres_step(hm, p, Q, G)
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            hist.append(info.res_l1)
            if (k + 1) % every == 0 or k >= args.steps - 10:
                cds.append((k + 1, cd(hm, p, Q, G)))
        traj[prec] = (Q, G, cds, np.array(hist), ms / args.steps)
    (Q64, G64, cd64, h64, ms64), (Q32, G32, cd32, h32, ms32) = traj[0], traj[1]
    last = lambda c: [v for k, v in c if k > args.steps - 10]
    out["full"] = {"n_cells": m.n_tet, "steps": args.steps,
                   "cd_fp64": cd64, "cd_mixed": cd32,
                   "cd_last10_fp64": {"mean": float(np.mean(last(cd64))), "min": min(last(cd64)), "max": max(last(cd64))},
                   "cd_last10_mixed": {"mean": float(np.mean(last(cd32))), "min": min(last(cd32)), "max": max(last(cd32))},
                   "cd_rel_diff": abs(np.mean(last(cd32)) - np.mean(last(cd64))) / abs(np.mean(last(cd64))),
                   "drop_fp64": (h64 / h64.max())[::every].tolist(), "drop_mixed": (h32 / h32.max())[::every].tolist(),
                   "final_drop_fp64": float(h64[-1] / h64.max()), "final_drop_mixed": float(h32[-1] / h32.max()),
                   "state_rel_l2": float(torch.linalg.norm(Q32 - Q64) / torch.linalg.norm(Q64)),
                   "ms_per_step_fp64": ms64, "ms_per_step_mixed": ms32,
                   "mcells_per_s_fp64": m.n_tet / ms64 / 1e3, "mcells_per_s_mixed": m.n_tet / ms32 / 1e3}
    del traj, Q64, G64, Q32, G32, hm
    if rank != 0:
        return 0
    res_line = {"metric": "precision: drag coefficient and state error, FP32 Krylov vs FP64", "value": out["full"]["cd_rel_diff"],
                "unit": "relative C_D difference (mean of the last 10 steps)", "n_gpus": world, "steps": args.steps,
                "warmup": 0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
                "data": "synthetic",
                "config": {"workload": "viscous sphere Re 118, Ma 0.2535, 6x24x24x48 (first layer 3e-2), HWENO, CFL 20, "
                                       "GMRES(10)x3, Jacobi 2, from the free stream",
                           "grad_relax": args.grad_relax}, **out}
    print(json.dumps(res_line))
    return 0


def run_hex(args, rank, world):
    """Hexahedral cells (Sec. 3.1): the sphere workload's solver settings
    (inviscid Ma 0.3, GMRES(20)x3, Jacobi 2, CFL 10, FP64) on n^3 hexahedra between
    tilted planes (planar faces, cells that are not parallelepipeds), far field
    all round, from a smooth perturbation of the free stream. For both schemes:
    residual and implicit-step throughput, per-kernel times of one step, and the
    flux kernel's fraction of the FP64 peak (its work per Gauss point is the
    tetrahedral flux's: the same flux function)."""
    import torch
    import paper_2304_09485_gb300 as H
    from paper_2304_09485_gb300 import inputs as I
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    fp64_peak = H.hgks_fp64_peak(local, 2.0)
    cond = I.sphere_conditions(0.3)
    m = I.hex_tilted_box_mesh(args.hex_n)
    t0 = time.time()
    hm = H.hgks_mesh_create(m, scheme_mask=3, device=local)
    setup_s = time.time() - t0
    F = H.hgks_mesh_info(hm).n_faces
    u = cond["u_inf"]
    Q0, G0 = I.smooth_state(m, amp=0.05, base=(cond["rho_inf"], u[0], u[1], u[2], cond["p_inf"]))
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    clocks = ClockSampler(local)
    clocks.start()
    for scheme in (0, 1):
        p = H.hgks_default_params(scheme=scheme, krylov_dim=20, restarts=3, jacobi_sweeps=2, cfl=10.0, **cond)
        Q, G = hm.to_internal(Q0, device=dev), hm.to_internal(G0, device=dev)
        R, Gn = torch.empty_like(Q), torch.empty_like(G)
        gargs = (G, R, Gn) if scheme else (None, R, None)
        for _ in range(3):
            H.hgks_residual(hm, p, Q, *gargs)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            H.hgks_residual(hm, p, Q, *gargs)
        e1.record(stream)
        torch.cuda.synchronize()
        res_ms = e0.elapsed_time(e1) / args.steps
        for _ in range(max(3, args.warmup)):
            H.hgks_gmres_step(hm, p, Q, G if scheme else None)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            H.hgks_gmres_step(hm, p, Q, G if scheme else None)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms = e0.elapsed_time(e1) / args.steps
        H.hgks_profile_begin()
        H.hgks_gmres_step(hm, p, Q, G if scheme else None)
        prof = H.hgks_profile_end()
        fl_ms, fl_n = prof["flux"][0], prof["flux"][1]
        flux_gflops = KERNEL_FLOPS["flux"][0] * 4 * F / (fl_ms / fl_n * 1e-3) / 1e9
        res[("weno", "hweno")[scheme]] = {
            "residual_ms": res_ms, "residual_mcells_per_s": m.n_cells / res_ms / 1e3,
            "step_ms": step_ms, "step_mcells_per_s": m.n_cells / step_ms / 1e3,
            "kernels_ms_one_step": {k: round(v[0], 3) for k, v in prof.items()},
            "flux_fp64_frac": flux_gflops / fp64_peak}
    clk = clocks.stop()
    if rank != 0:
        return 0
    line = {"metric": "hexahedral mesh: residual and implicit-step Mcells/s", "value": res["weno"]["step_mcells_per_s"],
            "unit": "Mcells/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.hex_n}^3 = {m.n_cells:,} hexahedra between tilted planes, far field, "
                                   "inviscid Ma 0.3, GMRES(20)x3, Jacobi 2, CFL 10, FP64", "n_faces": F,
                       "mesh_setup_s": setup_s, "l2": "inputs larger than L2"},
            "fp64_peak_gflops": fp64_peak, "clocks": clk, **res}
    print(json.dumps(line))
    return 0


def wake_and_separation(m, Qc, radii):
    """Closed wake length L (diameters, from the rear of the sphere to where u_x
    changes sign on the downstream axis) and separation angle theta (degrees from
    the front stagnation point, where the meridional velocity of the first cell
    layer, averaged over the azimuth in 2-degree bins, changes sign) from the cell
    states Qc [n, 5] (caller order) of a sphere of diameter 1 in a flow along +x."""
    cen = m.xyz[m.cells].mean(1)
    u = Qc[:, 1:4] / Qc[:, :1]
    r = np.linalg.norm(cen, axis=1)
    first = r < radii[1]
    c, uf = cen[first], u[first]
    cn = c / np.linalg.norm(c, axis=1)[:, None]
    th = np.degrees(np.arccos(np.clip(-cn[:, 0], -1.0, 1.0)))
    e = np.array([1.0, 0.0, 0.0])[None, :] - cn * cn[:, :1]
    e_th = e / np.maximum(np.linalg.norm(e, axis=1), 1e-30)[:, None]
    ut = np.einsum("ij,ij->i", uf, e_th)
    bins = np.linspace(0.0, 180.0, 91)
    idx = np.digitize(th, bins) - 1
    prof = np.array([ut[idx == k].mean() if np.any(idx == k) else np.nan for k in range(90)])
    mid = 0.5 * (bins[1:] + bins[:-1])
    theta = None
    for k in range(1, 90):
        if mid[k] > 60.0 and np.isfinite(prof[k - 1]) and np.isfinite(prof[k]) and prof[k - 1] > 0.0 >= prof[k]:
            theta = float(mid[k - 1] + (mid[k] - mid[k - 1]) * prof[k - 1] / (prof[k - 1] - prof[k]))
            break
    n = m.meta["n"]
    ax = (cen[:, 0] > 0.5) & (np.linalg.norm(cen[:, 1:], axis=1) < 0.8 * cen[:, 0] * (math.pi / 2) / n)
    xs, ux = cen[ax, 0], u[ax, 0]
    o = np.argsort(xs)
    xs, ux = xs[o], ux[o]
    L = None
    for k in range(1, len(xs)):
        if ux[k - 1] < 0.0 <= ux[k]:
            L = float(xs[k - 1] + (xs[k] - xs[k - 1]) * (-ux[k - 1]) / (ux[k] - ux[k - 1]) - 0.5)
            break
    return L, theta


def run_hexsphere(args, rank, world):
    """Sec. 5.2's viscous sphere on hexahedra: a cubed-sphere O-grid of 6 x 32 x
    32 x 31 = 190,464 hexahedra (the paper's cell count) with a first layer 3e-2
    thick, adiabatic no-slip wall, GMRES(10) x 3, Jacobi 2, from the free stream;
    Re 118, Ma 0.2535 with linear weights at CFL 20, or Re 300, Ma 1.5 with
    nonlinear weights at CFL 5 (the paper's two cases). Algorithm 1 to a 1e-10 drop
    (or the step limit) with both schemes in FP64 and the compact one with the
    FP32 Krylov part: steps, time, C_D, the closed wake length L and the
    separation angle theta, beside the values the paper prints for its own
    190,464-cell hexahedral grid (context: the grids differ)."""
    import torch
    import paper_2304_09485_gb300 as H
    from paper_2304_09485_gb300 import inputs as I
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    layers = 31
    stretch = I.sphere_stretch(layers, dr1=3e-2)
    m = I.hex_sphere_mesh(32, layers, stretch=stretch)
    radii = I.sphere_radii(layers, 0.5, 10.0, stretch)
    hm = H.hgks_mesh_create(m, scheme_mask=3, device=local)
    # the paper's two cases on this grid: Re 118, Ma 0.2535, linear weights, CFL 20;
    # Re 300, Ma 1.5, nonlinear weights, CFL 5
    sub = args.hexsphere_case == "re118"
    cond = I.sphere_conditions(0.2535, Re=118.0) if sub else I.sphere_conditions(1.5, Re=300.0)
    weights, cfl = (1, 20.0) if sub else (0, 5.0)
    paper = ({"GMRES-HWENO": {"L": 0.95, "theta_deg": 128.1}, "GMRES-WENO": {"L": 0.91, "theta_deg": 124.5}} if sub else
             {"GMRES-HWENO": {"L": 1.16, "theta_deg": 135.9}, "GMRES-WENO": {"L": 1.17, "theta_deg": 135.4}})
    qinf = 0.5 * cond["rho_inf"] * cond["u_inf"][0] ** 2 * math.pi * 0.25
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    res = {}
    for name, scheme, prec in (("GMRES-HWENO", 1, 0), ("GMRES-WENO", 0, 0), ("GMRES-HWENO, FP32 Krylov", 1, 1)):
        p = H.hgks_default_params(scheme=scheme, weights=weights, precision=prec, Pr=0.72, cfl=cfl, krylov_dim=10,
                                  restarts=3, jacobi_sweeps=2, **cond)
        Q = hm.to_internal(I.state_from_conditions(m.n_cells, cond), device=dev)
        G = torch.zeros((15, m.n_cells), dtype=torch.float64, device=dev)
        e0.record(stream)
        info, hist, conv = H.hgks_solve_steady(hm, p, Q, G if scheme else None, drop_tol=args.hexsphere_drop,
                                               max_steps=args.hexsphere_max_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        L, theta = wake_and_separation(m, hm.to_caller(Q), radii)
        cd = float(H.hgks_wall_force(hm, p, Q, G if scheme else None, I.BC_NOSLIP_ADIA)[0] / qinf)
        res[name] = {"converged": bool(conv), "steps": int(info.steps), "final_drop": float(hist[-1] / hist.max()),
                     "seconds": sec, "mcells_per_s": m.n_cells * info.steps / sec / 1e6, "C_D": cd, "L": L,
                     "theta_deg": theta, "state": Q}
    clk = clocks.stop()
    q64, q32 = res["GMRES-HWENO"].pop("state"), res["GMRES-HWENO, FP32 Krylov"].pop("state")
    res["GMRES-WENO"].pop("state")
    state_diff = float(torch.linalg.norm(q32 - q64) / torch.linalg.norm(q64))
    if rank != 0:
        return 0
    line = {"metric": "viscous sphere on hexahedra: closed wake length and separation angle at a converged steady state",
            "value": res["GMRES-HWENO"]["L"], "unit": "L (diameters), GMRES-HWENO", "n_gpus": world,
            "steps": res["GMRES-HWENO"]["steps"], "warmup": 0, "higher_is_better": None, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": ("sphere Re 118, Ma 0.2535, " if sub else "sphere Re 300, Ma 1.5, ") +
                                   "cubed-sphere O-grid 6x32x32x31 = 190,464 hexahedra, first layer 3e-2, adiabatic "
                                   "no-slip wall, " + ("linear weights, CFL 20" if sub else "nonlinear weights, CFL 5") +
                                   f", GMRES(10)x3, Jacobi 2, from the free stream, drop {args.hexsphere_drop:g}, "
                                   f"max {args.hexsphere_max_steps} steps"},
            "results": res, "fp32_vs_fp64_state_rel_l2": state_diff, "paper_190464_hex": paper,
            "clocks": clk}
    print(json.dumps(line))
    return 0


def run_serve(args, rank, world):
    """Steady-solve requests with Poisson arrivals served by the continuous-
    batching server (mixed precision) against the same requests solved one
    after another with the single-mesh FP64 solver (a live stream too: first
    come, first served, each waits for its arrival and for the one before).
    Time to convergence (TTC) runs from a request's arrival to its finished
    state; mesh building is included. Solves per hour count converged requests
    only; requests that hit the step limit or went non-finite are reported
    apart."""
    import torch
    import paper_2304_09485_gb300 as H
    from paper_2304_09485_gb300 import inputs as I
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    reqs = I.serving_requests(args.serve_requests, n_min=args.serve_min_tets, n_max=args.serve_max_tets,
                              rate=args.serve_rate, seed=I.BASE_SEED + 500 + 1000 * rank,
                              viscous_fraction=args.serve_viscous_fraction,
                              cavity_fraction=args.serve_cavity_fraction)
    kw = dict(scheme=0, krylov_dim=10, restarts=3, jacobi_sweeps=2)
    drop, max_steps = args.serve_drop, args.serve_max_steps
    for r in reqs:
        r["Q0"] = I.state_from_conditions(r["n_cells"], r["cond"])
        r["p"] = dict(r["cond"], Pr=0.72 if r["cond"]["viscous"] else 1.0, **kw)

    def pct(v, q):
        return float(np.percentile(np.asarray(v), q)) if v else None

    # (a) the server, mixed precision, arrivals in real time
    shared = H.hgks_default_params(precision=1, **kw)
    srv = H.hgks_server(shared, hbm_budget_bytes=int(args.serve_budget_gb * 1e9), max_inflight=64, device=local)
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()
    ids, nxt, rounds, done = {}, 0, 0, 0
    while done < len(reqs):
        now = time.perf_counter() - t0
        while nxt < len(reqs) and reqs[nxt]["arrival"] <= now:
            r = reqs[nxt]
            ids[nxt] = srv.submit(r["mesh"], H.hgks_default_params(precision=1, **r["p"]), r["Q0"], drop_tol=drop,
                                  max_steps=max_steps)
            nxt += 1
        fin, run, wait = srv.step()
        rounds += 1
        done += fin
        if run == 0:
            if wait == 0 and nxt < len(reqs):
                time.sleep(max(0.0, min(0.05, reqs[nxt]["arrival"] - (time.perf_counter() - t0))))
            else:
                time.sleep(0.002)
    clk = clocks.stop()
    served = []
    for k, rid in ids.items():
        st = srv.status(rid)
        served.append(dict(ttc=st.t_done - st.t_submit, steps=st.solve.steps, converged=bool(st.solve.converged),
                           failed=st.status == H.HGKS_ERR_NONPHYSICAL, admit_wait=st.t_admit - st.t_built,
                           done=st.t_done, submit=st.t_submit))
        srv.collect(rid)
    info = srv.info()
    del srv
    span_a = max(s["done"] for s in served) - min(s["submit"] for s in served)
    # (b) one after another, FP64, as a live stream: each request is taken when it
    # has arrived and the one before it is done (first come, first served)
    seq, end = [], 0.0
    t0b = time.perf_counter()
    for r in reqs:
        wait = r["arrival"] - (time.perf_counter() - t0b)
        if wait > 0:
            time.sleep(wait)
        t1 = time.perf_counter()
        hm = H.hgks_mesh_create(r["mesh"], scheme_mask=1, device=local)
        Q = hm.to_internal(r["Q0"], device=f"cuda:{local}")
        failed = False
        try:
            si, hist, conv = H.hgks_solve_steady(hm, H.hgks_default_params(**r["p"]), Q, None, drop_tol=drop,
                                                 max_steps=max_steps)
            steps = si.steps
        except H.HGKSError as e:
            if e.status != H.HGKS_ERR_NONPHYSICAL:
                raise
            failed, conv, steps = True, False, -1
        torch.cuda.synchronize()
        end = time.perf_counter() - t0b
        dur = time.perf_counter() - t1
        del hm, Q
        seq.append(dict(ttc=end - r["arrival"], steps=steps, converged=bool(conv), failed=failed, service=dur))
    span_b = end - reqs[0]["arrival"]
    if rank != 0:
        return 0
    conv_a = [s["ttc"] for s in served if s["converged"]]
    conv_b = [s["ttc"] for s in seq if s["converged"]]
    res = {"metric": "steady solves/hour (served, mixed)", "value": 3600.0 * len(conv_a) / span_a, "unit": "solves/h",
           "n_gpus": world, "steps": len(reqs), "warmup": 0, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
           "config": {"workload": f"{len(reqs)} steady-solve requests, Poisson arrivals at {args.serve_rate}/s, "
                                  f"meshes of {min(r['n_cells'] for r in reqs)}-{max(r['n_cells'] for r in reqs)} tets: "
                                  f"a fraction {args.serve_cavity_fraction} lid-driven cavities (lid Mach U(0.2,0.5), "
                                  f"Re logU(50,1000)), the rest spheres, "
                                  f"inviscid (Mach U(0.2,0.5), AoA U(0,10)) and a fraction {args.serve_viscous_fraction} "
                                  f"viscous (Re logU(50,1000)), "
                                  f"WENO, GMRES(10)x3, Jacobi 2, CFL 10, drop {drop:g}, max {max_steps} steps",
                      "kinds": {k: sum(r["kind"] == k for r in reqs) for k in sorted({r["kind"] for r in reqs})},
                      "hbm_budget_gb": args.serve_budget_gb, "arena_cells": int(info.n_cells),
                      "arena_gb": info.device_bytes / 1e9},
           "served_mixed": {"solves_per_hour": 3600.0 * len(conv_a) / span_a,
                            "finished_per_hour": 3600.0 * len(served) / span_a, "p50_ttc_s": pct([s["ttc"] for s in served], 50),
                            "p99_ttc_s": pct([s["ttc"] for s in served], 99), "converged": len(conv_a),
                            "failed_nonfinite": sum(s["failed"] for s in served),
                            "hit_max_steps": len(served) - len(conv_a) - sum(s["failed"] for s in served),
                            "p50_ttc_converged_s": pct(conv_a, 50),
                            "p99_ttc_converged_s": pct(conv_a, 99), "rounds": rounds, "span_s": span_a,
                            "mean_steps": float(np.mean([s["steps"] for s in served]))},
           "sequential_fp64": {"solves_per_hour": 3600.0 * len(conv_b) / span_b,
                               "finished_per_hour": 3600.0 * len(seq) / span_b, "p50_ttc_s": pct([s["ttc"] for s in seq], 50),
                               "p99_ttc_s": pct([s["ttc"] for s in seq], 99), "converged": len(conv_b),
                               "failed_nonfinite": sum(s["failed"] for s in seq),
                               "hit_max_steps": len(seq) - len(conv_b) - sum(s["failed"] for s in seq),
                               "p50_ttc_converged_s": pct(conv_b, 50),
                               "p99_ttc_converged_s": pct(conv_b, 99), "span_s": span_b,
                               "mean_steps": float(np.mean([s["steps"] for s in seq if s["steps"] >= 0])),
                               "mean_service_s": float(np.mean([s["service"] for s in seq]))},
           "requests": [{"kind": r["kind"], "n_cells": r["n_cells"], "served_steps": a["steps"],
                         "served_converged": a["converged"], "sequential_steps": b["steps"],
                         "sequential_converged": b["converged"]} for r, a, b in zip(reqs, served, seq)],
           "clocks": clk}
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
    ap.add_argument("--sphere-n", type=int, default=0, help="sphere of n x n patches and 2n layers (profiling runs)")
    ap.add_argument("--workload", default="sphere",
                    choices=["sphere", "batch", "serve", "precision", "hex", "hexsphere"],
                    help="sphere: the 2.36M-tet sphere (default); batch: many problems in one batch; "
                         "serve: Poisson-arriving solves through the request server")
    ap.add_argument("--serve-requests", type=int, default=96)
    ap.add_argument("--serve-rate", type=float, default=0.4,
                    help="requests per second (0.4: about 0.8 x the measured served capacity of ~0.5/s)")
    ap.add_argument("--serve-min-tets", type=float, default=30e3)
    ap.add_argument("--serve-max-tets", type=float, default=250e3)
    ap.add_argument("--serve-viscous-fraction", type=float, default=0.5)
    ap.add_argument("--serve-cavity-fraction", type=float, default=0.0,
                    help="serve workload: fraction of lid-driven cavity requests (the rest spheres)")
    ap.add_argument("--serve-drop", type=float, default=1e-2)
    ap.add_argument("--serve-max-steps", type=int, default=500)
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--batch-meshes", type=int, default=48)
    ap.add_argument("--batch-scheme", default="hweno", choices=["weno", "hweno"])
    ap.add_argument("--batch-precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--hex-n", type=int, default=72, help="hex workload: n^3 hexahedra")
    ap.add_argument("--hexsphere-case", default="re118", choices=["re118", "ma15"],
                    help="hexsphere workload: Re 118, Ma 0.2535 (linear weights, CFL 20) or Re 300, Ma 1.5 "
                         "(nonlinear weights, CFL 5)")
    ap.add_argument("--hexsphere-drop", type=float, default=1e-10)
    ap.add_argument("--hexsphere-max-steps", type=int, default=4000)
    ap.add_argument("--grad-relax", type=float, default=1.0,
                    help="precision workload: relaxation of the compact gradient update (1: Algorithm 1's)")
    ap.add_argument("--batch-drop", type=float, default=0.0,
                    help="batch workload: also solve every mesh from its start to this drop (0: skip)")
    ap.add_argument("--batch-max-steps", type=int, default=500)
    ap.add_argument("--launch-precision", default="fp64", choices=["fp64", "mixed"],
                    help="precision of the step timed by --launch-list")
    ap.add_argument("--launch-list", action="store_true",
                    help="warm-up then the timed steps only (no e2e, no residual-only pass): for ncu launch lists")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batch":
        return run_batch(args, rank, world)
    if args.workload == "serve":
        return run_serve(args, rank, world)
    if args.workload == "hex":
        return run_hex(args, rank, world)
    if args.workload == "hexsphere":
        return run_hexsphere(args, rank, world)
    if args.workload == "precision":
        return run_precision(args, rank, world)

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

    # the FP64 roofline of this GPU, measured (DFMA chains, about 2 s)
    peak_clk = ClockSampler(local)
    peak_clk.start()
    fp64_peak = H.hgks_fp64_peak(local, 2.0)
    peak_clk = peak_clk.stop()

    m, cond, kw, name = workload(small=args.small, sphere_n=args.sphere_n)
    hm = H.hgks_mesh_create(m, scheme_mask=1, device=local)
    p = H.hgks_default_params(**kw)
    if args.launch_list and args.launch_precision == "mixed":
        p = H.hgks_default_params(precision=1, **kw)
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

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.launch_list:                  # eager steps with an event pair around every launch
        barrier()
        H.hgks_launch_count(reset=True)
        H.hgks_profile_begin()
        ev0.record(stream)
        for _ in range(args.steps):
            H.hgks_gmres_step(hm, p, Q)
        ev1.record(stream)
        barrier()
        prof = H.hgks_profile_end()
        if rank == 0:
            print(json.dumps({"launch_list": True, "ms_per_step": ev0.elapsed_time(ev1) / args.steps,
                              "gpu_launches": int(H.hgks_launch_count()),
                              "kernels_ms": {k: round(v[0], 3) for k, v in prof.items()}, "n_cells": m.n_tet}))
        return 0

    # the timed steps: what a caller gets (the step's launches replayed from its CUDA graph)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    H.hgks_launch_count(reset=True)
    ev0.record(stream)
    for _ in range(args.steps):
        H.hgks_gmres_step(hm, p, Q)
    ev1.record(stream)
    barrier()
    launches = H.hgks_launch_count()
    clk = clocks.stop()
    ms, value = aggregate(ev0.elapsed_time(ev1), m.n_tet, args.steps, world, device=f"cuda:{local}")
    # per-kernel CUDA-event times: the same number of steps again, launched eagerly with
    # an event pair around every launch on the launching stream (events between the
    # launches would slow the timed steps down)
    H.hgks_profile_begin()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        H.hgks_gmres_step(hm, p, Q)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = H.hgks_profile_end()
    profiled_ms = e0.elapsed_time(e1) / args.steps
    # residual alone (the R(U) kernels), same stream, for the residual throughput
    Rt = torch.empty_like(Q)
    H.hgks_residual(hm, p, Q, None, Rt)
    torch.cuda.synchronize()
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
    H.hgks_profile_begin()
    H.hgks_gmres_step(hm, pm, Qm)
    mixed_prof = H.hgks_profile_end()
    del Qm

    # the same step with matrix-free products (Eq. (frechet)): one residual per Krylov vector
    pf = H.hgks_default_params(jv_mode=1, **kw)
    Qf = Q.clone()
    H.hgks_gmres_step(hm, pf, Qf)
    torch.cuda.synchronize()
    e0.record(stream)
    H.hgks_gmres_step(hm, pf, Qf)
    e1.record(stream)
    torch.cuda.synchronize()
    fd_ms = e0.elapsed_time(e1)
    del Qf

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

    # context: the paper's timing case (48,000-tet wall-clustered cavity, Re = 1000),
    # seconds per 100 implicit steps of Algorithm 1 with both schemes, FP64
    ctx = paper_timing_context(H, I, local) if rank == 0 and not args.small else None

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    # roofline of the dominant kernel
    F = int(H.hgks_mesh_info(hm).n_faces)

    def kroof(name):
        kms, kcnt = prof[name]
        avg_s = kms / kcnt / 1000.0
        r = {"kernel": name, "bound": "alu", "unit": "GFLOP/s", "peak": fp64_peak,
             "peak_source": "measured: FP64 FMA chains on this GPU in this run (hgks_fp64_peak), "
                            f"sm clock median {peak_clk.get('sm_mhz')} MHz during the measurement; "
                            f"nominal {FP64_NOMINAL_GFLOPS} (152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz)",
             "avg_launch_ms": avg_s * 1000.0, "launches": kcnt, "traffic": None}
        if name in KERNEL_FLOPS:
            per, units = KERNEL_FLOPS[name]
            fl = per * units(m.n_tet, F)
            r.update({"achieved": fl / avg_s / 1e9, "frac": fl / avg_s / 1e9 / fp64_peak, "flops_per_launch": fl})
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
        "config": step_config(name, m.n_tet, F, world),
        "residual_only": {"value": m.n_tet / (res_ms / 1000.0) / 1e6, "unit": "Mcells/s", "ms": res_ms},
        "mixed": {"value": world * m.n_tet / (mixed_ms / 1000.0) / 1e6, "unit": "Mcells/s", "ms_per_step": mixed_ms,
                  "note": "same step with FP32 Krylov basis, Arnoldi and Jacobi (FP64 residual and update)",
                  "kernels_ms_one_step": {k: round(v[0], 3) for k, v in sorted(mixed_prof.items(), key=lambda kv: -kv[1][0])}},
        "matrix_free": {"value": world * m.n_tet / (fd_ms / 1000.0) / 1e6, "unit": "Mcells/s", "ms_per_step": fd_ms,
                        "vs_assembled": ms / args.steps / fd_ms,
                        "note": "same step with the Frechet-difference products of Eq. (frechet) (jv_mode 1); "
                                "one residual per Krylov vector, the cost the paper avoids with the assembled A"},
        "e2e": {"value": e2e_val, "unit": "Mcells/s", "h2d_bytes_per_step": 5 * 8 * m.n_tet,
                "d2h_bytes_per_step": 5 * 8 * m.n_tet},
        "gmres_iterations_per_s": {
            "fp64": world * kw["krylov_dim"] * p.restarts / (ms / args.steps / 1000.0),
            "mixed": world * kw["krylov_dim"] * p.restarts / (mixed_ms / 1000.0),
            "note": "Arnoldi steps (Krylov vectors) per second, whole job, inside full implicit steps"},
        "gpu_launches": int(launches),
        "kernels_ms": {k: round(v[0], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])},
        "kernels_note": "per-kernel CUDA-event totals over a repeat of the timed steps launched eagerly with an "
                        "event pair around each launch (the timed steps replay the captured step graph)",
        "profiled_ms_per_step": profiled_ms,
        "roofline": roof,
        "roofline_frac_by_kernel": roof_all,
        "fp64_peak_gflops": {"measured": fp64_peak, "nominal": FP64_NOMINAL_GFLOPS, "clocks": peak_clk},
        "clocks": clk,
        "cpu_baseline": cb,
        "paper_timing_context": ctx,
    }
    print(json.dumps(result))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
