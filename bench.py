"""Benchmark of the GB300 charge-conserving FEM-PIC step.

One step = one full PIC cycle of the library (sort by tet, per-tet
coefficients, gather + push + walk + exact deposit, reduction to edges and
nodes, Newmark RHS, PCG to 1e-10, gradient completion, Faraday update,
diagnostics) over every particle of the workload.  The metric is
particle-steps/s over whole steps; the plain-FP64 GPU path is timed in the
same run for the comparison the metric names.

Default workload: the neutral plasma ball of 64^3 Kuhn cells (1,572,864 tets,
interior vertices jittered by up to 20% of h), 16M electrons + 16M protons
(mass ratio 1836) in a Gaussian sphere, Te = 10 eV, Ti = 0.1 eV, Debye length
2h at the peak density, PEC walls, wave-equation Newmark, Boris push,
dt = 4 x the explicit limit, Jacobi-PCG to 1e-10.  Synthetic seeded inputs.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
        [--workload plasma_ball|thermal_cube] [--cells C] [--particles P]
Under torchrun (N > 1) each rank runs an independent replica (the method's
field solve couples the whole mesh, so there is nothing to shard): weak scaling.
The side legs (learned preconditioner, beam, batch, single electron, pusher
sweep, MIXED against the oracle) and the CPU baseline run at N = 1 only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2102_06248_gb300 import workloads as W  # noqa: E402

METRIC = "particle-steps/s (gather+push+deposit) and step time vs plain FP64 GPU path"
FALLBACK_HBM_GBS = 6800.0
CLOCK_LOG = None   # --clock-log: where the clock samples of the timed region go ({gpu}: the GPU index)
FP64_NOMINAL_TFLOPS = 1.25   # GB300 dense FP64 (non-tensor) nominal rate
# DRAM bytes over algorithmic bytes of the MIXED Newmark launch
# (k_pcg_persistent<1>), from one ncu capture of that kernel (its current code)
# on the 64^3 plasma ball: 15.664 GB (dram__bytes_read.sum +
# dram__bytes_write.sum) for 60 FP32 + 2 FP64 iterations whose algorithmic
# bytes are 19.938 GB (below 1: with the matrix loaded evict-first, the
# vectors written each iteration stay in L2).  The FP64 Newmark form has no
# capture of its current code: its traffic is reported as null.
TRAFFIC_RATIO_MIXED = (15.561853 + 0.102376) / 19.937848
# DRAM bytes of one MIXED push launch (k_push_mixed<0>) on the 64^3 plasma-ball
# mesh with 4M + 4M particles, from one ncu capture of the current kernel:
# 0.408 + 0.336 GB (93 B per particle, per-tet bytes included); scaled to a
# launch by the particles it pushes
PUSH_TRAFFIC_SMALL = (0.408e9 + 0.336e9, 8_000_000)
# Warp instructions of the same capture (smsp__inst_executed.sum): 245M for the
# 8M particles, the push's binding resource being instruction issue
PUSH_WARP_INST_SMALL = (245.0e6, 8_000_000)
SCHEDULERS_PER_SM = 4   # warp schedulers per SM, one warp instruction issued per cycle each
TRAFFIC_RATIO_PLAIN = None


def dt_table():
    with open(os.path.join(ROOT, "tests", "golden", "dt_cfl.json")) as f:
        return json.load(f)


def workload_desc(name: str, cells: int, per_species: int) -> str:
    if name == "plasma_ball":
        return (f"plasma_ball {cells}^3 Kuhn cells ({6 * cells ** 3} tets, 20% jitter), "
                f"{per_species} e- + {per_species} p+ Gaussian sphere, Te=10 eV, Ti=0.1 eV, "
                f"WE Newmark, Boris, dt=4xCFL, Jacobi-PCG 1e-10, PEC walls")
    if name == "thermal_cube":
        return (f"thermal_cube {cells}^3 Kuhn cells, {per_species} e- Maxwellian 0.01c, "
                f"B0=0.1 T, WE Newmark, Boris, dt=2xCFL, Jacobi-PCG 1e-10")
    raise SystemExit(f"unknown workload {name}")


def make_workload(name: str, cells: int, per_species: int):
    tab = dt_table()
    desc = workload_desc(name, cells, per_species)
    if name == "plasma_ball":
        wl = W.plasma_ball(n_cells=cells, n_per_species=per_species)
        kappa = tab["kuhn_lattice_16^3_jitter0.2"]["kappa"]
        dt = wl.dt_cfl_multiple * kappa * wl.mesh.h / W.C0
    else:
        wl = W.thermal_plasma_cube(n_cells=cells, n_particles=per_species)
        dt = 2.0 * tab["thermal_plasma_cube_6^3"]["dt_cfl_s"] * (6.0 / cells)
    return wl, dt, desc


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as f:
                d = json.load(f)
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "of measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "of fallback"


class ClockSampler:
    """SM clock, power and clock-event reasons of one GPU while the timed region
    runs: NVML (the driver's libnvidia-ml, public API through ctypes) polled
    every 2 ms from a thread, else nvidia-smi every 50 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # nvmlClocksEventReason bits (nvml.h)
    REASON_BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
                   "hw_thermal_slowdown": 0x40, "hw_power_brake_slowdown": 0x80}

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.thread = None
        self.path = (CLOCK_LOG.replace("{gpu}", str(gpu)) if CLOCK_LOG
                     else os.path.join(tempfile.gettempdir(), f"fempic_clocks_gpu{gpu}.csv"))
        self.nvml = None
        try:
            import ctypes
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() == 0:
                h = ctypes.c_void_p()
                if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(gpu), ctypes.byref(h)) == 0:
                    self.nvml, self.handle, self.ct = lib, h, ctypes
        except Exception:
            self.nvml = None

    def _poll(self):
        ct, lib, h = self.ct, self.nvml, self.handle
        clk, mx, mw, rs = ct.c_uint(), ct.c_uint(), ct.c_uint(), ct.c_ulonglong()
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        lib.nvmlDeviceGetMaxClockInfo(h, 1, ct.byref(mx))
        while not self.stop_flag:
            if lib.nvmlDeviceGetClockInfo(h, 1, ct.byref(clk)) == 0:      # NVML_CLOCK_SM
                lib.nvmlDeviceGetPowerUsage(h, ct.byref(mw))
                get_reasons(h, ct.byref(rs))
                self.samples.append((clk.value, mx.value, mw.value / 1000.0, rs.value))
            time.sleep(0.002)

    def start(self):
        if os.path.dirname(self.path):
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
        if self.nvml is not None:
            import threading
            self.samples, self.stop_flag = [], False
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            return
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.stop_flag = True
            self.thread.join(timeout=5)
            sm = [c for c, _, _, _ in self.samples]
            smax = [m for _, m, _, _ in self.samples]
            reasons = {n for _, _, _, r in self.samples for n, bit in self.REASON_BITS.items() if r & bit}
            with open(self.path, "w") as fh:
                fh.write("sm_mhz,max_sm_mhz,power_w,reasons_mask\n")
                for c, m, w, r in self.samples:
                    fh.write(f"{c},{m},{w:.1f},{r:#x}\n")
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                    "sm_mhz_min": min(sm) if sm else None, "reasons": sorted(reasons), "samples": len(sm),
                    "source": "nvml, 2 ms"}
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi, 50 ms"}


def clock_rejected(clk: dict) -> bool:
    """A clock record that rejects a timing: hardware or thermal slowdown, or
    SM clocks well below their maximum with no reason (a leftover lock);
    sw_power_cap alone is kept (and shows in the record)."""
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "hw_power_brake_slowdown"}
    reasons = set(clk.get("reasons") or [])
    if reasons & bad:
        return True
    sm, smax = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    return bool(sm and smax and sm < 0.85 * smax and not reasons)


def dist_setup(n_gpus: int):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local, dist


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device])
        else:
            dist.barrier()


def max_over_ranks(dist, value: float, device) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value: float, device) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def push_bytes(n_particles: int, n_tets: int, precision: str, n_species: int = 1) -> float:
    """Algorithmic bytes of one launch of the fused push kernel: every live
    particle's state read (through the sort permutation) and written once,
    plus the per-tet geometry, coefficients and accumulators once."""
    r = 4 if precision == "mixed" else 8
    per_particle = 2 * (6 * r + 4 + 4) + 4 + 4      # x,v,key,id in and out; perm; sorted key
    acc = 80 * (n_species if precision == "mixed" else 1)
    per_tet = 12 * r + 10 * r + acc                 # barycentric map, coefficients, accumulator write
    return n_particles * per_particle + n_tets * per_tet


def measured_sm_mhz() -> float:
    """Maximum SM clock of the machine's GPUs from MEASURED_PEAKS.json (the
    nominal 2070 MHz when the file or the key is missing)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f).get("sm_max_mhz", 2070.0))
    except (OSError, ValueError, TypeError, AttributeError):
        return 2070.0


def issue_roofline(n_particles: float, avg_ms: float, sms: int, sm_mhz: float) -> dict:
    """The push against its binding resource, instruction issue: the warp
    instructions of one launch (the ncu count per particle of the captured
    launch times the particles pushed) over its duration, against every
    scheduler issuing one warp instruction per cycle at the given SM clock."""
    per_particle = PUSH_WARP_INST_SMALL[0] / PUSH_WARP_INST_SMALL[1]
    inst = per_particle * n_particles
    achieved = inst / (avg_ms / 1e3)
    peak = float(sms) * SCHEDULERS_PER_SM * sm_mhz * 1e6
    return {"bound": "issue", "warp_instructions_per_particle": round(per_particle, 2),
            "achieved_warp_inst_per_s": achieved, "peak_warp_inst_per_s": peak,
            "frac": round(achieved / peak, 4),
            "peak_source": f"{sms} SMs x {SCHEDULERS_PER_SM} schedulers x {sm_mhz:.0f} MHz",
            "source": "ncu smsp__inst_executed.sum of the same kernel on the same mesh with 8M particles, "
                      "scaled by the particles pushed"}


def pcg_iter_bytes(n_rows: int, nnz: int) -> float:
    """Algorithmic bytes of one iteration of the persistent Chronopoulos-Gear
    PCG on SELL-32: values + columns once (12 B/nnz) and two slice headers per
    32 rows; the SpMV reads u once and writes w; the vector phase reads u, w,
    p, s, x, r, D^-1 and writes p, s, x, r, u (14 vector passes of 8 B)."""
    return 12.0 * nnz + 8.0 * (n_rows + 31) / 32 + 8.0 * 14 * n_rows


def pcg_iter_flops(n_rows: int, nnz: int) -> float:
    """FP64 flops of one such iteration: a multiply-add per stored entry and
    per row the seven of the vector phase plus the one of (w, u)."""
    return 2.0 * nnz + 2.0 * 8 * n_rows


def refine_bytes(n_rows: int, nnz: int, inner_iters: float, outer: float) -> float:
    """Algorithmic bytes of one MIXED Newmark solve (FP64 refinement with FP32
    correction solves on the diagonally scaled system): per FP32 iteration 8 B
    per nonzero (FP32 value + column) + 11 vector passes of 4 B per row (SpMV:
    r read, w written; vector phase: w, p, s, x, r read, p, s, x, r written);
    per refinement step one FP64 residual (12 B per nonzero, b read, x
    gathered, r in FP32 written: 20 B per row) and the update x += d (20 B per
    row); plus the final residual check."""
    inner = inner_iters * (8.0 * nnz + 4.0 * 11 * n_rows)
    return inner + (outer + 1) * (12.0 * nnz + 20.0 * n_rows) + outer * 20.0 * n_rows


def beam_leg(F, torch, stream, args):
    """The non-neutral electron beam (MIXED): 32x32x128 Kuhn cells of 1.25 mm,
    2M electrons in flight, the steady-state injection at z = 0 before every
    step (pic_particles_inject with host arrays, generated before the timed
    region), dt = 4 x CFL.  Host wall clock around inject + step (both
    synchronise)."""
    tab = dt_table()
    wl = W.electron_beam(n_inflight=args.beam_particles)
    h = 1.25e-3
    dt = 4.0 * tab["kuhn_lattice_16^3"]["kappa"] * h / W.C0
    n_inj = W.inject_per_step(wl, dt)
    total = args.warmup + args.beam_steps
    inj = [W.beam_injection(wl, k, n_inj, dt) for k in range(total)]
    sim = F.sim_from_workload(wl, dt, precision="mixed", stream=stream, profile=True)
    for k in range(args.warmup):
        sim.particles_inject(0, *inj[k])
        sim.step()
    sim.profile_reset()
    torch.cuda.synchronize()
    alive0 = sim.diag()["n_alive"]
    t_inj = 0.0
    t0 = time.perf_counter()
    for k in range(args.warmup, total):
        a = time.perf_counter()
        sim.particles_inject(0, *inj[k])
        t_inj += time.perf_counter() - a
        sim.step()
    t1 = time.perf_counter()
    d = sim.diag()
    pr = sim.profile()
    ms = 1e3 * (t1 - t0) / args.beam_steps
    out = {"workload": "electron beam 32x32x128 Kuhn cells (786,432 tets), h = 1.25 mm, PEC; "
                       f"{args.beam_particles} electrons in flight, radial Gaussian sigma = 0.1 width, vz = 0.1c, "
                       f"1% spread, {n_inj} injected per step, 0.25 A, dt = 4xCFL, MIXED, Jacobi-PCG 1e-10",
           "steps": args.beam_steps, "ms_per_step": ms, "inject_ms_per_step": 1e3 * t_inj / args.beam_steps,
           "particles_alive": [alive0, d["n_alive"]],
           "value": 0.5 * (alive0 + d["n_alive"]) / (ms / 1e3), "unit": "particle-steps/s",
           "phases_ms_per_step": {k: round(v[0] / args.beam_steps, 4) for k, v in pr.items()},
           "continuity_rel": d["continuity_abs"] / max(d["rho_max"], 1e-300),
           "gauss_rel": d["gauss_abs"] / max(d["rho_max"], 1e-300),
           "timing": "host clock around synchronising calls"}
    del sim
    return out


def gnn_leg(F, torch, wl, dt, stream, args):
    """The headline workload (MIXED) with the learned preconditioner: three
    Jacobi steps, training on residuals of the last Newmark system with the
    library's own kernels, then steps whose Newmark solve is the flexible PCG
    with the network (CUDA events on the simulation's stream)."""
    sim = F.sim_from_workload(wl, dt, precision="mixed", stream=stream, profile=True, preconditioner="gnn")
    for _ in range(3):
        sim.step()
    jac_iters = sim.diag()["cg_iters"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = sim.gnn_train(steps=args.gnn_train_steps, lr=1e-3, samples=8)
    t1 = time.perf_counter()
    sim.profile_reset()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    iters = []
    for _ in range(args.gnn_steps):
        sim.step()
        iters.append(sim.diag()["cg_iters"])
    ev1.record(stream)
    torch.cuda.synchronize()
    pr = sim.profile()
    d = sim.diag()
    out = {"train_steps": args.gnn_train_steps, "train_s": t1 - t0, "train_loss": loss,
           "ms_per_step": ev0.elapsed_time(ev1) / args.gnn_steps,
           "cg_ms_per_step": pr["cg"][0] / args.gnn_steps, "cg_iters": iters, "jacobi_cg_iters_before": jac_iters,
           "continuity_rel": d["continuity_abs"] / max(d["rho_max"], 1e-300),
           "gauss_rel": d["gauss_abs"] / max(d["rho_max"], 1e-300),
           "solve": ("flexible PCG (Polak-Ribiere) with the network, 3 message-passing layers, hidden 32, bf16 weights; "
                     "inference layers on the tensor cores (mma.sync TF32 on split FP32 activations, FP32 sums)")}
    del sim
    return out


def batched_leg(F, torch, args):
    """64 independent thermal runs (cells 8^3..32^3, 1e4..1e6 electrons, log-
    uniform from a seed), MIXED, stepped as one batch (one stream per run, one
    persistent launch per solve over all runs, six-step CUDA graphs) and, for
    comparison, one after another with pic_step.  Host wall clock around
    calls that synchronise at their end, after a device synchronise."""
    runs = W.batched_runs(n_runs=args.batch_runs)
    dt6 = dt_table()["thermal_plasma_cube_6^3"]["dt_cfl_s"]
    sims = []
    for wl in runs:
        cells = round(len(wl.mesh.tets) / 6) ** (1.0 / 3.0)
        sims.append(F.sim_from_workload(wl, 2.0 * dt6 * 6.0 / round(cells), precision="mixed"))
    n_part = sum(wl.n_particles for wl in runs)
    batch = F.Batch(sims)
    batch.step(7)                      # warm-up: one eager step, tuning, capture, one graph launch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch.step(args.batch_steps)
    t1 = time.perf_counter()
    info = batch.info()
    # the same runs one by one (fewer steps: every pic_step synchronises)
    seq_steps = max(1, args.batch_steps // 5)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    for s in sims:
        s.step(seq_steps)
    t3 = time.perf_counter()
    ps_b = n_part * args.batch_steps / (t1 - t0)
    ps_s = n_part * seq_steps / (t3 - t2)
    ok = all(s.diag()["continuity_abs"] <= 1e-12 * max(s.diag()["rho_max"], 1e-300) for s in sims)
    del batch
    return {"workload": f"{len(runs)} thermal runs, cells 8^3..32^3, 1e4..1e6 electrons (log-uniform, seed 1005), "
                        f"MIXED, WE Newmark, Boris, dt = 2xCFL, Jacobi-PCG 1e-10",
            "particles": n_part, "steps": args.batch_steps, "ms_per_step": 1e3 * (t1 - t0) / args.batch_steps,
            "value": ps_b, "unit": "particle-steps/s",
            "one_by_one": {"steps": seq_steps, "ms_per_step": 1e3 * (t3 - t2) / seq_steps, "value": ps_s},
            "speedup_batched": ps_b / ps_s, "continuity_ok": ok, "timing": "host clock around synchronising calls",
            "graph": info["graph"], "graph_steps": info["graph_steps"], "graph_launches": info["graph_launches"],
            "tuned": {"newmark": {"blocks_per_sm": info["solver_blocks_per_sm"], "build": info["solver_build"]},
                      "completion": {"blocks_per_sm": info["completion_blocks_per_sm"],
                                     "build": info["completion_build"]},
                      "candidates": "blocks/SM 2, 3, 4 (64-register build), 2, 3 (80-register), 5, 6 (40-register), 7, 8 (32-register)",
                      "tune_newmark_ms": [round(v, 3) for v in info["tune_newmark_ms"]],
                      "tune_completion_ms": [round(v, 3) for v in info["tune_completion_ms"]]}}


def larmor_leg(F, torch, args):
    """Single electron gyrating in uniform B0 (0.05 T, v_perp = 0.05c), 20^3
    Kuhn-cell box of side 10 r_L, Maxwell-solver Newmark form, dt = T_c/64
    (Sec. IV.A analogue): FP64 and MIXED precision on the GPU, orbit radius
    about the fixed guiding centre and accumulated phase against the closed
    forms of the continuous orbit (r_L, w_c t) and of the Boris map (radius
    r_L sqrt(1 + (w_c dt/2)^2), phase 2 atan(w_c dt/2) per step)."""
    wl = W.larmor_orbit_box(n_cells=args.larmor_cells, steps=args.larmor_steps)
    wc = abs(W.Q_E) * wl.b0[2] / W.M_E
    vperp = 0.05 * W.C0
    r_l = vperp / wc
    h = wl.mesh.h
    centre = np.array([0.5 * wl.mesh.size[0], 0.5 * wl.mesh.size[1] + 0.137 * h])
    th_b = 2.0 * math.atan(0.5 * wc * wl.dt)
    r_boris = r_l * math.sqrt(1.0 + (0.5 * wc * wl.dt) ** 2)
    out = {"workload": f"larmor_orbit {args.larmor_cells}^3 Kuhn cells, side 10 r_L, 1 e-, B0=0.05 T, "
                       f"v_perp=0.05c, MFEM Newmark, Boris, dt=T_c/64", "steps": args.larmor_steps,
           "r_L_m": r_l, "boris_radius_closed_form_m": r_boris, "boris_phase_per_step": th_b}
    for prec in ("plain", "mixed"):
        sim = F.sim_from_workload(wl, wl.dt, precision=prec)
        x0, _, _, _ = sim.particles()
        ph0 = math.atan2(x0[0, 1] - centre[1], x0[0, 0] - centre[0])
        rads, phase, prev = [], 0.0, ph0
        t0 = time.perf_counter()
        for k in range(args.larmor_steps):
            sim.step()
            x, _, _, _ = sim.particles()
            dx, dy = x[0, 0] - centre[0], x[0, 1] - centre[1]
            rads.append(math.hypot(dx, dy))
            ph = math.atan2(dy, dx)
            d = ph - prev
            d -= 2.0 * math.pi * round(d / (2.0 * math.pi))
            phase += d
            prev = ph
        el = time.perf_counter() - t0
        n = args.larmor_steps
        # an electron (q < 0) in B0 z turns counter-clockwise: the phase grows
        r_mean = float(np.mean(rads))
        out[prec] = {"radius_mean_m": r_mean,
                     "radius_rel_err_vs_r_L": r_mean / r_l - 1.0,
                     "radius_rel_err_vs_boris": r_mean / r_boris - 1.0,
                     "radius_rel_spread": float((np.max(rads) - np.min(rads)) / r_l),
                     "phase_err_rad_vs_wc_t": phase - wc * wl.dt * n,
                     "phase_err_rad_vs_boris": phase - th_b * n,
                     "seconds": el}
        del sim
    out["mixed_minus_plain_radius_rel"] = out["mixed"]["radius_mean_m"] / out["plain"]["radius_mean_m"] - 1.0
    out["mixed_minus_plain_phase_rad"] = out["mixed"]["phase_err_rad_vs_wc_t"] - out["plain"]["phase_err_rad_vs_wc_t"]
    return out


def pusher_sweep_leg(F, args):
    """Sec. IV.A, Table I: the cyclotron orbit (B = 6.822756e-5 T, v0 = 3e6 m/s)
    in frozen fields on the GPU for Boris and Adams-Bashforth orders 1-5 at
    dt = T_c/N, with the exact start-up history; the paper's error
    ||r - r_a||_2 / ||r_a||_2 over one period, and its log-log slope."""
    with open(os.path.join(ROOT, "tests", "golden", "table1_cyclotron.json")) as f:
        tab = json.load(f)
    q, mass, bz = tab["q_C"], tab["m_kg"], tab["B_z_T"]
    v0 = np.array(tab["v0_m_per_s"])
    r0 = np.array(tab["r0_m"])
    wc = abs(q) * bz / mass
    t_c = 2.0 * math.pi / wc
    r_l = np.linalg.norm(v0) / wc
    cx, cy = r0[0] - r_l, r0[1]

    def exact(t):
        ph = wc * t
        return (np.array([cx + r_l * math.cos(ph), cy + r_l * math.sin(ph), 0.0]),
                np.array([-r_l * wc * math.sin(ph), r_l * wc * math.cos(ph), 0.0]))
    box = W.kuhn_box((4, 4, 4), (1.0, 1.0, 1.0))
    xyz = box.xyz.copy()
    xyz[:, 2] -= 0.5
    mesh = F.Mesh(xyz, box.tets)
    xs, tet = W.place_in_box(box, (r0 + np.array([0, 0, 0.5]))[None, :])
    xs = xs - np.array([0, 0, 0.5])
    out = {"workload": "Table I cyclotron (Sec. IV.A), frozen uniform B, one period", "errors": {}, "slopes": {}}
    ns = (128, 256, 512)
    for pusher in ("boris", "ab1", "ab2", "ab3", "ab4", "ab5"):
        errs = []
        for nsteps in ns:
            dt = t_c / nsteps
            sim = F.Sim(mesh, dt, pusher=pusher, b0=(0, 0, bz))
            if pusher == "boris":
                # Boris takes v^{-1/2}: the exact velocity half a step back
                _, vh = exact(-0.5 * dt)
                sim.particles_load(0, q, mass, 1.0, xs, vh[None, :], tet)
            else:
                sim.particles_load(0, q, mass, 1.0, xs, v0[None, :], tet)
            sim.init()
            sim.set_field("E", np.zeros(mesh.n_edges))
            sim.set_field("E_PREV", np.zeros(mesh.n_edges))
            order = 0 if pusher == "boris" else int(pusher[2:])
            if order > 1:
                ah, vh_ = [], []
                for j in range(1, order):
                    _, vj = exact(-j * dt)
                    ah.append((q / mass) * np.cross(vj, [0, 0, bz])[None, :])
                    vh_.append(vj[None, :])
                sim.set_ab_history(np.array(ah), np.array(vh_))
            num = den = 0.0
            for k in range(1, nsteps + 1):
                sim.particle_phase()
                x, _, _, _ = sim.particles()
                ra, _ = exact(k * dt)
                num += float(np.sum((x[0] - ra) ** 2))
                den += float(np.sum(ra ** 2))
            errs.append(math.sqrt(num / den))
            del sim
        out["errors"][pusher] = {f"T_c/{n}": e for n, e in zip(ns, errs)}
        out["slopes"][pusher] = math.log(errs[0] / errs[-1]) / math.log(ns[-1] / ns[0])
    return out


def mixed_error_leg(F, args):
    """MIXED precision against the FP64 oracle, per result, on reduced copies
    of the benchmark workloads (10 steps, Newmark solves at 1e-13 on both
    sides): the plasma ball at 16^3 cells with 2 x 65,536 particles and the
    electron beam at 8 x 8 x 32 cells with 20,000 electrons in flight.
    Errors are max |gpu - oracle| / max |oracle| per field; positions against
    the box side, velocities against the species' largest speed."""
    from oracle.oracle import from_workload
    tab = dt_table()
    cases = []
    wl = W.plasma_ball(n_cells=16, n_per_species=65536, seed=41)
    cases.append(("plasma_ball 16^3, 2 x 65536 e-/p+", wl,
                   4.0 * tab["kuhn_lattice_16^3_jitter0.2"]["kappa"] * wl.mesh.h / W.C0))
    wb = W.electron_beam(cells=(8, 8, 32), h=1.25e-3, n_inflight=20000, seed=1003)
    cases.append(("electron_beam 8x8x32, 20000 e-", wb, 4.0 * tab["kuhn_lattice_16^3"]["kappa"] * wb.mesh.h / W.C0))
    out = {}
    for name, w, dt in cases:
        o = from_workload(w, dt, cg_tol=1e-13)
        g = F.sim_from_workload(w, dt, precision="mixed", cg_tol=1e-13)
        worst = {}
        for _ in range(10):
            o.step()
            g.step()
            for f in ("E", "B", "G", "RHO", "WALL"):
                b = o.field(f)
                sc = max(np.abs(b).max(), 1e-300)
                worst[f] = max(worst.get(f, 0.0), float(np.abs(g.field(f) - b).max() / sc))
        gx, gv, gt, gid = g.particles()
        ox, ov, ot, alive = o.particles()
        ids = np.where(alive)[0]
        common = np.intersect1d(gid, ids)
        gi = np.searchsorted(gid, common)
        worst["x_rel_box"] = float(np.abs(gx[gi] - ox[common]).max() / max(w.mesh.size))
        worst["v_rel"] = float(np.abs(gv[gi] - ov[common]).max() / np.abs(ov).max())
        worst["tet_agree_frac"] = float(np.mean(gt[gi] == ot[common]))
        worst["alive_gpu_oracle"] = [int(len(gid)), int(len(ids))]
        d = g.diag()
        worst["continuity_rel"] = d["continuity_abs"] / d["rho_max"]
        worst["gauss_rel"] = d["gauss_abs"] / d["rho_max"]
        out[name] = worst
        del o, g
    return out


def time_gpu(F, wl, dt, precision, steps, warmup, stream, dist, device, torch, profile=True):
    sim = F.sim_from_workload(wl, dt, precision=precision, stream=stream, profile=profile)
    for _ in range(warmup):
        sim.step()
    sim.profile_reset()
    barrier(dist, device)
    torch.cuda.synchronize()
    l0 = F.launch_count()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        sim.step()
    stop.record(stream)
    torch.cuda.synchronize()
    barrier(dist, device)
    ms = start.elapsed_time(stop)
    launches = F.launch_count() - l0
    prof = sim.profile()
    diag = sim.diag()
    return sim, ms, launches, prof, diag


def gpu_arm(args):
    import torch
    from paper_2102_06248_gb300 import fempic as F

    rank, world, local, dist = dist_setup(args.gpus)
    if world > 1:
        # the side legs and the CPU baseline do not depend on N and are
        # reported by the N = 1 run; here they would hold every GPU meanwhile
        args.skip_gnn = args.skip_beam = args.skip_batched = True
        args.skip_larmor = args.skip_sweep = args.skip_mixed_error = True
        args.no_cpu_baseline = True
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    F.load()
    wl, dt, desc = make_workload(args.workload, args.cells, args.particles)
    n_part = wl.n_particles

    # ---- mixed precision (headline) with clocks sampled during the timed region ----
    clocks = ClockSampler(local)
    sim_m = F.sim_from_workload(wl, dt, precision="mixed", stream=stream, profile=True)
    mesh = sim_m.mesh
    for _ in range(args.warmup):
        sim_m.step()

    def timed_region():
        sim_m.profile_reset()
        d_start = sim_m.diag()
        barrier(dist, local if world > 1 else None)
        torch.cuda.synchronize()
        l_start = F.launch_count()
        clocks.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            sim_m.step()
        ev1.record(stream)
        torch.cuda.synchronize()
        clk_r = clocks.stop()
        barrier(dist, local if world > 1 else None)
        return ev0.elapsed_time(ev1), F.launch_count() - l_start, clk_r, d_start

    ms_mixed, launches, clk, d0 = timed_region()
    # a timed region that saw a hardware or thermal slowdown, or clocks well
    # below their maximum with no reason given, is measured once more (every
    # rank does when one rank saw it)
    if sum_over_ranks(dist, 1.0 if clock_rejected(clk) else 0.0, device) > 0:
        first_clk = clk
        ms_mixed, launches, clk, d0 = timed_region()
        clk = dict(clk, remeasured=True, first=first_clk)
    else:
        clk = dict(clk, remeasured=False)
    prof_m = sim_m.profile()
    diag_m = sim_m.diag()
    alive_m = diag_m["n_alive"]
    cg_iters_timed = diag_m["cg_iters_sum"] - d0["cg_iters_sum"]
    ms_max = max_over_ranks(dist, ms_mixed, device)
    total_ps = sum_over_ranks(dist, float(n_part) * args.steps, device)
    value = total_ps / (ms_max / 1e3)
    del sim_m

    # ---- plain FP64 GPU path, same workload ----
    if args.skip_plain:
        ms_plain, prof_p = float("nan"), {}
    else:
        sim_p, ms_plain, _, prof_p, diag_p = time_gpu(F, wl, dt, "plain", args.steps, args.warmup, stream, dist,
                                                       local if world > 1 else None, torch)
        del sim_p
    ms_plain_max = max_over_ranks(dist, ms_plain, device)
    value_plain = total_ps / (ms_plain_max / 1e3)

    # ---- end to end through the public API from host arrays ----
    if args.skip_e2e:
        e2e_s_max, h2d, d2h = float("nan"), 0, 0
    else:
        torch.cuda.synchronize()
        sim_e = F.Sim(F.Mesh(wl.mesh.xyz, wl.mesh.tets), dt, form=wl.form, pusher=wl.pusher, precision="mixed",
                      b0=wl.b0, rho_background=wl.rho_background, stream=stream)
        # the inputs sit in pinned host memory, as a data loader would leave them
        pinned = [tuple(torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
                        for a in (sp.x, sp.v, sp.tet.astype(np.int32)))
                  for sp in wl.species]
        t_mesh = time.perf_counter()
        for k, sp in enumerate(wl.species):
            px, pv, pt = pinned[k]
            sim_e.particles_load(k, sp.q, sp.m, sp.w, px, pv, pt)
        t_load = time.perf_counter()
        sim_e.init()
        t_setup = time.perf_counter()
        d2h = 0
        for _ in range(args.steps):
            sim_e.step()
            dg = sim_e.diag()                       # the step's result, read back every step
            d2h += 8 * len(dg)
        e_out = sim_e.field("E")
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        e2e_s = t1 - t_mesh
        e2e_setup_s = t_setup - t_mesh
        e2e_load_s, e2e_init_s = t_load - t_mesh, t_setup - t_load
        h2d = sum(sp.x.nbytes + sp.v.nbytes + sp.tet.nbytes for sp in wl.species)
        d2h += e_out.nbytes
        del sim_e, pinned
        e2e_s_max = max_over_ranks(dist, e2e_s, device)

    # ---- roofline of the dominant kernel (live CUDA-event times) ----
    peak, peak_src = measured_peak()
    push_ms, push_n = prof_m["push"]
    cg_ms, cg_n = prof_m["cg"]
    push_avg = push_ms / max(push_n, 1)
    cg_avg = cg_ms / max(cg_n, 1)
    nnz_A = int(getattr(mesh, "nnz_A", 0))
    fp64 = None
    traffic = None
    if push_ms >= cg_ms:
        kernel = "k_push_mixed (fused gather/push/walk/deposit)"
        alg = push_bytes(int(alive_m), mesh.n_tets, "mixed", len(wl.species))
        avg_ms = push_avg
    else:
        # one launch runs the whole Newmark solve: its algorithmic bytes are
        # the iterations it ran times the bytes of one iteration
        iters_per_launch = cg_iters_timed / max(cg_n, 1)
        avg_ms = cg_avg
        outer = diag_m.get("cg_outer", 0.0)
        if outer > 0:
            # MIXED: FP64 refinement steps (the last solve's count) around FP32 correction iterations
            kernel = ("k_pcg_persistent (Newmark: FP64 refinement, FP32 Chronopoulos-Gear corrections, "
                      "SELL-32)")
            alg = refine_bytes(mesh.n_int_edges, nnz_A, iters_per_launch, outer)
            traffic = alg * TRAFFIC_RATIO_MIXED if TRAFFIC_RATIO_MIXED else None
            fp64 = {"note": "the FP32 correction iterations issue no FP64 arithmetic", "outer_steps": outer,
                    "fp32_iters_per_launch": iters_per_launch}
        else:
            kernel = "k_pcg_persistent (Newmark PCG, Chronopoulos-Gear, SELL-32)"
            alg = iters_per_launch * pcg_iter_bytes(mesh.n_int_edges, nnz_A)
            traffic = alg * TRAFFIC_RATIO_PLAIN if TRAFFIC_RATIO_PLAIN else None
            flops = iters_per_launch * pcg_iter_flops(mesh.n_int_edges, nnz_A)
            fp64_tf = flops / (avg_ms / 1e3) / 1e12
            fp64 = {"achieved_tflops": round(fp64_tf, 4), "peak_tflops": FP64_NOMINAL_TFLOPS,
                    "frac": round(fp64_tf / FP64_NOMINAL_TFLOPS, 4), "peak_source": "nominal",
                    "iters_per_launch": iters_per_launch}
    achieved = alg / (avg_ms / 1e3) / 1e9
    roofline = {"kernel": kernel, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_src,
                "traffic": traffic, "traffic_source": "ncu DRAM/algorithmic ratio of the same kernel, scaled to this launch",
                "algorithmic_bytes_per_launch": alg, "avg_launch_ms": round(avg_ms, 5),
                "fp64": fp64}

    # the push, the other hot kernel (issue- and latency-bound: its fraction
    # of HBM is reported, not claimed as the bound)
    push_alg = push_bytes(int(alive_m), mesh.n_tets, "mixed", len(wl.species))
    push_ach = push_alg / (push_avg / 1e3) / 1e9
    roofline_push = {"kernel": "k_push_mixed (fused gather/push/walk/deposit)", "bound": "issue/latency",
                     "achieved": round(push_ach, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(push_ach / peak, 4), "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": push_alg, "avg_launch_ms": round(push_avg, 5),
                     "traffic": PUSH_TRAFFIC_SMALL[0] * alive_m / PUSH_TRAFFIC_SMALL[1] if args.cells == 64 else None,
                     "traffic_source": "ncu DRAM bytes of the same kernel on the same mesh with 8M particles, "
                                       "scaled by the particles pushed",
                     "issue": issue_roofline(alive_m, push_avg,
                                             torch.cuda.get_device_properties(device).multi_processor_count,
                                             measured_sm_mhz())
                     if args.cells == 64 and args.workload == "plasma_ball" else None}

    # ---- learned preconditioner on the same workload ----
    gnn = None
    if not args.skip_gnn:
        gnn = gnn_leg(F, torch, wl, dt, stream, args)

    # ---- electron beam with injection (32x32x128 cells, 2M electrons in flight) ----
    beam = None
    if not args.skip_beam:
        beam = beam_leg(F, torch, stream, args)

    # ---- batched runs: 64 uneven thermal runs stepped together vs one by one ----
    batched = None
    if not args.skip_batched:
        batched = batched_leg(F, torch, args)

    # ---- single electron (config 2), pusher sweep (Table I), MIXED vs oracle ----
    larmor = sweep = mixed_err = None
    if rank == 0 and not args.skip_larmor:
        larmor = larmor_leg(F, torch, args)
    if rank == 0 and not args.skip_sweep:
        sweep = pusher_sweep_leg(F, args)
    if rank == 0 and not args.skip_mixed_error:
        mixed_err = mixed_error_leg(F, args)

    # ---- CPU baseline: the oracle on a bounded, proportionally scaled sample ----
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, seconds=args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 push + int64 fixed-point deposit + f32 CG corrections in f64 refinement", "data": "synthetic",
            "config": {"workload": desc, "particles_per_gpu": n_part, "tets": mesh.n_tets,
                       "edges": mesh.n_edges, "interior_edges": mesh.n_int_edges, "dt_s": dt,
                       "precision": "mixed", "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (particle state > 1 GB per GPU)"},
            "plain_fp64": None if args.skip_plain else {
                "value": value_plain, "ms_per_step": ms_plain_max / args.steps,
                "speedup_mixed_over_plain": value / value_plain},
            "phases_ms_per_step": {k: round(v[0] / max(args.steps, 1), 4) for k, v in prof_m.items()},
            "phases_ms_per_step_plain": {k: round(v[0] / max(args.steps, 1), 4) for k, v in prof_p.items()},
            "cg_iters_last": diag_m["cg_iters"],
            "cg_outer_last": diag_m.get("cg_outer", 0.0),
            "completion_iters_last": diag_m["completion_iters"],
            "conservation_last": {"continuity_rel": diag_m["continuity_abs"] / max(diag_m["rho_max"], 1e-300),
                                  "gauss_rel": diag_m["gauss_abs"] / max(diag_m["rho_max"], 1e-300)},
            "roofline": roofline, "roofline_push": roofline_push,
            "cpu_baseline": cpu,
            "e2e": None if args.skip_e2e else {"value": total_ps / e2e_s_max, "unit": "particle-steps/s",
                    "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                    "seconds": e2e_s_max, "setup_seconds": e2e_setup_s, "load_seconds": e2e_load_s,
                    "init_seconds": e2e_init_s,
                    "what": "particles_load from pinned host arrays (H2D) + init + K steps, each followed by "
                            "its diagnostics read back (D2H), + the final E field read back"},
            "gpu_launches": launches,
            "clocks": clk,
            "gnn": gnn,
            "beam": beam,
            "batched": batched,
            "larmor": larmor,
            "pusher_sweep": sweep,
            "mixed_vs_oracle": mixed_err,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def host_cpu() -> dict:
    """The host's logical core count and CPU model (from /proc/cpuinfo or lscpu)."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"logical_cores": os.cpu_count(), "model": model or "unknown"}


def _oracle_replica(spec):
    """One process of the all-core oracle runs: builds the scaled sample, runs
    `warmup` steps, waits for the other replicas, then steps it for `steps`
    steps or until `seconds` have passed (whichever comes first)."""
    workload, cells, per, warmup, steps, seconds, barrier = spec
    from oracle.oracle import from_workload
    wl, dt, _ = make_workload(workload, cells, per)
    sim = from_workload(wl, dt)
    for _ in range(warmup):
        sim.step()
    if barrier is not None:
        barrier.wait()
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        sim.step()
        done += 1
        if seconds is not None and time.perf_counter() - t0 > seconds:
            break
    return wl.n_particles, done, time.perf_counter() - t0


def oracle_runs(workload: str, cells: int, per: int, warmup: int, steps: int, seconds, procs: int):
    """The oracle as it stands (one particle at a time, sequential sums: a
    single-threaded program) on `procs` host cores: that many independent
    replicas of the sample in spawned processes, started together after their
    warm-up.  Returns (particle-steps/s summed over the replicas, per-replica
    (particles, steps, seconds))."""
    if procs <= 1:
        r = _oracle_replica((workload, cells, per, warmup, steps, seconds, None))
        return r[0] * r[1] / r[2], [r]
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        barrier = mgr.Barrier(procs)
        with ctx.Pool(procs) as pool:
            res = pool.map(_oracle_replica, [(workload, cells, per, warmup, steps, seconds, barrier)] * procs)
    # every replica ran the same sample from a common start: the job's rate is
    # all particle-steps over the slowest replica's time
    return sum(n * k for n, k, _ in res) / max(el for _, _, el in res), res


def default_cpu_procs() -> int:
    return max(1, os.cpu_count() or 1)


def cpu_baseline(args, seconds: float = 20.0):
    """The FP64 oracle, as it stands, on the host cores: a proportionally
    scaled copy of the workload (cells / 4 per axis, particles / 64, same
    density and dt recipe), stepped for about `seconds`: one replica per core
    (the headline value) and, before that, a single thread."""
    cells = max(4, args.cells // 4)
    per = max(1000, args.particles // 64)
    v1, r1 = oracle_runs(args.workload, cells, per, 0, 200, seconds, 1)
    procs = args.cpu_procs or default_cpu_procs()
    vall, rall = oracle_runs(args.workload, cells, per, 0, 200, seconds, procs) if procs > 1 else (v1, r1)
    n = r1[0][0]
    steps = min(k for _, k, _ in rall)
    return {"value": vall, "unit": "particle-steps/s", "cores": procs, "kind": "oracle",
            "host": host_cpu(),
            "single_thread": {"value": v1, "steps": r1[0][1], "seconds": round(r1[0][2], 2)},
            "sample": f"{args.workload} scaled to {cells}^3 cells and {n} particles (same density and dt recipe): "
                      f"{procs} independent replicas, one per host core, each for about {seconds:.0f} s "
                      f"(at least {steps} full steps each); the oracle is timed as it stands, a single-threaded "
                      f"program (one particle at a time in load order, sequential sums)"}


def reference_arm(args):
    """The oracle as the reference arm: K timed steps (after W warm-up steps)
    of the bounded scaled sample of the same workload, one replica per host
    core (the oracle is single-threaded)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cells = max(4, args.cells // 4)
    per = max(1000, args.particles // 64)
    desc = workload_desc(args.workload, cells, per)
    procs = args.cpu_procs or default_cpu_procs()
    value, res = oracle_runs(args.workload, cells, per, args.warmup, args.steps, None, procs)
    n = res[0][0]
    el = max(r[2] for r in res)
    sample = (f"{desc}: each step one step of this scaled copy of the workload (same density and dt recipe, "
              f"{cells}^3 cells, {n} particles) in each of {procs} independent replicas, one per host core")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, cells, per),
                       "sample_of": workload_desc(args.workload, args.cells, args.particles),
                       "replicas": procs},
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": procs, "kind": "oracle",
                             "host": host_cpu(), "sample": sample},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="plasma_ball", choices=["plasma_ball", "thermal_cube"])
    ap.add_argument("--cells", type=int, default=64)
    ap.add_argument("--particles", type=int, default=16 * 1024 * 1024, help="particles per species")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-procs", type=int, default=0,
                    help="oracle replicas for the CPU baseline and the reference arm (0: one per host core)")
    ap.add_argument("--clock-log", default=None, help="CSV of the clock samples of the timed region ({gpu}: index)")
    ap.add_argument("--skip-plain", action="store_true", help="do not time the plain-FP64 path (profiling runs)")
    ap.add_argument("--skip-e2e", action="store_true", help="do not run the end-to-end leg (profiling runs)")
    ap.add_argument("--skip-batched", action="store_true", help="do not run the batched-runs leg")
    ap.add_argument("--skip-gnn", action="store_true", help="do not run the learned-preconditioner leg")
    ap.add_argument("--skip-beam", action="store_true", help="do not run the electron-beam leg")
    ap.add_argument("--beam-particles", type=int, default=2_000_000)
    ap.add_argument("--beam-steps", type=int, default=20)
    ap.add_argument("--gnn-train-steps", type=int, default=300)
    ap.add_argument("--gnn-steps", type=int, default=3)
    ap.add_argument("--batch-runs", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=60)
    ap.add_argument("--skip-larmor", action="store_true", help="do not run the single-electron leg")
    ap.add_argument("--larmor-cells", type=int, default=20)
    ap.add_argument("--larmor-steps", type=int, default=10000)
    ap.add_argument("--skip-sweep", action="store_true", help="do not run the Table I pusher sweep")
    ap.add_argument("--skip-mixed-error", action="store_true", help="do not compare MIXED with the oracle")
    args = ap.parse_args()
    global CLOCK_LOG
    CLOCK_LOG = args.clock_log
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
