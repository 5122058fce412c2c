#!/usr/bin/env python
"""Throughput benchmark of the boosted-frame PIC step on GB300.

One step = the whole hot path of the method: gather + Boris push + Esirkepov
deposit of the electrons (one fused kernel), deposit of the drifting ions,
laser antenna, binomial current filter, Yee update and injection of the
plasma entering the box.  Default workload: the 3D gamma_boost = 13 stage
(256 x 256 x 1024 cells, 2x2x2 electrons per cell, ~535M electrons plus as
many drifting ions), FP32.  The metric is electron particle-steps per second
of whole steps, with all state resident in HBM; `e2e` is the same metric
through the C ABI with the initial state restored from pinned host memory and
the on-axis field line read back to the host after every step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torchrun) every rank runs an independent replica of
the workload on its own GPU: the stage does not shard across GPUs here, the
replicas exchange nothing, and rank 0 prints one JSON line.  `--impl
reference` times the FP64 CPU oracle on a bounded slab of the same stage.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (gather+push+deposit+Yee), %HBM roofline, adjoint/forward time"
UNIT = "particle-steps/s"
# algorithmic bytes per electron particle-step of the fused gather/push/deposit
# kernel in 3D: particle state read 32 B + written 28 B, plus fields read
# (24 B/cell) and current written (12 B/cell) amortised over ppc = 8; the same
# kernel then moves each drifting-ion record of the tile: 20 B read + 20 B
# written (the record moves to its output slot)
BYTES_PER_PARTICLE_STEP_3D = 60.0 + 36.0 / 8.0
BYTES_PER_ION_STEP_3D = 40.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--slots-per-cell", type=float, default=10.0)
    ap.add_argument("--touched-advance", type=int, default=300,
                    help="steps further into the stage for the second push window that separates the cost of "
                         "a field-touched electron from that of a paired one (0: skip)")
    ap.add_argument("--tile", default="",
                    help="particle tile shape x,y,z (a compiled one; default: the library's)")
    ap.add_argument("--sort-every", type=int, default=0,
                    help="order every tile's particles by cell before every N-th step (0: never)")
    ap.add_argument("--advance", type=int, default=-1,
                    help="stage steps run before the warm-up (default: half the stage, so that the timed window "
                         "sits in the middle of the stage, where the laser has reached the plasma in the box)")
    ap.add_argument("--explicit-ions", action="store_true",
                    help="store every drifting ion as its own record (no electron-ion pairs)")
    ap.add_argument("--no-explicit-check", action="store_true",
                    help="skip the second, shorter timing of the same stage with explicit ion records")
    ap.add_argument("--btd", type=int, default=16,
                    help="lab-frame (x, z)-plane snapshots timed after the main measurement (0: none)")
    ap.add_argument("--adjoint-steps", type=int, default=400,
                    help="steps of the adjoint/forward timing on one c4 run (0: skip)")
    ap.add_argument("--c4", type=int, default=64,
                    help="runs of the batched scan timed after the main measurement (0: none)")
    ap.add_argument("--c4-only", action="store_true",
                    help="time only the batched scan of --c4 runs (launch forms of pic_batch_step)")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="time only the adjoint/forward leg (one c4 run, --adjoint-steps steps, a checkpoint "
                         "every --checkpoint-every) and print its record")
    ap.add_argument("--checkpoint-every", type=int, default=50)
    ap.add_argument("--adjoint-3d-steps", type=int, default=100,
                    help="steps of the adjoint/forward timing on a 3D slab of the c2 stage (0: skip)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [float(r[3]) for r in self.rows if r[3].replace(".", "", 1).isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows), "power_w_max": max(pw) if pw else None}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_from_profiles(kernel_key: str):
    """DRAM bytes per launch of the kernel from the committed ncu summary, if
    that summary is for the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "push_kernel_traffic_c2_small.txt")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel_key)
    if not e:
        return None
    from paper_1011_0917_gb300 import build
    import hashlib
    # the electron kernel's sources: its per-tile body and the kernel itself
    src = b"".join(open(os.path.join(build.CSRC, f), "rb").read() for f in ("pic_push.cuh", "pic_particles.cu"))
    h = hashlib.sha256(src).hexdigest()[:16]
    if e.get("source_sha") != h:
        return None
    return e.get("dram_bytes_per_launch")


# --------------------------------------------------------------------- ours


def whole_job(elapsed: float, work: float, world: int, device: str) -> tuple[float, float]:
    """Whole-job aggregation of N independent replicas: the slowest rank's
    elapsed time (any unit) and the work of all ranks summed (two scalar
    all-reduces outside the timed region; the replicas exchange nothing else).
    device: "cuda" under NCCL, "cpu" under gloo."""
    if world <= 1:
        return elapsed, work
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([work], device=device, dtype=torch.float64)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def run_ours(args, rank, world, local):
    import torch
    import paper_1011_0917_gb300 as P
    from paper_1011_0917_gb300 import workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    st = W.stage(args.workload)
    g = st.grid
    stream = torch.cuda.Stream()
    advance = st.steps // 2 if args.advance < 0 else args.advance
    tile = tuple(int(v) for v in args.tile.split(",")) if args.tile else (0, 0, 0)
    sim = make_sim(P, st, args.slots_per_cell, stream, args.explicit_ions, advance, tile)
    ctx = sim.ctx
    if args.sort_every > 0:
        P.pic_set_cell_sort(ctx, args.sort_every)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # warm-up (untimed)
    P.pic_step(ctx, args.warmup)
    d0 = sim.diagnostics()
    P.pic_profile(ctx, True)
    P.pic_profile_read(ctx)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    P.pic_step_async(ctx, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    barrier()
    ms = e0.elapsed_time(e1)
    sim_tile = tuple(sim.sizes.tile)
    phase_ms, phase_calls, kernels = P.pic_profile_read(ctx)
    P.pic_profile(ctx, False)
    d1 = sim.diagnostics()
    n_e = 0.5 * (d0.n_particles[0] + d1.n_particles[0])
    n_i = 0.5 * (d0.n_particles[1] + d1.n_particles[1])
    # ion records the electron kernel moves (ions of paired electrons have none;
    # explicit ions have their own kernel)
    n_ir = 0.0 if args.explicit_ions else 0.5 * (d0.n_particles[1] - d0.n_paired + d1.n_particles[1] - d1.n_paired)
    # electrons still paired with their ion (plasma no field has reached yet:
    # the pair's current is exactly zero and is not deposited)
    paired = [d0.n_paired / max(d0.n_particles[0], 1), d1.n_paired / max(d1.n_particles[0], 1)]
    psteps = n_e * args.steps

    # whole-job aggregation: max time, summed work
    ms, psteps = whole_job(ms, psteps, world, "cuda")
    value = psteps / (ms * 1e-3)

    # roofline of the dominant kernel (the fused electron gather/push/deposit)
    push_ms = phase_ms[1] / max(phase_calls[1], 1)
    algo_bytes = (BYTES_PER_PARTICLE_STEP_3D * n_e + BYTES_PER_ION_STEP_3D * n_ir if g["dim"] == 3
                  else (52.0 + 36.0 / 4) * n_e + 32.0 * n_ir)
    achieved = algo_bytes / (push_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    # (slot 7, the TIME phase's, holds the cell sorts)
    phases = ["zero_j", "push", "ions", "antenna", "filter", "yee", "inject", "cell_sort"]
    share = {phases[i]: round(phase_ms[i] / max(sum(phase_ms), 1e-30), 4) for i in range(8)
             if i < 7 or phase_calls[7] > 0}

    # end to end through the C ABI: restore the initial state from pinned host
    # memory, then each step read the on-axis E_z line back to the host
    e2e = None
    if not args.no_e2e:
        nbytes = P.pic_state_bytes(ctx)
        host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        P.pic_get_state(ctx, host.data_ptr(), nbytes, False)
        line = torch.empty(g["nz"] + 1, dtype=torch.float32, pin_memory=True)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P.pic_set_state(ctx, host.data_ptr(), nbytes, False)
        for _ in range(args.steps):
            P.pic_step_async(ctx, 1)
            P.pic_get_axis(ctx, 2, line.data_ptr(), line.numel() * 4, False)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        el, e2e_work = whole_job(t1 - t0, n_e * args.steps, world, "cuda")
        e2e = {"value": e2e_work / el, "unit": UNIT,
               "h2d_bytes_per_step": int(nbytes // args.steps), "d2h_bytes_per_step": int(line.numel() * 4),
               "note": "initial state restored from pinned host memory once per job of --steps steps; "
                       "on-axis Ez line read back after every step"}
        del host

    # lab-frame snapshots: the same steps with n (x, z)-plane snapshots whose
    # events the run is passing now, filled by the YEE phase
    btd = None
    if args.btd > 0 and g["gamma_boost"] > 1.0:
        k = max(1, min(args.steps, 8))
        P.pic_profile(ctx, True)
        P.pic_profile_read(ctx)
        P.pic_step(ctx, k)
        base_ms, base_calls, _ = P.pic_profile_read(ctx)
        sz = sim.sizes
        gam, beta = g["gamma_boost"], sz.beta
        lz = g["nz"] * sz.hz
        tnow = sim.diagnostics().t
        # snapshot j at lab time t_first + j (lambda0/c) covers lab z in
        # [beta T_j, beta T_j + Lz / gamma]; the run is passing the events at
        # the middle of the box for every one of them
        t_first = gam * (tnow + 0.5 * beta * lz)
        z0 = beta * t_first - 1.0
        nz_lab = int((lz / gam + 2.0 + args.btd * beta) / g["dz"])
        sim.btd_setup(args.btd, t_first, 1.0, z0, g["dz"], nz_lab, 1)
        P.pic_step(ctx, k)
        btd_ms, btd_calls, _ = P.pic_profile_read(ctx)
        P.pic_profile(ctx, False)
        filled = sum(int(sim.btd_snapshot(j)[1].sum()) for j in range(args.btd))
        yee = btd_ms[5] / max(btd_calls[5], 1)
        yee0 = base_ms[5] / max(base_calls[5], 1)
        btd = {"snapshots": args.btd, "plane": "(x, z) at y = Ly/2", "lab_points_per_snapshot": nz_lab,
               "columns": g["nx"], "steps": k, "lab_planes_filled": filled,
               "yee_phase_ms_with": yee, "yee_phase_ms_without": yee0, "added_ms_per_step": yee - yee0,
               "buffer_bytes": int(sim._btd.numel())}
        P.pic_btd_setup(ctx, None, 0, 0)

    # the cost of a field-touched electron: the push timed again further into
    # the stage, where fewer electrons are still paired with their ion; with
    # push time = a * paired + b * released (b: a released electron together
    # with the record of its ion), the two windows give a and b
    touched = None
    if args.touched_advance > 0 and g["gamma_boost"] > 1.0 and not args.explicit_ions:
        P.pic_step(ctx, args.touched_advance)
        k = max(1, min(args.steps, 8))
        d2 = sim.diagnostics()
        P.pic_profile(ctx, True)
        P.pic_profile_read(ctx)
        P.pic_step(ctx, k)
        ph2, calls2, _ = P.pic_profile_read(ctx)
        P.pic_profile(ctx, False)
        d3 = sim.diagnostics()
        p1 = 0.5 * (d0.n_paired + d1.n_paired)
        r1 = n_e - p1
        p2 = 0.5 * (d2.n_paired + d3.n_paired)
        r2 = 0.5 * (d2.n_particles[0] + d3.n_particles[0]) - p2
        t1, t2 = push_ms, ph2[1] / max(calls2[1], 1)
        det = p1 * r2 - p2 * r1
        if abs(det) > 1e-6 * max(p1 * r2, 1.0):
            a_ms = (t1 * r2 - t2 * r1) / det
            b_ms = (p1 * t2 - p2 * t1) / det
            touched = {"windows_steps_from": [advance + args.warmup, int(round(d2.t / sim.dt))],
                       "paired": [p1, p2], "released": [r1, r2], "push_ms": [t1, t2],
                       "ns_per_paired_electron": a_ms * 1e6, "ns_per_released_electron": b_ms * 1e6,
                       "released_electron_steps_per_s": 1e3 / b_ms if b_ms > 0 else None,
                       "note": "push time per launch = a * paired electrons + b * released electrons (each with "
                               "its released-ion record), solved from two windows of the stage"}
    sim.close()
    del sim
    torch.cuda.empty_cache()

    # the same stage with every ion stored as its own record from the start
    # (no electron-ion pairs), timed over fewer steps: what the step costs when
    # the ions are pushed and deposited like any other species
    explicit = None
    if not args.explicit_ions and not args.no_explicit_check and st.plasma["ions"]:
        k = max(1, min(args.steps, 8))
        sim = make_sim(P, st, args.slots_per_cell, stream, True, advance)
        P.pic_step(sim.ctx, args.warmup)
        P.pic_profile(sim.ctx, True)
        P.pic_profile_read(sim.ctx)
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        P.pic_step_async(sim.ctx, k)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        xph, xcalls, _ = P.pic_profile_read(sim.ctx)
        dx_ = sim.diagnostics()
        xms, xwork = whole_job(e0.elapsed_time(e1), dx_.n_particles[0] * k, world, "cuda")
        explicit = {"steps": k, "ms_per_step": xms / k, "value": xwork / (xms * 1e-3),
                    "n_ion_records": dx_.n_particles[1], "push_ms_per_launch": xph[1] / max(xcalls[1], 1),
                    "ions_ms_per_launch": xph[2] / max(xcalls[2], 1)}
        sim.close()

    c4 = run_c4(P, torch, args.c4, args.warmup, 200) if args.c4 > 0 else None
    adj = run_adjoint(P, torch, args.adjoint_steps, args.checkpoint_every) if args.adjoint_steps > 0 else None
    adj3 = run_adjoint_3d(P, torch, args.adjoint_3d_steps) if args.adjoint_3d_steps > 0 else None

    result = None
    if rank == 0:
        cpu = None if args.no_cpu_baseline else cpu_baseline(args.workload, steps=20)
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded lattice plasma + Gaussian laser antenna)",
            "config": {"workload": workload_name(args.workload), "n_electrons": n_e, "n_drift_ions": n_i,
                       "grid": [g["nx"], g["ny"], g["nz"]], "gamma_boost": g["gamma_boost"],
                       "filter_passes": g["filter_passes"], "shape_order": g["shape_order"],
                       "slots_per_cell": args.slots_per_cell, "cell_sort_every": args.sort_every,
                       "tile": list(sim_tile),
                       "timed_window": f"steps {advance + args.warmup}..{advance + args.warmup + args.steps - 1} "
                                       f"of the {st.steps}-step stage",
                       "ion_records": "explicit" if args.explicit_ions else "paired with electrons until released",
                       "paired_fraction_start_end": [round(paired[0], 4), round(paired[1], 4)],
                       "l2": "inputs larger than L2 (particle store >> 129 MB)",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": traffic_from_profiles("push_kernel<float,3,1>"),
                         "kernel": "push_kernel<float,3,1> (electrons: gather+Boris+Esirkepov+re-bucket; "
                                   "then the tile's drifting-ion records: move+Jz+re-bucket)",
                         "bytes_per_unit": {"electron particle-step": BYTES_PER_PARTICLE_STEP_3D,
                                            "ion record step": BYTES_PER_ION_STEP_3D},
                         "units_per_launch": {"electrons": n_e, "ion_records": n_ir},
                         "ms_per_launch": push_ms},
            "phase_share": share,
            "field_touched_electron_cost": touched,
            "e2e": e2e,
            "gpu_launches": int(kernels),
            "clocks": clock_info,
            "cpu_baseline": cpu,
            "adjoint_forward_ratio": adj["ratio"] if adj else None,
            "adjoint": adj,
            "adjoint_3d": adj3,
            "explicit_ion_records": explicit,
            "lab_frame_snapshots": btd,
            "batched_c4": c4,
        }
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return result


def run_c4(P, torch, nruns, warmup, steps, graph_steps=20):
    """The batched scan: nruns independent 2D3V boosted runs (c4 recipe), each
    on its own stream, stepped together by pic_batch_step; and the same runs
    stepped one after another on one stream.  Aggregate electron
    particle-steps/s of both."""
    from paper_1011_0917_gb300 import workloads as W
    sims = []
    for r in range(nruns):
        st = W.c4_run(r)
        g = st.grid
        sim = P.Simulation(dim=2, nx=g["nx"], ny=1, nz=g["nz"], dx=g["dx"], dz=g["dz"], cfl=g["cfl"],
                           gamma_boost=g["gamma_boost"], filter_passes=g["filter_passes"], precision=P.PIC_FP32,
                           seed=g["seed"], slots_per_cell=6.0, stream=torch.cuda.Stream())
        p = st.plasma
        sim.load_plasma(p["ne"], p["z_start"], p["z_end"], p["ramp"], p["ppc"], p["jitter"], p["profile"], p["ions"])
        l = st.laser
        sim.launch_laser(l["a0"], l["waist"], l["fwhm"], 0.0, -1.0, 1)
        sims.append(sim)
    batch = P.Batch(sims, graph_steps=0)
    batch.step(warmup)
    n0 = sum(s.diagnostics().n_particles[0] for s in sims)
    # launch by launch on the runs' streams
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch.step(steps)
    torch.cuda.synchronize()
    t_streams = time.perf_counter() - t0
    # the same steps as replays of a captured graph: a first call of
    # graph_steps steps captures it (timed on its own), the batch keeps it;
    # the per-context graph (every run's launches on its own stream), then
    # the fused one with 1, 2, 4 and 8 launch chains
    P.pic_batch_set_graph(batch.h, graph_steps)
    timings = {}
    for chains in (0, 1, 2, 4, 8):
        P.pic_batch_set_fused(batch.h, chains)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch.step(graph_steps)
        torch.cuda.synchronize()
        t_capture = time.perf_counter() - t0
        t0 = time.perf_counter()
        batch.step(steps)
        torch.cuda.synchronize()
        timings[chains] = (time.perf_counter() - t0, t_capture, batch.graph_info())
    best = min((c for c in timings if c > 0), key=lambda c: timings[c][0])
    t_batch, t_capture, info = timings[best]
    t_ctx, t_capture_ctx, info_ctx = timings[0]
    # the same runs one after another on a single stream (each pic_step waits)
    t0 = time.perf_counter()
    for s in sims:
        P.pic_step(s.ctx, steps)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    batch.close()
    for s in sims:
        s.close()
    torch.cuda.empty_cache()
    forms = {"streams": t_streams, "per_context_graph": t_ctx, f"fused_graph_{best}_chains": t_batch}
    fastest = min(forms, key=forms.get)
    return {"runs": nruns, "steps": steps, "electrons": n0, "value": n0 * steps / forms[fastest],
            "ms_per_step": 1e3 * forms[fastest] / steps, "form": fastest,
            "fused_value": n0 * steps / t_batch, "fused_ms_per_step": 1e3 * t_batch / steps,
            "graph_steps": graph_steps, "fused_chains": info["chains"],
            "fused_ms_per_step_by_chains": {c: round(1e3 * timings[c][0] / steps, 4) for c in timings if c > 0},
            "launches_per_step": info["launches_per_replay"] / graph_steps,
            "first_call_ms": 1e3 * t_capture,
            "per_context_graph_value": n0 * steps / t_ctx, "per_context_graph_ms_per_step": 1e3 * t_ctx / steps,
            "per_context_launches_per_step": info_ctx["launches_per_replay"] / graph_steps,
            "per_context_first_call_ms": 1e3 * t_capture_ctx,
            "streams_value": n0 * steps / t_streams, "streams_ms_per_step": 1e3 * t_streams / steps,
            "sequential_value": n0 * steps / t_seq, "speedup_vs_sequential": t_seq / forms[fastest],
            "note": "2D3V boosted runs, gamma in {5, 13, 30}, nz in [1024, 4096], nx = 128, 2x2 per cell, "
                    "8-coefficient profile, a0 in [0.5, 2]; host wall clock around pic_batch_step (graph: "
                    "graph_steps steps of all runs captured once as one CUDA graph by a first call, timed as "
                    "first_call_ms, and kept by the batch; the timed call replays it).  value: the fastest form "
                    "(form): streams (launch by launch on the runs' streams), per_context_graph (every run's "
                    "launches on its own stream inside the graph) or the fused graph with the fastest of 1, 2, "
                    "4, 8 launch chains (each chain one launch per phase over its runs, the push a persistent "
                    "grid over (run, tile) items; fused_value)"}


def run_adjoint(P, torch, steps, K, r=0):
    """Adjoint/forward time on run r of the c4 scan: the gradient of the
    on-axis Ez over planes 16..127 after `steps` steps with respect to the
    8 profile coefficients, a0 and the waist (forward with a checkpoint every
    K steps, then the reverse sweep recomputing each segment), against the
    library's forward step over the same steps; with the checkpoint interval
    fitted to the device's memory and with the fixed interval K.  CUDA events
    on the run's stream."""
    from paper_1011_0917_gb300 import workloads as W
    st = W.c4_run(r)
    g = st.grid

    def make():
        sim = P.Simulation(dim=2, nx=g["nx"], ny=1, nz=g["nz"], dx=g["dx"], dz=g["dz"], cfl=g["cfl"],
                           gamma_boost=g["gamma_boost"], filter_passes=g["filter_passes"], precision=P.PIC_FP32,
                           seed=g["seed"], slots_per_cell=6.0, stream=torch.cuda.Stream())
        p = st.plasma
        sim.load_plasma(p["ne"], p["z_start"], p["z_end"], p["ramp"], p["ppc"], p["jitter"], p["profile"], p["ions"])
        l = st.laser
        sim.launch_laser(l["a0"], l["waist"], l["fwhm"], 0.0, -1.0, 1)
        return sim

    def timed(sim, fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(sim.stream)
        out = fn()
        e1.record(sim.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    # untimed warm-up of both paths (the first launch of each kernel in a
    # process loads its module)
    w = make()
    with torch.cuda.stream(w.stream):
        f = w.adjoint_forward(4, 2)
        w.adjoint_backward(torch.zeros_like(f))
    w.close()
    w = make()
    P.pic_step(w.ctx, 4)
    w.close()
    del f
    sim = make()
    n_e = sim.diagnostics().n_particles[0]
    fwd_ms, _ = timed(sim, lambda: P.pic_step_async(sim.ctx, steps))
    sim.close()

    def adjoint(k):
        sim = make()
        if k is None:  # fitted to the device's memory
            k = sim.adjoint_checkpoint_interval(steps)
        with torch.cuda.stream(sim.stream):
            # the adjoint's buffer allocated before the timing, as the forward's are
            bufs = sim.adjoint_buffers(steps, k)
            a_fwd_ms, fields = timed(sim, lambda: sim.adjoint_forward(steps, k, buffers=bufs))
            cot = torch.zeros_like(fields)
            cot[2, 16:128, g["nx"] // 2] = 1.0
            a_bwd_ms, grad = timed(sim, lambda: sim.adjoint_backward(cot))
        nbytes = sim._adj.numel()
        sim.close()
        del fields, cot, bufs
        torch.cuda.empty_cache()
        return {"checkpoint_every": k, "adjoint_forward_ms": a_fwd_ms, "adjoint_reverse_ms": a_bwd_ms,
                "ratio": (a_fwd_ms + a_bwd_ms) / fwd_ms, "buffer_bytes": int(nbytes),
                "gradient": {"profile": grad[:-2], "a0": grad[-2], "w0": grad[-1]}}

    fixed = adjoint(K)
    fitted = adjoint(None)
    return {"run": f"c4[{r}]: gamma={g['gamma_boost']:g}, {g['nx']}x{g['nz']} cells, {n_e} electrons, {steps} steps",
            "forward_ms": fwd_ms, "ratio": fixed["ratio"], "checkpoint_every": K,
            "adjoint_forward_ms": fixed["adjoint_forward_ms"], "adjoint_reverse_ms": fixed["adjoint_reverse_ms"],
            "buffer_bytes": fixed["buffer_bytes"], "gradient": fixed["gradient"],
            "memory_fitted_interval": {k: v for k, v in fitted.items() if k != "gradient"},
            "objective": "sum of on-axis Ez over planes 16..127 (behind the antenna, inside the plasma) at the "
                         "last step",
            "note": "CUDA events on the run's stream around the library's forward steps and around the adjoint "
                    "forward and reverse calls; the adjoint's device buffer is allocated before its timing, as "
                    "the forward's buffers are at binding; both paths warmed up (module loading) before.  ratio: "
                    "with a checkpoint every --checkpoint-every steps; memory_fitted_interval: with the largest "
                    "interval whose buffer fits half of the free HBM (Simulation.adjoint_checkpoint_interval)"}


def run_adjoint_3d(P, torch, steps, K=25, K2=5):
    """Adjoint/forward time of a 3D run: the c2 stage (gamma = 13, CIC, 2
    passes, 2x2x2 per cell, FP32) on a 96 x 96 x 192 slab, the gradient of the
    on-axis Ez over planes 8..119 after `steps` steps with respect to a0 and
    the waist (the c2 plasma has no profile coefficients); one-level
    checkpoints every K steps and two-level ones (a sub-checkpoint every K2
    steps: a smaller buffer for one more forward pass)."""
    from paper_1011_0917_gb300 import workloads as W
    st = W.stage("c2")
    g = dict(st.grid, nx=96, ny=96, nz=192)

    def make():
        sim = P.Simulation(dim=3, nx=g["nx"], ny=g["ny"], nz=g["nz"], dx=g["dx"], dy=g["dy"], dz=g["dz"],
                           cfl=g["cfl"], gamma_boost=g["gamma_boost"], filter_passes=g["filter_passes"],
                           precision=P.PIC_FP32, seed=g["seed"], slots_per_cell=10.0, stream=torch.cuda.Stream())
        p = st.plasma
        sim.load_plasma(p["ne"], p["z_start"], p["z_end"], p["ramp"], p["ppc"], p["jitter"], (), p["ions"])
        l = st.laser
        sim.launch_laser(l["a0"], l["waist"], l["fwhm"], 0.0, 1.0, l["pol"])
        return sim

    def timed(sim, fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(sim.stream)
        out = fn()
        e1.record(sim.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    # untimed warm-up of both paths (module loading)
    w = make()
    with torch.cuda.stream(w.stream):
        f = w.adjoint_forward(4, 2)
        w.adjoint_backward(torch.zeros_like(f))
    w.close()
    w = make()
    P.pic_step(w.ctx, 4)
    w.close()
    del f
    sim = make()
    n_e = sim.diagnostics().n_particles[0]
    fwd_ms, _ = timed(sim, lambda: P.pic_step_async(sim.ctx, steps))
    sim.close()
    out = {"run": f"c2 stage on a {g['nx']}x{g['ny']}x{g['nz']} slab, {n_e} electrons, {steps} steps, FP32",
           "forward_ms": fwd_ms}
    for name, k2 in (("one_level", 0), ("two_level", K2)):
        sim = make()
        with torch.cuda.stream(sim.stream):
            bufs = sim.adjoint_buffers(steps, K, k2)
            a_fwd_ms, fields = timed(sim, lambda: sim.adjoint_forward(steps, K, k2, buffers=bufs))
            cot = torch.zeros_like(fields)
            cot[2, 8:120, g["ny"] // 2, g["nx"] // 2] = 1.0
            a_bwd_ms, grad = timed(sim, lambda: sim.adjoint_backward(cot))
        out[name] = {"checkpoint_every": K, "sub_checkpoint_every": k2, "adjoint_forward_ms": a_fwd_ms,
                     "adjoint_reverse_ms": a_bwd_ms, "ratio": (a_fwd_ms + a_bwd_ms) / fwd_ms,
                     "buffer_bytes": int(sim._adj.numel()), "gradient": {"a0": grad[-2], "w0": grad[-1]}}
        sim.close()
        del fields, cot, bufs
        torch.cuda.empty_cache()
    return out


def make_sim(P, st, slots_per_cell, stream, explicit_ions, advance, tile=(0, 0, 0)):
    g = st.grid
    sim = P.Simulation(dim=g["dim"], nx=g["nx"], ny=g["ny"], nz=g["nz"], dx=g["dx"], dy=g["dy"], dz=g["dz"],
                       cfl=g["cfl"], gamma_boost=g["gamma_boost"], shape_order=g["shape_order"],
                       filter_passes=g["filter_passes"], bc_z=g["bc_z"], precision=P.PIC_FP32, seed=g["seed"],
                       slots_per_cell=slots_per_cell, explicit_ions=explicit_ions, stream=stream, tile=tile)
    p = st.plasma
    sim.load_plasma(p["ne"], p["z_start"], p["z_end"], p["ramp"], p["ppc"], p["jitter"], (), p["ions"])
    l = st.laser
    sim.launch_laser(l["a0"], l["waist"], l["fwhm"], l["z_antenna"], -1.0, l["pol"])
    if advance > 0:
        P.pic_step(sim.ctx, advance)
    return sim


def workload_name(w: str) -> str:
    names = {
        "c2": "3D boosted frame gamma=13, 256x256x1024 cells, 2x2x2 electrons/cell (+drifting ions), CIC, "
              "2 binomial passes, FP32",
        "c1": "2D3V boosted frame gamma=13, 256x8192 cells, 2x2 electrons/cell, CIC, 2 passes, FP32",
        "c0": "2D3V lab frame, 64x512 cells, 2x2 electrons/cell, CIC, 1 pass, FP32",
        "c2_small": "3D boosted frame gamma=13, 128x128x256 cells (profiling slab of the 256x256x1024 stage), "
                    "2x2x2 electrons/cell (+drifting ions), CIC, 2 binomial passes, FP32",
    }
    return names.get(w, w)


# ------------------------------------------------------------------ oracle


def oracle_slab(workload: str):
    """A bounded slab of the workload for the FP64 CPU oracle: same cell
    sizes, boost, shape, filter, density and lattice, fewer cells."""
    import oracle.oracle as O
    st, g = oracle_slab_grid(workload)
    o = O.Oracle(O.GridParams(dim=g["dim"], nx=g["nx"], ny=g["ny"], nz=g["nz"], dx=g["dx"], dy=g["dy"], dz=g["dz"],
                              cfl=g["cfl"], gamma_boost=g["gamma_boost"], shape=g["shape_order"],
                              npass=g["filter_passes"], bc_z=g["bc_z"], seed=g["seed"]))
    p = st.plasma
    o.load_plasma(O.PlasmaParams(ne=p["ne"], z_start=p["z_start"], z_end=p["z_end"], ramp=p["ramp"], ppc=p["ppc"],
                                 jitter=p["jitter"], ions=p["ions"]))
    l = st.laser
    o.set_laser(O.LaserParams(a0=l["a0"], waist=l["waist"], fwhm=l["fwhm"], z_antenna=l["z_antenna"], pol=l["pol"]))
    return o, g


def cpu_model() -> str:
    """The host CPU's model name (lscpu), else the platform's processor string."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_copy(workload, warmup, steps, barrier, out):
    """One copy of the oracle's slab in its own process: warm-up steps, then
    (once every copy is ready) `steps` timed steps."""
    o, _ = oracle_slab(workload)
    o.step(warmup)
    n = o.num(0)
    barrier.wait()
    t0 = time.perf_counter()
    o.step(steps)
    out.put((n, time.perf_counter() - t0))


def oracle_timing(workload: str, warmup: int, steps: int, copies: int) -> dict:
    """Electron particle-steps/s of the FP64 oracle, as it stands, on the
    host: `copies` independent copies of the same slab run at once, one per
    process (started with spawn: the caller may hold a CUDA context), each
    single-threaded, so that `copies` cores work.  Returns the summed work over
    the slowest copy's elapsed time."""
    if copies <= 1:
        o, g = oracle_slab(workload)
        o.step(warmup)
        n = o.num(0)
        t0 = time.perf_counter()
        o.step(steps)
        el = time.perf_counter() - t0
        return {"value": n * steps / el, "elapsed_s": el, "electrons_per_copy": n, "ions_per_copy": o.num(1),
                "grid": [g["nx"], g["ny"], g["nz"]], "copies": 1}
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(copies)
    out = ctx.Queue()
    procs = [ctx.Process(target=_oracle_copy, args=(workload, warmup, steps, barrier, out)) for _ in range(copies)]
    for p in procs:
        p.start()
    res = [out.get() for _ in procs]
    for p in procs:
        p.join()
    el = max(r[1] for r in res)
    n = res[0][0]
    _, g = oracle_slab_grid(workload)
    return {"value": sum(r[0] for r in res) * steps / el, "elapsed_s": el, "electrons_per_copy": n,
            "grid": [g["nx"], g["ny"], g["nz"]], "copies": copies}


def oracle_slab_grid(workload: str):
    from paper_1011_0917_gb300 import workloads as W
    st = W.stage(workload)
    g = dict(st.grid)
    if g["dim"] == 3:
        g.update(nx=32, ny=32, nz=64)
    else:
        g.update(nx=min(g["nx"], 64), nz=min(g["nz"], 256))
    return st, g


def cpu_baseline(workload: str, steps: int = 20):
    """The oracle on the host cores: one thread, then every core (one copy of
    the slab per core); the all-cores figure is the value."""
    one = oracle_timing(workload, 0, steps, 1)
    cores = host_cores()
    allc = oracle_timing(workload, 0, steps, cores) if cores > 1 else one
    model = cpu_model()
    gx, gy, gz = one["grid"]
    return {"value": allc["value"], "unit": UNIT, "cores": allc["copies"], "kind": "oracle",
            "sample": f"{gx}x{gy}x{gz} slab of the same stage ({one['electrons_per_copy']} electrons, "
                      f"{one['ions_per_copy']} ions), {steps} steps, FP64 C oracle as it stands; "
                      f"{allc['copies']} single-threaded copies at once on {cores} cores ({model}), "
                      f"{allc['elapsed_s']:.1f} s",
            "single_thread": {"value": one["value"], "cores": 1, "elapsed_s": one["elapsed_s"]},
            "nproc": cores, "cpu_model": model}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    cores = host_cores()
    r = oracle_timing(args.workload, args.warmup, args.steps, cores)
    value = r["value"]
    gx, gy, gz = r["grid"]
    model = cpu_model()
    sample = (f"{gx}x{gy}x{gz} slab of the same stage per step ({r['electrons_per_copy']} electrons per copy), "
              f"FP64 C oracle as it stands, {r['copies']} single-threaded copies at once on {cores} cores "
              f"({model})")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["elapsed_s"] * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded lattice plasma + Gaussian laser antenna)",
            "config": {"workload": workload_name(args.workload).replace(", FP32", "")
                       + f"; timed on a {gx}x{gy}x{gz} slab of it in FP64",
                       "slab": [gx, gy, gz], "parallelism": "host cores, rank 0 only"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["copies"], "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.c4_only:
        out = None
        if rank == 0:
            import torch

            import paper_1011_0917_gb300 as P
            out = run_c4(P, torch, args.c4, args.warmup, 200)
    elif args.adjoint_only:
        out = None
        if rank == 0:
            import torch

            import paper_1011_0917_gb300 as P
            out = run_adjoint(P, torch, args.adjoint_steps, args.checkpoint_every)
    else:
        out = run_ours(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
