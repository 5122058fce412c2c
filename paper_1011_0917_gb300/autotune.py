"""Autotuner of a run's launch configuration.

Chooses, by timing a few steps of the run itself, among the configurations
the library offers at run time:

* the particle tile shape: in 2D 16 x 16, 32 x 8 or 8 x 32 cells (x, z; the
  last two with the CIC shape), in 3D 8 x 8 x 8 or (CIC) 8 x 8 x 4, which
  sets how many particles a CTA stages fields and accumulates currents for,
  and how many leave their tile per step;
* the bucket capacity (slots per cell), which sets the memory a tile's
  particle records span;
* for a batch of runs, the launch form: launch by launch on the runs'
  streams, or captured CUDA graphs of a number of steps, per context or
  fused with a number of launch chains (each chain one launch per phase
  over its runs, the particle push a persistent grid over (run, tile)
  items).

Particles are sorted into their tiles at every step, inside the push; the
order by cell inside a tile (pic_set_cell_sort) is a candidate too (its
interval, 0 for never).  The CTA shape (256 threads) is compiled.
A candidate whose buckets overflow during the trial is discarded.
"""
from __future__ import annotations

import itertools
import time

TILES_2D = ((16, 1, 16), (32, 1, 8), (8, 1, 32))
TILES_3D = ((8, 8, 8), (8, 8, 4))
SLOTS = (6.0, 8.0, 12.0)


def _build(P, settings: dict, tile, slots, stream):
    g = dict(settings["grid"])
    g.update(tile=tile, slots_per_cell=slots, stream=stream)
    sim = P.Simulation(**g)
    p = settings["plasma"]
    sim.load_plasma(p["ne"], p["z_start"], p["z_end"], p.get("ramp", 0.0), p.get("ppc", (2, 1, 2)),
                    p.get("jitter", 0.1), p.get("profile", ()), p.get("ions", 1))
    l = settings["laser"]
    sim.launch_laser(l["a0"], l["waist"], l["fwhm"], l.get("z_antenna", 0.0), l.get("t_peak", -1.0),
                     l.get("pol", P.PIC_POL_Y))
    return sim


def tune_run(settings: dict, steps: int = 8, warmup: int = 3, tiles=None, slots=SLOTS, sort_every=(0,)) -> dict:
    """Time every (tile, slots_per_cell, sort_every) candidate on `steps` steps
    of the run described by settings = {"grid": Simulation kwargs, "plasma":
    ..., "laser": ...} after `warmup` steps (sort_every: order the particle
    store by cell before every n-th step, 0 never).  Returns {"tile",
    "slots_per_cell", "sort_every", "ms_per_step", "trials": [...]} for the
    fastest candidate."""
    import torch

    import paper_1011_0917_gb300 as P
    g = settings["grid"]
    if tiles is None:
        cic = g.get("shape_order", 1) == 1
        tiles = (TILES_2D if g.get("dim", 2) == 2 else TILES_3D) if cic else ((0, 0, 0),)
    trials = []
    for tile, sl, srt in itertools.product(tiles, slots, sort_every):
        stream = torch.cuda.Stream()
        sim = None
        cand = {"tile": tuple(tile), "slots_per_cell": sl, "sort_every": srt}
        try:
            sim = _build(P, settings, tile, sl, stream)
            P.pic_step(sim.ctx, warmup)
            P.pic_set_cell_sort(sim.ctx, srt)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            P.pic_step_async(sim.ctx, steps)
            e1.record(stream)
            torch.cuda.synchronize()
            P.pic_step(sim.ctx, 0)  # the device error word of the timed steps
            trials.append(dict(cand, ms_per_step=e0.elapsed_time(e1) / steps))
        except P.PicError as e:
            trials.append(dict(cand, error=str(e)))
        finally:
            if sim is not None:
                sim.close()
    ok = [t for t in trials if "ms_per_step" in t]
    if not ok:
        raise RuntimeError("autotune: no candidate ran: " + "; ".join(t.get("error", "") for t in trials))
    best = min(ok, key=lambda t: t["ms_per_step"])
    return dict(best, trials=trials)


def tune_batch(settings_list, steps: int = 40, warmup: int = 3, graph_steps=(0, 20, 40), chains=(0, 1, 2, 4, 8),
               tile=(0, 0, 0), slots: float = 8.0) -> dict:
    """Time pic_batch_step of the runs for every launch form: launch by launch
    on the runs' streams (graph_steps 0), and for each number of steps per
    captured graph, the per-context graph (chains 0) and the fused graph with
    each number of launch chains.  Returns the fastest and all trials."""
    import torch

    import paper_1011_0917_gb300 as P
    sims = [_build(P, s, tile, slots, torch.cuda.Stream()) for s in settings_list]
    trials = []
    try:
        batch = P.Batch(sims, graph_steps=0)
        batch.step(warmup)
        forms = [(0, 0)] + [(k, m) for k in graph_steps if k > 0 for m in chains]
        for k, m in forms:
            # the runs' work spans their own streams: time on the host between
            # two device-wide synchronisations; a graph is captured by an
            # untimed first call of k steps and kept by the batch
            P.pic_batch_set_graph(batch.h, k)
            P.pic_batch_set_fused(batch.h, m)
            if k > 0:
                batch.step(k)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            batch.step(steps)
            torch.cuda.synchronize()
            info = P.pic_batch_graph_info(batch.h)
            trials.append({"graph_steps": k, "chains": info["chains"] if k > 0 else 0,
                           "ms_per_step": 1e3 * (time.perf_counter() - t0) / steps})
        batch.close()
    finally:
        for s in sims:
            s.close()
    best = min(trials, key=lambda t: t["ms_per_step"])
    return dict(best, trials=trials)
