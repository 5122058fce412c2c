"""The batched scan: independent boosted runs (different boosts, lengths,
density profiles and laser amplitudes, the c4 recipe on smaller grids) stepped
together through pic_batch_step: as replays of a captured CUDA graph in its
fused form (one launch per phase over all runs) or per context (each run's
launches on its own stream), or launch by launch on the runs' streams; every
run matches its own FP64 oracle run (full-step tolerances: 1e-4 FP32, 1e-10
FP64)."""
import pytest

from pairs import make_pair, vector_errors
from paper_1011_0917_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1
TOL = {FP32: 1e-4, FP64: 1e-10}


@pytest.fixture(scope="module")
def O():
    import oracle.oracle as O
    O.build_oracle()
    return O


@pytest.mark.parametrize("graph_steps,fused", [(10, 2), (10, 0), (0, 1)])
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_batch_matches_each_run(O, prec, graph_steps, fused):
    import torch

    import paper_1011_0917_gb300 as P
    runs = [W.c4_run(r, nz_range=(96, 200), nx=24, steps=32) for r in range(4)]
    sims, oracles = [], []
    for st in runs:
        g = dict(st.grid)
        sim, o = make_pair(O, g, prec)
        # a stream of its own for every run (make_pair's Simulation used the
        # current stream: rebuild it on a private one)
        sim.close()
        sim = P.Simulation(dim=2, nx=g["nx"], ny=1, nz=g["nz"], dx=g["dx"], dz=g["dz"], gamma_boost=g["gamma_boost"],
                           filter_passes=g["filter_passes"], precision=prec, seed=g["seed"], slots_per_cell=16.0,
                           stream=torch.cuda.Stream())
        p = dict(st.plasma, z_end=st.plasma["z_start"] + 300.0 * g["gamma_boost"])
        sim.load_plasma(p["ne"], p["z_start"], p["z_end"], p["ramp"], p["ppc"], p["jitter"], p["profile"], p["ions"])
        o.load_plasma(O.PlasmaParams(ne=p["ne"], z_start=p["z_start"], z_end=p["z_end"], ramp=p["ramp"], ppc=p["ppc"],
                                     jitter=p["jitter"], profile=p["profile"], ions=p["ions"]))
        l = st.laser
        sim.launch_laser(l["a0"], l["waist"], l["fwhm"], 0.0, 0.5, 1)
        o.set_laser(O.LaserParams(a0=l["a0"], waist=l["waist"], fwhm=l["fwhm"], t_peak=0.5, pol=1))
        sims.append(sim)
        oracles.append(o)
    assert len({st.grid["gamma_boost"] for st in runs}) >= 2
    # 32 steps in three calls.  With graphs of 10 steps: a capture and its
    # replay; the kept graph replayed again and one step launch by launch
    # (the double buffers now on their other halves); a new capture for the
    # other halves, its replay and one more step.  Or the stream path.
    batch = P.Batch(sims, graph_steps=graph_steps, fused=fused)
    for n in (10, 11, 11):
        batch.step(n)
    batch.close()
    for sim, o, st in zip(sims, oracles, runs):
        o.step(32)
        err = vector_errors(sim, o)
        assert max(err.values()) < TOL[prec], (st.name, err)
        d = sim.diagnostics()
        assert d.n_particles[0] == o.num(0) and d.n_particles[1] == o.num(1)


# ------------------------------------------------------------- fused form

GAM = 13.0
_BETA = (1 - 1 / GAM ** 2) ** 0.5
_HZ = (1 / 32) * GAM * (1 + _BETA)
# runs of one batch that take different kernel instances: three 2D tile
# shapes, the quadratic shape, explicit ions, another boost, a 3D run
MIXED = [
    dict(grid=dict(dim=2, nx=32, nz=256, gamma_boost=GAM, seed=17), opts=dict(tile=(16, 1, 16))),
    dict(grid=dict(dim=2, nx=32, nz=200, gamma_boost=GAM, seed=18), opts=dict(tile=(32, 1, 8))),
    dict(grid=dict(dim=2, nx=32, nz=224, gamma_boost=GAM, seed=19), opts=dict(tile=(8, 1, 32), explicit_ions=True)),
    dict(grid=dict(dim=2, nx=32, nz=160, gamma_boost=GAM, seed=20, shape_order=2), opts=dict()),
    dict(grid=dict(dim=2, nx=32, nz=256, gamma_boost=5.0, seed=21), opts=dict()),
    dict(grid=dict(dim=3, nx=16, ny=16, nz=64, gamma_boost=GAM, seed=22), opts=dict()),
]


def _mixed_run(P, torch, O, spec, prec, with_oracle):
    g = dict(dx=1.0, dy=1.0, dz=1 / 32, filter_passes=2, **spec["grid"])
    gam = g["gamma_boost"]
    hz = (1 / 32) * gam * (1 + (1 - 1 / gam ** 2) ** 0.5)
    sim = P.Simulation(dim=g["dim"], nx=g["nx"], ny=g.get("ny", 1), nz=g["nz"], dx=g["dx"], dy=g["dy"], dz=g["dz"],
                       gamma_boost=gam, shape_order=g.get("shape_order", 1), filter_passes=g["filter_passes"],
                       precision=prec, seed=g["seed"], slots_per_cell=16.0, stream=torch.cuda.Stream(),
                       **spec["opts"])
    p = dict(ne=0.004, z_start=gam * 10 * hz, z_end=gam * 400 * hz, ramp=2.0,
             ppc=(2, 2, 2) if g["dim"] == 3 else (2, 1, 2), jitter=0.1, ions=1)
    laser = dict(a0=4.0, waist=8.0, fwhm=2.0, t_peak=0.5)
    sim.load_plasma(p["ne"], p["z_start"], p["z_end"], p["ramp"], p["ppc"], p["jitter"], (), p["ions"])
    sim.launch_laser(laser["a0"], laser["waist"], laser["fwhm"], 0.0, laser["t_peak"], 1)
    o = None
    if with_oracle:
        from pairs import oracle_grid
        o = O.Oracle(oracle_grid(O, g))
        o.load_plasma(O.PlasmaParams(ne=p["ne"], z_start=p["z_start"], z_end=p["z_end"], ramp=p["ramp"],
                                     ppc=p["ppc"], jitter=p["jitter"], ions=p["ions"]))
        o.set_laser(O.LaserParams(a0=laser["a0"], waist=laser["waist"], fwhm=laser["fwhm"], t_peak=laser["t_peak"],
                                  pol=1))
    return sim, o


def _rel_vectors(a, b):
    import numpy as np
    fa, fb = a.fields(), b.fields()
    out = {}
    for name, comps in (("E", ("Ex", "Ey", "Ez")), ("B", ("Bx", "By", "Bz")), ("J", ("Jx", "Jy", "Jz"))):
        num = sum(float(((fa[c].double() - fb[c].double()) ** 2).sum()) for c in comps)
        den = sum(float((fb[c].double() ** 2).sum()) for c in comps)
        out[name] = (num / den) ** 0.5 if den > 0 else num ** 0.5
    return out


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_fused_batch_mixed_kernels(O, prec):
    """One batch whose runs take six different particle-kernel instances (2D
    tile shapes 16 x 16, 32 x 8, 8 x 32, the quadratic shape, explicit ions,
    a 3D run) and two boosts: the fused graph (one launch per phase and
    kernel instance over all runs; the push a persistent grid over (run,
    tile) items) against the per-context graph from the same start, and both
    against each run's oracle.  The two GPU forms differ only by the order of
    the floating-point atomics that add tiles into J (tolerances 1e-12 FP64,
    2e-6 FP32); every run meets the full-step oracle tolerances."""
    import torch

    import paper_1011_0917_gb300 as P
    STEPS, K = 20, 10
    fused = [_mixed_run(P, torch, O, spec, prec, True) for spec in MIXED]
    plain = [_mixed_run(P, torch, O, spec, prec, False)[0] for spec in MIXED]
    bf = P.Batch([s for s, _ in fused], graph_steps=K, fused=1)
    bp = P.Batch(plain, graph_steps=K, fused=False)
    bf.step(STEPS)
    bp.step(STEPS)
    info_f, info_p = bf.graph_info(), bp.graph_info()
    bf.close()
    bp.close()
    assert info_f["chains"] == 1 and not info_p["fused"] and info_f["steps"] == K
    # one launch per phase and instance, a counter reset per particle launch
    assert 0 < info_f["launches_per_replay"] < info_p["launches_per_replay"], (info_f, info_p)
    assert info_f["launches_per_replay"] <= K * (1 + 2 * 7 + 1 + 1 + 2 * 2 + 2 + 2 + 1), info_f
    tight = 1e-12 if prec == FP64 else 2e-6
    for (sim, o), other, spec in zip(fused, plain, MIXED):
        d = _rel_vectors(sim, other)
        assert max(d.values()) < tight, (spec, d)
        o.step(STEPS)
        err = vector_errors(sim, o)
        assert max(err.values()) < TOL[prec], (spec, err)
        dg = sim.diagnostics()
        assert dg.n_particles[0] == o.num(0) and dg.n_particles[1] == o.num(1), spec
        assert other.diagnostics().n_particles[0] == dg.n_particles[0]
