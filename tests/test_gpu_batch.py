"""The batched scan: independent boosted runs (different boosts, lengths,
density profiles and laser amplitudes, the c4 recipe on smaller grids) stepped
together through pic_batch_step, each on its own stream, as replays of a
captured CUDA graph or launch by launch; every run matches its own FP64
oracle run (full-step tolerances: 1e-4 FP32, 1e-10 FP64)."""
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


@pytest.mark.parametrize("graph_steps", [10, 0])
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_batch_matches_each_run(O, prec, graph_steps):
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
    batch = P.Batch(sims, graph_steps=graph_steps)
    for n in (10, 11, 11):
        batch.step(n)
    batch.close()
    for sim, o, st in zip(sims, oracles, runs):
        o.step(32)
        err = vector_errors(sim, o)
        assert max(err.values()) < TOL[prec], (st.name, err)
        d = sim.diagnostics()
        assert d.n_particles[0] == o.num(0) and d.n_particles[1] == o.num(1)
