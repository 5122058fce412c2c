"""Full-run agreement with the FP64 oracle: the c0 stage (lab frame, 64 x 512,
a0 = 1 laser into n = 0.01 plasma), all 512 steps.

Trajectories are chaotic over such a horizon, so the run is compared through
its physical outcomes, each within 1%: the peak on-axis wake field E_z over
the run (sampled every 16 steps) and the energy the laser has given the
plasma electrons by the end (their kinetic energy, sum w (gamma - 1); with the
same laser energy and propagation distance on both sides this fixes the
depletion length, which is inversely proportional to it)."""
import numpy as np
import pytest

from pairs import make_pair
from paper_1011_0917_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1
SAMPLE = 16


def _peak_and_energy_gpu(sim, nsteps, nx):
    peak = 0.0
    for _ in range(nsteps // SAMPLE):
        sim.step(SAMPLE)
        ez = sim.fields(1 << 2)["Ez"][:, 0, nx // 2].double().cpu().numpy()
        peak = max(peak, float(np.abs(ez).max()))
    st, _ = sim.particles(0)
    u2 = st[3] ** 2 + st[4] ** 2 + st[5] ** 2
    ke = float(np.sum(st[6] * u2 / (np.sqrt(1 + u2) + 1)))
    return peak, ke


@pytest.fixture(scope="module")
def oracle_run():
    import oracle.oracle as O
    O.build_oracle()
    st = W.stage("c0")
    g = st.grid
    o = O.Oracle(O.GridParams(dim=2, nx=g["nx"], nz=g["nz"], dx=g["dx"], dz=g["dz"], npass=g["filter_passes"],
                              seed=g["seed"]))
    o.load_plasma(O.PlasmaParams(**{k: st.plasma[k] for k in ("ne", "z_start", "z_end", "ramp", "ppc", "jitter",
                                                                 "ions")}))
    l = st.laser
    o.set_laser(O.LaserParams(a0=l["a0"], waist=l["waist"], fwhm=l["fwhm"], pol=l["pol"]))
    peak = 0.0
    for _ in range(st.steps // SAMPLE):
        o.step(SAMPLE)
        peak = max(peak, float(np.abs(o.field("Ez")[:, 0, g["nx"] // 2]).max()))
    p = o.particles(0)
    u2 = p["ux"] ** 2 + p["uy"] ** 2 + p["uz"] ** 2
    ke = float(np.sum(p["w"] * u2 / (np.sqrt(1 + u2) + 1)))
    return O, st, peak, ke


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_c0_full_run_peak_wake_and_depletion(oracle_run, prec):
    O, st, peak_o, ke_o = oracle_run
    g = st.grid
    sim, _ = make_pair(O, g, prec)
    p = st.plasma
    sim.load_plasma(p["ne"], p["z_start"], p["z_end"], p["ramp"], p["ppc"], p["jitter"], (), p["ions"])
    l = st.laser
    sim.launch_laser(l["a0"], l["waist"], l["fwhm"], l["z_antenna"], -1.0, l["pol"])
    peak, ke = _peak_and_energy_gpu(sim, st.steps, g["nx"])
    assert peak_o > 1e-2 and ke_o > 0
    assert abs(peak - peak_o) <= 1e-2 * peak_o, (peak, peak_o)
    assert abs(ke - ke_o) <= 1e-2 * ke_o, (ke, ke_o)


# ------------------------------------------------------ boosted-frame stages

def _golden(name):
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_runs.json")
    with open(path) as f:
        return json.load(f)[name]


def _run_stage(name, sample, slots=8.0):
    """The stage in FP32 on the GPU: the peak on-axis |E_z| every `sample`
    steps, the electrons and ions at the end."""
    import torch

    import paper_1011_0917_gb300 as P
    st = W.stage(name)
    g = st.grid
    sim = P.Simulation(dim=g["dim"], nx=g["nx"], ny=g["ny"], nz=g["nz"], dx=g["dx"], dy=g["dy"], dz=g["dz"],
                       cfl=g["cfl"], gamma_boost=g["gamma_boost"], shape_order=g["shape_order"],
                       filter_passes=g["filter_passes"], bc_z=g["bc_z"], precision=FP32, seed=g["seed"],
                       slots_per_cell=slots)
    p = st.plasma
    sim.load_plasma(p["ne"], p["z_start"], p["z_end"], p["ramp"], p["ppc"], p["jitter"], (), p["ions"])
    l = st.laser
    sim.launch_laser(l["a0"], l["waist"], l["fwhm"], l["z_antenna"], -1.0, l["pol"])
    line = torch.empty(g["nz"] + 1, dtype=torch.float32)
    steps, hist = [], []
    for s in range(st.steps // sample):
        sim.step(sample)
        P.pic_get_axis(sim.ctx, 2, line.data_ptr(), line.numel() * 4, False)
        steps.append((s + 1) * sample)
        hist.append(float(line.abs().max()))
    e, _ = sim.particles(0)
    i, _ = sim.particles(1)
    sim.close()
    return st, steps, hist, e, i


def test_c1_full_run_matches_oracle():
    """The gamma = 13 stage (c1: 256 x 8192, 1800 steps, until the pulse peak
    has crossed the 2000 lambda0 plasma), FP32, against the outcomes of the
    FP64 oracle's own whole run (tests/golden/full_runs.json, written by
    tests/golden/make_full_runs.py from the oracle alone): the peak on-axis
    wake field over the run and the energy the plasma electrons took from the
    laser, each within 1%."""
    import fullrun
    ref = _golden("c1")
    st, steps, hist, e, i = _run_stage("c1", ref["sample"])
    assert ref["steps"] == st.steps
    peak = max(hist)
    U = float(i[5, 0])  # the drift momentum as this side holds it
    energy = fullrun.plasma_energy(e[6], e[3], e[4], e[5], U)
    assert ref["peak_ez"] > 0 and ref["plasma_energy"] > 0
    assert abs(peak - ref["peak_ez"]) <= 1e-2 * ref["peak_ez"], (peak, ref)
    assert abs(energy - ref["plasma_energy"]) <= 1e-2 * ref["plasma_energy"], (energy, ref)


def test_c3_small_instability_growth_matches_oracle():
    """The gamma = 130 stage on its 4x coarser grid (c3_small: 128 x 4096,
    quadratic shape, 4 filter passes, 6500 steps), FP32.  In this frame the
    streaming plasma is numerically unstable with 4 binomial passes (the
    instability the paper's mitigation section treats): the on-axis E_z is
    exactly zero until it grows from round-off, exponentially, long before
    the pulse peak (emitted after ~5000 steps by the antenna) meets the
    plasma.  Outcomes of the wake cannot be compared then; what both sides
    must share is the instability's growth rate once its fastest mode
    dominates (|E_z| from 1e-7 to 1e-5: two decades below saturation, above
    either side's round-off), a property of the discrete scheme rather than
    of the round-off that seeds it (FP32 seeds it later and with another
    spectrum, so its onset transient differs): within 15% of the rate of the
    FP64 oracle's own run (tests/golden/full_runs.json)."""
    import math

    import fullrun
    ref = _golden("c3_small")
    st, steps, hist, _, _ = _run_stage("c3_small", ref["sample"], slots=24.0)
    assert ref["steps"] == st.steps
    rate, used = fullrun.growth_rate(steps, hist)
    assert ref["ez_growth_samples"] >= 6 and used >= 6, (used, ref["ez_growth_samples"])
    assert ref["ez_growth_rate"] > 0.005
    assert abs(rate - ref["ez_growth_rate"]) <= 0.15 * ref["ez_growth_rate"], (rate, ref["ez_growth_rate"])
    # it is an instability: growth by orders of magnitude, not a wake
    assert max(hist) > 1e3 * min(v for v in hist if v > 0) and math.isfinite(max(hist))
