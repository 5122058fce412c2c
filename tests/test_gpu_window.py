"""Parity of the moving window with the FP64 oracle: the same stage, the same
window, the same moves at the same steps; fields (full-step tolerances: 1e-4
FP32, 1e-10 FP64 relative L2), particles by id and the window displacement."""
import math

import numpy as np
import pytest

from pairs import gpu_particles, make_pair, oracle_particles, vector_errors
from paper_1011_0917_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1
TOL = {FP32: 1e-4, FP64: 1e-10}


@pytest.fixture(scope="module")
def O():
    import oracle.oracle as O
    O.build_oracle()
    return O


def _both(O, g, p, laser, window, nsteps, prec, rel=0):
    sim, o = make_pair(O, g, prec, z_relative=rel)
    sim.set_moving_window(*window)
    o.set_window(*window)
    if p is not None:
        sim.load_plasma(p["ne"], p["z_start"], p["z_end"], p["ramp"], p["ppc"], p["jitter"], (), p["ions"])
        o.load_plasma(O.PlasmaParams(ne=p["ne"], z_start=p["z_start"], z_end=p["z_end"], ramp=p["ramp"],
                                     ppc=p["ppc"], jitter=p["jitter"], ions=p["ions"]))
    sim.launch_laser(laser["a0"], laser["waist"], laser["fwhm"], 0.0, laser.get("t_peak", -1.0), 1)
    o.set_laser(O.LaserParams(a0=laser["a0"], waist=laser["waist"], fwhm=laser["fwhm"], z_antenna=0.0,
                              t_peak=laser.get("t_peak", -1.0), pol=1))
    sim.step(nsteps)
    o.step(nsteps)
    return sim, o


def _check(sim, o, prec):
    d = sim.diagnostics()
    assert d.z_window == o.z_window
    err = vector_errors(sim, o)
    assert max(err.values()) < TOL[prec], err
    for sp in (0, 1) if o.num(1) > 0 else (0,):
        a, ia = gpu_particles(sim, sp)
        b, ib = oracle_particles(o, sp)
        assert np.array_equal(ia, ib), (sp, len(ia), len(ib))


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_window_lab_frame_2d(O, prec):
    # the c0 stage (lab frame): window at 0.99 c from t = 6 (the pulse is in)
    # in moves of one tile layer (16 cells); plasma ahead of the box enters
    # through the moves
    st = W.stage("c0")
    g = dict(st.grid, nz=256)
    p = dict(st.plasma, z_end=60.0)
    sim, o = _both(O, g, p, st.laser, (0.99, 6.0, 16), 260, prec)
    assert o.z_window >= 8.0 and o.num(0) > 0
    _check(sim, o, prec)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("rel", [0, 1])
def test_window_boosted_2d(O, prec, rel):
    # gamma = 5 with the window at the laser's group velocity seen in that
    # frame (v_g' ~ 0.74 for gamma_g ~ 13); plasma drifting in at -beta
    g = dict(dim=2, nx=24, nz=128, dx=1.0, dz=1 / 32, gamma_boost=5.0, filter_passes=1, seed=47)
    beta = math.sqrt(1 - 1 / 25.0)
    hz = (1 / 32) * 5 * (1 + beta)
    p = dict(ne=0.004, z_start=5 * 8 * hz, z_end=5 * 900 * hz, ramp=1.0, ppc=(2, 1, 2), jitter=0.1, ions=1)
    laser = dict(a0=2.0, waist=6.0, fwhm=2.0, t_peak=0.5)
    sim, o = _both(O, g, p, laser, (0.74, 3.0, 16), 120, prec, rel)
    assert o.z_window > 0
    _check(sim, o, prec)


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_window_3d(O, prec):
    g = dict(dim=3, nx=12, ny=10, nz=40, dx=1.0, dy=1.0, dz=1 / 16, filter_passes=1, seed=49)
    p = dict(ne=0.01, z_start=0.5, z_end=12.0, ramp=0.5, ppc=(2, 2, 2), jitter=0.1, ions=1)
    laser = dict(a0=1.0, waist=3.0, fwhm=1.5, t_peak=0.5)
    sim, o = _both(O, g, p, laser, (1.0, 1.0, 8), 60, prec)
    assert o.z_window > 0
    _check(sim, o, prec)
