"""Parity of the lab-frame (back-transformed) snapshots with the FP64 oracle.

Both sides run the same boosted stage and take the same snapshots; the set of
filled lab points must be identical (the event times are FP64 on both sides)
and the lab fields agree within the full-step tolerances (relative L2 over the
filled points of all snapshots: 1e-4 FP32, 1e-10 FP64).
"""
import math

import numpy as np
import pytest

from pairs import make_pair

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1
TOL = {FP32: 1e-4, FP64: 1e-10}
NAMES = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")


@pytest.fixture(scope="module")
def O():
    import oracle.oracle as O
    O.build_oracle()
    return O


def _run(O, g, p, laser, btd, nsteps, prec):
    sim, o = make_pair(O, g, prec)
    if p is not None:
        sim.load_plasma(p["ne"], p["z_start"], p["z_end"], p["ramp"], p["ppc"], p["jitter"], (), p["ions"])
        o.load_plasma(O.PlasmaParams(ne=p["ne"], z_start=p["z_start"], z_end=p["z_end"], ramp=p["ramp"],
                                     ppc=p["ppc"], jitter=p["jitter"], ions=p["ions"]))
    sim.launch_laser(laser["a0"], laser["waist"], laser["fwhm"], 0.0, laser.get("t_peak", -1.0), laser.get("pol", 1))
    o.set_laser(O.LaserParams(a0=laser["a0"], waist=laser["waist"], fwhm=laser["fwhm"], z_antenna=0.0,
                              t_peak=laser.get("t_peak", -1.0), pol=laser.get("pol", 1)))
    sim.btd_setup(btd["nsnap"], btd["t0"], btd["dt"], btd["z0"], btd["dz"], btd["nz"], btd["plane"])
    o.btd_setup(O.BtdParams(**btd))
    sim.step(nsteps)
    o.step(nsteps)
    return sim, o


def _compare(sim, o, nsnap, prec):
    num = den = 0.0
    nfilled = 0
    for j in range(nsnap):
        fg, mg = sim.btd_snapshot(j)
        fo, mo = o.btd_snapshot(j)
        assert np.array_equal(mg, mo), (j, int(mg.sum()), int(mo.sum()))
        nfilled += int(mo.sum())
        for c in NAMES:
            a, b = fg[c][mo], fo[c][mo]
            num += float(np.sum((a - b) ** 2))
            den += float(np.sum(b ** 2))
            assert not np.any(fg[c][~mo]), "unfilled points stay zero"
    assert nfilled > 0 and den > 0
    return math.sqrt(num / den), nfilled


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_btd_plane_boosted_2d_with_plasma(O, prec):
    # gamma = 2, a plasma streaming in from 10 cells ahead of the antenna, the
    # laser meeting it; six lab snapshots of the (x, z) plane
    g = dict(dim=2, nx=24, nz=96, dx=1.0, dz=1 / 32, gamma_boost=2.0, filter_passes=1, seed=41)
    beta = math.sqrt(1 - 1 / 4.0)
    hz = (1 / 32) * 2 * (1 + beta)
    Lz = 96 * hz
    p = dict(ne=0.01, z_start=2 * 10 * hz, z_end=2 * 400 * hz, ramp=1.0, ppc=(2, 1, 2), jitter=0.1, ions=1)
    laser = dict(a0=2.0, waist=6.0, fwhm=2.0, t_peak=0.5)
    T0 = 2 * beta * Lz
    btd = dict(nsnap=6, t0=T0, dt=1.5, z0=beta * T0 - 1.0, dz=1 / 32, nz=400, plane=1)
    # steps: until the last snapshot's latest event
    t_end = 2 * (T0 + 5 * 1.5 - beta * btd["z0"]) + 1.0
    sim, o = _run(O, g, p, laser, btd, 0, prec)
    n = int(t_end / o.dt) + 1
    sim.step(n)
    o.step(n)
    err, nfilled = _compare(sim, o, btd["nsnap"], prec)
    assert nfilled > 800
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_btd_axis_boosted_3d(O, prec):
    g = dict(dim=3, nx=12, ny=10, nz=48, dx=1.0, dy=1.0, dz=1 / 32, gamma_boost=3.0, filter_passes=1, seed=43)
    beta = math.sqrt(1 - 1 / 9.0)
    hz = (1 / 32) * 3 * (1 + beta)
    Lz = 48 * hz
    laser = dict(a0=1.0, waist=4.0, fwhm=2.0, t_peak=0.5)
    T0 = 3 * beta * Lz
    btd = dict(nsnap=4, t0=T0, dt=2.0, z0=beta * T0 - 1.0, dz=1 / 64, nz=900, plane=0)
    t_end = 3 * (T0 + 3 * 2.0 - beta * btd["z0"]) + 1.0
    sim, o = _run(O, g, None, laser, btd, 0, prec)
    n = int(t_end / o.dt) + 1
    sim.step(n)
    o.step(n)
    err, nfilled = _compare(sim, o, btd["nsnap"], prec)
    assert nfilled > 300
    assert err < TOL[prec], err
