"""Oracle pins of the lab-frame (back-transformed) snapshots of a boosted run.

What fixes them, independently of the oracle's own transformation code:
* fields static in a frame moving at v = beta z (the simulation frame) are, in
  the lab frame, the fields of uniformly moving sources: E_parallel unchanged,
  E_perp and B_perp scaled by gamma, and B = v x E for an electrostatic field,
  E = -v x B for a magnetostatic one (textbook special relativity); the
  invariants E^2 - B^2 and E.B are the simulation-frame ones;
* which lab points a run covers: a lab event (T, Z) is seen in the simulation
  frame at t' = gamma (T - beta Z), z' = gamma (Z - beta T), and a snapshot
  point is filled once the run has passed t' while z' lies between the planes
  of every component;
* the paper's comparison (section "Effect of the hyperbolic rotation in
  Minkowski space", Fig. 2): one laser pulse computed in the lab frame and in a
  boosted frame, the boosted data transformed to the lab, agree.
"""
import math

import numpy as np
import pytest


def _static_run(O, e, b, gam=3.0):
    g = O.GridParams(dim=2, nx=4, nz=96, dx=1.0, dz=1 / 16, gamma_boost=gam, npass=0, bc_z=1)
    o = O.Oracle(g)
    for c, v in zip(("Ex", "Ey", "Ez"), e):
        o.field(c)[...] = v
    for c, v in zip(("Bx", "By", "Bz"), b):
        o.field(c)[...] = v
    T0 = gam * o.beta * o.Lz
    bt = O.BtdParams(nsnap=3, t0=T0, dt=4.0, z0=o.beta * T0 - 2.0, dz=1 / 16, nz=400, plane=1)
    o.btd_setup(bt)
    t_end = gam * (T0 + 2 * bt.dt) + 5.0
    nsteps = int(t_end / o.dt) + 1
    o.step(nsteps)
    return o, bt, nsteps


@pytest.mark.parametrize("e,b", [((0.3, -0.7, 0.25), (0.0, 0.0, 0.0)), ((0.0, 0.0, 0.0), (0.4, 0.9, -0.2)),
                                 ((0.3, -0.7, 0.25), (-0.5, 0.2, 0.6))])
def test_static_fields_seen_from_the_lab(oracle_mod, e, b):
    O = oracle_mod
    o, bt, _ = _static_run(O, e, b)
    gam, beta = 3.0, o.beta
    v = np.array([0.0, 0.0, beta])
    nfilled = 0
    for j in range(bt.nsnap):
        f, m = o.btd_snapshot(j)
        nfilled += int(m.sum())
        E = np.stack([f["Ex"][m], f["Ey"][m], f["Ez"][m]], axis=-1)
        B = np.stack([f["Bx"][m], f["By"][m], f["Bz"][m]], axis=-1)
        if not m.any():
            continue
        # parallel components unchanged, perpendicular ones of the pure cases scaled by gamma
        assert np.allclose(E[..., 2], e[2], atol=1e-13) and np.allclose(B[..., 2], b[2], atol=1e-13)
        if not any(b):
            assert np.allclose(E[..., :2], gam * np.array(e[:2]), atol=1e-12)
            assert np.allclose(B, np.cross(v, E), atol=1e-12)
        if not any(e):
            assert np.allclose(B[..., :2], gam * np.array(b[:2]), atol=1e-12)
            assert np.allclose(E, -np.cross(v, B), atol=1e-12)
        # invariants
        e2, b2 = float(np.dot(e, e)), float(np.dot(b, b))
        assert np.allclose((E * E).sum(-1) - (B * B).sum(-1), e2 - b2, atol=1e-12)
        assert np.allclose((E * B).sum(-1), float(np.dot(e, b)), atol=1e-12)
    assert nfilled > 100


def test_snapshot_coverage(oracle_mod):
    # the filled lab points are exactly those whose event the run has passed
    # and that lie between the planes of every component
    O = oracle_mod
    o, bt, nsteps = _static_run(O, (0.1, 0.2, 0.3), (0.0, 0.0, 0.0))
    gam, beta = 3.0, o.beta
    t_end = nsteps * o.dt
    for j in range(bt.nsnap):
        _, m = o.btd_snapshot(j)
        T = bt.t0 + j * bt.dt
        Z = bt.z0 + np.arange(bt.nz) * bt.dz
        tp = gam * (T - beta * Z)
        zp = gam * (Z - beta * T)
        expect = (tp >= 0) & (tp < t_end - 1e-9) & (zp >= 0.5 * o.hz) & (zp <= (o.grid.nz - 0.5) * o.hz)
        # points within rounding of a boundary may go either way
        edge = (np.abs(zp - 0.5 * o.hz) < 1e-9) | (np.abs(zp - (o.grid.nz - 0.5) * o.hz) < 1e-9) | \
               (np.abs(tp - t_end) < 1e-6)
        assert np.array_equal(m[~edge], expect[~edge]), j
        assert expect.sum() > 50


def test_lab_and_boosted_runs_of_one_pulse_agree(oracle_mod):
    # a plane laser pulse launched by an antenna two lab cells from z = 0, once
    # in the lab frame and once in a frame boosted to gamma = 1.5 whose data are
    # transformed to the lab: the lab-frame Ey(Z) at T = 60 lambda0/c agrees
    # within the two grids' discretisation (relative L2 1.6% measured)
    O = oracle_mod
    dzl = 1 / 32
    T = 60.0
    laser = O.LaserParams(a0=1.0, waist=1e9, fwhm=4.0, z_antenna=0.0, pol=1)
    lab = O.Oracle(O.GridParams(dim=2, nx=4, nz=int(32 * (T + 8)), dx=1.0, dz=dzl, npass=0, bc_z=1))
    lab.set_laser(laser)
    n0 = int(T / lab.dt)
    Tj = n0 * lab.dt
    gam = 1.5
    bst = O.Oracle(O.GridParams(dim=2, nx=4, nz=400, dx=1.0, dz=dzl, gamma_boost=gam, npass=0, bc_z=1))
    bst.set_laser(laser)
    bst.btd_setup(O.BtdParams(nsnap=1, t0=Tj, dt=1.0, z0=0.0, dz=dzl, nz=lab.grid.nz + 1, plane=0))
    t_end = gam * (Tj - bst.beta * (bst.beta * Tj)) + 2.0
    bst.step(int(t_end / bst.dt) + 2)
    f, m = bst.btd_snapshot(0)
    lab.step(n0)
    ey = lab.field("Ey")[:, 0, 2]
    k = np.where(m)[0]
    assert len(k) > 500
    a, b = f["Ey"][k, 0], ey[k]
    # the pulse peak (Z ~ T - 3 tau) lies inside the boosted box at T
    assert np.abs(b).max() > 0.99
    assert abs(np.abs(a).max() - np.abs(b).max()) < 0.02
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 0.03
    # and the pulse is not displaced: a one-cell shift is far worse
    worse = np.linalg.norm(a - ey[k + 1]) / np.linalg.norm(ey[k + 1])
    assert worse > 0.1
