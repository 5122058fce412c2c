"""Oracle pins of the moving window (in the paper's gamma = 1 and 5 runs the
box moves with the laser at its group velocity; section "Effect of the
hyperbolic rotation in Minkowski space").

What fixes them: a window moving at c over a pulse that travels at c sees the
same fields as a long fixed box at the same absolute positions (up to the
pulse's Gaussian tails reaching the window's ends), a plasma at rest seen
through the window is the lattice of a long box, point for point, and so is
a boosted plasma drifting through a moving window.
"""
import math

import numpy as np


def test_pulse_in_window_matches_long_box(oracle_mod):
    O = oracle_mod
    dz, nz, S = 1 / 16, 512, 16
    laser = O.LaserParams(a0=1.0, waist=1e9, fwhm=3.0, z_antenna=0.0, pol=1)
    win = O.Oracle(O.GridParams(dim=2, nx=4, nz=nz, dx=1.0, dz=dz, npass=0, bc_z=1))
    big = O.Oracle(O.GridParams(dim=2, nx=4, nz=3 * nz, dx=1.0, dz=dz, npass=0, bc_z=1))
    for o in (win, big):
        o.set_laser(laser)
    win.set_window(1.0, 20.0, S)
    n = int(40 / win.dt)
    win.step(n)
    big.step(n)
    zw = win.z_window
    kw = int(round(zw / dz))
    assert abs(kw * dz - zw) < 1e-12 and kw % S == 0 and kw > 0
    inner = slice(4, nz - 4)
    for c in ("Ey", "Bx"):
        a, b = win.field(c)[inner], big.field(c)[kw:kw + nz + 1][inner]
        assert np.abs(b).max() > 0.9
        # the pulse's tails at 3.5 tau reach the window's ends: exp(-12.5) ~ 4e-6
        assert np.abs(a - b).max() < 2e-5 * np.abs(b).max(), c


def test_static_plasma_through_window_is_the_lattice(oracle_mod):
    O = oracle_mod
    g = dict(dim=2, nx=8, dx=0.5, dz=1 / 16, npass=0, bc_z=1)
    p = O.PlasmaParams(ne=0.01, z_start=1.0, z_end=30.0, ramp=0.5, ppc=(2, 1, 3), jitter=0.2, ions=0)
    win = O.Oracle(O.GridParams(nz=128, **g))
    big = O.Oracle(O.GridParams(nz=640, **g))
    win.set_window(0.9, 1.5, 16)
    win.load_plasma(p)
    big.load_plasma(p)
    n = int(20.0 / win.dt)
    win.step(n)
    big.step(n)
    zw = win.z_window
    assert zw > 10.0
    a, b = win.particles(0), big.particles(0)
    inwin = (b["z"] >= zw) & (b["z"] < zw + win.Lz)
    ia, ib = np.argsort(a["id"]), np.argsort(b["id"][inwin])
    assert np.array_equal(a["id"][ia], b["id"][inwin][ib])
    assert np.allclose(a["z"][ia] + zw, b["z"][inwin][ib], atol=1e-12, rtol=0)
    assert np.array_equal(a["x"][ia], b["x"][inwin][ib])
    assert np.array_equal(a["w"][ia], b["w"][inwin][ib])


def test_boosted_plasma_through_window_matches_long_box(oracle_mod):
    # a boosted plasma (drifting at -beta, streaming in at the top) seen
    # through a window moving at +v: every particle the window holds is where
    # the same lattice particle is in a long fixed box, both the ones that
    # drifted in through the window's top and the ones the window moved over
    O = oracle_mod
    g = dict(dim=2, nx=4, dx=1.0, dz=1 / 16, gamma_boost=5.0, npass=0, bc_z=1)
    win = O.Oracle(O.GridParams(nz=96, **g))
    big = O.Oracle(O.GridParams(nz=480, **g))
    p = O.PlasmaParams(ne=0.01, z_start=0.0, z_end=5.0 * big.Lz * 2, ramp=0.0, ppc=(2, 1, 2), jitter=0.1, ions=1)
    win.set_window(0.6, 0.5, 8)
    win.load_plasma(p)
    big.load_plasma(p)
    mask = O.PH_PUSH | O.PH_IONS | O.PH_INJECT | O.PH_TIME   # field-free: every particle drifts at -beta
    for _ in range(int(60.0 / win.dt)):
        win.step_phases(mask)
        big.step_phases(mask)
    zw = win.z_window
    assert zw >= 5 * 8 * win.hz - 1e-9 and zw + win.Lz < big.Lz   # several moves, inside the long box
    for sp in (0, 1):
        a, b = win.particles(sp), big.particles(sp)
        pos = dict(zip(b["id"].tolist(), b["z"]))
        assert len(a["id"]) > 1000
        for pid, z in zip(a["id"].tolist(), a["z"]):
            assert abs(z + zw - pos[pid]) < 1e-9, (sp, pid, z + zw, pos[pid])
        # and nothing the long box holds inside the window is missing from it
        ids = set(a["id"].tolist())
        inner = (b["z"] > zw + 1e-9) & (b["z"] < zw + win.Lz - 1e-9)
        assert all(i in ids for i in b["id"][inner].tolist())


def test_antenna_stays_put_as_the_window_moves(oracle_mod):
    # the window starts moving (at c) while the antenna, 25 lambda0 into the
    # box, is still emitting: the antenna stays at its launch position, so the
    # forward pulse in the window's upper half is the long box's, node for
    # node; and the window has moved by whole steps of S cells, one each time
    # v (t - t0) reached the next multiple of S hz
    O = oracle_mod
    dz, nz, S = 1 / 16, 512, 16
    laser = O.LaserParams(a0=1.0, waist=1e9, fwhm=3.0, z_antenna=25.0, pol=1)
    win = O.Oracle(O.GridParams(dim=2, nx=4, nz=nz, dx=1.0, dz=dz, npass=0, bc_z=1))
    big = O.Oracle(O.GridParams(dim=2, nx=4, nz=3 * nz, dx=1.0, dz=dz, npass=0, bc_z=1))
    for o in (win, big):
        o.set_laser(laser)
    v, t0 = 1.0, 4.0
    win.set_window(v, t0, S)
    n = int(30 / win.dt)
    win.step(n)
    big.step(n)
    zw = win.z_window
    assert zw == S * dz * math.floor(v * (n * win.dt - t0) / (S * dz))
    kw = int(round(zw / dz))
    up = slice(nz // 2, nz - 4)                 # the forward pulse; the backward one left through the bottom
    for c in ("Ey", "Bx"):
        a, b = win.field(c)[up], big.field(c)[kw:kw + nz + 1][up]
        assert np.abs(b).max() > 0.9
        assert np.abs(a - b).max() < 1e-12 * np.abs(b).max(), c


def test_lab_plasma_with_immobile_ions_stays_neutral_through_the_window(oracle_mod):
    # the immobile ions of a lab plasma are its neutralising background: the
    # plasma a moving window brings into view brings its background along, so
    # the charge density stays zero as the window moves, on every node but
    # the bottom one (whose electrons just below the window have left it
    # while their background share on that node stays)
    O = oracle_mod
    o = O.Oracle(O.GridParams(dim=2, nx=8, nz=128, dx=0.5, dz=1 / 16, npass=0, bc_z=1))
    o.load_plasma(O.PlasmaParams(ne=0.01, z_start=1.0, z_end=30.0, ramp=0.5, ppc=(2, 1, 3), jitter=0.2, ions=1))
    o.set_window(0.9, 1.5, 16)
    assert np.abs(o.rho()).max() <= 1e-14 * 0.01
    o.step(int(20.0 / o.dt))
    assert o.z_window > 10.0
    assert np.abs(o.rho_background()).max() > 0.5 * 0.01
    assert np.abs(o.rho()[1:]).max() <= 1e-14 * 0.01
