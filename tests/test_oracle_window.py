"""Oracle pins of the moving window (in the paper's gamma = 1 and 5 runs the
box moves with the laser at its group velocity; section "Effect of the
hyperbolic rotation in Minkowski space").

What fixes them: a window moving at c over a pulse that travels at c sees the
same fields as a long fixed box at the same absolute positions (up to the
pulse's Gaussian tails reaching the window's ends), and a plasma at rest seen
through the window is the lattice of a long box, point for point.
"""
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
