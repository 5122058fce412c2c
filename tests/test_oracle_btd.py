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


def _wake_lab_vs_boost(O, gam, dzl=1 / 32, ne=0.01, zs=4.0, a0=1.0, fwhm=5.0, ahead=12.0):
    """A plane laser pulse (a0, intensity FWHM `fwhm`) driving a wake in a
    cold plasma at rest in the lab from z = zs (2 lambda0 ramp): the on-axis
    Ez(Z) of a lab-frame run once the pulse peak is `ahead` lambda0 into the
    plasma, and the same lab-frame line from a run boosted to `gam`, read off
    its back-transformed snapshot.  The boosted run's antenna moves in the lab
    (it is at rest in the boosted frame), so its plasma is placed `delta`
    further along (the pulse is emitted in vacuum, the plasma enters the box
    through z = Lz) and the lab events (Z, T) of the first run correspond to
    (Z + delta, T + delta) of the second: a plane pulse in vacuum and a
    plasma at rest are both unchanged by that shift."""
    tau = fwhm / math.sqrt(2 * math.log(2))
    lab = O.Oracle(O.GridParams(dim=2, nx=4, nz=int(round((zs + ahead + 8) / dzl)), dx=1.0, dz=dzl, npass=1,
                                bc_z=1, seed=5))
    lab.load_plasma(O.PlasmaParams(ne=ne, z_start=zs, z_end=zs + 400, ramp=2.0, ppc=(2, 1, 2), jitter=0.0, ions=1))
    lab.set_laser(O.LaserParams(a0=a0, waist=1e9, fwhm=fwhm, pol=1))
    lab.step(int(math.ceil((zs + ahead + 3 * tau) / lab.dt)))
    T_lab = lab.t
    ez_lab = lab.field("Ez")[:, 0, 2]
    z_ez = (np.arange(len(ez_lab)) + 0.5) * lab.hz      # Ez sits at k + 1/2
    beta = math.sqrt(1 - 1 / gam ** 2)
    # the lab events to compare must lie ahead of the boosted antenna
    # (z' > 0): (1 - beta) delta > beta T_lab - zs, with a margin
    delta = math.ceil((beta * T_lab - zs + 4) / (1 - beta))
    Ts, Z0, span = T_lab + delta, zs + delta - 2.0, ahead + 6.0
    nzl = int(round(span / dzl))
    hz = dzl * gam * (1 + beta)
    nz = int(math.ceil((gam * (Z0 + span - beta * Ts) + 20) / hz))
    bst = O.Oracle(O.GridParams(dim=2, nx=4, nz=nz, dx=1.0, dz=dzl, gamma_boost=gam, npass=1, bc_z=1, seed=5))
    assert (zs + delta) / gam > bst.Lz  # all of the plasma is injected
    bst.load_plasma(O.PlasmaParams(ne=ne, z_start=zs + delta, z_end=zs + delta + 400, ramp=2.0, ppc=(2, 1, 2),
                                   jitter=0.0, ions=1))
    bst.set_laser(O.LaserParams(a0=a0, waist=1e9, fwhm=fwhm, pol=1))
    bst.btd_setup(O.BtdParams(nsnap=1, t0=Ts, dt=1.0, z0=Z0, dz=dzl, nz=nzl, plane=0))
    bst.step(int(math.ceil((gam * (Ts - beta * Z0) + 2 * bst.dt) / bst.dt)))
    f, filled = bst.btd_snapshot(0)
    Z = Z0 + np.arange(nzl) * dzl - delta               # back in the first run's coordinates
    ez_b = f["Ez"][:, 0]
    ez_l = np.interp(Z, z_ez, ez_lab)
    wake = filled & (Z >= zs) & (Z <= zs + ahead)       # behind the pulse peak
    return Z, ez_l, ez_b, wake, filled


@pytest.mark.parametrize("gam", [2.0, 3.0, 5.0])
def test_boosted_wake_back_transformed_matches_lab_wake(oracle_mod, gam):
    # The paper's central claim (section "Effect of the hyperbolic rotation in
    # Minkowski space", Fig. 2): a stage computed in a boosted frame and
    # transformed back to the lab reproduces the lab-frame computation.  Here
    # with plasma: the peak wake field behind a plane a0 = 1 pulse in an
    # n = 0.01 n_c plasma, computed at gamma = 1 and at gamma = 2, 3, 5
    # (plasma contracted and drifting at -beta, injected through z = Lz,
    # drifting ions, Doppler-shifted antenna, lab snapshot), agrees within 5%
    # at the same lab position.  At 32 cells per wavelength the measured gap
    # is 2.2%, 2.6%, 4.0% (it is discretisation: 7%, 8%, 19% at 16 cells); a
    # wrong boosted density, drift or injection time moves or rescales the
    # wake far beyond this.
    O = oracle_mod
    Z, ez_l, ez_b, wake, filled = _wake_lab_vs_boost(O, gam)
    assert filled.mean() > 0.95
    assert wake.sum() > 300
    il = int(np.argmax(np.abs(ez_l * wake)))
    ib = int(np.argmax(np.abs(ez_b * wake)))
    assert abs(ez_l[il]) > 0.02                          # a nonlinear wake is there
    assert abs(abs(ez_b[ib]) - abs(ez_l[il])) / abs(ez_l[il]) < 0.05
    assert np.sign(ez_b[ib]) == np.sign(ez_l[il])
    assert abs(Z[ib] - Z[il]) <= 2 * (1 / 32)            # the same lab position (two lab cells)


def test_snapshots_of_a_windowed_run_match_the_long_box(oracle_mod):
    # A boosted pulse followed by a window moving at c once the antenna has
    # stopped emitting: the lab snapshot points the window fills carry the
    # same fields as those of a long fixed box (the window holds the long
    # box's fields at the same absolute positions), so both snapshots agree
    # wherever both are filled.
    O = oracle_mod
    gam, dzl = 1.5, 1 / 32
    laser = O.LaserParams(a0=1.0, waist=1e9, fwhm=1.0, z_antenna=0.0, pol=1)
    win = O.Oracle(O.GridParams(dim=2, nx=4, nz=400, dx=1.0, dz=dzl, gamma_boost=gam, npass=0, bc_z=1))
    big = O.Oracle(O.GridParams(dim=2, nx=4, nz=1200, dx=1.0, dz=dzl, gamma_boost=gam, npass=0, bc_z=1))
    T, Z0, nzl = 97.0, 80.0, int(30 / dzl)
    for o in (win, big):
        o.set_laser(laser)
        o.btd_setup(O.BtdParams(nsnap=1, t0=T, dt=1.0, z0=Z0, dz=dzl, nz=nzl, plane=0))
    win.set_window(1.0, 16.0, 16)
    beta = win.beta
    t_last = gam * (T - beta * Z0) + 2.0                 # the latest event of the snapshot
    n = int(t_last / win.dt) + 2
    win.step(n)
    big.step(n)
    assert win.z_window > 0.5 * win.Lz
    fa, ma = win.btd_snapshot(0)
    fb, mb = big.btd_snapshot(0)
    both = ma & mb
    assert both.sum() > 300
    for c in ("Ey", "Bx"):
        a, b = fa[c][both, 0], fb[c][both, 0]
        assert np.abs(b).max() > 0.5
        assert np.abs(a - b).max() < 1e-4 * np.abs(b).max(), c


def test_on_axis_snapshot_is_the_middle_column(oracle_mod):
    # an electrostatic field varying across x, Ex'(x) = cos(2 pi x / Lx) at
    # Ex's own staggered x (static: its curl is zero), seen from the lab: the
    # on-axis snapshot is the column nx/2 of the full-plane one, and both are
    # gamma Ex' with By = gamma beta Ex' there
    O = oracle_mod
    gam, nx = 3.0, 8
    g = O.GridParams(dim=2, nx=nx, nz=96, dx=1.0, dz=1 / 16, gamma_boost=gam, npass=0, bc_z=1)
    runs = []
    for plane in (0, 1):
        o = O.Oracle(g)
        x = (np.arange(nx) + 0.5) * o.hx
        o.field("Ex")[...] = np.cos(2 * math.pi * x / o.Lx)
        T0 = gam * o.beta * o.Lz
        o.btd_setup(O.BtdParams(nsnap=1, t0=T0, dt=1.0, z0=o.beta * T0 - 2.0, dz=1 / 16, nz=200, plane=plane))
        o.step(int((gam * T0 + 5.0) / o.dt) + 1)
        runs.append(o.btd_snapshot(0))
    (f0, m0), (f1, m1) = runs
    assert m0.sum() > 50 and np.array_equal(m0, m1)
    ex_mid = math.cos(2 * math.pi * (nx // 2 + 0.5) / nx)
    assert np.allclose(f0["Ex"][m0, 0], f1["Ex"][m1, nx // 2], atol=1e-13, rtol=0)
    assert np.allclose(f0["Ex"][m0, 0], gam * ex_mid, atol=1e-12, rtol=0)
    assert np.allclose(f0["By"][m0, 0], gam * o.beta * ex_mid, atol=1e-12, rtol=0)
