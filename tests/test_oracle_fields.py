"""Oracle pins for the field side: Yee dispersion, Mur absorption, binomial
filter transfer function and the antenna's radiated amplitude.

Closed forms used:
* Yee leapfrog: a plane wave exp(i(k.r - w t)) with every component sampled at
  its own staggered point is an exact discrete solution iff
  (2/dt) sin(w dt/2) = |K|,  K_d = (2/h_d) sin(k_d h_d / 2)     (Yee 1966);
  B at integer times is the mean of the two half steps, i.e. B_hat cos(w dt/2).
* binomial pass (1/4, 1/2, 1/4): multiplies a mode by cos^2(k h / 2).
* discrete current sheet in 1D Yee: a harmonic source J at one node radiates
  E = -pi h J / cos(kappa/2) each way (kappa = k h, vacuum discrete k), in
  phase with J when J is centred at the half step: the field at node k is
  the discrete plane wave with phase -kappa |k - k_a|.
"""
import math

import numpy as np
import pytest


def set_mode(o, g, kvec, ehat, n=0):
    """Fill E, B with the discrete Yee eigenmode at integer time n."""
    h = np.array([o.hx, o.hy, o.hz])
    K = 2.0 / h * np.sin(np.array(kvec) * h / 2.0)
    if g.dim == 2:
        K[1] = 0.0
    Om = math.sqrt(K @ K)
    w = 2.0 / o.dt * math.asin(Om * o.dt / 2.0)
    bhat = np.cross(K, ehat) / Om
    stag = {0: (0.5, 0, 0), 1: (0, 0.5, 0), 2: (0, 0, 0.5), 3: (0, 0.5, 0.5), 4: (0.5, 0, 0.5), 5: (0.5, 0.5, 0)}
    k, j, i = np.meshgrid(np.arange(g.nz + 1), np.arange(o.ny), np.arange(g.nx), indexing="ij")
    out = {}
    for c in range(6):
        sx, sy, sz = stag[c]
        ph = kvec[0] * (i + sx) * o.hx + kvec[2] * (k + sz) * o.hz
        if g.dim == 3:
            ph = ph + kvec[1] * (j + sy) * o.hy
        amp = ehat[c] if c < 3 else bhat[c - 3] * math.cos(w * o.dt / 2)
        out[c] = amp * np.cos(ph - w * n * o.dt)
    return out, w


@pytest.mark.parametrize("dim,pol", [(2, "TE"), (2, "TM"), (3, "A"), (3, "B")])
def test_yee_discrete_eigenmode(oracle_mod, dim, pol):
    G = oracle_mod.GridParams
    if dim == 2:
        g = G(dim=2, nx=16, nz=24, dx=0.5, dz=0.25, cfl=0.95, bc_z=0, npass=0)
    else:
        g = G(dim=3, nx=10, ny=8, nz=12, dx=0.5, dy=0.6, dz=0.4, cfl=0.95, bc_z=0, npass=0)
    o = oracle_mod.Oracle(g)
    kvec = np.array([2 * math.pi * 2 / o.Lx, 2 * math.pi * (1 if dim == 3 else 0) / o.Ly, 2 * math.pi * 3 / o.Lz])
    h = np.array([o.hx, o.hy, o.hz])
    K = 2.0 / h * np.sin(kvec * h / 2.0)
    if dim == 2:
        K[1] = 0.0
    if pol == "TE":
        e = np.array([0.0, 1.0, 0.0])
    elif pol == "TM":
        e = np.array([K[2], 0.0, -K[0]])
    else:
        a = np.array([1.0, 0.3, -0.2]) if pol == "A" else np.array([-0.4, 1.0, 0.5])
        e = np.cross(K, a)
    e = e / np.linalg.norm(e)
    f0, w = set_mode(o, g, kvec, e, 0)
    for c in range(6):
        o.field(c)[...] = f0[c]
    nsteps = 600
    for _ in range(nsteps):
        o.step_phases(oracle_mod.PH_YEE | oracle_mod.PH_TIME)
    fN, _ = set_mode(o, g, kvec, e, nsteps)
    kmax = g.nz  # periodic z: plane nz is unused
    err = max(np.abs(o.field(c)[:kmax] - fN[c][:kmax]).max() for c in range(6))
    assert err < 1e-10, err
    # the continuum dispersion w = |k| would be visibly wrong after 600 steps
    wc = float(np.linalg.norm(kvec if dim == 3 else kvec * [1, 0, 1]))
    phase_gap = abs(wc - w) * nsteps * o.dt
    assert phase_gap > 1e-2


def test_filter_transfer_function(oracle_mod):
    G = oracle_mod.GridParams
    for npass in (1, 2, 4):
        g = G(dim=3, nx=16, ny=12, nz=20, dx=0.5, dy=0.5, dz=0.5, bc_z=0, npass=npass)
        o = oracle_mod.Oracle(g)
        k, j, i = np.meshgrid(np.arange(g.nz + 1), np.arange(g.ny), np.arange(g.nx), indexing="ij")
        mx, my, mz = 3, 2, 5
        ax, ay, az = 2 * math.pi * mx / g.nx, 2 * math.pi * my / g.ny, 2 * math.pi * mz / g.nz
        stag = {6: (0.5, 0, 0), 7: (0, 0.5, 0), 8: (0, 0, 0.5)}
        for c, (sx, sy, sz) in stag.items():
            o.field(c)[...] = np.cos(ax * (i + sx) + ay * (j + sy) + az * (k + sz) + 0.3 * c)
            o.field(c)[g.nz] = 0.0
        ref = {c: o.field(c).copy() for c in stag}
        o.filter()
        gain = (math.cos(ax / 2) ** 2 * math.cos(ay / 2) ** 2 * math.cos(az / 2) ** 2) ** npass
        for c in stag:
            np.testing.assert_allclose(o.field(c)[: g.nz], gain * ref[c][: g.nz], atol=1e-14)


def test_filter_absorbing_z_boundary_and_dc(oracle_mod):
    # zero values outside the valid z range; a constant is preserved inside
    G = oracle_mod.GridParams
    g = G(dim=2, nx=8, nz=10, dx=0.5, dz=0.5, bc_z=1, npass=1)
    o = oracle_mod.Oracle(g)
    o.field("Jy")[0, 0, 3] = 1.0      # node k = 0 (valid range 0..nz)
    o.field("Jz")[g.nz - 1, 0, 5] = 1.0  # half node nz-1/2 (valid range 0..nz-1)
    o.field("Jx")[...] = 2.0
    o.filter()
    jy = o.field("Jy")[:, 0, :]
    assert abs(jy[0, 3] - 0.25) < 1e-15 and abs(jy[1, 3] - 0.125) < 1e-15
    assert abs(jy[0, 2] - 0.125) < 1e-15 and abs(jy.sum() - 0.75) < 1e-15
    jz = o.field("Jz")[:, 0, :]
    assert abs(jz[g.nz - 1, 5] - 0.25) < 1e-15 and jz[g.nz, 5] == 0.0
    jx = o.field("Jx")[:, 0, :]
    assert np.allclose(jx[1:g.nz], 2.0) and abs(jx[0, 0] - 1.5) < 1e-15


def _plane_wave_box(oracle_mod, nz, dz, fwhm=3.0, a0=1.0, z_ant=0.0, pol=1, dx=0.5):
    G = oracle_mod.GridParams
    g = G(dim=2, nx=4, nz=nz, dx=dx, dz=dz, cfl=0.99, bc_z=1, npass=0)
    o = oracle_mod.Oracle(g)
    o.set_laser(oracle_mod.LaserParams(a0=a0, waist=1e9, fwhm=fwhm, z_antenna=z_ant, pol=pol))
    return g, o


def test_antenna_amplitude_and_carrier(oracle_mod):
    from scipy.signal import hilbert
    fwhm = 10.0
    g, o = _plane_wave_box(oracle_mod, nz=640, dz=1.0 / 32, fwhm=fwhm)
    probe = 400
    tau = fwhm / math.sqrt(2 * math.log(2))
    nsteps = int((6 * tau + probe * o.hz + 2.0) / o.dt)
    hist = np.zeros(nsteps)
    for n in range(nsteps):
        o.step(1)
        hist[n] = o.field("Ey")[probe, 0, 0]
    # discrete vacuum wavenumber of the carrier and the sheet amplitude factor
    r = o.dt / o.hz
    kappa = 2 * math.asin(math.sin(2 * math.pi * o.dt / 2) / r)
    expect = 1.0 / math.cos(kappa / 2)
    env = np.abs(hilbert(hist))
    peak = env[nsteps // 4: 3 * nsteps // 4].max()
    assert abs(peak - expect) / expect < 2e-3, (peak, expect)
    # envelope peak arrives 3 tau + (travel time) after the start, and the
    # carrier just after the envelope peak is positive-going (sin phase)
    t = (np.arange(nsteps) + 1) * o.dt
    tpk = t[np.argmax(env)]
    travel = (probe - o_ka(o)) * o.hz
    assert abs(tpk - (3 * tau + travel)) < 0.5
    # carrier period 1 lambda0/c from the phase slope of the analytic signal
    ph = np.unwrap(np.angle(hilbert(hist)))
    core = slice(int((tpk - tau) / o.dt), int((tpk + tau) / o.dt))
    slope = np.polyfit(t[core], ph[core], 1)[0]
    assert abs(slope / (2 * math.pi) - 1.0) < 2e-3


def test_antenna_carrier_phase_and_plane(oracle_mod):
    # A sheet current centred at t^{n+1/2} on the node plane nearest
    # z_antenna radiates, on the Yee lattice, exactly the discrete plane wave
    # sin(2 pi (t - s_pk) - kappa (k - k_a)) (kappa the discrete vacuum
    # wavenumber per cell): its carrier phase at a probe agrees with that to
    # well below the half-step (pi dt) or one-cell (kappa) shifts a
    # mis-centred time or plane would give.
    from scipy.signal import hilbert
    fwhm = 10.0
    z_cells = 10.7                                       # rounds to plane 11 (floor would give 10)
    g, o = _plane_wave_box(oracle_mod, nz=640, dz=1.0 / 32, fwhm=fwhm)
    o.set_laser(oracle_mod.LaserParams(a0=1.0, waist=1e9, fwhm=fwhm, z_antenna=z_cells * o.hz, pol=1))
    ka, probe = 11, 400
    tau = fwhm / math.sqrt(2 * math.log(2))
    nsteps = int((6 * tau + probe * o.hz + 2.0) / o.dt)
    hist = np.zeros(nsteps)
    for n in range(nsteps):
        o.step(1)
        hist[n] = o.field("Ey")[probe, 0, 0]
    t = (np.arange(nsteps) + 1) * o.dt
    kappa = 2 * math.asin(math.sin(math.pi * o.dt) / (o.dt / o.hz))
    expect = 2 * math.pi * (t - 3 * tau) - kappa * (probe - ka) - math.pi / 2   # phase of the analytic signal
    an = hilbert(hist)
    tpk = t[np.argmax(np.abs(an))]
    core = (t > tpk - tau) & (t < tpk + tau)
    res = np.angle(np.exp(1j * (np.angle(an[core]) - expect[core])))
    assert min(math.pi * o.dt, kappa) > 0.05
    assert np.abs(res).max() < 5e-3, (res.mean(), np.abs(res).max())


def o_ka(o):
    """antenna plane index: nearest node to z_antenna, at least 2 nodes in"""
    return 2


@pytest.mark.parametrize("pol", [0, 1])
def test_mur_absorbs_normal_pulse(oracle_mod, pol):
    # The antenna, mid-box, sends one pulse towards z = 0 and one towards
    # z = Lz.  The run stops once both have left but before anything they
    # reflected could have crossed the box, so what is left is the reflection.  dx = dz makes
    # dt/dz ~ 0.7, where the Mur coefficient (dt - dz)/(dt + dz) is far from
    # zero and a plain outflow condition would reflect ~18%.
    fwhm = 3.0
    g, o = _plane_wave_box(oracle_mod, nz=1200, dz=1.0 / 32, pol=pol, dx=1.0 / 32, fwhm=fwhm,
                           z_ant=600 / 32)
    comp = "Ex" if pol == 0 else "Ey"
    tau = fwhm / math.sqrt(2 * math.log(2))
    t_end = 6 * tau + 0.5 * o.Lz + 2.0
    assert t_end < 6 * tau + 1.5 * o.Lz - 1.0
    peak = 0.0
    for n in range(int(t_end / o.dt)):
        o.step(1)
        peak = max(peak, np.abs(o.field(comp)).max())
    left = np.abs(o.field(comp)).max()
    assert peak > 0.9
    assert left / peak < 1e-2, left / peak


@pytest.mark.parametrize("dim,bc", [(2, 1), (2, 0), (3, 1)])
@pytest.mark.parametrize("npass", [1, 2, 4])
def test_filter_is_its_own_transpose(oracle_mod, dim, bc, npass):
    # the reverse sweep of the adjoint applies the filter to the current
    # cotangent as its own transpose: <F x, y> = <x, F y> over the valid nodes
    # of each component (zero outside the absorbing z range, wrapped when
    # periodic)
    G = oracle_mod.GridParams
    g = G(dim=dim, nx=12, ny=6 if dim == 3 else 1, nz=14, dx=0.5, dy=0.5, dz=0.5, bc_z=bc, npass=npass)
    rng = np.random.default_rng(7 + 10 * dim + bc + 100 * npass)

    def valid(c):
        m = np.ones((g.nz + 1, g.ny, g.nx), bool)
        if bc == 0 or c == "Jz":
            m[g.nz] = False  # plane nz: unused when periodic, outside the half-integer range of Jz
        return m

    def apply(vals):
        o = oracle_mod.Oracle(g)
        for c, v in vals.items():
            o.field(c)[...] = v
        o.filter()
        return {c: o.field(c).copy() for c in vals}

    comps = ("Jx", "Jy", "Jz")
    x = {c: rng.normal(size=(g.nz + 1, g.ny, g.nx)) * valid(c) for c in comps}
    y = {c: rng.normal(size=(g.nz + 1, g.ny, g.nx)) * valid(c) for c in comps}
    fx, fy = apply(x), apply(y)
    for c in comps:
        m = valid(c)
        lhs = float(np.sum(fx[c][m] * y[c][m]))
        rhs = float(np.sum(x[c][m] * fy[c][m]))
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs) + 1.0), (c, lhs, rhs)


@pytest.mark.parametrize("pol", [0, 1])
def test_antenna_beam_has_the_waist(oracle_mod, pol):
    # A Gaussian beam launched by the antenna with field 1/e radius w0 = 4
    # lambda0 keeps that transverse profile a wavelength ahead of it (the
    # Rayleigh length pi w0^2 is 50 lambda0): the peak |E| over time at each
    # transverse node of the probe plane follows exp(-(x - xc)^2 / w0^2), with
    # x the node's own staggered position (Ex on half-integer x).
    G, L = oracle_mod.GridParams, oracle_mod.LaserParams
    w0 = 4.0
    g = G(dim=2, nx=64, nz=256, dx=0.5, dz=1.0 / 16, cfl=0.99, bc_z=1, npass=0)
    o = oracle_mod.Oracle(g)
    o.set_laser(L(a0=1.0, waist=w0, fwhm=2.0, z_antenna=1.0, pol=pol))
    comp = "Ex" if pol == 0 else "Ey"
    kp = int(round(2.0 / o.hz))  # one wavelength ahead of the antenna
    peak = np.zeros(g.nx)
    while o.t < 14.0:
        o.step(1)
        peak = np.maximum(peak, np.abs(o.field(comp)[kp, 0, :]))
    x = (np.arange(g.nx) + (0.5 if pol == 0 else 0.0)) * o.hx
    xc = 0.5 * g.nx * o.hx
    expect = np.exp(-((x - xc) / w0) ** 2)
    near = np.abs(x - xc) < 2.0 * w0
    ratio = peak / peak[np.argmin(np.abs(x - xc))]
    assert peak.max() > 0.5
    assert np.abs(ratio[near] - expect[near]).max() < 0.02, np.abs(ratio[near] - expect[near]).max()



def test_antenna_beam_has_the_waist_across_y(oracle_mod):
    # the same in 3D for a beam polarised along y: its Ey sits on
    # half-integer y, and the peak |Ey| a wavelength ahead follows
    # exp(-((x - xc)^2 + (y - yc)^2) / w0^2) at those staggered points
    G, L = oracle_mod.GridParams, oracle_mod.LaserParams
    w0 = 4.0
    g = G(dim=3, nx=24, ny=48, nz=128, dx=1.0, dy=0.5, dz=1.0 / 16, cfl=0.99, bc_z=1, npass=0)
    o = oracle_mod.Oracle(g)
    o.set_laser(L(a0=1.0, waist=w0, fwhm=2.0, z_antenna=1.0, pol=1))
    kp = int(round(2.0 / o.hz))
    peak = np.zeros((g.ny, g.nx))
    while o.t < 12.0:
        o.step(1)
        peak = np.maximum(peak, np.abs(o.field("Ey")[kp]))
    x = np.arange(g.nx) * o.hx
    y = (np.arange(g.ny) + 0.5) * o.hy
    xc, yc = 0.5 * g.nx * o.hx, 0.5 * g.ny * o.hy
    ic = int(np.argmin(np.abs(x - xc)))
    col = peak[:, ic]                                    # the profile across y through the axis
    expect = np.exp(-((y - yc) / w0) ** 2)
    near = np.abs(y - yc) < 2.0 * w0
    ratio = col / col.max() * expect[np.argmax(col)]
    assert peak.max() > 0.5
    assert np.abs(ratio[near] - expect[near]).max() < 0.02, np.abs(ratio[near] - expect[near]).max()