"""Oracle pins for the particle side: Boris rotation, uniform-E acceleration,
E x B drift, and Esirkepov's charge conservation.

Closed forms used:
* Boris in uniform B (no E): |u| is conserved and u turns by exactly
  theta = 2 atan(w_c dt / 2) per step, w_c = 2 pi |q| B / gamma in lambda0/c
  units; the sense of rotation is fixed by the sign of q.
* uniform E (no B): u_n = u_0 + 2 pi q E n dt, exactly.
* Esirkepov: (rho(x1) - rho(x0)) / dt + div J = 0 at every node, with rho the
  plain nodal deposit q w S S S / V of the same shape, and
  sum(J_d) V = q w (x1 - x0)_d / dt; a particle that does not move deposits
  no current.
"""
import math

import numpy as np
import pytest


def test_boris_uniform_b_rotation(oracle_mod):
    Bz, dt = 2.0, 0.05
    u0 = np.array([3.0, 0.0, 0.4])
    u = u0.copy()
    g = math.sqrt(1 + u0 @ u0)
    wc = 2 * math.pi * Bz / g
    theta = 2 * math.atan(wc * dt / 2)
    for n in range(1, 401):
        u = oracle_mod.boris(u, [0, 0, 0], [0, 0, Bz], -1.0, dt)
        assert abs(np.linalg.norm(u) - np.linalg.norm(u0)) < 1e-12
    ang = math.atan2(u[1], u[0])
    expect = math.remainder(400 * theta, 2 * math.pi)  # electrons turn counter-clockwise about +B
    assert abs(math.remainder(ang - expect, 2 * math.pi)) < 1e-11
    assert abs(u[2] - 0.4) < 1e-14
    # a positive charge turns the other way
    v = oracle_mod.boris(u0, [0, 0, 0], [0, 0, Bz], +1.0, dt)
    assert abs(math.atan2(v[1], v[0]) + theta) < 1e-13


def test_boris_orbit_radius_through_step(oracle_mod):
    # gather of a uniform field + Boris + position update, run through the
    # oracle's step: the discrete orbit is a circle of radius
    # R = (v_perp / w_c) sqrt(1 + (w_c dt/2)^2) (chord geometry).
    G = oracle_mod.GridParams
    g = G(dim=3, nx=16, ny=16, nz=16, dx=1.0, dy=1.0, dz=1.0, cfl=0.5, bc_z=0, npass=0)
    o = oracle_mod.Oracle(g)
    Bz = 0.05
    o.field("Bz")[...] = Bz
    u = np.array([0.5, 0.0, 0.0])
    o.add_particles(0, [8.0], [8.0], [8.0], [u[0]], [u[1]], [u[2]], [1.0], [0])
    gam = math.sqrt(1 + u @ u)
    wc = 2 * math.pi * Bz / gam
    vperp = np.linalg.norm(u) / gam
    R = vperp / wc * math.sqrt(1 + (wc * o.dt / 2) ** 2)
    pts = []
    for n in range(300):
        o.step_phases(oracle_mod.PH_PUSH | oracle_mod.PH_TIME)
        p = o.particles(0)
        pts.append((p["x"][0], p["y"][0]))
    pts = np.array(pts)
    # centre: fit the circle algebraically
    A = np.c_[2 * pts, np.ones(len(pts))]
    bb = (pts ** 2).sum(1)
    cx, cy, c0 = np.linalg.lstsq(A, bb, rcond=None)[0]
    r = np.sqrt(((pts - [cx, cy]) ** 2).sum(1))
    assert np.abs(r - R).max() < 1e-10, (r.min(), r.max(), R)


def test_boris_uniform_e(oracle_mod):
    E = np.array([0.3, -0.1, 0.2])
    u = np.array([0.1, 0.2, -0.3])
    dt = 0.07
    for n in range(1, 201):
        u = oracle_mod.boris(u, E, [0, 0, 0], -1.0, dt)
    np.testing.assert_allclose(u, np.array([0.1, 0.2, -0.3]) - 2 * math.pi * E * 200 * dt, atol=1e-12)


def test_boris_exb_drift(oracle_mod):
    # E_x with B_y: mean velocity E x B / B^2 = (E_x B_y / B^2) z for |E| << |B|
    Ex, By, dt = 0.01, 1.0, 0.01
    u = np.zeros(3)
    vs = []
    for n in range(20000):
        u = oracle_mod.boris(u, [Ex, 0, 0], [0, By, 0], -1.0, dt)
        vs.append(u / math.sqrt(1 + u @ u))
    vmean = np.mean(vs[-(len(vs) // 2):], axis=0)
    assert abs(vmean[2] - Ex / By) < 2e-4 and abs(vmean[0]) < 2e-4


def _one_particle_rho(oracle_mod, g, x, w):
    o = oracle_mod.Oracle(g)
    o.add_particles(0, [x[0]], [x[1]], [x[2]], [0.0], [0.0], [0.0], [w], [0])
    return o.rho()


def _div_j(o, g):
    Jx, Jy, Jz = o.field("Jx"), o.field("Jy"), o.field("Jz")
    nz = g.nz
    d = (Jx[:nz] - np.roll(Jx[:nz], 1, axis=2)) / o.hx
    d = d + (Jz[:nz] - np.roll(Jz[:nz], 1, axis=0)) / o.hz
    if g.dim == 3:
        d = d + (Jy[:nz] - np.roll(Jy[:nz], 1, axis=1)) / o.hy
    return d


@pytest.mark.parametrize("dim,order", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_esirkepov_continuity_and_total_current(oracle_mod, dim, order):
    G = oracle_mod.GridParams
    g = G(dim=dim, nx=8, ny=7 if dim == 3 else 1, nz=9, dx=0.6, dy=0.7, dz=0.5, cfl=0.9,
          shape=order, bc_z=0, npass=0)
    probe = oracle_mod.Oracle(g)
    rng = np.random.default_rng(11 + dim * 10 + order)
    h = np.array([probe.hx, probe.hy, probe.hz])
    L = np.array([probe.Lx, probe.Ly, probe.Lz])
    for trial in range(60):
        x0 = rng.uniform(0, 1, 3) * L
        if trial % 3 == 0:  # start right next to the periodic edge
            x0[0] = L[0] - 1e-3 * h[0]
        # |dx| < h per axis; every third move crosses a cell face in each axis
        d = rng.uniform(-0.95, 0.95, 3) * h
        if dim == 2:
            x0[1] = 0.0
            d[1] = 0.0
        x1 = x0 + d
        w = rng.uniform(0.5, 2.0)
        vy = rng.uniform(-0.5, 0.5)
        o = oracle_mod.Oracle(g)
        o.deposit_current(-w, x0, x1, vy)
        x1w = np.mod(x1, L)
        rho0 = _one_particle_rho(oracle_mod, g, x0, w)[: g.nz]
        rho1 = _one_particle_rho(oracle_mod, g, x1w, w)[: g.nz]
        resid = (rho1 - rho0) / probe.dt + _div_j(o, g)
        scale = np.abs(rho0).max() / probe.dt
        assert np.abs(resid).max() < 1e-12 * scale, (trial, np.abs(resid).max() / scale)
        vol = h[0] * h[2] * (h[1] if dim == 3 else 1.0)
        jx = o.field("Jx")[: g.nz].sum() * vol
        jz = o.field("Jz")[: g.nz].sum() * vol
        assert abs(jx - (-w) * d[0] / probe.dt) < 1e-12 * w * h[0] / probe.dt
        assert abs(jz - (-w) * d[2] / probe.dt) < 1e-12 * w * h[2] / probe.dt
        jy = o.field("Jy")[: g.nz].sum() * vol
        expect_jy = (-w) * d[1] / probe.dt if dim == 3 else (-w) * vy
        assert abs(jy - expect_jy) < 1e-12 * w * max(1.0, h[1] / probe.dt)


def test_esirkepov_static_and_one_axis(oracle_mod):
    G = oracle_mod.GridParams
    g = G(dim=3, nx=6, ny=6, nz=6, dx=1.0, dy=1.0, dz=1.0, cfl=0.9, shape=1, bc_z=0)
    o = oracle_mod.Oracle(g)
    o.deposit_current(-1.0, [2.3, 3.1, 1.7], [2.3, 3.1, 1.7], 0.0)
    for c in ("Jx", "Jy", "Jz"):
        assert np.count_nonzero(o.field(c)) == 0
    # motion along x only, inside one cell, CIC: Jx on the two x-faces of the
    # cell... at (i+1/2) equals q w vx times the (y, z) bilinear weights / V
    o = oracle_mod.Oracle(g)
    x0, x1 = np.array([2.2, 3.25, 1.5]), np.array([2.6, 3.25, 1.5])
    o.deposit_current(-1.0, x0, x1, 0.0)
    vx = (x1[0] - x0[0]) / o.dt
    jx = o.field("Jx")
    # nodes j = 3, 4 with weights 0.75, 0.25; k = 1, 2 with 0.5, 0.5; i + 1/2 = 2.5
    for (j, wy) in ((3, 0.75), (4, 0.25)):
        for (k, wz) in ((1, 0.5), (2, 0.5)):
            assert abs(jx[k, j, 2] - (-1.0) * vx * wy * wz) < 1e-13
    assert np.count_nonzero(o.field("Jy")) == 0 and np.count_nonzero(o.field("Jz")) == 0


@pytest.mark.parametrize("sp", [0, 1])
def test_particles_leaving_through_absorbing_ends_are_removed(oracle_mod, sp):
    # without fields every particle moves by dt u / gamma; with absorbing z
    # exactly those whose new z lies outside [0, Lz) leave the store, at
    # either end, and the others are where the free motion puts them
    O = oracle_mod
    o = O.Oracle(O.GridParams(dim=2, nx=4, nz=16, dx=1.0, dz=0.25, bc_z=1, npass=0))
    rng = np.random.default_rng(5 + sp)
    n = 400
    z = np.concatenate([rng.uniform(0, 0.3, n // 2), rng.uniform(o.Lz - 0.3, o.Lz, n // 2)])
    uz = np.concatenate([rng.uniform(-20, 5, n // 2), rng.uniform(-5, 20, n // 2)])
    x = rng.uniform(0, o.Lx, n)
    ids = np.arange(n)
    o.add_particles(sp, x, 0 * x, z, 0 * x, 0 * x, uz, np.full(n, 1e-3), ids)
    o.step_phases(O.PH_PUSH if sp == 0 else O.PH_IONS)
    z1 = z + o.dt * uz / np.sqrt(1 + uz ** 2)
    stay = (z1 >= 0) & (z1 < o.Lz)
    assert 0 < stay.sum() < n and (z1 >= o.Lz).any() and (z1 < 0).any()
    p = o.particles(sp)
    assert np.array_equal(np.sort(p["id"]), ids[stay])
    got = dict(zip(p["id"].tolist(), p["z"]))
    assert max(abs(got[i] - z1[i]) for i in ids[stay]) < 1e-12


def test_boris_step_satisfies_its_implicit_form(oracle_mod):
    # Boris (1970): with u- = u + eps E and u+ = u_new - eps E (eps = pi (q/m)
    # dt, the half impulse), the magnetic part is the rotation defined
    # implicitly by u+ - u- = (u+ + u-) x t, t = eps B / gamma(u-), so that
    # |u+| = |u-|.  Checked on relativistic particles in strong fields, where
    # taking gamma anywhere else than at u- is far outside round-off.
    rng = np.random.default_rng(23)
    dt = 0.05
    for q_over_m in (-1.0, 1.0):
        eps = math.pi * q_over_m * dt
        for _ in range(50):
            u = rng.normal(scale=5.0, size=3)
            e = rng.normal(scale=10.0, size=3)
            b = rng.normal(scale=10.0, size=3)
            un = np.asarray(oracle_mod.boris(u, e, b, q_over_m, dt))
            um, up = u + eps * e, un - eps * e
            t = eps * b / math.sqrt(1.0 + um @ um)
            assert abs(up @ up - um @ um) <= 1e-12 * (um @ um)
            assert np.abs((up - um) - np.cross(up + um, t)).max() <= 1e-12 * (1.0 + np.abs(um).max())
