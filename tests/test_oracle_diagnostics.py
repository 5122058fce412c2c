"""Pins of the oracle's FP64 diagnostics (field energy, electron kinetic
energy, charge) and of its lab-frame view of the simulation-frame fields.

Closed forms and invariants used:
* a single Fourier mode cos(2 pi m i / n) sums to n/2 in square over a period
  (discrete orthogonality), a uniform field to n; each component counts only
  its own valid planes (half-integer-z components one plane fewer with
  absorbing z);
* a cold plasma at rest in the lab, seen from a frame boosted to gamma, has
  density gamma n and every electron the Lorentz factor gamma: kinetic energy
  (gamma - 1) gamma n V, net charge 0 with its drifting ions; in the lab
  frame its charge is -n times the volume it fills;
* a compensated sum keeps terms below half an ulp of the running total that a
  plain running sum drops (one unit term followed by many of 1e-17);
* energy moves between the electrons and the field in a plasma oscillation:
  the field energy at the turning point equals the initial kinetic energy
  (this fixes the relative normalisation of the two sums);
* a static field seen from a frame moving at +beta along z: E_par unchanged,
  E_perp = gamma E'_perp, B = v x E; the invariants E.B and E^2 - B^2; a field
  linear in z lands on each component's own staggered position.
"""
import math

import numpy as np
import pytest

COMPS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")
HALF_Z = {"Ez", "Bx", "By"}


def _planes(c, nz, bc_z):
    return nz if (bc_z == 0 or c in HALF_Z) else nz + 1


@pytest.mark.parametrize("dim,bc_z", [(2, 1), (2, 0), (3, 1)])
def test_field_energy_of_modes_and_uniform_fields(oracle_mod, dim, bc_z):
    O = oracle_mod
    nx, ny, nz = 16, (6 if dim == 3 else 1), 20
    o = O.Oracle(O.GridParams(dim=dim, nx=nx, ny=ny, nz=nz, dx=0.5, dy=0.7, dz=0.25, bc_z=bc_z))
    i = np.arange(nx)
    A = {"Ex": 0.3, "Ey": 0.0, "Ez": 1.1, "Bx": 0.0, "By": 0.7, "Bz": 0.2}
    o.field("Ex")[...] = A["Ex"] * np.cos(2 * math.pi * 3 * i / nx)      # a mode: n/2 per row
    o.field("Ez")[...] = A["Ez"] * np.sin(2 * math.pi * 5 * i / nx)      # half-integer z
    o.field("By")[...] = A["By"]                                         # uniform, half-integer z
    o.field("Bz")[...] = A["Bz"] * np.cos(2 * math.pi * 1 * i / nx)
    # values on the plane a component does not use are not part of the state
    if bc_z == 1:
        for c in ("Ez", "By"):
            o.field(c)[nz] = 123.0
    rows = {c: ny * _planes(c, nz, bc_z) for c in COMPS}
    sums = {"Ex": A["Ex"] ** 2 * nx / 2, "Ez": A["Ez"] ** 2 * nx / 2, "By": A["By"] ** 2 * nx,
            "Bz": A["Bz"] ** 2 * nx / 2}
    V = o.hx * o.hy * o.hz if dim == 3 else o.hx * o.hz
    expect = 0.5 * V * sum(sums[c] * rows[c] for c in sums)
    got = o.diagnostics()["field_energy"]
    assert abs(got - expect) <= 1e-13 * expect, (got, expect)


@pytest.mark.parametrize("gam", [1.0, 13.0])
def test_kinetic_energy_and_charge_of_a_cold_plasma(oracle_mod, gam):
    O = oracle_mod
    ne = 0.004
    o = O.Oracle(O.GridParams(dim=2, nx=12, nz=40, dx=1.0, dz=1 / 32, gamma_boost=gam, seed=3))
    if gam == 1.0:
        # at rest in the lab over [0.25, 0.75) lambda0 (box: 1.25), immobile ions (a background)
        o.load_plasma(O.PlasmaParams(ne=ne, z_start=0.25, z_end=0.75, ramp=0.0, ppc=(2, 1, 2), jitter=0.0, ions=1))
        d = o.diagnostics()
        assert d["kinetic_energy"] == 0.0
        expect_q = -ne * o.Lx * 0.5
        assert abs(d["charge"] - expect_q) <= 1e-12 * abs(expect_q)
    else:
        # filling the boosted box (lab z from 0 to gamma Lz and beyond)
        o.load_plasma(O.PlasmaParams(ne=ne, z_start=0.0, z_end=gam * o.Lz * 2, ramp=0.0, ppc=(2, 1, 2),
                                     jitter=0.0, ions=1))
        d = o.diagnostics()
        V = o.Lx * o.Lz
        n_boost = gam * ne                           # Lorentz contraction of the density
        expect_ke = (gam - 1.0) * n_boost * V        # each electron at gamma
        assert abs(d["kinetic_energy"] - expect_ke) <= 1e-12 * expect_ke, (d, expect_ke)
        assert abs(d["charge"]) <= 1e-12 * n_boost * V   # electrons and their drifting ions
        assert o.num(0) == o.num(1) == 2 * 2 * o.grid.nx * o.grid.nz


def test_field_energy_sum_is_compensated(oracle_mod):
    # one node of unit field first in storage order, every other valid node a
    # value whose square is below half an ulp of 1: a plain running sum stays
    # at exactly 1, the compensated sum keeps all N - 1 small terms
    O = oracle_mod
    nx, nz = 128, 256
    o = O.Oracle(O.GridParams(dim=2, nx=nx, nz=nz, dx=0.5, dz=0.25, bc_z=1))
    v = math.sqrt(1e-17)
    for c in COMPS:
        o.field(c)[...] = v
    o.field("Ex")[0, 0, 0] = 1.0
    n_small = sum(_planes(c, nz, 1) * nx for c in COMPS) - 1
    V = o.hx * o.hz
    expect = 0.5 * V * (1.0 + n_small * (v * v))
    got = o.diagnostics()["field_energy"]
    assert n_small * v * v > 1e-12                       # far above the sum's own rounding
    assert abs(got - expect) <= 1e-14 * expect, (got, expect, 0.5 * V)


def test_energy_moves_between_electrons_and_field(oracle_mod):
    # a cold plasma oscillation (periodic z, longest mode): the initial
    # kinetic energy reappears as field energy at the turning point, and the
    # electrons give (nearly) all of it up there
    O = oracle_mod
    g = O.GridParams(dim=2, nx=2, nz=128, dx=0.5, dz=0.25, cfl=0.9, bc_z=0, npass=0, shape=1)
    o = O.Oracle(g)
    n0, ppc = 0.01, 4
    zs = (np.arange(g.nz * ppc) + 0.5) * (o.hz / ppc)
    xs = (np.arange(g.nx * 2) + 0.5) * (o.hx / 2)
    X, Z = np.meshgrid(xs, zs)
    X, Z = X.ravel(), Z.ravel()
    w = n0 * o.hx * o.hz / (2 * ppc)
    uz = 1e-2 * np.sin(2 * math.pi * Z / o.Lz)
    o.add_particles(0, X, 0 * X, Z, 0 * X, 0 * X, uz, np.full_like(X, w))
    ke0 = o.diagnostics()["kinetic_energy"]
    assert abs(ke0 - 0.5 * w * float(np.sum(uz ** 2))) < 1e-4 * ke0     # (gamma - 1) ~ u^2 / 2
    fe, ke = [], []
    for _ in range(int(12.0 / o.dt)):                # past the first turning point
        o.step(1)
        d = o.diagnostics()
        fe.append(d["field_energy"])
        ke.append(d["kinetic_energy"])
    fe, ke = np.array(fe), np.array(ke)
    assert abs(fe.max() / ke0 - 1.0) < 0.02, fe.max() / ke0
    assert ke.min() < 0.02 * ke0


@pytest.mark.parametrize("gam", [1.0, 3.0, 130.0])
def test_lab_fields_of_uniform_fields(oracle_mod, gam):
    O = oracle_mod
    o = O.Oracle(O.GridParams(dim=3, nx=6, ny=5, nz=12, dx=1.0, dy=1.0, dz=0.25, gamma_boost=gam, bc_z=1))
    beta = o.beta
    e, b = np.array([0.3, -0.2, 0.5]), np.array([0.1, 0.4, -0.25])
    for q, c in enumerate(COMPS):
        o.field(c)[...] = (e if q < 3 else b)[q % 3]
    lab = o.fields_lab()
    E = np.array([lab[c][4:8].mean() for c in COMPS[:3]])
    B = np.array([lab[c][4:8].mean() for c in COMPS[3:]])
    for c in COMPS:
        assert np.ptp(lab[c][1:-2]) < 1e-14  # uniform stays uniform
    # invariants of the transformation
    assert abs(E @ B - e @ b) < 1e-12 * max(1.0, gam * gam)
    assert abs((E @ E - B @ B) - (e @ e - b @ b)) < 1e-12 * max(1.0, gam * gam)
    # parallel components unchanged
    assert E[2] == e[2] and B[2] == b[2]
    # a purely electric field in the moving frame: the lab sees gamma E'_perp
    # and B = v x E with v = +beta z
    for c in COMPS[3:]:
        o.field(c)[...] = 0.0
    lab = o.fields_lab()
    E = np.array([lab[c][4:8].mean() for c in COMPS[:3]])
    B = np.array([lab[c][4:8].mean() for c in COMPS[3:]])
    assert np.allclose(E, [gam * e[0], gam * e[1], e[2]], rtol=1e-14, atol=0)
    assert np.allclose(B, np.cross([0.0, 0.0, beta], E), rtol=1e-13, atol=1e-15)


def test_lab_fields_pair_each_component_with_its_staggered_partner(oracle_mod):
    # By' linear in z at its half-integer planes, Ex' zero: the lab Ex at the
    # integer plane k is gamma beta By'(k hz) exactly (the mean of the planes
    # k - 1/2 and k + 1/2); and Ex' linear, By' zero: the lab By at k + 1/2 is
    # gamma beta Ex'((k + 1/2) hz)
    O = oracle_mod
    gam = 2.0
    o = O.Oracle(O.GridParams(dim=2, nx=4, nz=16, dx=1.0, dz=0.25, gamma_boost=gam, bc_z=1))
    beta, hz, nz = o.beta, o.hz, o.grid.nz
    k = np.arange(nz + 1)
    by_at = lambda z: 0.2 + 0.03 * z
    o.field("By")[:, 0, :] = by_at((k[:, None] + 0.5) * hz)
    lab = o.fields_lab()
    inner = slice(1, nz)
    assert np.allclose(lab["Ex"][inner, 0, :], gam * beta * by_at(k[inner, None] * hz), rtol=1e-14, atol=0)
    o.field("By")[...] = 0.0
    ex_at = lambda z: -0.1 + 0.05 * z
    o.field("Ex")[:, 0, :] = ex_at(k[:, None] * hz)
    lab = o.fields_lab()
    inner = slice(0, nz - 1)
    assert np.allclose(lab["By"][inner, 0, :], gam * beta * ex_at((k[inner, None] + 0.5) * hz), rtol=1e-14,
                       atol=0)
    # at gamma = 1 the view is the identity
    o1 = O.Oracle(O.GridParams(dim=2, nx=4, nz=16, dx=1.0, dz=0.25, bc_z=1))
    rng = np.random.default_rng(1)
    for c in COMPS:
        o1.field(c)[...] = rng.normal(size=o1.field(c).shape)
        if c in HALF_Z:
            o1.field(c)[nz] = 0.0
    lab = o1.fields_lab()
    for c in COMPS:
        assert np.array_equal(lab[c], o1.field(c)), c
