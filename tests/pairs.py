"""Helpers that run the CUDA library and the FP64 oracle side by side on the
same seeded inputs (test infrastructure)."""
from __future__ import annotations

import math

import numpy as np

COMPONENTS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz")
HALF_Z = {"Ez", "Bx", "By", "Jz"}


def oracle_grid(O, g: dict):
    return O.GridParams(dim=g["dim"], nx=g["nx"], ny=g.get("ny", 1), nz=g["nz"], dx=g["dx"], dy=g.get("dy", 1.0),
                        dz=g["dz"], cfl=g.get("cfl", 0.99), gamma_boost=g.get("gamma_boost", 1.0),
                        shape=g.get("shape_order", 1), npass=g.get("filter_passes", 1), bc_z=g.get("bc_z", 1),
                        seed=g.get("seed", 1))


def make_pair(O, g: dict, precision: int, track_ids: bool = True, slots_per_cell: float = 16.0, tile=(0, 0, 0),
              explicit_ions: bool = False, z_relative: int = 0):
    """GPU context and oracle on the same grid.  z_relative: 0 automatic
    (relative electron positions from gamma_boost 50 on), 1 on, 2 off."""
    import paper_1011_0917_gb300 as P
    sim = P.Simulation(dim=g["dim"], nx=g["nx"], ny=g.get("ny", 1), nz=g["nz"], dx=g["dx"], dy=g.get("dy", 1.0),
                       dz=g["dz"], cfl=g.get("cfl", 0.99), gamma_boost=g.get("gamma_boost", 1.0),
                       shape_order=g.get("shape_order", 1), filter_passes=g.get("filter_passes", 1),
                       bc_z=g.get("bc_z", 1), precision=precision, seed=g.get("seed", 1),
                       slots_per_cell=slots_per_cell, track_ids=track_ids, tile=tile, explicit_ions=explicit_ions,
                       z_relative=z_relative)
    o = O.Oracle(oracle_grid(O, g))
    assert sim.dt == o.dt
    return sim, o


def zmax(c: str, nz: int, bc_z: int) -> int:
    if bc_z == 0:
        return nz - 1
    return nz - 1 if c in HALF_Z else nz


def set_fields_both(sim, o, fields: dict, bc_z: int):
    nz = o.grid.nz
    clean = {}
    for c, v in fields.items():
        v = np.array(v, dtype=np.float64)
        v[zmax(c, nz, bc_z) + 1:] = 0.0
        clean[c] = v
        o.field(c)[...] = v
    sim.set_fields(clean)


def gpu_fields(sim) -> dict:
    return {c: t.double().cpu().numpy() for c, t in sim.fields().items()}


def field_errors(sim, o, comps=COMPONENTS, bc_z: int = 1) -> dict:
    """relative L2 error of each component over its valid planes"""
    g = gpu_fields(sim)
    nz = o.grid.nz
    out = {}
    for c in comps:
        km = zmax(c, nz, bc_z) + 1
        a, b = g[c][:km], o.field(c)[:km]
        nb = np.linalg.norm(b)
        out[c] = np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)
    return out


def field_maxrel(sim, o, comps=COMPONENTS, bc_z: int = 1) -> dict:
    """max |a - b| / max |b| of each component over its valid planes"""
    g = gpu_fields(sim)
    nz = o.grid.nz
    out = {}
    for c in comps:
        km = zmax(c, nz, bc_z) + 1
        a, b = g[c][:km], o.field(c)[:km]
        m = np.abs(b).max()
        out[c] = np.abs(a - b).max() / m if m > 0 else np.abs(a).max()
    return out


def gpu_particles(sim, sp: int = 0):
    st, ids = sim.particles(sp, with_ids=True)
    order = np.argsort(ids, kind="stable")
    return st[:, order], ids[order]


def oracle_particles(o, sp: int = 0):
    p = o.particles(sp)
    st = np.stack([p["x"], p["y"], p["z"], p["ux"], p["uy"], p["uz"], p["w"]])
    order = np.argsort(p["id"], kind="stable")
    return st[:, order], p["id"][order]


def periodic_delta(a, b, L):
    d = a - b
    return d - L * np.round(d / L)


def vector_errors(sim, o, bc_z: int = 1, floor: float = 0.1) -> dict:
    """Relative L2 of the E field and of the B field as vectors (all three
    components together), plus the relative L2 of every component that carries
    at least `floor` of its vector field's norm.  A component the physics
    leaves at zero (e.g. Ez where no wake has formed yet) holds round-off only
    on both sides; its own relative error says nothing about the method."""
    g = gpu_fields(sim)
    nz = o.grid.nz
    out = {}
    for name, comps in (("E", ("Ex", "Ey", "Ez")), ("B", ("Bx", "By", "Bz"))):
        num = den = 0.0
        norms = {}
        for c in comps:
            km = zmax(c, nz, bc_z) + 1
            a, b = g[c][:km], o.field(c)[:km]
            num += float(np.sum((a - b) ** 2))
            den += float(np.sum(b ** 2))
            norms[c] = (float(np.linalg.norm(a - b)), float(np.linalg.norm(b)))
        out[name] = math.sqrt(num / den) if den > 0 else math.sqrt(num)
        vn = math.sqrt(den)
        for c, (dn, bn) in norms.items():
            if vn > 0 and bn >= floor * vn:
                out[c] = dn / bn
    return out
