"""Cell order of the particle store (pic_sort_cells, pic_set_cell_sort):
after a sort the records of every tile come out cell by cell, the particle
set is unchanged (compared by id), and runs that sort every few steps match
the FP64 oracle exactly as runs that do not (the deposit is order-free)."""
import math

import numpy as np
import pytest

from pairs import gpu_particles, make_pair, vector_errors

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1
TOL = {FP32: 1e-4, FP64: 1e-10}
GAM = 13.0
BETA = math.sqrt(1 - 1 / GAM ** 2)
HZ = (1 / 32) * GAM * (1 + BETA)
G2 = dict(dim=2, nx=32, nz=256, dx=1.0, dz=1 / 32, gamma_boost=GAM, filter_passes=2, seed=31)
G3 = dict(dim=3, nx=16, ny=16, nz=64, dx=1.0, dy=1.0, dz=1 / 32, gamma_boost=GAM, filter_passes=2, seed=32)
LASER = dict(a0=4.0, waist=8.0, fwhm=2.0, t_peak=0.5)


def plasma(dim):
    return dict(ne=0.004, z_start=GAM * 10 * HZ, z_end=GAM * 600 * HZ, ramp=2.0,
                ppc=(2, 2, 2) if dim == 3 else (2, 1, 2), jitter=0.1, ions=1)


@pytest.fixture(scope="module")
def O():
    import oracle.oracle as O
    O.build_oracle()
    return O


def _setup(O, g, prec, **kw):
    sim, o = make_pair(O, g, prec, **kw)
    p = plasma(g["dim"])
    sim.load_plasma(p["ne"], p["z_start"], p["z_end"], p["ramp"], p["ppc"], p["jitter"], (), p["ions"])
    o.load_plasma(O.PlasmaParams(ne=p["ne"], z_start=p["z_start"], z_end=p["z_end"], ramp=p["ramp"], ppc=p["ppc"],
                                 jitter=p["jitter"], ions=p["ions"]))
    sim.launch_laser(LASER["a0"], LASER["waist"], LASER["fwhm"], 0.0, LASER["t_peak"], 1)
    o.set_laser(O.LaserParams(a0=LASER["a0"], waist=LASER["waist"], fwhm=LASER["fwhm"], t_peak=LASER["t_peak"],
                              pol=1))
    return sim, o


def _tile_cell_keys(sim, st):
    """(tile, cell in tile) of each particle, x fastest, from its position"""
    s = sim.sizes
    g = sim.params
    # (the positions are (cell + offset) h in FP64: an offset of exactly 0
    # may come back a rounding below the cell's edge)
    cell = [np.floor(st[0] / s.hx + 1e-9).astype(np.int64),
            np.floor(st[1] / s.hy + 1e-9).astype(np.int64) if g.dim == 3 else np.zeros(st.shape[1], np.int64),
            np.floor(st[2] / s.hz + 1e-9).astype(np.int64)]
    lt = [int(round(math.log2(t))) for t in s.tile]
    nt = [(n + t - 1) // t for n, t in zip((g.nx, g.ny if g.dim == 3 else 1, g.nz), s.tile)]
    tile = ((cell[2] >> lt[2]) * nt[1] + (cell[1] >> lt[1])) * nt[0] + (cell[0] >> lt[0])
    lc = ((((cell[2] & ((1 << lt[2]) - 1)) << lt[1]) | (cell[1] & ((1 << lt[1]) - 1))) << lt[0]) | \
        (cell[0] & ((1 << lt[0]) - 1))
    return tile, lc


@pytest.mark.parametrize("g", [G2, G3], ids=["2d", "3d"])
def test_sort_orders_each_tile_by_cell(O, g):
    sim, _ = _setup(O, g, FP64)
    sim.step(12)
    before, ids_b = gpu_particles(sim, 0)
    ions_b, iids_b = gpu_particles(sim, 1)
    import paper_1011_0917_gb300 as P
    P.pic_sort_cells(sim.ctx)
    st, ids = sim.particles(0, with_ids=True)
    tile, lc = _tile_cell_keys(sim, st)
    key = tile * 4096 + lc
    # records come out tile by tile (each tile's bucket in cell order)
    assert np.all(np.diff(key) >= 0)
    after, ids_a = gpu_particles(sim, 0)
    assert np.array_equal(ids_a, ids_b) and np.array_equal(after, before)
    ions_a, iids_a = gpu_particles(sim, 1)
    assert np.array_equal(iids_a, iids_b) and np.array_equal(ions_a, ions_b)


@pytest.mark.parametrize("g", [G2, G3], ids=["2d", "3d"])
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_sorting_run_matches_oracle(O, g, prec):
    import paper_1011_0917_gb300 as P
    sim, o = _setup(O, g, prec)
    P.pic_set_cell_sort(sim.ctx, 4)
    sim.step(30)
    o.step(30)
    err = vector_errors(sim, o)
    assert max(err.values()) < TOL[prec], err
    d = sim.diagnostics()
    assert d.n_particles[0] == o.num(0) and d.n_particles[1] == o.num(1)
