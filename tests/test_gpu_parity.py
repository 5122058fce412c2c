"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Single phases on random inputs, then whole steps.  Tolerances:
* FP64 build: round-off only.  Single phases: max |gpu - oracle| / max |oracle|
  <= 1e-12; full-step windows: relative L2 <= 1e-10.
* FP32 build: single phases <= 2e-6 (fields) / 1e-5 (currents, which sum many
  rounded contributions through shared-memory atomics in any order); full-step
  windows (50 steps or fewer): relative L2 <= 1e-4.
Full-step windows compare the E and B fields as vectors, and each component
that carries at least 10% of its field's norm on its own (see
pairs.vector_errors): a component the physics leaves at zero holds only
round-off on both sides.
Grids are chosen to span several tiles with ragged last tiles.  Cases marked
"rel" run the electrons in relative form (reference path + departure, the
currents in FP64; include/pic.h), which the library selects on its own from
gamma_boost 50 on.
"""
import math

import numpy as np
import pytest

from pairs import (COMPONENTS, field_errors, field_maxrel, gpu_particles, make_pair, oracle_particles,
                   periodic_delta, set_fields_both, vector_errors)
from paper_1011_0917_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1
TOL1 = {FP32: 2e-6, FP64: 1e-12}
TOLJ = {FP32: 1e-5, FP64: 1e-12}

G2 = dict(dim=2, nx=24, nz=40, dx=0.5, dz=0.125, cfl=0.95, filter_passes=2, seed=7)
G3 = dict(dim=3, nx=12, ny=10, nz=20, dx=0.5, dy=0.6, dz=0.25, cfl=0.95, filter_passes=1, seed=8)


def test_bounded_wait_reports_timeout():
    # the wait primitive of the TMA pipelines: completes when the arrival is
    # made, runs out (PIC_ERR_TIMEOUT, no fault) when nothing ever arrives;
    # the device stays usable
    import torch

    import paper_1011_0917_gb300 as P
    s = torch.cuda.current_stream().cuda_stream
    assert P.pic_wait_check(True, 100.0, s) == P.PIC_OK
    assert P.pic_wait_check(False, 50.0, s) == P.PIC_ERR_TIMEOUT
    assert P.pic_wait_check(True, 100.0, s) == P.PIC_OK
    x = torch.ones(1024, device="cuda")
    assert float(x.sum()) == 1024.0


def shape3(g):
    return (g["nz"] + 1, g.get("ny", 1) if g["dim"] == 3 else 1, g["nx"])


@pytest.fixture(scope="module")
def O():
    import oracle.oracle as O
    O.build_oracle()
    return O


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("g,bc", [(G2, 1), (G2, 0), (G3, 1), (G3, 0)])
def test_yee_phase(O, g, bc, prec):
    g = dict(g, bc_z=bc)
    sim, o = make_pair(O, g, prec)
    set_fields_both(sim, o, W.random_fields(shape3(g), seed=11), bc)
    for _ in range(3):
        sim.step_phases(32)
        o.step_phases(O.PH_YEE)
    err = field_maxrel(sim, o, COMPONENTS[:6], bc)
    assert max(err.values()) < TOL1[prec], err


# 3D grids whose rows are a multiple of 16 bytes: the filter stages its planes
# with tensor (TMA) copies there, with ragged last columns in x and y
G3T = dict(dim=3, nx=48, ny=20, nz=24, dx=0.5, dy=0.6, dz=0.25, cfl=0.95, filter_passes=1, seed=9)
G3W = dict(dim=3, nx=72, ny=12, nz=16, dx=0.5, dy=0.6, dz=0.25, cfl=0.95, filter_passes=1, seed=10)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("g,bc,npass", [(G2, 1, 1), (G2, 0, 3), (G3, 1, 2), (G3, 0, 1), (G2, 1, 5), (G3, 1, 4),
                                        (G3T, 1, 1), (G3T, 0, 2), (G3T, 1, 3), (G3W, 1, 4), (G3W, 0, 2)])
def test_filter_phase(O, g, bc, npass, prec):
    g = dict(g, bc_z=bc, filter_passes=npass)
    sim, o = make_pair(O, g, prec)
    set_fields_both(sim, o, W.random_fields(shape3(g), seed=12), bc)
    sim.step_phases(16)
    o.step_phases(O.PH_FILTER)
    err = field_maxrel(sim, o, ("Jx", "Jy", "Jz"), bc)
    assert max(err.values()) < TOL1[prec], err


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("g,pol,gam", [(G2, 1, 1.0), (G2, 0, 1.0), (G3, 1, 1.0), (G3, 0, 5.0)])
def test_antenna_phase(O, g, pol, gam, prec):
    g = dict(g, gamma_boost=gam)
    sim, o = make_pair(O, g, prec)
    lp = dict(a0=1.3, waist=2.0, fwhm=2.0, z_antenna=1.0, t_peak=0.4)
    sim.launch_laser(lp["a0"], lp["waist"], lp["fwhm"], lp["z_antenna"], lp["t_peak"], pol)
    o.set_laser(O.LaserParams(a0=lp["a0"], waist=lp["waist"], fwhm=lp["fwhm"], z_antenna=lp["z_antenna"],
                              t_peak=lp["t_peak"], pol=pol))
    c = "Jx" if pol == 0 else "Jy"
    for _ in range(4):  # the sheet at t + dt/2 for four successive times
        sim.step_phases(1 | 8 | 128)
        o.step_phases(O.PH_ZERO_J | O.PH_ANTENNA | O.PH_TIME)
        err = field_maxrel(sim, o, ("Jx", "Jy"), 1)
        assert np.abs(o.field(c)).max() > 0
        assert max(err.values()) < TOL1[prec], err


def _random_state(o, g, n, seed, margin_cells=2.0, u_scale=0.5):
    return W.random_particles(n, (o.Lx, o.Ly, o.Lz), seed, u_scale=u_scale, dim=g["dim"],
                              margin_z=margin_cells * o.hz)


def _load_both(sim, o, sp, st, ids):
    sim.load_particles(sp, st, ids)
    o.add_particles(sp, st[0], st[1], st[2], st[3], st[4], st[5], st[6], ids)


def _compare_particles(sim, o, sp, prec, pos_tol=None, u_tol=None):
    a, ia = gpu_particles(sim, sp)
    b, ib = oracle_particles(o, sp)
    assert np.array_equal(ia, ib), (len(ia), len(ib))
    pos_tol = pos_tol if pos_tol is not None else (1e-12 if prec == FP64 else 2e-6)
    u_tol = u_tol if u_tol is not None else (1e-12 if prec == FP64 else 1e-5)
    dx = np.abs(periodic_delta(a[0], b[0], o.Lx)) / o.hx
    dz = np.abs(a[2] - b[2]) / o.hz
    assert dx.max() < pos_tol and dz.max() < pos_tol, (dx.max(), dz.max())
    if o.grid.dim == 3:
        dy = np.abs(periodic_delta(a[1], b[1], o.Ly)) / o.hy
        assert dy.max() < pos_tol, dy.max()
    du = np.abs(a[3:6] - b[3:6]).max() / max(1.0, np.abs(b[3:6]).max())
    assert du < u_tol, du
    assert np.abs(a[6] - b[6]).max() <= (1e-15 if prec == FP64 else 1e-7) * np.abs(b[6]).max()


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("g,shape,bc,rel", [(G2, 1, 1, 2), (G2, 2, 1, 2), (G2, 1, 0, 2), (G3, 1, 1, 2),
                                            (G3, 2, 0, 2), (G2, 2, 1, 1), (G2, 1, 0, 1), (G3, 1, 1, 1),
                                            (G3, 2, 0, 1)])
def test_push_deposit_phase(O, g, shape, bc, rel, prec):
    g = dict(g, shape_order=shape, bc_z=bc)
    sim, o = make_pair(O, g, prec, z_relative=rel)
    n = 3000 if g["dim"] == 2 else 6000
    st = _random_state(o, g, n, seed=21 + shape)
    ids = np.arange(n, dtype=np.int64) * 7 + 3
    _load_both(sim, o, 0, st, ids)
    set_fields_both(sim, o, W.random_fields((g["nz"] + 1, g.get("ny", 1) if g["dim"] == 3 else 1, g["nx"]),
                                            seed=22, scale=0.3), bc)
    for _ in range(2):
        sim.step_phases(1 | 2)
        o.step_phases(O.PH_ZERO_J | O.PH_PUSH)
    _compare_particles(sim, o, 0, prec)
    err = field_maxrel(sim, o, ("Jx", "Jy", "Jz"), bc)
    assert max(err.values()) < TOLJ[prec], err


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("g,shape,rel", [(G2, 1, 2), (G2, 2, 2), (G3, 1, 2), (G2, 2, 1), (G3, 1, 1)])
def test_drifting_ion_phase(O, g, shape, rel, prec):
    g = dict(g, shape_order=shape, gamma_boost=5.0)
    sim, o = make_pair(O, g, prec, z_relative=rel)
    n = 2000
    st = _random_state(o, g, n, seed=31)
    uz0 = -(5.0 * o.beta)
    st[3:6] = 0.0
    st[5] = uz0
    ids = np.arange(n, dtype=np.int64)
    _load_both(sim, o, 1, st, ids)
    for _ in range(3):
        sim.step_phases(1 | 4)
        o.step_phases(O.PH_ZERO_J | O.PH_IONS)
    _compare_particles(sim, o, 1, prec, u_tol=1e-6)
    err = field_maxrel(sim, o, ("Jx", "Jy", "Jz"), 1)
    assert max(err.values()) < TOLJ[prec], err


def _plasma_both(sim, o, O, p):
    sim.load_plasma(p["ne"], p["z_start"], p["z_end"], p["ramp"], p["ppc"], p["jitter"], p.get("profile", ()),
                    p["ions"])
    return o.load_plasma(O.PlasmaParams(ne=p["ne"], z_start=p["z_start"], z_end=p["z_end"], ramp=p["ramp"],
                                        ppc=p["ppc"], jitter=p["jitter"], profile=p.get("profile", ()),
                                        ions=p["ions"]))


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("case,explicit", [("c0", False), ("boost2d", False), ("boost3d", False),
                                           ("boost3d", True), ("profile", False)])
def test_plasma_load_matches_lattice(O, case, explicit, prec):
    if case == "c0":
        st = W.stage("c0")
        g, p = st.grid, st.plasma
    elif case == "boost2d":
        g = dict(dim=2, nx=40, nz=300, dx=1.0, dz=1 / 32, gamma_boost=13.0, filter_passes=2, seed=5)
        p = dict(ne=0.001, z_start=1200.0, z_end=3500.0, ramp=2.0, ppc=(2, 1, 2), jitter=0.1, ions=1)
    elif case == "boost3d":
        g = dict(dim=3, nx=12, ny=10, nz=40, dx=1.0, dy=1.0, dz=1 / 32, gamma_boost=13.0, seed=6)
        p = dict(ne=0.001, z_start=100.0, z_end=900.0, ramp=2.0, ppc=(2, 2, 2), jitter=0.1, ions=1)
    else:
        g = dict(dim=2, nx=16, nz=200, dx=1.0, dz=1 / 16, gamma_boost=5.0, seed=9)
        p = dict(ne=0.002, z_start=50.0, z_end=400.0, ramp=3.0, ppc=(2, 1, 3), jitter=0.2, ions=1,
                 profile=(0.1, -0.05, 0.02, 0.0, 0.01, -0.02, 0.03, -0.01))
    sim, o = make_pair(O, g, prec, explicit_ions=explicit)
    n = _plasma_both(sim, o, O, p)
    assert n > 100
    if explicit or g.get("gamma_boost", 1.0) == 1.0:
        assert sim.diagnostics().n_paired == 0
    _compare_particles(sim, o, 0, prec)
    if g.get("gamma_boost", 1.0) > 1.0:
        _compare_particles(sim, o, 1, prec)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("explicit,rel", [(False, 2), (True, 2), (False, 1)])
def test_injection_matches_oracle(O, explicit, rel, prec):
    g = dict(dim=2, nx=12, nz=120, dx=1.0, dz=1 / 16, gamma_boost=5.0, filter_passes=1, seed=13)
    sim, o = make_pair(O, g, prec, explicit_ions=explicit, z_relative=rel)
    zs = 5.0 * (o.Lz - 2.0)
    p = dict(ne=0.002, z_start=zs, z_end=zs + 5.0 * 40.0, ramp=1.0, ppc=(2, 1, 2), jitter=0.1, ions=1)
    _plasma_both(sim, o, O, p)
    assert o.pending() > 0
    mask_gpu = 2 | 4 | 64 | 128
    nsteps = 40
    for _ in range(nsteps):
        sim.step_phases(1 | mask_gpu)
        o.step_phases(O.PH_ZERO_J | O.PH_PUSH | O.PH_IONS | O.PH_INJECT | O.PH_TIME)
    # a field-free drift repeats the same rounded displacement v dt / hz every
    # step: in FP32, v = u/gamma carries up to ~1 ulp (1.2e-7 relative), so the
    # position error grows like steps x (cells per step) x 1.2e-7
    tol = 1e-12 if prec == FP64 else 2e-6 + nsteps * 0.61 * 1.2e-7 * 1.5
    _compare_particles(sim, o, 0, prec, pos_tol=tol)
    _compare_particles(sim, o, 1, prec, pos_tol=tol)


def _run_steps_parity(O, g, p, laser, nsteps, prec, slots=16.0, explicit=False, rel=0):
    sim, o = make_pair(O, g, prec, slots_per_cell=slots, explicit_ions=explicit, z_relative=rel)
    if p is not None:
        _plasma_both(sim, o, O, p)
    if laser is not None:
        sim.launch_laser(laser["a0"], laser["waist"], laser["fwhm"], laser.get("z_antenna", 0.0),
                         laser.get("t_peak", -1.0), laser.get("pol", 1))
        o.set_laser(O.LaserParams(a0=laser["a0"], waist=laser["waist"], fwhm=laser["fwhm"],
                                  z_antenna=laser.get("z_antenna", 0.0), t_peak=laser.get("t_peak", -1.0),
                                  pol=laser.get("pol", 1)))
    sim.step(nsteps)
    o.step(nsteps)
    return sim, o


TOL50 = {FP32: 1e-4, FP64: 1e-10}


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_c0_first_50_steps(O, prec):
    st = W.stage("c0")
    sim, o = _run_steps_parity(O, st.grid, st.plasma, st.laser, 50, prec)
    err = vector_errors(sim, o)
    assert max(err.values()) < TOL50[prec], err


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_c0_window_laser_in_plasma(O, prec):
    # the oracle runs c0 to step 330 (laser well inside the plasma), the GPU
    # starts from that state, then both run 50 more steps
    st = W.stage("c0")
    g = st.grid
    o = O.Oracle(O.GridParams(dim=2, nx=g["nx"], nz=g["nz"], dx=g["dx"], dz=g["dz"], npass=g["filter_passes"],
                              seed=g["seed"]))
    o.load_plasma(O.PlasmaParams(**{k: st.plasma[k] for k in ("ne", "z_start", "z_end", "ramp", "ppc", "jitter",
                                                                "ions")}))
    o.set_laser(O.LaserParams(a0=1.0, waist=8.0, fwhm=5.0, pol=1))
    o.step(330)
    sim, _ = make_pair(O, g, prec)
    fld = {c: o.field(c).copy() for c in COMPONENTS}
    sim.set_fields(fld)
    pst, pid = oracle_particles(o, 0)
    sim.load_particles(0, pst, pid)
    sim.launch_laser(1.0, 8.0, 5.0, 0.0, -1.0, 1)
    # carry the oracle's clock over through a snapshot header edit-free path:
    # step the GPU's time forward with TIME-only phases
    for _ in range(330):
        sim.step_phases(128)
    assert abs(sim.diagnostics().t - o.t) < 1e-12
    sim.step(50)
    o.step(50)
    err = vector_errors(sim, o)
    assert np.abs(o.field("Ez")).max() > 1e-3  # a wake is there
    assert max(err.values()) < TOL50[prec], err
    # the wake field, small next to the laser, is checked on its own
    assert field_errors(sim, o, ("Ez",))["Ez"] < TOL50[prec]


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("explicit,rel", [(False, 0), (True, 0), (False, 1), (True, 1)])
def test_boosted_2d_50_steps_with_injection(O, explicit, rel, prec):
    # gamma = 13, plasma 10 cells from the antenna streaming in through z = Lz;
    # the laser meets the plasma within the window
    g = dict(dim=2, nx=32, nz=256, dx=1.0, dz=1 / 32, gamma_boost=13.0, filter_passes=2, seed=17)
    beta = math.sqrt(1 - 1 / 169.0)
    hz = (1 / 32) * 13 * (1 + beta)
    p = dict(ne=0.004, z_start=13 * 10 * hz, z_end=13 * 600 * hz, ramp=2.0, ppc=(2, 1, 2), jitter=0.1, ions=1)
    laser = dict(a0=4.0, waist=8.0, fwhm=2.0, t_peak=0.5)
    sim, o = _run_steps_parity(O, g, p, laser, 50, prec, explicit=explicit, rel=rel)
    err = vector_errors(sim, o)
    assert max(err.values()) < TOL50[prec], err
    # the plasma's own Ez (the wake the laser starts), far below the laser's
    # Ey, on its own
    assert np.abs(o.field("Ez")).max() > 1e-6 * np.abs(o.field("Ey")).max()
    assert field_errors(sim, o, ("Ez",))["Ez"] < TOL50[prec]
    d = sim.diagnostics()
    assert d.n_particles[0] == o.num(0) and d.n_particles[1] == o.num(1)
    if explicit:
        assert d.n_paired == 0
    else:
        assert 0 < d.n_paired < d.n_particles[0]  # some pairs were released by the laser


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("explicit,rel", [(False, 0), (True, 0), (False, 1)])
def test_3d_boosted_30_steps(O, explicit, rel, prec):
    g = dict(dim=3, nx=16, ny=16, nz=48, dx=1.0, dy=1.0, dz=1 / 32, gamma_boost=13.0, filter_passes=2, seed=19)
    beta = math.sqrt(1 - 1 / 169.0)
    hz = (1 / 32) * 13 * (1 + beta)
    p = dict(ne=0.004, z_start=13 * 6 * hz, z_end=13 * 200 * hz, ramp=2.0, ppc=(2, 2, 2), jitter=0.1, ions=1)
    laser = dict(a0=4.0, waist=4.0, fwhm=2.0, t_peak=0.5)
    sim, o = _run_steps_parity(O, g, p, laser, 30, prec, explicit=explicit, rel=rel)
    err = vector_errors(sim, o)
    assert max(err.values()) < TOL50[prec], err
    assert np.abs(o.field("Ez")).max() > 1e-6 * np.abs(o.field("Ey")).max()
    assert field_errors(sim, o, ("Ez",))["Ez"] < TOL50[prec]


# the wake on its own: at gamma = 130 the oracle's own FP64 wake carries
# ~1e-8 (the species' currents it subtracts are 1/(2 gamma^2) ~ 3e-8 of the
# plasma response apart), so the FP64 build is held to 1e-7 there
TOL_WAKE = {FP32: 1e-3, FP64: 1e-7}


def _c3_small_window(O, a0, prec, explicit):
    # the gamma = 130, quadratic-shape, 4-pass stage on a 4x coarser grid; the
    # plasma starts 3 cells from the antenna so the laser reaches it
    g = dict(dim=2, nx=32, nz=200, dx=4.0, dz=4 / 32, gamma_boost=130.0, shape_order=2, filter_passes=4, seed=23)
    beta = math.sqrt(1 - 1 / 130.0 ** 2)
    hz = (4 / 32) * 130 * (1 + beta)
    p = dict(ne=5.7e-5, z_start=130 * 3 * hz, z_end=130 * 400 * hz, ramp=5.0, ppc=(2, 1, 2), jitter=0.1, ions=1)
    laser = dict(a0=a0, waist=20.0, fwhm=4.0, t_peak=0.2)
    return _run_steps_parity(O, g, p, laser, 50, prec, explicit=explicit)


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_quadratic_high_boost_small(O, prec):
    # a strong drive (a0 = 20): relative electron positions are selected
    # automatically at this boost
    sim, o = _c3_small_window(O, 20.0, prec, False)
    err = vector_errors(sim, o)
    assert max(err.values()) < TOL50[prec], err
    wake = field_errors(sim, o, ("Ex", "Ez", "By"))
    assert max(wake.values()) < TOL_WAKE[prec], wake


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("explicit", [False, True])
def test_c3_stage_a0_1_5(O, explicit, prec):
    # the gamma = 130 stage at its own drive (a0 = 1.5) on the 4x coarser grid:
    # the plasma's wake current is ~3e-8 of either species' current in this
    # frame; with electrons in relative form and the currents formed in FP64,
    # FP32 meets the same bar as everywhere else, and the wake fields (Ex, Ez,
    # By: about a thousandth of the laser's) are checked on their own
    sim, o = _c3_small_window(O, 1.5, prec, explicit)
    err = vector_errors(sim, o)
    assert max(err.values()) < TOL50[prec], err
    wake = field_errors(sim, o, ("Ex", "Ez"))
    assert np.abs(o.field("Ez")).max() > 1e-3 * np.abs(o.field("Ey")).max()  # a wake is there
    assert max(wake.values()) < TOL_WAKE[prec] * (10 if prec == FP32 else 1), wake


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_c3_stage_absolute_positions_fall_short(O, prec):
    # the same window with absolute FP32 offsets and FP32 currents (z_relative
    # = 2): the wake drowns in rounding (measured: E as a vector 1e-3, Ez on
    # its own ~70%); FP64 is unaffected
    g = dict(dim=2, nx=32, nz=200, dx=4.0, dz=4 / 32, gamma_boost=130.0, shape_order=2, filter_passes=4, seed=23)
    beta = math.sqrt(1 - 1 / 130.0 ** 2)
    hz = (4 / 32) * 130 * (1 + beta)
    p = dict(ne=5.7e-5, z_start=130 * 3 * hz, z_end=130 * 400 * hz, ramp=5.0, ppc=(2, 1, 2), jitter=0.1, ions=1)
    laser = dict(a0=1.5, waist=20.0, fwhm=4.0, t_peak=0.2)
    sim, o = _run_steps_parity(O, g, p, laser, 50, prec, rel=2)
    err = vector_errors(sim, o)
    if prec == FP64:
        assert max(err.values()) < TOL50[prec], err
    else:
        assert err["E"] > 1e-4, err  # the reason the relative form exists


def test_c2_slab_at_bench_settings(O):
    # the benchmarked 3D gamma = 13 stage (256 x 256 x 1024 in the bench) on a
    # 32 x 32 x 64 slab with the bench's own settings: FP32, 10 slots per
    # cell, electron-ion pairs, the stage's plasma (filling the box and
    # streaming in) and laser (a0 = 1, waist 20, FWHM 10), its peak emitted
    # early so that it drives the plasma within the window; compared after 40
    # and after 60 steps, the wake field Ez also on its own
    st = W.stage("c2")
    g = dict(st.grid, nx=32, ny=32, nz=64)
    laser = dict(st.laser, t_peak=1.0)
    sim, o = make_pair(O, g, FP32, slots_per_cell=10.0)
    _plasma_both(sim, o, O, st.plasma)
    sim.launch_laser(laser["a0"], laser["waist"], laser["fwhm"], 0.0, laser["t_peak"], laser["pol"])
    o.set_laser(O.LaserParams(a0=laser["a0"], waist=laser["waist"], fwhm=laser["fwhm"], z_antenna=0.0,
                              t_peak=laser["t_peak"], pol=laser["pol"]))
    for nsteps in (40, 20):
        sim.step(nsteps)
        o.step(nsteps)
        err = vector_errors(sim, o)
        assert max(err.values()) < TOL50[FP32], err
        assert field_errors(sim, o, ("Ez",))["Ez"] < TOL50[FP32]
    assert np.abs(o.field("Ez")).max() > 1e-3
    d = sim.diagnostics()
    assert d.n_particles[0] == o.num(0) and d.n_particles[1] == o.num(1)
    assert 0 < d.n_paired < d.n_particles[0]


class _FieldView:  # oracle-shaped view of GPU fields for the residual helpers
    def __init__(self, f, hx, hy, hz):
        self.f, self.hx, self.hy, self.hz = f, hx, hy, hz

    def field(self, c):
        return self.f[c]


def _residual(sim, o, dim, npass, bc_z):
    """div E - 2 pi F(rho) on the GPU's state, planes 6..nz-6 (away from the
    antenna sheet, the Mur ends and the plasma entering through z = Lz)"""
    from test_oracle_physics import _div_e, _filtered
    f = {c: t.double().cpu().numpy() for c, t in sim.fields().items()}
    rho = sim.rho().double().cpu().numpy()
    v = _FieldView(f, o.hx, o.hy, o.hz)
    return _div_e(v, dim)[6:-6] - 2 * math.pi * _filtered(rho, npass, dim, bc_z)[6:-6]


def test_continuity_residual_fp32(O):
    # div E - 2 pi F(rho) stays constant; F = the same binomial passes on rho
    from test_oracle_physics import _filtered
    g = dict(dim=2, nx=32, nz=96, dx=0.5, dz=0.125, filter_passes=2, seed=29)
    sim, o = make_pair(O, g, FP32)
    st = W.random_particles(20000, (o.Lx, 1.0, 7.0), seed=30, u_scale=0.3)
    st[2] += 2.5
    st[6] = 0.02 * o.hx * o.hz / 4
    sim.load_particles(0, st, np.arange(st.shape[1]))
    r0 = _residual(sim, o, 2, 2, 1)
    rho0 = sim.rho().double().cpu().numpy()
    sim.step(30)
    r1 = _residual(sim, o, 2, 2, 1)
    scale = 2 * math.pi * np.abs(_filtered(rho0, 2, 2, 1)).max()
    assert np.abs(r1 - r0).max() < 1e-5 * scale, np.abs(r1 - r0).max() / scale


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("dim,shape,explicit,rel", [(2, 1, False, 0), (2, 2, False, 0), (2, 1, True, 0),
                                                    (3, 1, False, 0), (3, 1, True, 0), (3, 2, False, 0),
                                                    (2, 2, False, 1), (3, 1, False, 1)])
def test_continuity_residual_boosted(O, dim, shape, explicit, rel, prec):
    # the boosted frame (gamma = 13): plasma loaded and injected with drifting
    # ions (paired or explicit records), a laser releasing pairs, CIC and
    # quadratic shapes, 2D and 3D, absolute and relative electron positions:
    # the residual's change over 30 steps, relative to the plasma's charge
    # density 2 pi gamma n, stays at round-off (1e-5 FP32, 1e-13 FP64)
    gam = 13.0
    beta = math.sqrt(1 - 1 / gam ** 2)
    dzl = 1 / 32
    hz = dzl * gam * (1 + beta)
    if dim == 2:
        g = dict(dim=2, nx=32, nz=96, dx=1.0, dz=dzl, gamma_boost=gam, filter_passes=2, shape_order=shape, seed=41)
        laser = dict(a0=4.0, waist=8.0, fwhm=2.0, t_peak=0.5, pol=1)
    else:
        g = dict(dim=3, nx=16, ny=16, nz=48, dx=1.0, dy=1.0, dz=dzl, gamma_boost=gam, filter_passes=2,
                 shape_order=shape, seed=42)
        laser = dict(a0=4.0, waist=4.0, fwhm=2.0, t_peak=0.5, pol=0)
    ne = 0.004
    p = dict(ne=ne, z_start=gam * 8 * hz, z_end=gam * 2000 * hz, ramp=0.0, ppc=(2, 2, 2) if dim == 3 else (2, 1, 2),
             jitter=0.1, ions=1)
    sim, o = make_pair(O, g, prec, explicit_ions=explicit, z_relative=rel)
    _plasma_both(sim, o, O, p)
    sim.launch_laser(laser["a0"], laser["waist"], laser["fwhm"], 0.0, laser["t_peak"], laser["pol"])
    sim.step(5)
    r0 = _residual(sim, o, dim, 2, 1)
    sim.step(30)
    r1 = _residual(sim, o, dim, 2, 1)
    d = sim.diagnostics()
    assert d.n_particles[0] > 1000
    if not explicit:
        assert d.n_paired < d.n_particles[0]  # the laser released pairs
    scale = 2 * math.pi * gam * ne
    tol = 1e-5 if prec == FP32 else 1e-13
    assert np.abs(r1 - r0).max() < tol * scale, np.abs(r1 - r0).max() / scale


def test_capacity_overflow_is_reported(O):
    import paper_1011_0917_gb300 as P
    g = dict(dim=2, nx=16, nz=32, dx=0.5, dz=0.125, seed=3)
    sim, o = make_pair(O, g, FP32, slots_per_cell=0.05)
    with pytest.raises(P.PicError) as e:
        sim.load_plasma(0.01, 0.0, 4.0, 0.0, (4, 1, 4), 0.1, (), 1)
    assert e.value.status == P.PIC_ERR_CAPACITY


@pytest.mark.parametrize("on_device,rel", [(False, 0), (True, 0), (True, 1)])
def test_state_roundtrip(O, on_device, rel):
    import torch
    import paper_1011_0917_gb300 as P
    g = dict(dim=2, nx=32, nz=256, dx=1.0, dz=1 / 32, gamma_boost=13.0, filter_passes=2, seed=17)
    p = dict(ne=0.001, z_start=13 * 30 * 0.81, z_end=13 * 600 * 0.81, ramp=2.0, ppc=(2, 1, 2), jitter=0.1, ions=1)
    laser = dict(a0=2.0, waist=8.0, fwhm=2.0, t_peak=0.5)
    sim, _ = _run_steps_parity(O, g, p, laser, 20, FP64, rel=rel)
    nb = P.pic_state_bytes(sim.ctx)
    buf = torch.empty(nb, dtype=torch.uint8, device="cuda" if on_device else "cpu")
    P.pic_get_state(sim.ctx, buf.data_ptr(), nb, on_device)
    sim2, _ = make_pair(O, g, FP64, z_relative=rel)
    sim2.load_plasma(p["ne"], p["z_start"], p["z_end"], p["ramp"], p["ppc"], p["jitter"], (), 1)
    P.pic_set_state(sim2.ctx, buf.data_ptr(), nb, on_device)
    sim.step(10)
    sim2.step(10)
    a, b = sim.fields(), sim2.fields()
    for c in COMPONENTS[:6]:
        den = max(float(a[c].abs().max()), 1e-30)
        assert float((a[c] - b[c]).abs().max()) / den < 1e-12, c
    assert sim.diagnostics().n_particles[0] == sim2.diagnostics().n_particles[0]
