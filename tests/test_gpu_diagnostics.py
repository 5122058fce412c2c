"""The FP64 Kahan-compensated diagnostics (field energy, electron kinetic
energy, charge) and the lab-frame view of the fields, through the C ABI,
against the oracle on the same seeded inputs.

Tolerances: FP64 build 1e-10 relative (the sums are taken in different
orders on the two sides); FP32 build: the state itself differs from the FP64
oracle by the run's rounding, so the field energy (a quadratic form of fields
held to 1e-4 relative L2) is held to 2e-4, the kinetic energy and the charge
(weights and momenta in FP32) to 1e-6.  The lab-frame view is compared on
identical fields (set on both sides), so it checks the transformation alone:
1e-13 in FP64, 2e-6 in FP32 (the FP32 inputs are the FP64 values rounded).
"""
import math

import numpy as np
import pytest

from pairs import make_pair, set_fields_both
from paper_1011_0917_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1
TOL_FE = {FP32: 2e-4, FP64: 1e-10}
TOL_KQ = {FP32: 1e-6, FP64: 1e-10}


@pytest.fixture(scope="module")
def O():
    import oracle.oracle as O
    O.build_oracle()
    return O


def _stage(O, sim, o, p, laser):
    sim.load_plasma(p["ne"], p["z_start"], p["z_end"], p["ramp"], p["ppc"], p["jitter"], (), p["ions"])
    o.load_plasma(O.PlasmaParams(ne=p["ne"], z_start=p["z_start"], z_end=p["z_end"], ramp=p["ramp"], ppc=p["ppc"],
                                 jitter=p["jitter"], ions=p["ions"]))
    sim.launch_laser(laser["a0"], laser["waist"], laser["fwhm"], 0.0, laser.get("t_peak", -1.0), laser.get("pol", 1))
    o.set_laser(O.LaserParams(a0=laser["a0"], waist=laser["waist"], fwhm=laser["fwhm"], z_antenna=0.0,
                              t_peak=laser.get("t_peak", -1.0), pol=laser.get("pol", 1)))


def _compare(sim, o, prec, n_charge_scale):
    d = sim.diagnostics()
    ref = o.diagnostics()
    assert ref["field_energy"] > 0 and ref["kinetic_energy"] > 0
    fe = abs(d.field_energy - ref["field_energy"]) / ref["field_energy"]
    ke = abs(d.kinetic_energy - ref["kinetic_energy"]) / ref["kinetic_energy"]
    q = abs(d.charge - ref["charge"]) / n_charge_scale
    # (the measured errors, for the record: pytest -s shows them)
    print(f"diagnostics vs oracle ({'FP64' if prec == FP64 else 'FP32'}): field energy {fe:.2e}, "
          f"kinetic energy {ke:.2e}, charge {q:.2e}")
    assert fe < TOL_FE[prec] and ke < TOL_KQ[prec] and q < TOL_KQ[prec], (fe, ke, q, d.field_energy, ref)
    return fe, ke, q


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("case,explicit", [("lab2d", False), ("boost2d", False), ("boost2d", True),
                                           ("boost3d", False), ("c3", False)])
def test_diagnostics_match_oracle(O, case, explicit, prec):
    if case == "lab2d":
        st = W.stage("c0")
        g, p, laser, n = dict(st.grid, nz=256), dict(st.plasma, z_start=2.0), dict(st.laser, t_peak=1.0), 60
    elif case == "boost2d":
        g = dict(dim=2, nx=32, nz=256, dx=1.0, dz=1 / 32, gamma_boost=13.0, filter_passes=2, seed=17)
        hz = (1 / 32) * 13 * (1 + math.sqrt(1 - 1 / 169.0))
        p = dict(ne=0.004, z_start=13 * 10 * hz, z_end=13 * 600 * hz, ramp=2.0, ppc=(2, 1, 2), jitter=0.1, ions=1)
        laser, n = dict(a0=4.0, waist=8.0, fwhm=2.0, t_peak=0.5), 40
    elif case == "boost3d":
        g = dict(dim=3, nx=16, ny=16, nz=48, dx=1.0, dy=1.0, dz=1 / 32, gamma_boost=13.0, filter_passes=2, seed=19)
        hz = (1 / 32) * 13 * (1 + math.sqrt(1 - 1 / 169.0))
        p = dict(ne=0.004, z_start=13 * 6 * hz, z_end=13 * 200 * hz, ramp=2.0, ppc=(2, 2, 2), jitter=0.1, ions=1)
        laser, n = dict(a0=4.0, waist=4.0, fwhm=2.0, t_peak=0.5), 30
    else:  # the gamma = 130 stage on its 4x coarser grid (relative electron positions)
        g = dict(dim=2, nx=32, nz=200, dx=4.0, dz=4 / 32, gamma_boost=130.0, shape_order=2, filter_passes=4,
                 seed=23)
        hz = (4 / 32) * 130 * (1 + math.sqrt(1 - 1 / 130.0 ** 2))
        p = dict(ne=5.7e-5, z_start=130 * 3 * hz, z_end=130 * 400 * hz, ramp=5.0, ppc=(2, 1, 2), jitter=0.1, ions=1)
        laser, n = dict(a0=1.5, waist=20.0, fwhm=4.0, t_peak=0.2), 50
    sim, o = make_pair(O, g, prec, explicit_ions=explicit)
    _stage(O, sim, o, p, laser)
    sim.step(n)
    o.step(n)
    # the charge is compared against the electrons' own total |q w|
    scale = float(np.sum(o.particles(0)["w"]))
    _compare(sim, o, prec, scale)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("dim,gam,bc", [(2, 13.0, 1), (3, 5.0, 1), (2, 130.0, 0), (3, 1.0, 1)])
def test_lab_frame_fields_match_oracle(O, dim, gam, bc, prec):
    if dim == 2:
        g = dict(dim=2, nx=24, nz=40, dx=0.5, dz=0.125, gamma_boost=gam, bc_z=bc, seed=7)
        shape = (41, 1, 24)
    else:
        g = dict(dim=3, nx=12, ny=10, nz=20, dx=0.5, dy=0.6, dz=0.25, gamma_boost=gam, bc_z=bc, seed=8)
        shape = (21, 10, 12)
    sim, o = make_pair(O, g, prec)
    set_fields_both(sim, o, W.random_fields(shape, seed=71, scale=0.3), bc)
    lab = {c: t.double().cpu().numpy() for c, t in sim.fields(0x3F, frame=1).items()}
    ref = o.fields_lab()
    tol = 1e-13 if prec == FP64 else 2e-6
    for c, v in ref.items():
        m = np.abs(v).max()
        assert np.abs(lab[c] - v).max() <= tol * m, (c, np.abs(lab[c] - v).max() / m)
    if gam == 1.0:
        boost = {c: t.double().cpu().numpy() for c, t in sim.fields(0x3F, frame=0).items()}
        for c in ref:
            assert np.array_equal(lab[c], boost[c])


def test_lab_frame_rejects_currents(O):
    import paper_1011_0917_gb300 as P
    sim, _ = make_pair(O, dict(dim=2, nx=16, nz=32, dx=0.5, dz=0.125, gamma_boost=5.0), FP32)
    with pytest.raises(P.PicError) as e:
        sim.fields(0x1FF, frame=1)
    assert e.value.status == P.PIC_ERR_ARG
    with pytest.raises(P.PicError):
        sim.fields(0x3F, frame=2)
