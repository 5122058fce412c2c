"""Free electrons in a boosted frame, against the closed form.

A field-free particle moves with constant velocity: after N steps it has
moved by N dt v, v = u / sqrt(1 + u^2).  In the boosted frame every plasma
electron starts at the drift momentum u_d = (0, 0, -gamma beta) and its
response to the fields is a small change du, which moves v_z by only
~du / gamma^3.  What the fields see is the electron's displacement relative to
its ion, which moves with the drift: so each electron here is loaded with an
ion at the same point, and the electron-ion separation after N steps is held
against N dt (v - v_d).  (Zero weights: no current, no field, so the
momenta stay as loaded.)  An error in the drift-relative
velocity (a dropped term, a wrong sign) shows at once in FP64; FP32 with
absolute in-cell offsets is held to their rounding bound, and FP32 with
relative positions (the departure from the reference path in its own word)
to the relative precision of the departure itself.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1

# du of each electron (x, y, z); the ion of each sits at the same point
DU = [(0.0, 0.0, 1e-3), (0.0, 0.0, -1e-3), (0.0, 0.0, 3e-3), (0.0, 0.0, 1e-2), (0.02, 0.0, 2e-3),
      (-0.01, 0.005, -5e-3), (0.0, 0.0, 0.0), (0.0, 0.0, 2e-2)]


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("rel", [2, 1])
def test_separation_from_the_drift(prec, rel):
    import paper_1011_0917_gb300 as P
    gam = 13.0
    sim = P.Simulation(dim=2, nx=16, nz=512, dx=1.0, dz=1 / 32, gamma_boost=gam, filter_passes=1,
                       precision=prec, track_ids=True, explicit_ions=True, slots_per_cell=4.0, z_relative=rel)
    beta = math.sqrt(1 - 1 / gam ** 2)
    # the drift as the working precision holds it (the ions move with it)
    U = -gam * beta if prec == FP64 else float(np.float32(-gam * beta))
    hz = sim.sizes.hz
    n = len(DU)
    x0 = 3.3 + np.arange(n) * 1.37
    z0 = hz * (480.0 + 0.37 * np.arange(n))
    e = np.zeros((7, n))
    e[0], e[2], e[6] = x0, z0, 0.0
    for i, (ux, uy, duz) in enumerate(DU):
        e[3, i], e[4, i], e[5, i] = ux, uy, U + duz
    ions = np.zeros((7, n))
    ions[0], ions[2], ions[5], ions[6] = x0, z0, U, 0.0
    ids = np.arange(n, dtype=np.int64)
    sim.load_particles(0, e, ids)
    sim.load_particles(1, ions, ids)
    nsteps = 400
    sim.step(nsteps)
    (pe, ie), (pi, ii) = sim.particles(0, True), sim.particles(1, True)
    pe, pi = pe[:, np.argsort(ie)], pi[:, np.argsort(ii)]
    assert pe.shape[1] == n and pi.shape[1] == n
    T = nsteps * sim.dt
    assert pi[5, 0] == U
    vd = U / math.sqrt(1 + U * U)
    for i in range(n):
        u = pe[3:6, i]
        g = math.sqrt(1 + float(u @ u))
        dz_exact = T * (u[2] / g - vd)
        dx_exact = T * u[0] / g
        dz, dx = pe[2, i] - pi[2, i], pe[0, i] - pi[0, i]
        if DU[i] == (0.0, 0.0, 0.0):
            # an electron at the drift momentum stays on its ion, bit for bit
            assert dz == 0.0 and dx == 0.0
            continue
        # the position update rounds twice per step (the drift's displacement,
        # then the departure from it), each by at most half an ulp of an
        # in-cell offset: 2^-24 cell per step bounds the error (FP32; the
        # rounding is systematic for a constant velocity, so the bound is
        # linear in the steps).  FP64 resolves the formula itself.
        # Relative positions: the electron's reference is its ion's path, so
        # the separation is the departure alone, summed in its own FP32 word
        # (at most ~ulp of the sum per step: 400 x 6e-8 relative).
        if prec == FP64:
            bound = 1e-9 * abs(dz_exact)
        elif rel == 1:
            bound = 4e-5 * abs(dz_exact)
        else:
            bound = nsteps * 2.0 ** -24 * hz + 1e-6 * abs(dz_exact)
        assert abs(dz - dz_exact) <= bound, (i, dz, dz_exact)
        if DU[i][0] != 0.0:  # one rounding of the offset per step (hx = 1)
            if prec == FP64:
                bx = 1e-9 * abs(dx_exact)
            elif rel == 1:
                bx = 4e-5 * abs(dx_exact)
            else:
                bx = nsteps * 2.0 ** -25 + 1e-6 * abs(dx_exact)
            assert abs(dx - dx_exact) <= bx, (i, dx, dx_exact)
    sim.close()
