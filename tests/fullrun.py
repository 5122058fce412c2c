"""Outcomes of a whole stage run, computed the same way from the GPU's and the
oracle's state (test infrastructure).

Over a full stage, particle trajectories are chaotic and cannot be compared
one by one; the stage is compared through its physical outcomes:
* peak_ez: the largest |E_z| on the axis line (i = nx/2) over the run,
  sampled every `sample` steps; E_z is unchanged by the boost along z, so this
  is the lab-frame peak wake field as well;
* plasma_energy: the energy the plasma electrons hold above the drift at the
  end, sum w (gamma(u) - gamma(U)) with U the plasma's drift momentum (0 in
  the lab frame, -gamma beta boosted) as each side holds it: an electron no
  field has touched contributes exactly zero.  The laser's energy and
  propagation distance being the same on both sides, this fixes the depletion
  length, which is inversely proportional to it.
"""
from __future__ import annotations

import numpy as np


def gamma_excess(ux, uy, uz, U: float) -> np.ndarray:
    """gamma(u) - gamma((0, 0, U)) without cancellation."""
    ux, uy, uz = (np.asarray(a, dtype=np.float64) for a in (ux, uy, uz))
    num = (uz - U) * (uz + U) + ux * ux + uy * uy
    return num / (np.sqrt(1.0 + ux * ux + uy * uy + uz * uz) + np.sqrt(1.0 + U * U))


def growth_rate(steps, values, lo: float = 1e-7, hi: float = 1e-5):
    """Exponential growth rate per step of a sampled amplitude over the samples
    in (lo, hi) (least-squares slope of its logarithm), and the number of
    samples used.  The on-axis Ez of the gamma = 130 stage holds only
    round-off until the numerical instability of the streaming plasma sets
    in; once its fastest mode dominates (the default window: two decades
    below saturation, well above either side's round-off) the rate of growth
    is a property of the discrete scheme, not of the round-off that seeds it."""
    s = np.asarray(steps, dtype=np.float64)
    v = np.asarray(values, dtype=np.float64)
    m = (v > lo) & (v < hi)
    if m.sum() < 3:
        return float("nan"), int(m.sum())
    slope = np.polyfit(s[m], np.log(v[m]), 1)[0]
    return float(slope), int(m.sum())


def plasma_energy(w, ux, uy, uz, U: float) -> float:
    return float(np.sum(np.asarray(w, dtype=np.float64) * gamma_excess(ux, uy, uz, U)))


def stage_objects(O, name: str):
    """Oracle grid/plasma/laser of a stage of the workload recipes."""
    from paper_1011_0917_gb300 import workloads as W
    st = W.stage(name)
    g = st.grid
    grid = O.GridParams(dim=g["dim"], nx=g["nx"], ny=g.get("ny", 1), nz=g["nz"], dx=g["dx"], dy=g.get("dy", 1.0),
                        dz=g["dz"], cfl=g["cfl"], gamma_boost=g["gamma_boost"], shape=g["shape_order"],
                        npass=g["filter_passes"], bc_z=g["bc_z"], seed=g["seed"])
    p = st.plasma
    plasma = O.PlasmaParams(ne=p["ne"], z_start=p["z_start"], z_end=p["z_end"], ramp=p["ramp"], ppc=p["ppc"],
                            jitter=p["jitter"], ions=p["ions"])
    l = st.laser
    laser = O.LaserParams(a0=l["a0"], waist=l["waist"], fwhm=l["fwhm"], z_antenna=l["z_antenna"], pol=l["pol"])
    return st, grid, plasma, laser
