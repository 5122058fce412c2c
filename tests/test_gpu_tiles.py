"""The tile-shape variants of the particle kernels (2D: 16 x 16, 32 x 8, 8 x 32
cells; 3D: 8 x 8 x 8, 8 x 8 x 4) against the FP64 oracle, and the autotuners
that pick among them and among the batch's launch forms.

The tile shape changes only how particles are grouped for staging, deposit
and re-bucketing, so every variant must match the oracle to the full-step
tolerances (relative L2 1e-4 FP32, 1e-10 FP64) on the boosted 2D stage with
plasma streaming in and a laser meeting it."""
import math

import pytest

from pairs import make_pair, vector_errors

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1
TOL = {FP32: 1e-4, FP64: 1e-10}
GAM = 13.0
BETA = math.sqrt(1 - 1 / GAM ** 2)
HZ = (1 / 32) * GAM * (1 + BETA)
G = dict(dim=2, nx=32, nz=256, dx=1.0, dz=1 / 32, gamma_boost=GAM, filter_passes=2, seed=17)
PLASMA = dict(ne=0.004, z_start=GAM * 10 * HZ, z_end=GAM * 600 * HZ, ramp=2.0, ppc=(2, 1, 2), jitter=0.1, ions=1)
LASER = dict(a0=4.0, waist=8.0, fwhm=2.0, t_peak=0.5)


@pytest.fixture(scope="module")
def O():
    import oracle.oracle as O
    O.build_oracle()
    return O


@pytest.mark.parametrize("tile", [(32, 1, 8), (8, 1, 32)])
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_tile_variant_matches_oracle(O, prec, tile):
    sim, o = make_pair(O, G, prec, tile=tile)
    assert tuple(sim.sizes.tile) == tile
    p = PLASMA
    sim.load_plasma(p["ne"], p["z_start"], p["z_end"], p["ramp"], p["ppc"], p["jitter"], (), p["ions"])
    o.load_plasma(O.PlasmaParams(ne=p["ne"], z_start=p["z_start"], z_end=p["z_end"], ramp=p["ramp"], ppc=p["ppc"],
                                 jitter=p["jitter"], ions=p["ions"]))
    sim.launch_laser(LASER["a0"], LASER["waist"], LASER["fwhm"], 0.0, LASER["t_peak"], 1)
    o.set_laser(O.LaserParams(a0=LASER["a0"], waist=LASER["waist"], fwhm=LASER["fwhm"], t_peak=LASER["t_peak"],
                              pol=1))
    sim.step(50)
    o.step(50)
    err = vector_errors(sim, o)
    assert max(err.values()) < TOL[prec], err
    d = sim.diagnostics()
    assert d.n_particles[0] == o.num(0) and d.n_particles[1] == o.num(1)


def test_autotune_picks_a_compiled_configuration():
    from paper_1011_0917_gb300 import autotune
    settings = {"grid": dict(G, precision=FP32), "plasma": PLASMA, "laser": dict(LASER, pol=1)}
    best = autotune.tune_run(settings, steps=4, warmup=2)
    assert best["tile"] in autotune.TILES_2D and best["slots_per_cell"] in autotune.SLOTS
    assert len(best["trials"]) == len(autotune.TILES_2D) * len(autotune.SLOTS)
    assert best["ms_per_step"] == min(t["ms_per_step"] for t in best["trials"] if "ms_per_step" in t)


def test_autotune_batch_tries_every_launch_form():
    """The batch autotuner times the stream path and, per graph length, the
    per-context graph and the fused graph with 1 and 2 launch chains, and
    returns the fastest."""
    from paper_1011_0917_gb300 import autotune
    runs = [{"grid": dict(G, precision=FP32, seed=17 + r), "plasma": PLASMA, "laser": dict(LASER, pol=1)}
            for r in range(3)]
    best = autotune.tune_batch(runs, steps=10, warmup=2, graph_steps=(10,), chains=(0, 1, 2))
    forms = {(t["graph_steps"], t["chains"]) for t in best["trials"]}
    assert forms == {(0, 0), (10, 0), (10, 1), (10, 2)}, best["trials"]
    assert best["ms_per_step"] == min(t["ms_per_step"] for t in best["trials"])


def test_autotune_tries_the_cell_sort_interval():
    from paper_1011_0917_gb300 import autotune
    settings = {"grid": dict(G, precision=FP32), "plasma": PLASMA, "laser": dict(LASER, pol=1)}
    best = autotune.tune_run(settings, steps=4, warmup=2, tiles=((16, 1, 16),), slots=(8.0,), sort_every=(0, 2))
    assert {t["sort_every"] for t in best["trials"]} == {0, 2}
    assert best["sort_every"] in (0, 2) and all("ms_per_step" in t for t in best["trials"])


G3 = dict(dim=3, nx=16, ny=16, nz=48, dx=1.0, dy=1.0, dz=1 / 32, gamma_boost=GAM, filter_passes=2, seed=19)
PLASMA3 = dict(ne=0.004, z_start=GAM * 6 * HZ, z_end=GAM * 200 * HZ, ramp=2.0, ppc=(2, 2, 2), jitter=0.1, ions=1)


@pytest.mark.parametrize("explicit", [False, True])
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_3d_tile_variant_matches_oracle(O, prec, explicit):
    """The 8 x 8 x 4 tile of the 3D CIC kernels against the oracle (30 steps,
    the laser in the plasma, both ion modes)."""
    sim, o = make_pair(O, G3, prec, tile=(8, 8, 4), explicit_ions=explicit)
    assert tuple(sim.sizes.tile) == (8, 8, 4)
    p = PLASMA3
    sim.load_plasma(p["ne"], p["z_start"], p["z_end"], p["ramp"], p["ppc"], p["jitter"], (), p["ions"])
    o.load_plasma(O.PlasmaParams(ne=p["ne"], z_start=p["z_start"], z_end=p["z_end"], ramp=p["ramp"], ppc=p["ppc"],
                                 jitter=p["jitter"], ions=p["ions"]))
    sim.launch_laser(LASER["a0"], 4.0, LASER["fwhm"], 0.0, LASER["t_peak"], 1)
    o.set_laser(O.LaserParams(a0=LASER["a0"], waist=4.0, fwhm=LASER["fwhm"], t_peak=LASER["t_peak"], pol=1))
    sim.step(30)
    o.step(30)
    err = vector_errors(sim, o)
    assert max(err.values()) < TOL[prec], err
    d = sim.diagnostics()
    assert d.n_particles[0] == o.num(0) and d.n_particles[1] == o.num(1)
