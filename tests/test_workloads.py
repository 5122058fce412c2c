"""The seeded workload recipes hold the stage parameters the benchmark and the
parity tests are quoted on (grid, boost, shape, filter passes, plasma, laser,
step counts) and are deterministic: the same run index gives the same run."""
import math

import pytest

from paper_1011_0917_gb300 import workloads as W


def test_lab_stage_c0():
    st = W.stage("c0")
    g, p, l = st.grid, st.plasma, st.laser
    assert (g["dim"], g["nx"], g["nz"], g["dx"], g["dz"]) == (2, 64, 512, 0.5, 1 / 16)
    assert (g["cfl"], g["gamma_boost"], g["shape_order"], g["filter_passes"]) == (0.99, 1.0, 1, 1)
    assert (p["ne"], p["z_start"], p["z_end"], p["ramp"], p["ppc"], p["jitter"]) == (0.01, 4.0, 32.0, 2.0,
                                                                                       (2, 1, 2), 0.1)
    assert (l["a0"], l["waist"], l["fwhm"]) == (1.0, 8.0, 5.0) and st.steps == 512


def test_boosted_stages_c1_c2():
    c1, c2 = W.stage("c1"), W.stage("c2")
    for st in (c1, c2):
        g, p, l = st.grid, st.plasma, st.laser
        assert g["gamma_boost"] == 13.0 and g["filter_passes"] == 2 and g["shape_order"] == 1
        assert g["dz"] == 1 / 32 and g["dx"] == 1.0 and p["ne"] == 0.001
        assert (l["a0"], l["waist"], l["fwhm"]) == (1.0, 20.0, 10.0)
    assert (c1.grid["nx"], c1.grid["nz"]) == (256, 8192)
    assert c1.plasma["z_end"] - c1.plasma["z_start"] == 2000.0
    assert (c2.grid["dim"], c2.grid["nx"], c2.grid["ny"], c2.grid["nz"]) == (3, 256, 256, 1024)
    assert c2.plasma["ppc"] == (2, 2, 2) and c2.steps == 1000
    # c2_small is the same stage on a smaller box
    s = W.stage("c2_small")
    assert (s.grid["nx"], s.grid["ny"], s.grid["nz"]) == (128, 128, 256)
    assert {k: v for k, v in s.grid.items() if k not in ("nx", "ny", "nz")} == \
        {k: v for k, v in c2.grid.items() if k not in ("nx", "ny", "nz")}


def test_high_boost_stage_c3():
    st = W.stage("c3")
    g, p, l = st.grid, st.plasma, st.laser
    assert (g["gamma_boost"], g["nx"], g["nz"], g["shape_order"], g["filter_passes"]) == (130.0, 512, 16384, 2, 4)
    assert (p["ne"], p["ramp"]) == (5.7e-5, 5.0)
    assert (l["a0"], l["waist"], l["fwhm"]) == (1.5, 50.0, 30.0)
    small = W.stage("c3_small")
    assert (small.grid["nx"] * 4, small.grid["nz"] * 4) == (g["nx"], g["nz"])


@pytest.mark.parametrize("r", range(64))
def test_scan_run_c4(r):
    st = W.c4_run(r)
    g, p, l = st.grid, st.plasma, st.laser
    assert g["gamma_boost"] in (5.0, 13.0, 30.0)
    assert 1024 <= g["nz"] <= 4096 and g["nx"] == 128 and p["ppc"] == (2, 1, 2)
    assert len(p["profile"]) == 8 and sum(abs(c) for c in p["profile"]) <= 0.2 + 1e-12
    assert 0.5 <= l["a0"] <= 2.0 and st.steps == 400 and g["filter_passes"] == 2
    # the plasma starts 10 boosted cells ahead of the antenna
    gam = g["gamma_boost"]
    hz = g["dz"] * gam * (1 + math.sqrt(1 - 1 / gam ** 2))
    assert math.isclose(p["z_start"], gam * 10 * hz)
    again = W.c4_run(r)
    assert (again.grid, again.plasma, again.laser) == (g, p, l)


def test_scan_mixes_boosts_and_lengths():
    runs = [W.c4_run(r) for r in range(64)]
    assert {st.grid["gamma_boost"] for st in runs} == {5.0, 13.0, 30.0}
    assert len({st.grid["nz"] for st in runs}) > 32
    assert len({st.grid["seed"] for st in runs}) == 64
