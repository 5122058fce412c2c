"""Writes tests/golden/full_runs.json: the outcomes (tests/fullrun.py) of the
FP64 oracle's whole runs of the c1 stage (gamma = 13, 2D3V, 256 x 8192, until
the pulse peak has crossed the 2000 lambda0 plasma) and of the c3 stage on
its 4x coarser grid (gamma = 130, 128 x 4096, quadratic shape, 4 passes, 6500
steps), with the history of the peak on-axis E_z and the growth rate of the
numerical instability that sets it at gamma = 130.  It calls only the oracle
and the workload recipes; each run takes tens of minutes on one core.

    python tests/golden/make_full_runs.py [c1] [c3_small]
    python tests/golden/make_full_runs.py --rates-only   (rates from the stored histories)
"""
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import fullrun  # noqa: E402
import oracle.oracle as O  # noqa: E402

SAMPLE = 20


def run(name: str) -> dict:
    st, grid, plasma, laser = fullrun.stage_objects(O, name)
    o = O.Oracle(grid)
    o.load_plasma(plasma)
    o.set_laser(laser)
    nx = grid.nx
    jc = (grid.ny if grid.dim == 3 else 1) // 2
    peak, peak_step = 0.0, 0
    hist_steps, hist_ez = [], []
    t0 = time.time()
    for s in range(st.steps // SAMPLE):
        o.step(SAMPLE)
        ez = float(np.abs(o.field("Ez")[:, jc, nx // 2]).max())
        hist_steps.append((s + 1) * SAMPLE)
        hist_ez.append(ez)
        if ez > peak:
            peak, peak_step = ez, (s + 1) * SAMPLE
    U = -(grid.gamma_boost * o.beta)
    p = o.particles(0)
    rate, used = fullrun.growth_rate(hist_steps, hist_ez)
    return {"steps": st.steps, "sample": SAMPLE, "peak_ez": peak, "peak_step": peak_step,
            "plasma_energy": fullrun.plasma_energy(p["w"], p["ux"], p["uy"], p["uz"], U),
            "ez_growth_rate": rate, "ez_growth_samples": used, "ez_history": hist_ez,
            "electrons_end": o.num(0), "ions_end": o.num(1), "seconds": round(time.time() - t0, 1),
            "host": platform.machine()}


def rates_only(path):
    """Recompute the growth rates from the stored oracle histories (after a
    change of the fit window; no oracle run)."""
    out = json.load(open(path))
    for name, res in out.items():
        if isinstance(res, dict) and "ez_history" in res:
            steps = [(i + 1) * res["sample"] for i in range(len(res["ez_history"]))]
            res["ez_growth_rate"], res["ez_growth_samples"] = fullrun.growth_rate(steps, res["ez_history"])
            print(name, res["ez_growth_rate"], res["ez_growth_samples"])
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


def main():
    names = sys.argv[1:] or ["c1", "c3_small"]
    path = os.path.join(HERE, "full_runs.json")
    if names == ["--rates-only"]:
        rates_only(path)
        return
    O.build_oracle()
    for name in names:
        res = run(name)
        # read the file again just before writing: other stages' entries
        # may have been written meanwhile
        out = json.load(open(path)) if os.path.exists(path) else {}
        out[name] = res
        out["_note"] = ("outcomes of whole runs of the FP64 oracle (tests/fullrun.py), written by "
                        "tests/golden/make_full_runs.py")
        with open(path, "w") as f:
            json.dump(out, f, indent=1, sort_keys=True)
        print(name, res, flush=True)


if __name__ == "__main__":
    main()
