"""The allocation-free current filter against the filter phase of a context.

Callers that cannot allocate device memory (all of it owned by another
framework's allocator, a fixed memory budget, a loop that must never
allocate) have no scratch buffer to bind; pic_filter_current_noalloc runs the
same binomial filter with its scratch in a fixed device array inside the
library.  These tests call it through the C ABI twice in a row on different
inputs and compare each result with the FILTER phase of a context (which uses
the caller-bound scratch), within the single-phase tolerances of the parity
tests.  The file name sorts last so that a run stopping at the first failure
has run every other test first; it passes alone in a fresh process too.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [
    dict(dim=2, nx=48, ny=1, nz=96, dx=0.5, dy=1.0, dz=0.125, bc_z=1, passes=2, prec=0),
    dict(dim=3, nx=20, ny=12, nz=40, dx=0.5, dy=0.6, dz=0.25, bc_z=0, passes=1, prec=1),
    dict(dim=3, nx=16, ny=16, nz=24, dx=1.0, dy=1.0, dz=0.5, bc_z=1, passes=2, prec=0),
]
TOL = {0: 2e-6, 1: 1e-12}
J_NAMES = ("Jx", "Jy", "Jz")


def _filter_phase(P, case, J):
    sim = P.Simulation(dim=case["dim"], nx=case["nx"], ny=case["ny"], nz=case["nz"], dx=case["dx"],
                       dy=case["dy"], dz=case["dz"], filter_passes=case["passes"], bc_z=case["bc_z"],
                       precision=case["prec"])
    sim.set_fields(J)
    sim.step_phases(P.PH_FILTER)
    out = {c: t.double().cpu().numpy() for c, t in sim.fields(0x1C0).items()}
    sim.close()
    return out


def test_noalloc_filter_matches_filter_phase_two_calls_in_a_row():
    import torch

    import paper_1011_0917_gb300 as P
    from paper_1011_0917_gb300 import workloads as W

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    for case in CASES:
        shape3 = (case["nz"] + 1, case["ny"], case["nx"])
        dtype = torch.float32 if case["prec"] == 0 else torch.float64
        for call, seed in enumerate((101, 202)):
            J = {c: v for c, v in W.random_fields(shape3, seed=seed).items() if c in J_NAMES}
            ref = _filter_phase(P, case, J)
            dev = {c: torch.tensor(J[c], dtype=dtype, device="cuda").contiguous() for c in J_NAMES}
            P.pic_filter_current_noalloc(case["dim"], case["nx"], case["ny"], case["nz"], case["bc_z"],
                                         case["passes"], case["prec"], dev["Jx"].data_ptr(), dev["Jy"].data_ptr(),
                                         dev["Jz"].data_ptr(), stream.cuda_stream)
            torch.cuda.synchronize()
            for c in J_NAMES:
                got = dev[c].double().cpu().numpy()
                err = np.abs(got - ref[c]).max() / np.abs(ref[c]).max()
                assert err < TOL[case["prec"]], (case, call, c, err)


def test_noalloc_filter_rejects_sizes_beyond_its_scratch():
    import paper_1011_0917_gb300 as P
    nx = 2048
    nz = P.PIC_NOALLOC_MAX_NODES // nx  # (nz + 1) * nx nodes: one plane too many
    with pytest.raises(P.PicError) as e:
        P.pic_filter_current_noalloc(2, nx, 1, nz, 1, 1, 0, 1 << 20, 1 << 20, 1 << 20, 0)
    assert e.value.status == P.PIC_ERR_ARG
    assert "exceed" in str(e.value)
