"""The adjoint (reverse-mode gradient) of boosted 2D3V and 3D runs, and of a
lab-frame 2D3V run, against central finite differences of the FP64 oracle.

The objective is linear in the final fields, L = sum(lambda . (E^N, B^N)),
with lambda on a few nodes behind the laser; its gradient is taken with
respect to the plasma profile coefficients (through every particle weight),
the laser's a0 and its waist (through the antenna current).  The oracle knows
nothing of the adjoint: its objective is evaluated at theta +- h and the
difference quotient is the reference.  Also checked: the adjoint's own forward
run (a fixed-order particle store) reproduces the oracle's fields, the
gradient does not depend on the checkpoint interval, and the FP32 gradient
agrees with the FP64 one.
"""
import math

import numpy as np
import pytest

from pairs import make_pair

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1
GAM = 5.0
BETA = math.sqrt(1 - 1 / GAM ** 2)
G = dict(dim=2, nx=16, nz=128, dx=1.0, dz=1 / 16, gamma_boost=GAM, filter_passes=1, seed=61)
HZ = (1 / 16) * GAM * (1 + BETA)
PLASMA = dict(ne=0.01, z_start=GAM * 8 * HZ, z_end=GAM * 2000 * HZ, ramp=1.0, ppc=(2, 1, 2), jitter=0.1, ions=1)
LASER = dict(a0=2.0, waist=5.0, fwhm=2.0, t_peak=0.5, pol=1)
COEF = (0.1, -0.05)
NSTEPS = 60


@pytest.fixture(scope="module")
def O():
    import oracle.oracle as O
    O.build_oracle()
    return O


def cotangent(nz, nx):
    lam = np.zeros((6, nz + 1, nx))
    lam[2, 20:44, nx // 2] = 1.0            # Ez on axis behind the pulse
    lam[0, 24:40, nx // 2 + 2] = 0.5        # Ex off axis
    lam[1, 30:34, :] = 0.05                 # Ey across
    return lam


def oracle_objective(O, coef, a0, w0):
    o = O.Oracle(O.GridParams(dim=2, nx=G["nx"], nz=G["nz"], dx=G["dx"], dz=G["dz"], gamma_boost=GAM,
                              npass=G["filter_passes"], bc_z=1, seed=G["seed"]))
    o.load_plasma(O.PlasmaParams(ne=PLASMA["ne"], z_start=PLASMA["z_start"], z_end=PLASMA["z_end"],
                                 ramp=PLASMA["ramp"], ppc=PLASMA["ppc"], jitter=PLASMA["jitter"],
                                 profile=tuple(coef), ions=1))
    o.set_laser(O.LaserParams(a0=a0, waist=w0, fwhm=LASER["fwhm"], z_antenna=0.0, t_peak=LASER["t_peak"], pol=1))
    o.step(NSTEPS)
    lam = cotangent(G["nz"], G["nx"])
    f = np.stack([o.field(c)[:, 0, :] for c in ("Ex", "Ey", "Ez", "Bx", "By", "Bz")])
    return float(np.sum(lam * f)), f


def gpu_run(O, prec, coef=COEF, a0=LASER["a0"], w0=LASER["waist"], K=20):
    import torch
    sim, _ = make_pair(O, G, prec)
    sim.load_plasma(PLASMA["ne"], PLASMA["z_start"], PLASMA["z_end"], PLASMA["ramp"], PLASMA["ppc"],
                    PLASMA["jitter"], coef, 1)
    sim.launch_laser(a0, w0, LASER["fwhm"], 0.0, LASER["t_peak"], 1)
    fields = sim.adjoint_forward(NSTEPS, K)
    lam = torch.as_tensor(cotangent(G["nz"], G["nx"]), dtype=fields.dtype, device=fields.device)
    grad = sim.adjoint_backward(lam)
    return fields.double().cpu().numpy(), grad


@pytest.fixture(scope="module")
def reference(O):
    """(L, fields) at theta and the central differences of the oracle."""
    L0, f0 = oracle_objective(O, COEF, LASER["a0"], LASER["waist"])
    fd = []
    h = 1e-4
    for m in range(len(COEF)):
        cp, cm = list(COEF), list(COEF)
        cp[m] += h
        cm[m] -= h
        fd.append((oracle_objective(O, cp, LASER["a0"], LASER["waist"])[0] -
                   oracle_objective(O, cm, LASER["a0"], LASER["waist"])[0]) / (2 * h))
    ha = 1e-4 * LASER["a0"]
    fd.append((oracle_objective(O, COEF, LASER["a0"] + ha, LASER["waist"])[0] -
               oracle_objective(O, COEF, LASER["a0"] - ha, LASER["waist"])[0]) / (2 * ha))
    hw = 1e-4 * LASER["waist"]
    fd.append((oracle_objective(O, COEF, LASER["a0"], LASER["waist"] + hw)[0] -
               oracle_objective(O, COEF, LASER["a0"], LASER["waist"] - hw)[0]) / (2 * hw))
    return L0, f0, np.array(fd)


def test_adjoint_forward_matches_oracle(O, reference):
    # the run the adjoint differentiates is the oracle's run (FP64: 1e-10)
    _, f0, _ = reference
    f, _ = gpu_run(O, FP64)
    for q in range(6):
        n = np.linalg.norm(f0[q])
        if n > 1e-3 * np.linalg.norm(f0):
            assert np.linalg.norm(f[q] - f0[q]) / n < 1e-10, q


def test_gradient_matches_oracle_finite_differences(O, reference):
    _, _, fd = reference
    _, g = gpu_run(O, FP64)
    g = np.array(g)
    assert np.all(np.abs(fd) > 0)
    rel = np.abs(g - fd) / np.abs(fd)
    assert np.all(rel < 1e-3), (g, fd, rel)


def test_gradient_independent_of_checkpoint_interval(O):
    _, g1 = gpu_run(O, FP64, K=NSTEPS)
    _, g2 = gpu_run(O, FP64, K=7)
    assert np.allclose(g1, g2, rtol=1e-11, atol=0)


@pytest.mark.parametrize("K,K2", [(20, 5), (NSTEPS, 7), (25, 4)])
def test_two_level_checkpoints_same_gradient_less_memory(O, K, K2):
    # segments recomputed in two levels (a sub-checkpoint every K2 steps):
    # the same gradient as with every state of a segment kept, from a
    # smaller buffer (K2 + 1 + ceil(K / K2) states instead of K + 1)
    import torch

    import paper_1011_0917_gb300 as P
    _, g1 = gpu_run(O, FP64, K=NSTEPS)
    sim, _ = make_pair(O, G, FP64)
    sim.load_plasma(PLASMA["ne"], PLASMA["z_start"], PLASMA["z_end"], PLASMA["ramp"], PLASMA["ppc"],
                    PLASMA["jitter"], COEF, 1)
    sim.launch_laser(LASER["a0"], LASER["waist"], LASER["fwhm"], 0.0, LASER["t_peak"], 1)
    one = P.pic_adjoint_bytes(sim.ctx, P.AdjointParams(NSTEPS, K, 0))
    two = P.pic_adjoint_bytes(sim.ctx, P.AdjointParams(NSTEPS, K, K2))
    assert two < one
    fields = sim.adjoint_forward(NSTEPS, K, K2)
    assert sim._adj.numel() == two
    lam = torch.as_tensor(cotangent(G["nz"], G["nx"]), dtype=fields.dtype, device=fields.device)
    g2 = sim.adjoint_backward(lam)
    assert np.allclose(g1, g2, rtol=1e-11, atol=0), (g1, g2)


def test_lab_frame_gradient_matches_oracle_finite_differences(O):
    # the same objective in the lab frame (gamma = 1: immobile ions, no
    # injection) on the c0 grid spacing, plasma from 6 cells on
    g = dict(dim=2, nx=16, nz=96, dx=0.5, dz=1 / 16, gamma_boost=1.0, filter_passes=1, seed=63)
    pl = dict(ne=0.01, z_start=6 / 16, z_end=40.0, ramp=0.5, ppc=(2, 1, 2), jitter=0.1)
    # a short horizon and a gentle drive (a0 = 0.5), where the oracle's central
    # differences agree across h = 1e-3 .. 1e-5 to 2e-5
    coef, a0, w0, nsteps = (0.15,), 0.5, 3.0, 40
    lam = np.zeros((6, g["nz"] + 1, g["nx"]))
    lam[2, 10:60, :] = 1.0
    lam[1, 20:40, :] = 0.1

    def objective(c, a, w):
        o = O.Oracle(O.GridParams(dim=2, nx=g["nx"], nz=g["nz"], dx=g["dx"], dz=g["dz"], npass=1, bc_z=1,
                                  seed=g["seed"]))
        o.load_plasma(O.PlasmaParams(profile=tuple(c), ions=1, **pl))
        o.set_laser(O.LaserParams(a0=a, waist=w, fwhm=2.0, z_antenna=0.0, t_peak=0.5, pol=1))
        o.step(nsteps)
        return float(np.sum(lam * np.stack([o.field(q)[:, 0, :] for q in ("Ex", "Ey", "Ez", "Bx", "By", "Bz")])))

    import torch
    sim, _ = make_pair(O, g, FP64)
    sim.load_plasma(pl["ne"], pl["z_start"], pl["z_end"], pl["ramp"], pl["ppc"], pl["jitter"], coef, 1)
    sim.launch_laser(a0, w0, 2.0, 0.0, 0.5, 1)
    sim.adjoint_forward(nsteps, 16)
    grad = np.array(sim.adjoint_backward(torch.as_tensor(lam, device="cuda")))
    h = 1e-4
    fd = np.array([(objective((coef[0] + h,), a0, w0) - objective((coef[0] - h,), a0, w0)) / (2 * h),
                   (objective(coef, a0 + h, w0) - objective(coef, a0 - h, w0)) / (2 * h),
                   (objective(coef, a0, w0 + h) - objective(coef, a0, w0 - h)) / (2 * h)])
    assert np.all(np.abs(fd) > 0)
    rel = np.abs(grad - fd) / np.abs(fd)
    assert np.all(rel < 1e-3), (grad, fd, rel)


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_3d_gradient_matches_oracle_finite_differences(O, prec):
    # a 3D boosted run (gamma = 5, 8 x 8 x 48 cells, 2 x 2 x 2 per cell);
    # the objective is Ez over a slab behind the antenna plus an Ey band
    gam = 5.0
    hz = (1 / 16) * gam * (1 + math.sqrt(1 - 1 / gam ** 2))
    g = dict(dim=3, nx=8, ny=8, nz=48, dx=1.0, dy=1.0, dz=1 / 16, gamma_boost=gam, filter_passes=1, seed=65)
    pl = dict(ne=0.01, z_start=gam * 6 * hz, z_end=gam * 600 * hz, ramp=1.0, ppc=(2, 2, 2), jitter=0.1)
    coef, a0, w0, nsteps = (0.1,), 1.0, 3.0, 20
    lam = np.zeros((6, g["nz"] + 1, g["ny"], g["nx"]))
    lam[2, 4:36] = 1.0
    lam[1, 10:30] = 0.05

    def objective(c, a, w):
        o = O.Oracle(O.GridParams(dim=3, nx=g["nx"], ny=g["ny"], nz=g["nz"], dx=g["dx"], dy=g["dy"], dz=g["dz"],
                                  gamma_boost=gam, npass=1, bc_z=1, seed=g["seed"]))
        o.load_plasma(O.PlasmaParams(profile=tuple(c), ions=1, **pl))
        o.set_laser(O.LaserParams(a0=a, waist=w, fwhm=2.0, z_antenna=0.0, t_peak=0.5, pol=1))
        o.step(nsteps)
        return float(np.sum(lam * np.stack([o.field(q) for q in ("Ex", "Ey", "Ez", "Bx", "By", "Bz")])))

    import torch
    sim, _ = make_pair(O, g, prec)
    sim.load_plasma(pl["ne"], pl["z_start"], pl["z_end"], pl["ramp"], pl["ppc"], pl["jitter"], coef, 1)
    sim.launch_laser(a0, w0, 2.0, 0.0, 0.5, 1)
    fields = sim.adjoint_forward(nsteps, 8)
    cot = torch.as_tensor(lam.reshape(6, g["nz"] + 1, g["ny"] * g["nx"]), dtype=fields.dtype, device="cuda")
    grad = np.array(sim.adjoint_backward(cot.reshape(fields.shape)))
    # where the oracle's differences agree across h = 1e-3 .. 1e-5 to 2e-6
    h = 1e-4
    fd = np.array([(objective((coef[0] + h,), a0, w0) - objective((coef[0] - h,), a0, w0)) / (2 * h),
                   (objective(coef, a0 + h, w0) - objective(coef, a0 - h, w0)) / (2 * h),
                   (objective(coef, a0, w0 + h) - objective(coef, a0, w0 - h)) / (2 * h)])
    rel = np.abs(grad - fd) / np.abs(fd)
    assert np.all(rel < 1e-3), (grad, fd, rel)


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_quadratic_shape_gradient_matches_oracle_finite_differences(O, prec):
    # the quadratic shape (3-node supports, 4-node Esirkepov windows) with two
    # filter passes, boosted 2D3V (gamma = 5)
    gam = 5.0
    hz = (1 / 16) * gam * (1 + math.sqrt(1 - 1 / gam ** 2))
    g = dict(dim=2, nx=16, nz=128, dx=1.0, dz=1 / 16, gamma_boost=gam, shape_order=2, filter_passes=2, seed=67)
    pl = dict(ne=0.01, z_start=gam * 8 * hz, z_end=gam * 2000 * hz, ramp=1.0, ppc=(2, 1, 2), jitter=0.1)
    coef, a0, w0, nsteps = (0.1, -0.05), 1.5, 4.0, 40
    lam = np.zeros((6, g["nz"] + 1, g["nx"]))
    lam[2, 16:48] = 1.0
    lam[1, 20:40] = 0.05

    def objective(c, a, w):
        o = O.Oracle(O.GridParams(dim=2, nx=g["nx"], nz=g["nz"], dx=g["dx"], dz=g["dz"], gamma_boost=gam, shape=2,
                                  npass=2, bc_z=1, seed=g["seed"]))
        o.load_plasma(O.PlasmaParams(profile=tuple(c), ions=1, **pl))
        o.set_laser(O.LaserParams(a0=a, waist=w, fwhm=2.0, z_antenna=0.0, t_peak=0.5, pol=1))
        o.step(nsteps)
        return float(np.sum(lam * np.stack([o.field(q)[:, 0, :] for q in ("Ex", "Ey", "Ez", "Bx", "By", "Bz")])))

    import torch
    sim, _ = make_pair(O, g, prec)
    sim.load_plasma(pl["ne"], pl["z_start"], pl["z_end"], pl["ramp"], pl["ppc"], pl["jitter"], coef, 1)
    sim.launch_laser(a0, w0, 2.0, 0.0, 0.5, 1)
    fields = sim.adjoint_forward(nsteps, 16)
    grad = np.array(sim.adjoint_backward(torch.as_tensor(lam, dtype=fields.dtype, device="cuda")))
    # the oracle's differences agree across h = 1e-3 .. 1e-5 to 3e-6 here
    h = 1e-4
    fd = np.array([(objective((coef[0] + h, coef[1]), a0, w0) - objective((coef[0] - h, coef[1]), a0, w0)) / (2 * h),
                   (objective((coef[0], coef[1] + h), a0, w0) - objective((coef[0], coef[1] - h), a0, w0)) / (2 * h),
                   (objective(coef, a0 + h, w0) - objective(coef, a0 - h, w0)) / (2 * h),
                   (objective(coef, a0, w0 + h) - objective(coef, a0, w0 - h)) / (2 * h)])
    rel = np.abs(grad - fd) / np.abs(fd)
    assert np.all(rel < 1e-3), (grad, fd, rel)


def test_fp32_gradient_against_fp64(O):
    _, g64 = gpu_run(O, FP64)
    _, g32 = gpu_run(O, FP32)
    g64, g32 = np.array(g64), np.array(g32)
    rel = np.abs(g32 - g64) / np.abs(g64)
    assert np.all(rel < 1e-3), (g32, g64, rel)


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_stage_gradient_autograd_matches_oracle_finite_differences(O, reference, prec):
    """The torch.autograd.Function face of the adjoint: coefficients, a0 and
    w0 as CUDA tensors with requires_grad, the objective built in torch from
    the returned fields, .backward(); each .grad lands on its input's device
    and dtype and matches the oracle's central differences (1e-3)."""
    import torch

    import paper_1011_0917_gb300 as P
    _, _, fd = reference
    dev = torch.device("cuda")
    coef = torch.tensor(COEF, dtype=torch.float64, device=dev, requires_grad=True)
    a0 = torch.tensor(LASER["a0"], dtype=torch.float64, device=dev, requires_grad=True)
    w0 = torch.tensor(LASER["waist"], dtype=torch.float64, device=dev, requires_grad=True)
    settings = dict(grid=dict(dim=2, nx=G["nx"], nz=G["nz"], dx=G["dx"], dz=G["dz"], gamma_boost=GAM,
                              filter_passes=G["filter_passes"], seed=G["seed"], precision=prec, slots_per_cell=16.0),
                    plasma=dict(ne=PLASMA["ne"], z_start=PLASMA["z_start"], z_end=PLASMA["z_end"],
                                ramp=PLASMA["ramp"], ppc=PLASMA["ppc"], jitter=PLASMA["jitter"], ions=1),
                    laser=dict(waist=LASER["waist"], fwhm=LASER["fwhm"], t_peak=LASER["t_peak"], pol=1),
                    nsteps=NSTEPS, checkpoint_every=20)
    out = P.StageGradient.apply(coef, a0, w0, settings)
    assert out.is_cuda and out.shape == (6, G["nz"] + 1, G["nx"])
    lam = torch.as_tensor(cotangent(G["nz"], G["nx"]), dtype=out.dtype, device=dev)
    (lam * out).sum().backward()
    for t in (coef, a0, w0):
        assert t.grad is not None and t.grad.device == t.device and t.grad.dtype == t.dtype
    g = np.concatenate([coef.grad.cpu().numpy(), [a0.grad.item(), w0.grad.item()]])
    rel = np.abs(g - fd) / np.abs(fd)
    assert np.all(rel < 1e-3), (g, fd, rel)


def test_stage_gradient_without_waist_input(O, reference):
    """w0 = None keeps the waist of the settings: its gradient slot is None."""
    import torch

    import paper_1011_0917_gb300 as P
    _, _, fd = reference
    coef = torch.tensor(COEF, dtype=torch.float64, device="cuda", requires_grad=True)
    a0 = torch.tensor(LASER["a0"], dtype=torch.float64, device="cuda", requires_grad=True)
    settings = dict(grid=dict(dim=2, nx=G["nx"], nz=G["nz"], dx=G["dx"], dz=G["dz"], gamma_boost=GAM,
                              filter_passes=G["filter_passes"], seed=G["seed"], precision=FP64, slots_per_cell=16.0),
                    plasma=dict(ne=PLASMA["ne"], z_start=PLASMA["z_start"], z_end=PLASMA["z_end"],
                                ramp=PLASMA["ramp"], ppc=PLASMA["ppc"], jitter=PLASMA["jitter"], ions=1),
                    laser=dict(waist=LASER["waist"], fwhm=LASER["fwhm"], t_peak=LASER["t_peak"], pol=1),
                    nsteps=NSTEPS, checkpoint_every=NSTEPS)
    out = P.StageGradient.apply(coef, a0, None, settings)
    lam = torch.as_tensor(cotangent(G["nz"], G["nx"]), dtype=out.dtype, device="cuda")
    (lam * out).sum().backward()
    g = np.concatenate([coef.grad.cpu().numpy(), [a0.grad.item()]])
    assert np.all(np.abs(g - fd[:-1]) / np.abs(fd[:-1]) < 1e-3)


# ------------------------------------------------------------ batched

BATCH_RUNS = [
    dict(coef=COEF, a0=LASER["a0"], w0=LASER["waist"]),
    dict(coef=(-0.08, 0.04, 0.02), a0=1.5, w0=6.0),
    dict(coef=(0.05,), a0=2.5, w0=4.5),
]


def _oracle_fd(O, coef, a0, w0):
    h = 1e-4
    fd = []
    for m in range(len(coef)):
        cp, cm = list(coef), list(coef)
        cp[m] += h
        cm[m] -= h
        fd.append((oracle_objective(O, cp, a0, w0)[0] - oracle_objective(O, cm, a0, w0)[0]) / (2 * h))
    ha, hw = 1e-4 * a0, 1e-4 * w0
    fd.append((oracle_objective(O, coef, a0 + ha, w0)[0] - oracle_objective(O, coef, a0 - ha, w0)[0]) / (2 * ha))
    fd.append((oracle_objective(O, coef, a0, w0 + hw)[0] - oracle_objective(O, coef, a0, w0 - hw)[0]) / (2 * hw))
    return np.array(fd)


def test_batch_adjoint_matches_oracle_finite_differences(O, reference):
    """The reverse mode of a scan: three runs with different profiles (M = 2,
    3, 1 coefficients), laser amplitudes and waists, all gradients from one
    pic_batch_adjoint call (every run's forward and reverse sweep queued on its
    own stream), each against central differences of its own FP64 oracle
    runs (1e-3), and run 0 the same as its single-run gradient."""
    import torch

    import paper_1011_0917_gb300 as P
    sims = []
    for r in BATCH_RUNS:
        sim = P.Simulation(dim=2, nx=G["nx"], nz=G["nz"], dx=G["dx"], dz=G["dz"], gamma_boost=GAM,
                           filter_passes=G["filter_passes"], precision=FP64, seed=G["seed"], slots_per_cell=16.0,
                           stream=torch.cuda.Stream())
        sim.load_plasma(PLASMA["ne"], PLASMA["z_start"], PLASMA["z_end"], PLASMA["ramp"], PLASMA["ppc"],
                        PLASMA["jitter"], r["coef"], 1)
        sim.launch_laser(r["a0"], r["w0"], LASER["fwhm"], 0.0, LASER["t_peak"], 1)
        sims.append(sim)
    batch = P.Batch(sims, graph_steps=0)
    lam = cotangent(G["nz"], G["nx"])
    grads = batch.adjoint(NSTEPS, [lam] * len(sims), checkpoint_every=20, sub_checkpoint_every=5)
    batch.close()
    _, single = gpu_run(O, FP64)
    assert np.allclose(grads[0], single, rtol=1e-11, atol=0), (grads[0], single)
    _, _, fd0 = reference
    for i, r in enumerate(BATCH_RUNS):
        fd = fd0 if i == 0 else _oracle_fd(O, r["coef"], r["a0"], r["w0"])
        g = np.array(grads[i])
        assert g.shape == fd.shape == (len(r["coef"]) + 2,)
        rel = np.abs(g - fd) / np.abs(fd)
        assert np.all(rel < 1e-3), (i, g, fd, rel)


def test_checkpoint_interval_fits_the_budget(O):
    """The memory-fitted checkpoint interval: the whole run when it fits, and
    otherwise the largest halving of it whose buffer fits the budget."""
    import paper_1011_0917_gb300 as P
    sim, _ = make_pair(O, G, FP64)
    sim.load_plasma(PLASMA["ne"], PLASMA["z_start"], PLASMA["z_end"], PLASMA["ramp"], PLASMA["ppc"],
                    PLASMA["jitter"], COEF, 1)
    sim.launch_laser(LASER["a0"], LASER["waist"], LASER["fwhm"], 0.0, LASER["t_peak"], 1)
    nbytes = lambda k: P.pic_adjoint_bytes(sim.ctx, P.AdjointParams(NSTEPS, k, 0))
    assert sim.adjoint_checkpoint_interval(NSTEPS, budget_bytes=nbytes(NSTEPS)) == NSTEPS
    k = sim.adjoint_checkpoint_interval(NSTEPS, budget_bytes=nbytes(NSTEPS) - 1)
    assert k < NSTEPS and nbytes(k) <= nbytes(NSTEPS) - 1
    _, g = gpu_run(O, FP64, K=k)
    _, g1 = gpu_run(O, FP64, K=NSTEPS)
    assert np.allclose(g, g1, rtol=1e-11, atol=0)


def test_backward_refused_after_the_run_changed(O):
    """A new laser (or plasma) after the adjoint's forward run makes its
    gradient another run's: the backward pass is refused with PIC_ERR_STATE."""
    import torch
    import paper_1011_0917_gb300 as P
    sim, _ = make_pair(O, G, FP64)
    sim.load_plasma(PLASMA["ne"], PLASMA["z_start"], PLASMA["z_end"], PLASMA["ramp"], PLASMA["ppc"],
                    PLASMA["jitter"], COEF, 1)
    sim.launch_laser(LASER["a0"], LASER["waist"], LASER["fwhm"], 0.0, LASER["t_peak"], 1)
    fields = sim.adjoint_forward(8, 4)
    sim.launch_laser(LASER["a0"] * 1.5, LASER["waist"], LASER["fwhm"], 0.0, LASER["t_peak"], 1)
    with pytest.raises(P.PicError) as e:
        sim.adjoint_backward(torch.zeros_like(fields))
    assert e.value.status == 2
