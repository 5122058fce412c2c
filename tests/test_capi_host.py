"""Host-side checks of the C-ABI library that need no GPU: it builds for
sm_103a, loads, exports every function include/pic.h declares, validates its
arguments, and derives the simulation-frame quantities exactly as the oracle
does (bit for bit)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import paper_1011_0917_gb300 as P
    P.lib()
    return P


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pic_init_grid", "pic_load_plasma", "pic_launch_laser", "pic_step", "pic_get_fields",
                     "pic_get_particles"):
        assert required in names


def test_library_exports_every_declared_symbol(P):
    lib = C.CDLL(P.library_path())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_every_declared_call(P):
    # the Python binding carries each C-ABI call under the same name
    missing = [n for n in declared_functions() if not callable(getattr(P, n, None))]
    assert not missing, missing


def test_library_targets_sm_103a(P):
    # the build line passes exactly one -gencode for compute_103a / sm_103a
    from paper_1011_0917_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def grid(P, **kw):
    d = dict(dim=2, nx=64, ny=1, nz=512, dx=0.5, dy=1.0, dz=1 / 16, cfl=0.99, gamma_boost=1.0, shape_order=1,
             filter_passes=1, bc_z=1, precision=0, seed=1, slots_per_cell=8.0, tile=(0, 0, 0), track_ids=0,
             z_relative=0)
    d.update(kw)
    return P.GridParams(d["dim"], d["nx"], d["ny"], d["nz"], d["dx"], d["dy"], d["dz"], d["cfl"], d["gamma_boost"],
                        d["shape_order"], d["filter_passes"], d["bc_z"], d["precision"], d["seed"],
                        d["slots_per_cell"], (C.c_int * 3)(*d["tile"]), d["track_ids"], 0, d["z_relative"], None)


@pytest.mark.parametrize("bad,status", [
    (dict(cfl=1.0), 5), (dict(cfl=1.2), 5), (dict(cfl=0.0), 1), (dict(dim=4), 1), (dict(nx=0), 1),
    (dict(ny=2), 1), (dict(shape_order=3), 1), (dict(gamma_boost=0.5), 1), (dict(tile=(3, 0, 0)), 1),
    (dict(precision=7), 1), (dict(slots_per_cell=0.0), 1), (dict(filter_passes=-1), 1), (dict(nz=2), 1),
    (dict(tile=(8, 1, 8)), 1), (dict(z_relative=3), 1), (dict(z_relative=-1), 1),
    (dict(dim=3, ny=4, dy=-1.0), 1),
])
def test_init_grid_rejects_invalid_parameters(P, bad, status):
    with pytest.raises(P.PicError) as e:
        P.pic_init_grid(grid(P, **bad))
    assert e.value.status == status


@pytest.mark.parametrize("tile", [(16, 1, 16), (32, 1, 8), (8, 1, 32), (32, 0, 8)])
def test_compiled_2d_tile_shapes_are_accepted(P, tile):
    ctx = P.pic_init_grid(grid(P, tile=tile))
    try:
        s = P.pic_query_sizes(ctx)
        assert (s.tile[0], s.tile[2]) == (tile[0], tile[2])
        assert s.tile_capacity % 32 == 0 and s.tile_capacity >= 8 * tile[0] * tile[2]
    finally:
        P.pic_destroy(ctx)


@pytest.mark.parametrize("tile,shape", [((32, 1, 8), 2), ((8, 1, 32), 2), ((32, 1, 16), 1), ((64, 1, 4), 1)])
def test_other_2d_tile_shapes_are_rejected(P, tile, shape):
    with pytest.raises(P.PicError) as e:
        P.pic_init_grid(grid(P, tile=tile, shape_order=shape))
    assert e.value.status == 1


@pytest.mark.parametrize("kw", [
    dict(), dict(gamma_boost=13.0, dx=1.0, dz=1 / 32, nx=256, nz=8192),
    dict(dim=3, nx=32, ny=16, nz=64, dx=1.0, dy=1.0, dz=1 / 32, gamma_boost=13.0),
    dict(gamma_boost=130.0, dx=1.0, dz=1 / 32, nx=512, nz=16384, shape_order=2, filter_passes=4),
])
def test_derived_quantities_match_oracle(P, oracle_mod, kw):
    g = grid(P, **kw)
    ctx = P.pic_init_grid(g)
    try:
        s = P.pic_query_sizes(ctx)
        o = oracle_mod.Oracle(oracle_mod.GridParams(dim=g.dim, nx=g.nx, ny=g.ny, nz=g.nz, dx=g.dx, dy=g.dy, dz=g.dz,
                                                    cfl=g.cfl, gamma_boost=g.gamma_boost, shape=g.shape_order,
                                                    npass=g.filter_passes))
        assert (s.dt, s.hx, s.hz, s.beta) == (o.dt, o.hx, o.hz, o.beta)
        if g.dim == 3:
            assert s.hy == o.hy
        # buffers: 9 field components, two bucket sides per species
        es = s.elem_bytes
        assert s.field_bytes == 9 * (g.nz + 1) * (g.ny if g.dim == 3 else 1) * g.nx * es
        assert s.slots[0] == s.ntiles * s.tile_capacity and s.tile_capacity % 32 == 0
        assert (s.species_bytes[1] > 0) == (g.gamma_boost > 1.0)
    finally:
        P.pic_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dim", [2, 3])
def test_relative_positions_add_departure_columns(P, prec, dim):
    # z_relative: automatic (on from gamma_boost 50), forced on, forced off;
    # on, the electron store holds one departure column per axis (x, z in
    # 2D; x, y, z in 3D) of elem_bytes per slot and side (256-byte aligned);
    # the ion store is unchanged
    extra = dict(dim=3, ny=16, nz=64, dy=1.0) if dim == 3 else {}

    def sizes(gam, mode):
        ctx = P.pic_init_grid(grid(P, gamma_boost=gam, precision=prec, z_relative=mode, **extra))
        try:
            return P.pic_query_sizes(ctx)
        finally:
            P.pic_destroy(ctx)

    off, on = sizes(130.0, 2), sizes(130.0, 1)
    col = -(-off.slots[0] * off.elem_bytes // 256) * 256
    assert on.species_bytes[0] == off.species_bytes[0] + 2 * dim * col
    assert on.species_bytes[1] == off.species_bytes[1]
    assert sizes(130.0, 0).species_bytes[0] == on.species_bytes[0]
    assert sizes(50.0, 0).species_bytes[0] == sizes(50.0, 1).species_bytes[0]
    assert sizes(30.0, 0).species_bytes[0] == sizes(30.0, 2).species_bytes[0]


def test_calls_before_bind_are_rejected(P):
    ctx = P.pic_init_grid(grid(P))
    try:
        with pytest.raises(P.PicError) as e:
            P.pic_step(ctx, 1)
        assert e.value.status == 2
        assert "bind" in P.pic_last_error(ctx)
    finally:
        P.pic_destroy(ctx)


def test_status_strings(P):
    for s in range(8):
        assert P.pic_status_string(s)


def test_btd_bytes_and_validation(P):
    # lab-frame snapshots: [nsnap][6][nz][nxs] elements, then nsnap * nz int32
    # flags at a 256-byte boundary; an unboosted grid has none
    g = grid(P, gamma_boost=5.0, dx=1.0, dz=1 / 32, nx=48, nz=256)
    ctx = P.pic_init_grid(g)
    try:
        for plane, nxs in ((0, 1), (1, 48)):
            p = P.BtdParams(4, 100.0, 5.0, 10.0, 1 / 32, 300, plane)
            data = 4 * 6 * 300 * nxs * 4
            align = lambda b: (b + 255) // 256 * 256
            assert P.pic_btd_bytes(ctx, p) == align(data) + align(4 * 4 * 300)
        for bad in (P.BtdParams(0, 0.0, 1.0, 0.0, 0.1, 10, 0), P.BtdParams(65, 0.0, 1.0, 0.0, 0.1, 10, 0),
                    P.BtdParams(2, 0.0, 1.0, 0.0, -0.1, 10, 0), P.BtdParams(2, 0.0, 1.0, 0.0, 0.1, 10, 2)):
            with pytest.raises(P.PicError):
                P.pic_btd_bytes(ctx, bad)
    finally:
        P.pic_destroy(ctx)
    ctx = P.pic_init_grid(grid(P))
    try:
        with pytest.raises(P.PicError):
            P.pic_btd_bytes(ctx, P.BtdParams(1, 0.0, 1.0, 0.0, 0.1, 10, 0))
    finally:
        P.pic_destroy(ctx)


def test_moving_window_validation(P):
    ctx = P.pic_init_grid(grid(P, nz=512))
    try:
        P.pic_set_moving_window(ctx, 0.99, 1.0, 16)      # one 2D tile layer
        P.pic_set_moving_window(ctx, 1.0, 0.0, 32)
        P.pic_set_moving_window(ctx, 0.0, 0.0, 0)        # off
        for v, s in ((1.2, 16), (-0.5, 16), (0.9, 8), (0.9, 24), (0.9, 512)):
            with pytest.raises(P.PicError):
                P.pic_set_moving_window(ctx, v, 0.0, s)
    finally:
        P.pic_destroy(ctx)
    ctx = P.pic_init_grid(grid(P, bc_z=0))
    try:
        with pytest.raises(P.PicError):
            P.pic_set_moving_window(ctx, 0.9, 0.0, 16)   # periodic z has no window
    finally:
        P.pic_destroy(ctx)


def test_batch_validation(P):
    # a batch needs bound contexts, at least one, none twice; graphs of an
    # even number of steps
    ctx = P.pic_init_grid(grid(P))
    try:
        with pytest.raises(P.PicError) as e:
            P.pic_batch_create([ctx])
        assert e.value.status == 2  # PIC_ERR_STATE: not bound
        with pytest.raises(P.PicError) as e:
            P.pic_batch_create([])
        assert e.value.status == 1
    finally:
        P.pic_destroy(ctx)
    for k in (-2, 3):
        with pytest.raises(P.PicError) as e:
            P.pic_batch_set_graph(None, k)
        assert e.value.status == 1


def test_cell_order_and_fused_batch_validation(P):
    # cell sorting needs bound buffers and a non-negative interval; the fused
    # form of a batch needs a batch and a non-negative chain count
    ctx = P.pic_init_grid(grid(P))
    try:
        with pytest.raises(P.PicError) as e:
            P.pic_sort_cells(ctx)
        assert e.value.status == 2 and "bind" in P.pic_last_error(ctx)
        with pytest.raises(P.PicError) as e:
            P.pic_set_cell_sort(ctx, -1)
        assert e.value.status == 1
        P.pic_set_cell_sort(ctx, 0)
    finally:
        P.pic_destroy(ctx)
    for chains in (2, -1):
        with pytest.raises(P.PicError) as e:
            P.pic_batch_set_fused(None, chains)
        assert e.value.status == 1
    with pytest.raises(P.PicError) as e:
        P.pic_batch_graph_info(None)
    assert e.value.status == 1


def test_adjoint_validation(P):
    # the adjoint needs bound buffers, then a loaded plasma and no step taken
    ctx = P.pic_init_grid(grid(P, gamma_boost=5.0, dx=1.0, dz=1 / 32, nx=48, nz=256))
    try:
        with pytest.raises(P.PicError) as e:
            P.pic_adjoint_bytes(ctx, P.AdjointParams(40, 20))
        assert e.value.status == 2
        assert "bind" in P.pic_last_error(ctx)
    finally:
        P.pic_destroy(ctx)


def test_adjoint_backward_needs_a_forward_run(P):
    ctx = P.pic_init_grid(grid(P, gamma_boost=5.0, dx=1.0, dz=1 / 32, nx=48, nz=256))
    try:
        cot = (C.c_double * 8)()
        with pytest.raises(P.PicError) as e:
            P.pic_adjoint_backward(ctx, C.addressof(cot), 2)
        assert e.value.status == 2
        assert "pic_adjoint_forward" in P.pic_last_error(ctx)
    finally:
        P.pic_destroy(ctx)


def test_simulation_refuses_without_a_gpu(P):
    # the product path has no CPU fallback: without a CUDA device it raises
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(RuntimeError, match="no CPU path"):
        P.Simulation(dim=2, nx=16, ny=1, nz=64, dx=0.5, dz=1 / 16)


@pytest.mark.parametrize("tile,shape,ok", [((8, 8, 8), 1, True), ((8, 8, 4), 1, True), ((0, 0, 4), 1, True),
                                           ((8, 8, 4), 2, False), ((8, 8, 16), 1, False), ((16, 8, 4), 1, False)])
def test_3d_tile_shapes(P, tile, shape, ok):
    g = grid(P, dim=3, nx=32, ny=16, nz=64, dx=1.0, dy=1.0, dz=1 / 32, gamma_boost=13.0, tile=tile,
             shape_order=shape)
    if not ok:
        with pytest.raises(P.PicError) as e:
            P.pic_init_grid(g)
        assert e.value.status == 1
        return
    ctx = P.pic_init_grid(g)
    try:
        s = P.pic_query_sizes(ctx)
        assert (s.tile[0], s.tile[1], s.tile[2]) == (8, 8, tile[2] if tile[2] else 8)
    finally:
        P.pic_destroy(ctx)
