"""GB300 (sm_103a) boosted-frame electromagnetic PIC library -- Python binding.

Thin ctypes binding of the C ABI in ``include/pic.h``: the functions below
carry the same names and marshal arguments only; every step of the PIC loop
runs in the CUDA kernels of ``libpic.so``.  PyTorch provides the device memory
(the caller-owned buffers the library asks for) and the CUDA stream.

There is no CPU fallback: importing the binding when ``libpic.so`` cannot be
built or loaded raises, and a context cannot be created without a CUDA device.
"""
from __future__ import annotations

import ctypes as C
import math
import os

from . import build as _build

__all__ = [
    "PIC_OK", "PicError", "GridParams", "PlasmaParams", "LaserParams", "Sizes", "Buffers", "Diag",
    "pic_init_grid", "pic_query_sizes", "pic_bind_buffers", "pic_load_plasma", "pic_load_particles",
    "pic_launch_laser", "pic_step", "pic_step_async", "pic_step_phases", "pic_get_fields", "pic_set_fields",
    "pic_get_axis", "pic_get_particles", "pic_get_rho", "pic_get_diagnostics", "pic_state_bytes",
    "pic_get_state", "pic_set_state", "pic_last_error", "pic_status_string", "pic_destroy", "pic_profile",
    "pic_profile_read", "pic_filter_current_noalloc", "PIC_NOALLOC_MAX_NODES", "BtdParams", "pic_btd_bytes",
    "pic_btd_setup", "pic_btd_get", "pic_set_moving_window", "pic_batch_create", "pic_batch_step",
    "pic_batch_destroy", "Simulation", "Batch", "library_path", "AdjointParams", "pic_adjoint_bytes",
    "pic_adjoint_forward", "pic_adjoint_backward", "StageGradient", "pic_batch_set_graph", "pic_wait_check",
    "pic_batch_set_fused", "pic_batch_graph_info", "pic_batch_adjoint", "pic_sort_cells", "pic_set_cell_sort",
    "PIC_FRAME_BOOST", "PIC_FRAME_LAB",
]

PIC_OK, PIC_ERR_ARG, PIC_ERR_STATE, PIC_ERR_CUDA = 0, 1, 2, 3
PIC_ERR_CAPACITY, PIC_ERR_CFL, PIC_ERR_NAN, PIC_ERR_TIMEOUT = 4, 5, 6, 7
PIC_BC_PERIODIC, PIC_BC_MUR = 0, 1
PIC_FP32, PIC_FP64 = 0, 1
PIC_ELECTRONS, PIC_IONS = 0, 1
PIC_POL_X, PIC_POL_Y = 0, 1
PIC_FRAME_BOOST, PIC_FRAME_LAB = 0, 1
COMPONENTS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz")
PH_ZERO_J, PH_PUSH, PH_IONS, PH_ANTENNA = 1, 2, 4, 8
PH_FILTER, PH_YEE, PH_INJECT, PH_TIME = 16, 32, 64, 128
PH_ALL = 255
PIC_NOALLOC_MAX_NODES = 4194304


class PicError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"pic status {status}: {detail}")
        self.status = status


class GridParams(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("cfl", C.c_double),
                ("gamma_boost", C.c_double), ("shape_order", C.c_int), ("filter_passes", C.c_int),
                ("bc_z", C.c_int), ("precision", C.c_int), ("seed", C.c_uint64),
                ("slots_per_cell", C.c_double), ("tile", C.c_int * 3), ("track_ids", C.c_int),
                ("explicit_ions", C.c_int), ("z_relative", C.c_int), ("stream", C.c_void_p)]


class Sizes(C.Structure):
    _fields_ = [("field_bytes", C.c_size_t), ("species_bytes", C.c_size_t * 2), ("scratch_bytes", C.c_size_t),
                ("slots", C.c_int64 * 2), ("ntiles", C.c_int64), ("tile_capacity", C.c_int),
                ("tile", C.c_int * 3), ("elem_bytes", C.c_int), ("dt", C.c_double), ("hx", C.c_double),
                ("hy", C.c_double), ("hz", C.c_double), ("beta", C.c_double)]


class Buffers(C.Structure):
    _fields_ = [("fields", C.c_void_p), ("species", C.c_void_p * 2), ("scratch", C.c_void_p)]


class PlasmaParams(C.Structure):
    _fields_ = [("ne_over_nc", C.c_double), ("z_start", C.c_double), ("z_end", C.c_double),
                ("ramp_len", C.c_double), ("ppc", C.c_int * 3), ("jitter", C.c_double),
                ("n_profile", C.c_int), ("profile", C.POINTER(C.c_double)), ("ions", C.c_int)]


class LaserParams(C.Structure):
    _fields_ = [("a0", C.c_double), ("waist", C.c_double), ("fwhm", C.c_double), ("z_antenna", C.c_double),
                ("t_peak", C.c_double), ("polarization", C.c_int), ("x_center", C.c_double),
                ("y_center", C.c_double)]


class Diag(C.Structure):
    _fields_ = [("t", C.c_double), ("step", C.c_int64), ("n_particles", C.c_int64 * 2), ("n_paired", C.c_int64),
                ("field_energy", C.c_double), ("kinetic_energy", C.c_double), ("charge", C.c_double), ("z_window", C.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


class BtdParams(C.Structure):
    """pic_btd_params: lab snapshots T_j = t0 + j dt, Z_k = z0 + k dz."""
    _fields_ = [("n_snapshots", C.c_int), ("t0", C.c_double), ("dt", C.c_double), ("z0", C.c_double),
                ("dz", C.c_double), ("nz", C.c_int), ("plane", C.c_int)]


class AdjointParams(C.Structure):
    """pic_adjoint_params: N steps, a checkpoint every K."""
    _fields_ = [("nsteps", C.c_int), ("checkpoint_every", C.c_int), ("sub_checkpoint_every", C.c_int)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    lib = C.CDLL(path)
    P, S, I, U = C.c_void_p, C.c_int, C.c_int, C.c_uint
    sig = {
        "pic_init_grid": (S, [C.POINTER(GridParams), C.POINTER(C.c_void_p)]),
        "pic_query_sizes": (S, [P, C.POINTER(Sizes)]),
        "pic_bind_buffers": (S, [P, C.POINTER(Buffers)]),
        "pic_load_plasma": (S, [P, C.POINTER(PlasmaParams)]),
        "pic_load_particles": (S, [P, I, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
        "pic_launch_laser": (S, [P, C.POINTER(LaserParams)]),
        "pic_step": (S, [P, I]),
        "pic_step_async": (S, [P, I]),
        "pic_step_phases": (S, [P, U]),
        "pic_get_fields": (S, [P, U, I, P, C.c_size_t, I]),
        "pic_set_fields": (S, [P, U, P, C.c_size_t, I]),
        "pic_get_axis": (S, [P, I, P, C.c_size_t, I]),
        "pic_get_particles": (S, [P, I, C.POINTER(C.c_double), C.c_size_t, C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int64)]),
        "pic_get_rho": (S, [P, P, C.c_size_t, I]),
        "pic_get_diagnostics": (S, [P, C.POINTER(Diag)]),
        "pic_state_bytes": (S, [P, C.POINTER(C.c_size_t)]),
        "pic_get_state": (S, [P, P, C.c_size_t, I]),
        "pic_set_state": (S, [P, P, C.c_size_t, I]),
        "pic_last_error": (C.c_char_p, [P]),
        "pic_status_string": (C.c_char_p, [S]),
        "pic_destroy": (None, [P]),
        "pic_profile": (S, [P, I]),
        "pic_profile_read": (S, [P, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "pic_filter_current_noalloc": (S, [I, I, I, I, I, I, I, P, P, P, P]),
        "pic_set_moving_window": (S, [P, C.c_double, C.c_double, I]),
        "pic_batch_create": (S, [C.POINTER(C.c_void_p), I, C.POINTER(C.c_void_p)]),
        "pic_batch_step": (S, [P, I]),
        "pic_batch_destroy": (None, [P]),
        "pic_batch_set_graph": (S, [P, I]),
        "pic_batch_set_fused": (S, [P, I]),
        "pic_sort_cells": (S, [P]),
        "pic_set_cell_sort": (S, [P, I]),
        "pic_batch_adjoint": (S, [P, C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_size_t),
                                  C.POINTER(C.c_void_p), C.POINTER(C.c_double), I]),
        "pic_batch_graph_info": (S, [P, C.POINTER(I), C.POINTER(C.c_int64), C.POINTER(I)]),
        "pic_btd_bytes": (S, [P, C.POINTER(BtdParams), C.POINTER(C.c_size_t)]),
        "pic_btd_setup": (S, [P, C.POINTER(BtdParams), P, C.c_size_t]),
        "pic_btd_get": (S, [P, I, P, C.c_size_t, I]),
        "pic_adjoint_bytes": (S, [P, C.POINTER(AdjointParams), C.POINTER(C.c_size_t)]),
        "pic_adjoint_forward": (S, [P, C.POINTER(AdjointParams), P, C.c_size_t, P]),
        "pic_adjoint_backward": (S, [P, P, C.POINTER(C.c_double)]),
        "pic_wait_check": (S, [I, C.c_double, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def lib():
    return _load()


def _check(ctx, status: int):
    if status != PIC_OK:
        detail = _load().pic_last_error(ctx).decode() if ctx else _load().pic_status_string(status).decode()
        raise PicError(status, detail or _load().pic_status_string(status).decode())


# ------------------------------------------------------ C-ABI, same names


def pic_init_grid(params: GridParams):
    ctx = C.c_void_p()
    st = _load().pic_init_grid(C.byref(params), C.byref(ctx))
    _check(None, st)
    return ctx


def pic_query_sizes(ctx) -> Sizes:
    s = Sizes()
    _check(ctx, _load().pic_query_sizes(ctx, C.byref(s)))
    return s


def pic_bind_buffers(ctx, bufs: Buffers):
    _check(ctx, _load().pic_bind_buffers(ctx, C.byref(bufs)))


def pic_load_plasma(ctx, p: PlasmaParams):
    _check(ctx, _load().pic_load_plasma(ctx, C.byref(p)))


def pic_load_particles(ctx, species: int, state, ids=None):
    """state: float64 array (7, n) = x, y, z, ux, uy, uz, w (host memory)."""
    import numpy as np
    st = np.ascontiguousarray(np.asarray(state, dtype=np.float64))
    n = st.shape[1] if st.ndim == 2 else 0
    idp = None
    if ids is not None:
        ids = np.ascontiguousarray(np.asarray(ids, dtype=np.int64))
        idp = ids.ctypes.data_as(C.POINTER(C.c_int64))
    _check(ctx, _load().pic_load_particles(ctx, species, n, st.ctypes.data_as(C.POINTER(C.c_double)), idp))


def pic_launch_laser(ctx, p: LaserParams):
    _check(ctx, _load().pic_launch_laser(ctx, C.byref(p)))


def pic_step(ctx, nsteps: int = 1):
    _check(ctx, _load().pic_step(ctx, int(nsteps)))


def pic_step_async(ctx, nsteps: int = 1):
    _check(ctx, _load().pic_step_async(ctx, int(nsteps)))


def pic_step_phases(ctx, mask: int):
    _check(ctx, _load().pic_step_phases(ctx, int(mask)))


def pic_get_fields(ctx, mask: int, frame: int, dst_ptr: int, dst_bytes: int, dst_is_device: bool):
    _check(ctx, _load().pic_get_fields(ctx, mask, int(frame), C.c_void_p(dst_ptr), dst_bytes, int(dst_is_device)))


def pic_set_fields(ctx, mask: int, src_ptr: int, src_bytes: int, src_is_device: bool):
    _check(ctx, _load().pic_set_fields(ctx, mask, C.c_void_p(src_ptr), src_bytes, int(src_is_device)))


def pic_get_axis(ctx, comp: int, dst_ptr: int, dst_bytes: int, dst_is_device: bool):
    _check(ctx, _load().pic_get_axis(ctx, comp, C.c_void_p(dst_ptr), dst_bytes, int(dst_is_device)))


def pic_get_particles(ctx, species: int, with_ids: bool = False):
    """Returns (state (7, n) float64, ids or None)."""
    import numpy as np
    n = C.c_int64(0)
    _check(ctx, _load().pic_get_particles(ctx, species, None, 0, C.byref(n), None))
    out = np.zeros((7, n.value), dtype=np.float64)
    ids = np.zeros(n.value, dtype=np.int64) if with_ids else None
    if n.value:
        _check(ctx, _load().pic_get_particles(ctx, species, out.ctypes.data_as(C.POINTER(C.c_double)), out.nbytes,
                                              C.byref(n), ids.ctypes.data_as(C.POINTER(C.c_int64))
                                              if ids is not None else None))
    return out, ids


def pic_get_rho(ctx, dst_ptr: int, dst_bytes: int, dst_is_device: bool):
    _check(ctx, _load().pic_get_rho(ctx, C.c_void_p(dst_ptr), dst_bytes, int(dst_is_device)))


def pic_get_diagnostics(ctx) -> Diag:
    d = Diag()
    _check(ctx, _load().pic_get_diagnostics(ctx, C.byref(d)))
    return d


def pic_state_bytes(ctx) -> int:
    n = C.c_size_t(0)
    _check(ctx, _load().pic_state_bytes(ctx, C.byref(n)))
    return n.value


def pic_get_state(ctx, dst_ptr: int, dst_bytes: int, dst_is_device: bool):
    _check(ctx, _load().pic_get_state(ctx, C.c_void_p(dst_ptr), dst_bytes, int(dst_is_device)))


def pic_set_state(ctx, src_ptr: int, src_bytes: int, src_is_device: bool):
    _check(ctx, _load().pic_set_state(ctx, C.c_void_p(src_ptr), src_bytes, int(src_is_device)))


def pic_last_error(ctx) -> str:
    return _load().pic_last_error(ctx).decode()


def pic_status_string(status: int) -> str:
    return _load().pic_status_string(status).decode()


def pic_destroy(ctx):
    _load().pic_destroy(ctx)


def pic_profile(ctx, enable: bool):
    _check(ctx, _load().pic_profile(ctx, int(enable)))


def pic_profile_read(ctx):
    """Returns (ms[8], calls[8], kernels) accumulated since the last read."""
    ms = (C.c_double * 8)()
    calls = (C.c_int64 * 8)()
    k = C.c_int64(0)
    _check(ctx, _load().pic_profile_read(ctx, ms, calls, C.byref(k)))
    return list(ms), list(calls), k.value


def pic_filter_current_noalloc(dim: int, nx: int, ny: int, nz: int, bc_z: int, passes: int, precision: int,
                               jx_ptr: int, jy_ptr: int, jz_ptr: int, stream_ptr: int = 0):
    """Filter Jx, Jy, Jz (device pointers, the library's layout) in place
    without any device allocation; see include/pic.h.  Raises PicError on a
    non-OK status, naming the size limit when that is the cause."""
    st = _load().pic_filter_current_noalloc(dim, nx, ny, nz, bc_z, passes, precision, C.c_void_p(jx_ptr),
                                            C.c_void_p(jy_ptr), C.c_void_p(jz_ptr), C.c_void_p(stream_ptr))
    if st != PIC_OK:
        nodes = (nz + 1) * ny * nx
        detail = _load().pic_status_string(st).decode()
        if st == PIC_ERR_ARG and nodes > PIC_NOALLOC_MAX_NODES:
            detail = f"{nodes} nodes per component exceed the static scratch of {PIC_NOALLOC_MAX_NODES} nodes"
        raise PicError(st, detail)


def pic_wait_check(arrive: bool, budget_ms: float, stream_ptr: int = 0) -> int:
    """Status of the bounded-wait self-check (PIC_OK or PIC_ERR_TIMEOUT)."""
    return int(_load().pic_wait_check(int(arrive), float(budget_ms), C.c_void_p(stream_ptr)))


def pic_batch_create(ctxs) -> int:
    arr = (C.c_void_p * len(ctxs))(*ctxs)
    out = C.c_void_p()
    st = _load().pic_batch_create(arr, len(ctxs), C.byref(out))
    if st != PIC_OK:
        raise PicError(st, _load().pic_status_string(st).decode())
    return out.value


def pic_batch_step(batch, nsteps: int):
    st = _load().pic_batch_step(batch, nsteps)
    if st != PIC_OK:
        raise PicError(st, _load().pic_status_string(st).decode())


def pic_batch_set_graph(batch, steps_per_graph: int):
    s = _load().pic_batch_set_graph(batch, int(steps_per_graph))
    if s != PIC_OK:
        raise PicError(s, "pic_batch_set_graph: " + pic_status_string(s))


def pic_sort_cells(ctx):
    _check(ctx, _load().pic_sort_cells(ctx))


def pic_set_cell_sort(ctx, every: int):
    _check(ctx, _load().pic_set_cell_sort(ctx, int(every)))


def pic_batch_set_fused(batch, chains):
    """chains: launch chains of the fused graph (0 or False: the per-context
    graph; True: the library's default of 4)."""
    n = (4 if chains else 0) if isinstance(chains, bool) else int(chains)
    s = _load().pic_batch_set_fused(batch, n)
    if s != PIC_OK:
        raise PicError(s, "pic_batch_set_fused: " + pic_status_string(s))


def pic_batch_graph_info(batch) -> dict:
    """{"fused", "chains", "launches_per_replay", "steps"} of the graph the
    batch keeps (chains: launch chains of the fused form, 0 per context)."""
    f, n, k = C.c_int(), C.c_int64(), C.c_int()
    s = _load().pic_batch_graph_info(batch, C.byref(f), C.byref(n), C.byref(k))
    if s != PIC_OK:
        raise PicError(s, "pic_batch_graph_info: " + pic_status_string(s))
    return {"fused": f.value > 0, "chains": int(f.value), "launches_per_replay": int(n.value),
            "steps": int(k.value)}


def pic_batch_adjoint(batch, params, buf_ptrs, nbytes, cot_ptrs, grad_stride: int):
    """Gradients of all runs of a batch (pic_batch_adjoint): a list of
    grad_stride doubles per run."""
    n = len(params)
    parr = (AdjointParams * n)(*params)
    bufs = (C.c_void_p * n)(*buf_ptrs)
    sizes = (C.c_size_t * n)(*nbytes)
    cots = (C.c_void_p * n)(*cot_ptrs)
    g = (C.c_double * (n * grad_stride))()
    s = _load().pic_batch_adjoint(batch, C.cast(parr, C.c_void_p), bufs, sizes, cots, g, int(grad_stride))
    if s != PIC_OK:
        raise PicError(s, "pic_batch_adjoint: " + pic_status_string(s))
    return [list(g[i * grad_stride:(i + 1) * grad_stride]) for i in range(n)]


def pic_batch_destroy(batch):
    _load().pic_batch_destroy(batch)


def pic_set_moving_window(ctx, v: float, t0: float, shift_cells: int):
    _check(ctx, _load().pic_set_moving_window(ctx, v, t0, shift_cells))


def pic_btd_bytes(ctx, p: BtdParams) -> int:
    n = C.c_size_t(0)
    _check(ctx, _load().pic_btd_bytes(ctx, C.byref(p), C.byref(n)))
    return n.value


def pic_btd_setup(ctx, p, buf_ptr: int, nbytes: int):
    """Start (p a BtdParams) or stop (p None) the lab-frame snapshots."""
    _check(ctx, _load().pic_btd_setup(ctx, C.byref(p) if p is not None else None, C.c_void_p(buf_ptr), nbytes))


def pic_btd_get(ctx, j: int, dst_ptr: int, dst_bytes: int, dst_is_device: bool):
    _check(ctx, _load().pic_btd_get(ctx, j, C.c_void_p(dst_ptr), dst_bytes, int(dst_is_device)))


def pic_adjoint_bytes(ctx, p: AdjointParams) -> int:
    n = C.c_size_t(0)
    _check(ctx, _load().pic_adjoint_bytes(ctx, C.byref(p), C.byref(n)))
    return n.value


def pic_adjoint_forward(ctx, p: AdjointParams, buf_ptr: int, nbytes: int, fields_out_ptr: int):
    _check(ctx, _load().pic_adjoint_forward(ctx, C.byref(p), C.c_void_p(buf_ptr), nbytes,
                                            C.c_void_p(fields_out_ptr) if fields_out_ptr else None))


def pic_adjoint_backward(ctx, cot_ptr: int, n_grad: int):
    g = (C.c_double * n_grad)()
    _check(ctx, _load().pic_adjoint_backward(ctx, C.c_void_p(cot_ptr), g))
    return list(g)


# --------------------------------------------------- torch-owned buffers


class Simulation:
    """Owns one context and the torch device buffers it is bound to."""

    def __init__(self, *, dim=2, nx=64, ny=1, nz=512, dx=0.5, dy=1.0, dz=1.0 / 16, cfl=0.99,
                 gamma_boost=1.0, shape_order=1, filter_passes=1, bc_z=PIC_BC_MUR, precision=PIC_FP32,
                 seed=10110917, slots_per_cell=8.0, tile=(0, 0, 0), track_ids=False, explicit_ions=False,
                 z_relative=0, device="cuda", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the PIC library needs a CUDA device; there is no CPU path")
        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.params = GridParams(dim, nx, ny, nz, dx, dy, dz, cfl, gamma_boost, shape_order, filter_passes, bc_z,
                                 precision, seed, slots_per_cell, (C.c_int * 3)(*tile), int(track_ids),
                                 int(explicit_ions), int(z_relative), C.c_void_p(self.stream.cuda_stream))
        self.ctx = pic_init_grid(self.params)
        self.sizes = pic_query_sizes(self.ctx)
        s = self.sizes

        def alloc(n):
            return torch.empty(max(int(n), 256), dtype=torch.uint8, device=self.device)

        self.fields_buf = alloc(s.field_bytes)
        self.species_buf = [alloc(s.species_bytes[0]), alloc(s.species_bytes[1]) if s.species_bytes[1] else None]
        self.scratch_buf = alloc(s.scratch_bytes)
        b = Buffers(self.fields_buf.data_ptr(),
                    (C.c_void_p * 2)(self.species_buf[0].data_ptr(),
                                     self.species_buf[1].data_ptr() if self.species_buf[1] is not None else None),
                    self.scratch_buf.data_ptr())
        pic_bind_buffers(self.ctx, b)
        self.dtype = torch.float64 if s.elem_bytes == 8 else torch.float32
        self.shape3 = (nz + 1, ny if dim == 3 else 1, nx)
        # profile coefficients loaded, and those of the adjoint forward run
        # (the library reports a backward pass without a forward one)
        self._prof_n = 0
        self._adj_n = 0

    # derived
    @property
    def dt(self):
        return self.sizes.dt

    def close(self):
        if getattr(self, "ctx", None):
            pic_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_plasma(self, ne, z_start, z_end, ramp=0.0, ppc=(2, 1, 2), jitter=0.1, profile=(), ions=1):
        prof = (C.c_double * max(1, len(profile)))(*profile) if len(profile) else None
        self._prof = prof
        self._prof_n = len(profile)
        p = PlasmaParams(ne, z_start, z_end, ramp, (C.c_int * 3)(*ppc), jitter, len(profile),
                         C.cast(prof, C.POINTER(C.c_double)) if prof is not None else None, ions)
        pic_load_plasma(self.ctx, p)

    def launch_laser(self, a0, waist, fwhm, z_antenna=0.0, t_peak=-1.0, polarization=PIC_POL_Y,
                     x_center=math.nan, y_center=math.nan):
        pic_launch_laser(self.ctx, LaserParams(a0, waist, fwhm, z_antenna, t_peak, polarization, x_center, y_center))

    def step(self, n=1):
        pic_step(self.ctx, n)

    def step_phases(self, mask):
        pic_step_phases(self.ctx, mask)

    def fields(self, mask=0x1FF, frame=0):
        """dict component -> torch tensor (nz+1, ny, nx) on the device; frame
        PIC_FRAME_LAB (1) gives the lab-frame E, B on the grid (mask <= 0x3F)."""
        comps = [c for q, c in enumerate(COMPONENTS) if mask >> q & 1]
        out = self.torch.empty((len(comps),) + self.shape3, dtype=self.dtype, device=self.device)
        pic_get_fields(self.ctx, mask, frame, out.data_ptr(), out.numel() * out.element_size(), True)
        return {c: out[q] for q, c in enumerate(comps)}

    def set_fields(self, values: dict):
        for c, v in values.items():
            q = COMPONENTS.index(c)
            t = self.torch.as_tensor(v, dtype=self.dtype, device=self.device).contiguous().reshape(self.shape3)
            pic_set_fields(self.ctx, 1 << q, t.data_ptr(), t.numel() * t.element_size(), True)

    def rho(self):
        out = self.torch.empty(self.shape3, dtype=self.dtype, device=self.device)
        pic_get_rho(self.ctx, out.data_ptr(), out.numel() * out.element_size(), True)
        return out

    def particles(self, species=PIC_ELECTRONS, with_ids=False):
        return pic_get_particles(self.ctx, species, with_ids)

    def load_particles(self, species, state, ids=None):
        pic_load_particles(self.ctx, species, state, ids)

    def diagnostics(self) -> Diag:
        return pic_get_diagnostics(self.ctx)

    def set_moving_window(self, v, t0, shift_cells):
        pic_set_moving_window(self.ctx, v, t0, shift_cells)

    def btd_setup(self, n_snapshots, t0, dt, z0, dz, nz, plane=0):
        """Lab-frame snapshots into a torch device buffer owned by this object."""
        p = BtdParams(n_snapshots, t0, dt, z0, dz, nz, plane)
        nbytes = pic_btd_bytes(self.ctx, p)
        self._btd = self.torch.empty(nbytes, dtype=self.torch.uint8, device=self.device)
        self._btd_p = p
        pic_btd_setup(self.ctx, p, self._btd.data_ptr(), nbytes)

    def btd_snapshot(self, j):
        """({Ex..Bz: (nz, nxs) float64 arrays}, filled (nz,) bool) of lab snapshot j."""
        import numpy as np
        p = self._btd_p
        nxs = self.params.nx if p.plane else 1
        es = self.sizes.elem_bytes
        nd = 6 * p.nz * nxs * es
        host = np.zeros(nd + 4 * p.nz, dtype=np.uint8)
        pic_btd_get(self.ctx, j, host.ctypes.data, host.nbytes, False)
        vals = host[:nd].view(np.float32 if es == 4 else np.float64).astype(np.float64).reshape(6, p.nz, nxs)
        filled = host[nd:].view(np.int32) != 0
        names = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")
        return {c: vals[q] for q, c in enumerate(names)}, filled


    def adjoint_checkpoint_interval(self, nsteps, budget_bytes=None):
        """The largest checkpoint interval K (nsteps, then halved) whose one-level
        adjoint buffer fits budget_bytes (default: half of the device memory
        free now): recomputation is traded for HBM only as far as needed."""
        if budget_bytes is None:
            free, _ = self.torch.cuda.mem_get_info(self.device)
            budget_bytes = free // 2
        k = int(nsteps)
        while k > 1 and pic_adjoint_bytes(self.ctx, AdjointParams(int(nsteps), k, 0)) > budget_bytes:
            k = (k + 1) // 2
        return k

    def adjoint_buffers(self, nsteps, checkpoint_every=50, sub_checkpoint_every=0):
        """The device buffers of an adjoint run (checkpoints and states; E^N,
        B^N), to be passed to adjoint_forward (allocated by it otherwise)."""
        p = AdjointParams(int(nsteps), int(checkpoint_every), int(sub_checkpoint_every))
        buf = self.torch.empty(pic_adjoint_bytes(self.ctx, p), dtype=self.torch.uint8, device=self.device)
        shape = (6,) + (self.shape3 if self.params.dim == 3 else (self.shape3[0], self.shape3[2]))
        return buf, self.torch.empty(shape, dtype=self.dtype, device=self.device)

    def adjoint_forward(self, nsteps, checkpoint_every=50, sub_checkpoint_every=0, buffers=None):
        """Forward run of the adjoint (from right after load_plasma and
        launch_laser): returns E^N, B^N as a (6, nz+1, nx) device tensor in 2D,
        (6, nz+1, ny, nx) in 3D, and keeps the checkpoints for adjoint_backward.
        buffers: those of adjoint_buffers (same arguments), else allocated here."""
        p = AdjointParams(int(nsteps), int(checkpoint_every), int(sub_checkpoint_every))
        if buffers is None:
            buffers = self.adjoint_buffers(nsteps, checkpoint_every, sub_checkpoint_every)
        self._adj, out = buffers
        self._adj_n = self._prof_n
        pic_adjoint_forward(self.ctx, p, self._adj.data_ptr(), self._adj.numel(), out.data_ptr())
        return out

    def adjoint_backward(self, cot):
        """Gradient of sum(cot * (E^N, B^N)) (cot shaped like adjoint_forward's
        output) with respect to the profile coefficients, a0 and the waist:
        a list [dL/dc_1, ..., dL/dc_M, dL/da0, dL/dw0]."""
        cot = self.torch.as_tensor(cot, dtype=self.dtype, device=self.device).contiguous()
        return pic_adjoint_backward(self.ctx, cot.data_ptr(), self._adj_n + 2)


class StageGradient:
    """torch.autograd.Function over one stage run: inputs the profile
    coefficients (M,) and the laser's a0 and w0 (0-d tensors, or None for w0
    to keep the waist of ``settings``); output E^N, B^N (6, nz+1, nx) in 2D,
    (6, nz+1, ny, nx) in 3D, on the device.  The forward builds the run from
    the fixed settings given to apply() and runs the library's adjoint forward
    (checkpoints kept in a device buffer); the backward runs the reverse sweep
    and returns each gradient on the device and in the dtype of its input, then
    releases the run."""

    @staticmethod
    def _function():
        import torch

        def _like(v, x):
            return torch.as_tensor(v, dtype=x.dtype, device=x.device) if isinstance(x, torch.Tensor) else None

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(ctx, coef, a0, w0, settings):
                sim = Simulation(**settings["grid"])
                p = settings["plasma"]
                sim.load_plasma(p["ne"], p["z_start"], p["z_end"], p.get("ramp", 0.0), p.get("ppc", (2, 1, 2)),
                                p.get("jitter", 0.1), [float(v) for v in coef.detach().cpu()], p.get("ions", 1))
                l = settings["laser"]
                sim.launch_laser(float(a0), l["waist"] if w0 is None else float(w0), l["fwhm"],
                                 l.get("z_antenna", 0.0), l.get("t_peak", -1.0), l.get("pol", PIC_POL_Y))
                out = sim.adjoint_forward(settings["nsteps"], settings.get("checkpoint_every", 50),
                                          settings.get("sub_checkpoint_every", 0))
                ctx.sim = sim
                ctx.m = coef.numel()
                ctx.inputs = (coef, a0, w0)
                return out.clone()

            @staticmethod
            def backward(ctx, grad_out):
                sim = ctx.sim
                try:
                    g = sim.adjoint_backward(grad_out)
                finally:
                    sim.close()
                    ctx.sim = None
                m = ctx.m
                coef, a0, w0 = ctx.inputs
                dc = torch.as_tensor(g[:m], dtype=coef.dtype, device=coef.device).reshape(coef.shape)
                return dc, _like(g[m], a0), _like(g[m + 1], w0), None

        return _F

    @classmethod
    def apply(cls, coef, a0, w0, settings):
        return cls._function().apply(coef, a0, w0, settings)


class Batch:
    """Steps several Simulations together: captured graphs of graph_steps
    steps, in the batched form when fused (the runs split into `fused` launch
    chains, True: 4, each chain one launch per phase over its runs), else
    each run's launches on its own stream."""

    def __init__(self, sims, graph_steps=20, fused=True):
        self.sims = list(sims)
        self.h = pic_batch_create([s.ctx for s in self.sims])
        pic_batch_set_graph(self.h, graph_steps)
        pic_batch_set_fused(self.h, fused)

    def graph_info(self) -> dict:
        return pic_batch_graph_info(self.h)

    def adjoint(self, nsteps, cots, checkpoint_every=50, sub_checkpoint_every=0):
        """Gradient of every run's objective sum(cot_r * (E^N, B^N)) (cot_r
        shaped like Simulation.adjoint_forward's output) with respect to its
        profile coefficients, a0 and waist, all runs' forward and reverse
        sweeps queued together (each run from right after its load_plasma and
        launch_laser): a list per run [dL/dc_1 .. dL/dc_M, dL/da0, dL/dw0]."""
        ps, bufs, cs = [], [], []
        for sim, cot in zip(self.sims, cots):
            p = AdjointParams(int(nsteps), int(checkpoint_every), int(sub_checkpoint_every))
            nb = pic_adjoint_bytes(sim.ctx, p)
            bufs.append(sim.torch.empty(nb, dtype=sim.torch.uint8, device=sim.device))
            cs.append(sim.torch.as_tensor(cot, dtype=sim.dtype, device=sim.device).contiguous())
            ps.append(p)
        m = [sim._prof_n for sim in self.sims]
        stride = max(m) + 2
        g = pic_batch_adjoint(self.h, ps, [b.data_ptr() for b in bufs], [b.numel() for b in bufs],
                              [c.data_ptr() for c in cs], stride)
        return [g[i][:m[i] + 2] for i in range(len(self.sims))]

    def step(self, nsteps: int = 1):
        pic_batch_step(self.h, nsteps)

    def close(self):
        if getattr(self, "h", None):
            pic_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
