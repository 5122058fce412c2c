"""ctypes wrapper of the FP64 C oracle (pic_oracle.c) -- TEST INFRASTRUCTURE ONLY.

Arrays come back as numpy views of the oracle's own memory: field component c is
shaped (nz+1, ny, nx) (ny = 1 in 2D) in the oracle's index order (k, j, i).
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liboracle.so")

PH_ZERO_J, PH_PUSH, PH_IONS, PH_ANTENNA = 1, 2, 4, 8
PH_FILTER, PH_YEE, PH_INJECT, PH_TIME = 16, 32, 64, 128
PH_ALL = 255
COMPONENTS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc: -O2, strict IEEE (no contraction into FMA)."""
    src = os.path.join(HERE, "pic_oracle.c")
    os.makedirs(os.path.dirname(LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(src),
                                                   os.path.getmtime(os.path.join(HERE, "pic_oracle.h")))):
        return LIB_PATH
    tmp = LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                    "-shared", "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class _Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("cfl", C.c_double), ("gamma_boost", C.c_double),
                ("shape", C.c_int), ("npass", C.c_int), ("bc_z", C.c_int),
                ("seed", C.c_uint64)]


class _Plasma(C.Structure):
    _fields_ = [("ne", C.c_double), ("z_start", C.c_double), ("z_end", C.c_double),
                ("ramp", C.c_double), ("ppc", C.c_int * 3), ("jitter", C.c_double),
                ("nprof", C.c_int), ("prof", C.POINTER(C.c_double)), ("ions", C.c_int)]


class _Btd(C.Structure):
    _fields_ = [("nsnap", C.c_int), ("t0", C.c_double), ("dt", C.c_double), ("z0", C.c_double),
                ("dz", C.c_double), ("nz", C.c_int), ("plane", C.c_int)]


class _Laser(C.Structure):
    _fields_ = [("a0", C.c_double), ("waist", C.c_double), ("fwhm", C.c_double),
                ("z_antenna", C.c_double), ("t_peak", C.c_double), ("pol", C.c_int),
                ("xc", C.c_double), ("yc", C.c_double)]


@dataclasses.dataclass
class GridParams:
    dim: int = 2
    nx: int = 64
    ny: int = 1
    nz: int = 512
    dx: float = 0.5
    dy: float = 1.0
    dz: float = 1.0 / 16
    cfl: float = 0.99
    gamma_boost: float = 1.0
    shape: int = 1
    npass: int = 1
    bc_z: int = 1          # 0 periodic, 1 Mur
    seed: int = 10110917


@dataclasses.dataclass
class PlasmaParams:
    ne: float = 0.01
    z_start: float = 4.0
    z_end: float = 32.0
    ramp: float = 2.0
    ppc: tuple = (2, 1, 2)
    jitter: float = 0.1
    profile: tuple = ()
    ions: int = 1


@dataclasses.dataclass
class BtdParams:
    """Lab-frame snapshots: T_j = t0 + j dt (j < nsnap), Z_k = z0 + k dz (k < nz);
    plane 0 the axis line, 1 the (x, z) plane through the box centre."""
    nsnap: int = 4
    t0: float = 0.0
    dt: float = 10.0
    z0: float = 0.0
    dz: float = 1.0 / 32
    nz: int = 256
    plane: int = 0


@dataclasses.dataclass
class LaserParams:
    a0: float = 1.0
    waist: float = 8.0
    fwhm: float = 5.0
    z_antenna: float = 0.0
    t_peak: float = -1.0
    pol: int = 1
    xc: float = math.nan
    yc: float = math.nan


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build_oracle())
        P = C.c_void_p
        D = C.POINTER(C.c_double)
        lib.opic_create.restype = P
        lib.opic_create.argtypes = [C.POINTER(_Grid)]
        lib.opic_destroy.argtypes = [P]
        lib.opic_info.argtypes = [P, D]
        lib.opic_time.restype = C.c_double
        lib.opic_time.argtypes = [P]
        lib.opic_steps.restype = C.c_int64
        lib.opic_steps.argtypes = [P]
        lib.opic_load_plasma.restype = C.c_int64
        lib.opic_load_plasma.argtypes = [P, C.POINTER(_Plasma)]
        lib.opic_pending.restype = C.c_int64
        lib.opic_pending.argtypes = [P]
        lib.opic_set_laser.argtypes = [P, C.POINTER(_Laser)]
        lib.opic_add_particles.restype = C.c_int
        lib.opic_add_particles.argtypes = [P, C.c_int, C.c_int64] + [D] * 7 + [C.POINTER(C.c_int64)]
        lib.opic_num.restype = C.c_int64
        lib.opic_num.argtypes = [P, C.c_int]
        lib.opic_particles.restype = D
        lib.opic_particles.argtypes = [P, C.c_int, C.c_int]
        lib.opic_ids.restype = C.POINTER(C.c_int64)
        lib.opic_ids.argtypes = [P, C.c_int]
        lib.opic_field.restype = D
        lib.opic_field.argtypes = [P, C.c_int]
        lib.opic_rho_background.restype = D
        lib.opic_rho_background.argtypes = [P]
        lib.opic_step.argtypes = [P, C.c_int]
        lib.opic_step_phases.argtypes = [P, C.c_uint]
        lib.opic_gather.argtypes = [P, C.c_int64, D, D, D, D]
        lib.opic_boris.argtypes = [D, D, D, C.c_double, C.c_double]
        lib.opic_deposit_current.argtypes = [P, C.c_double, D, D, C.c_double]
        lib.opic_deposit_rho.argtypes = [P, D]
        lib.opic_filter.argtypes = [P]
        lib.opic_density.restype = C.c_double
        lib.opic_density.argtypes = [C.POINTER(_Plasma), C.c_double]
        lib.opic_shape.restype = C.c_double
        lib.opic_shape.argtypes = [C.c_int, C.c_double]
        lib.opic_splitmix64.restype = C.c_uint64
        lib.opic_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        lib.opic_uniform.restype = C.c_double
        lib.opic_uniform.argtypes = [C.c_uint64, C.c_uint64]
        lib.opic_set_window.restype = C.c_int
        lib.opic_set_window.argtypes = [P, C.c_double, C.c_double, C.c_int]
        lib.opic_window.restype = C.c_double
        lib.opic_window.argtypes = [P]
        lib.opic_btd_setup.restype = C.c_int
        lib.opic_btd_setup.argtypes = [P, C.POINTER(_Btd)]
        lib.opic_btd_data.restype = D
        lib.opic_btd_data.argtypes = [P, C.c_int]
        lib.opic_diagnostics.argtypes = [P, D]
        lib.opic_fields_lab.argtypes = [P, D]
        lib.opic_btd_filled.restype = C.POINTER(C.c_ubyte)
        lib.opic_btd_filled.argtypes = [P, C.c_int]
        _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _plasma_struct(p: PlasmaParams):
    prof = np.ascontiguousarray(np.asarray(p.profile, dtype=np.float64))
    st = _Plasma(p.ne, p.z_start, p.z_end, p.ramp, (C.c_int * 3)(*p.ppc), p.jitter,
                 len(prof), _dptr(prof) if len(prof) else None, p.ions)
    return st, prof


def lib():
    return _load()


class Oracle:
    """One FP64 simulation state."""

    def __init__(self, grid: GridParams):
        self.lib = _load()
        self.grid = grid
        g = _Grid(grid.dim, grid.nx, grid.ny, grid.nz, grid.dx, grid.dy, grid.dz, grid.cfl,
                  grid.gamma_boost, grid.shape, grid.npass, grid.bc_z, grid.seed)
        self.h = self.lib.opic_create(C.byref(g))
        if not self.h:
            raise ValueError(f"oracle rejected grid {grid}")
        info = np.zeros(8)
        self.lib.opic_info(self.h, _dptr(info))
        (self.dt, self.hx, self.hy, self.hz, self.beta, self.Lx, self.Ly, self.Lz) = info.tolist()
        self.ny = grid.ny if grid.dim == 3 else 1
        self.shape3 = (grid.nz + 1, self.ny, grid.nx)

    def close(self):
        if self.h:
            self.lib.opic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- state
    @property
    def t(self) -> float:
        return self.lib.opic_time(self.h)

    def field(self, c) -> np.ndarray:
        ci = COMPONENTS.index(c) if isinstance(c, str) else int(c)
        ptr = self.lib.opic_field(self.h, ci)
        n = int(np.prod(self.shape3))
        return np.ctypeslib.as_array(ptr, shape=(n,)).reshape(self.shape3)

    def fields(self) -> dict:
        return {c: self.field(c) for c in COMPONENTS}

    def rho_background(self) -> np.ndarray:
        ptr = self.lib.opic_rho_background(self.h)
        return np.ctypeslib.as_array(ptr, shape=(int(np.prod(self.shape3)),)).reshape(self.shape3)

    def num(self, sp: int = 0) -> int:
        return int(self.lib.opic_num(self.h, sp))

    def pending(self) -> int:
        return int(self.lib.opic_pending(self.h))

    def particles(self, sp: int = 0) -> dict:
        """Copies of x, y, z, ux, uy, uz, w (lambda0 units) and ids."""
        n = self.num(sp)
        out = {}
        if n == 0:
            for k in ("x", "y", "z", "ux", "uy", "uz", "w"):
                out[k] = np.zeros(0)
            out["id"] = np.zeros(0, dtype=np.int64)
            return out
        for a, k in enumerate(("x", "y", "z", "ux", "uy", "uz", "w")):
            ptr = self.lib.opic_particles(self.h, sp, a)
            out[k] = np.ctypeslib.as_array(ptr, shape=(n,)).copy()
        ptr = self.lib.opic_ids(self.h, sp)
        out["id"] = np.ctypeslib.as_array(ptr, shape=(n,)).copy()
        return out

    def add_particles(self, sp: int, x, y, z, ux, uy, uz, w, ids=None):
        arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in (x, y, z, ux, uy, uz, w)]
        n = len(arrs[0])
        idp = None
        if ids is not None:
            ids = np.ascontiguousarray(np.asarray(ids, dtype=np.int64))
            idp = ids.ctypes.data_as(C.POINTER(C.c_int64))
        rc = self.lib.opic_add_particles(self.h, sp, n, *[_dptr(a) for a in arrs], idp)
        if rc != 0:
            raise ValueError("opic_add_particles failed")

    def load_plasma(self, p: PlasmaParams) -> int:
        st, keep = _plasma_struct(p)
        n = self.lib.opic_load_plasma(self.h, C.byref(st))
        del keep
        if n < 0:
            raise ValueError(f"oracle rejected plasma {p}")
        return int(n)

    def set_laser(self, l: LaserParams):
        st = _Laser(l.a0, l.waist, l.fwhm, l.z_antenna, l.t_peak, l.pol, l.xc, l.yc)
        self.lib.opic_set_laser(self.h, C.byref(st))

    # ----------------------------------------------------------------- run
    def step(self, n: int = 1):
        self.lib.opic_step(self.h, int(n))

    def step_phases(self, mask: int):
        self.lib.opic_step_phases(self.h, int(mask))

    def gather(self, x, y, z) -> np.ndarray:
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
        y = np.ascontiguousarray(np.asarray(y, dtype=np.float64))
        z = np.ascontiguousarray(np.asarray(z, dtype=np.float64))
        out = np.zeros((len(x), 6))
        self.lib.opic_gather(self.h, len(x), _dptr(x), _dptr(y), _dptr(z), _dptr(out))
        return out

    def deposit_current(self, qw, x0, x1, vy=0.0):
        a = np.ascontiguousarray(np.asarray(x0, dtype=np.float64))
        b = np.ascontiguousarray(np.asarray(x1, dtype=np.float64))
        self.lib.opic_deposit_current(self.h, float(qw), _dptr(a), _dptr(b), float(vy))

    def rho(self) -> np.ndarray:
        out = np.zeros(self.shape3)
        self.lib.opic_deposit_rho(self.h, _dptr(out))
        return out

    def filter(self):
        self.lib.opic_filter(self.h)

    def zero_fields(self):
        for c in COMPONENTS:
            self.field(c)[...] = 0.0

    # --------------------------------------------------------- diagnostics
    def diagnostics(self) -> dict:
        """FP64 Kahan sums: field_energy, kinetic_energy (electrons), charge."""
        out = np.zeros(3)
        self.lib.opic_diagnostics(self.h, _dptr(out))
        return {"field_energy": float(out[0]), "kinetic_energy": float(out[1]), "charge": float(out[2])}

    def fields_lab(self) -> dict:
        """Lab-frame E, B on the simulation grid at the current time:
        {Ex..Bz: (nz+1, ny, nx)} (a copy)."""
        out = np.zeros((6,) + self.shape3)
        self.lib.opic_fields_lab(self.h, _dptr(out))
        return {c: out[q] for q, c in enumerate(COMPONENTS[:6])}

    # ------------------------------------------------------- moving window
    def set_window(self, v: float, t0: float, shift_cells: int):
        """Window moving at v along +z from t0, in moves of shift_cells cells
        (v = 0: off)."""
        if self.lib.opic_set_window(self.h, v, t0, shift_cells) != 0:
            raise ValueError("oracle rejected the moving window")

    @property
    def z_window(self) -> float:
        return self.lib.opic_window(self.h)

    # ------------------------------------------------ back-transformed data
    def btd_setup(self, b: "BtdParams | None"):
        if b is None:
            self.lib.opic_btd_setup(self.h, None)
            self.btd = None
            return
        s = _Btd(b.nsnap, b.t0, b.dt, b.z0, b.dz, b.nz, b.plane)
        if self.lib.opic_btd_setup(self.h, C.byref(s)) != 0:
            raise ValueError(f"oracle rejected snapshot parameters {b}")
        self.btd = b

    def btd_snapshot(self, j: int):
        """(fields {Ex..Bz: (nz, nxs)}, filled (nz,) bool) of lab snapshot j."""
        b = self.btd
        nxs = self.grid.nx if b.plane else 1
        d = np.ctypeslib.as_array(self.lib.opic_btd_data(self.h, j), shape=(6 * b.nz * nxs,))
        f = np.ctypeslib.as_array(self.lib.opic_btd_filled(self.h, j), shape=(b.nz,))
        d = d.reshape(6, b.nz, nxs).copy()
        return {c: d[q] for q, c in enumerate(COMPONENTS[:6])}, f.astype(bool).copy()


def boris(u, e, b, q_over_m, dt):
    """Single Boris step on a copy of u (3-vector)."""
    lib_ = _load()
    u = np.array(u, dtype=np.float64)
    e = np.ascontiguousarray(np.asarray(e, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
    lib_.opic_boris(_dptr(u), _dptr(e), _dptr(b), float(q_over_m), float(dt))
    return u


def density(p: PlasmaParams, z: float) -> float:
    st, keep = _plasma_struct(p)
    v = _load().opic_density(C.byref(st), float(z))
    del keep
    return v


def shape(order: int, d: float) -> float:
    return _load().opic_shape(int(order), float(d))


def splitmix64(seed: int, counter: int) -> int:
    return int(_load().opic_splitmix64(C.c_uint64(seed), C.c_uint64(counter)))


def uniform(seed: int, counter: int) -> float:
    return float(_load().opic_uniform(C.c_uint64(seed), C.c_uint64(counter)))
