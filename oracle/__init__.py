"""CPU oracle for the progressive spatio-temporal filtering hot path.

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this package and shares no code with it.  See psf_oracle.cpp for the
definitions it follows and how each function is pinned.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psf_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

STATUS_TABLE_FULL = 1
STATUS_RANGE = 2
STATUS_SUM_RANGE = 8

RECORD_DTYPE = np.dtype([("key", "<u8"), ("sum", "<i8", (3,)), ("c_new", "<i8"), ("c_old", "<i8"),
                         ("L", "<f8", (3,))])
# the YCoCg two-band SH payload: sums Y, Co, Cg, c_new, n(3), Y n(3), n n(xx, xy, xz, yy, yz, zz);
# coefficients a, g_x, g_y, g_z, Co, Cg (luminance a + g . n)
SH_RECORD_DTYPE = np.dtype([("key", "<u8"), ("sum", "<i8", (16,)), ("c_old", "<i8"), ("coef", "<f8", (6,))])


class _Config(ctypes.Structure):
    _fields_ = [("pos_bits_q", ctypes.c_uint32), ("dir_bits_d", ctypes.c_uint32),
                ("use_normal", ctypes.c_uint32), ("frac_bits", ctypes.c_uint32),
                ("blend_mode", ctypes.c_uint32), ("cv_max_depth", ctypes.c_uint32),
                ("alpha_min", ctypes.c_double), ("beta", ctypes.c_double), ("levels", ctypes.c_uint32),
                ("pad", ctypes.c_uint32)]


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (IEEE single-rounding semantics: no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = f"{_LIB}.{os.getpid()}.tmp"  # concurrent test workers each build their own copy
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    """The oracle library; PSF_ORACLE_LIB names another build of it (the mutation tests
    point it at deliberately broken copies to check that the pins catch them)."""
    global _lib
    if _lib is None:
        L = ctypes.CDLL(os.environ.get("PSF_ORACLE_LIB") or build())
        vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        L.oracle_create.restype = vp
        L.oracle_create.argtypes = [ctypes.POINTER(_Config)]
        L.oracle_destroy.argtypes = [vp]
        L.oracle_key.restype = ctypes.c_int
        L.oracle_key.argtypes = [ctypes.POINTER(_Config), vp, ctypes.POINTER(u64)]
        L.oracle_key_at.restype = ctypes.c_int
        L.oracle_key_at.argtypes = [ctypes.POINTER(_Config), vp, u32, ctypes.POINTER(u64)]
        L.oracle_insert.restype = u32
        L.oracle_insert.argtypes = [vp, vp, u64]
        L.oracle_insert_progressive.restype = u32
        L.oracle_insert_progressive.argtypes = [vp, vp, u32, u32, u32]
        L.oracle_update.restype = u32
        L.oracle_update.argtypes = [vp]
        L.oracle_reset.argtypes = [vp]
        L.oracle_query_cv.argtypes = [vp, vp, u32, u32, vp]
        L.oracle_lookup.argtypes = [vp, vp, u64, vp]
        L.oracle_lookup_paths.argtypes = [vp, vp, u32, u32, vp]
        L.oracle_query_biased.argtypes = [vp, vp, u32, u32, ctypes.c_double, u32, u32, vp]
        L.oracle_size.restype = u64
        L.oracle_size.argtypes = [vp]
        L.oracle_counters.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.oracle_export.restype = u64
        L.oracle_export.argtypes = [vp, vp, u64]
        L.oracle_import.argtypes = [vp, vp, u64]
        L.oracle_sh_create.restype = vp
        L.oracle_sh_create.argtypes = [ctypes.POINTER(_Config), ctypes.c_double]
        L.oracle_sh_destroy.argtypes = [vp]
        L.oracle_sh_insert.restype = u32
        L.oracle_sh_insert.argtypes = [vp, vp, u64]
        L.oracle_sh_update.restype = u32
        L.oracle_sh_update.argtypes = [vp]
        L.oracle_sh_reset.argtypes = [vp]
        L.oracle_sh_lookup.argtypes = [vp, vp, u64, vp]
        L.oracle_sh_query_cv.argtypes = [vp, vp, u32, u32, vp]
        L.oracle_sh_size.restype = u64
        L.oracle_sh_size.argtypes = [vp]
        L.oracle_sh_counters.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.oracle_sh_export.restype = u64
        L.oracle_sh_export.argtypes = [vp, vp, u64]
        _lib = L
    return _lib


def make_config(pos_bits: int = 4, dir_bits: int = 2, use_normal: bool = True, frac_bits: int = 24,
                blend_mode: int = 0, cv_max_depth: int = 0xFFFFFFFF, alpha_min: float = 0.1,
                beta: float = 1.0, levels: int = 1) -> _Config:
    return _Config(pos_bits, dir_bits, int(bool(use_normal)), frac_bits, blend_mode, cv_max_depth,
                   float(alpha_min), float(beta), levels, 0)


def _verts(v: np.ndarray) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.float32)
    if v.ndim != 2 or v.shape[1] != 16:
        raise ValueError("vertices must be (n, 16) float32")
    return v


def vertex_key(cfg: _Config, v16, level: int = 0) -> int | None:
    """Packed cell key of one vertex record at a hierarchy level, or None if the vertex has
    no valid cell."""
    v = np.ascontiguousarray(v16, dtype=np.float32).reshape(16)
    out = ctypes.c_uint64()
    if level == 0:
        ok = lib().oracle_key(ctypes.byref(cfg), v.ctypes.data, ctypes.byref(out))
    else:
        ok = lib().oracle_key_at(ctypes.byref(cfg), v.ctypes.data, level, ctypes.byref(out))
    return int(out.value) if ok else None


class Oracle:
    """std::map-backed reference table (one render session)."""

    def __init__(self, cfg: _Config | None = None, **kw):
        self.cfg = cfg if cfg is not None else make_config(**kw)
        self._h = lib().oracle_create(ctypes.byref(self.cfg))
        if not self._h:
            raise ValueError("invalid oracle configuration")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oracle_destroy(h)
            self._h = None

    def insert(self, verts: np.ndarray) -> int:
        v = _verts(verts)
        return int(lib().oracle_insert(self._h, v.ctypes.data, v.shape[0]))

    def insert_progressive(self, verts: np.ndarray, P: int, D: int, field: int = 0) -> int:
        """Scatter with update values from the approximant at the next vertex (eq. 9)."""
        v = _verts(verts)
        if v.shape[0] != P * D:
            raise ValueError("vertex count must be P*D")
        return int(lib().oracle_insert_progressive(self._h, v.ctypes.data, P, D, field))

    def update(self) -> int:
        return int(lib().oracle_update(self._h))

    def reset(self) -> None:
        lib().oracle_reset(self._h)

    def query_cv(self, verts: np.ndarray, P: int, D: int) -> np.ndarray:
        v = _verts(verts)
        if v.shape[0] != P * D:
            raise ValueError("vertex count must be P*D")
        out = np.empty((P * D, 3), dtype=np.float64)
        lib().oracle_query_cv(self._h, v.ctypes.data, P, D, out.ctypes.data)
        return out

    def query_biased(self, verts: np.ndarray, P: int, D: int, gamma: float, j_begin: int = 0,
                     j_end: int = 0xFFFFFFFF) -> np.ndarray:
        v = _verts(verts)
        if v.shape[0] != P * D:
            raise ValueError("vertex count must be P*D")
        out = np.empty((P * D, 3), dtype=np.float64)
        lib().oracle_query_biased(self._h, v.ctypes.data, P, D, float(gamma), j_begin, j_end, out.ctypes.data)
        return out

    def lookup(self, verts: np.ndarray, P: int | None = None, D: int | None = None) -> np.ndarray:
        """(n, 3) approximant of each vertex's cell, 0 where the cell is absent; given P and D
        (depth-major paths) vertex j reads the level a query reads, min(j, levels - 1)."""
        v = _verts(verts)
        out = np.empty((v.shape[0], 3), dtype=np.float64)
        if P is None:
            lib().oracle_lookup(self._h, v.ctypes.data, v.shape[0], out.ctypes.data)
        else:
            lib().oracle_lookup_paths(self._h, v.ctypes.data, P, D, out.ctypes.data)
        return out

    def __len__(self) -> int:
        return int(lib().oracle_size(self._h))

    def counters(self) -> tuple[int, int]:
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        lib().oracle_counters(self._h, ctypes.byref(a), ctypes.byref(b))
        return int(a.value), int(b.value)

    def export(self) -> np.ndarray:
        n = len(self)
        out = np.zeros(n, dtype=RECORD_DTYPE)
        got = lib().oracle_export(self._h, out.ctypes.data, n)
        return out[:got]

    def import_records(self, recs: np.ndarray) -> None:
        r = np.ascontiguousarray(recs, dtype=RECORD_DTYPE)
        lib().oracle_import(self._h, r.ctypes.data, r.shape[0])


class ShOracle:
    """std::map-backed reference table with the YCoCg two-band SH payload: per cell, luminance
    fitted over the normal (a + g . n, ridge on g) and constant chroma (see psf_oracle.cpp)."""

    def __init__(self, cfg: _Config | None = None, ridge: float = 0.01, **kw):
        self.cfg = cfg if cfg is not None else make_config(**kw)
        self.ridge = float(ridge)
        self._h = lib().oracle_sh_create(ctypes.byref(self.cfg), self.ridge)
        if not self._h:
            raise ValueError("invalid oracle configuration")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oracle_sh_destroy(h)
            self._h = None

    def insert(self, verts: np.ndarray) -> int:
        v = _verts(verts)
        return int(lib().oracle_sh_insert(self._h, v.ctypes.data, v.shape[0]))

    def update(self) -> int:
        return int(lib().oracle_sh_update(self._h))

    def reset(self) -> None:
        lib().oracle_sh_reset(self._h)

    def lookup(self, verts: np.ndarray) -> np.ndarray:
        """(n, 3) RGB of each vertex's cell fit at the vertex's normal, 0 where absent."""
        v = _verts(verts)
        out = np.empty((v.shape[0], 3), dtype=np.float64)
        lib().oracle_sh_lookup(self._h, v.ctypes.data, v.shape[0], out.ctypes.data)
        return out

    def query_cv(self, verts: np.ndarray, P: int, D: int) -> np.ndarray:
        v = _verts(verts)
        if v.shape[0] != P * D:
            raise ValueError("vertex count must be P*D")
        out = np.empty((P * D, 3), dtype=np.float64)
        lib().oracle_sh_query_cv(self._h, v.ctypes.data, P, D, out.ctypes.data)
        return out

    def __len__(self) -> int:
        return int(lib().oracle_sh_size(self._h))

    def counters(self) -> tuple[int, int]:
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        lib().oracle_sh_counters(self._h, ctypes.byref(a), ctypes.byref(b))
        return int(a.value), int(b.value)

    def export(self) -> np.ndarray:
        n = len(self)
        out = np.zeros(n, dtype=SH_RECORD_DTYPE)
        got = lib().oracle_sh_export(self._h, out.ctypes.data, n)
        return out[:got]
