"""ctypes declarations of the C ABI in include/psf.h (argument marshalling only).

The library is built in-tree (paper_2005_07547_b300/libpsf.so); there is no
fallback: if it is missing, load() raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpsf.so")

PSF_OK = 0
PSF_ERR_INVALID_ARG = -1
PSF_ERR_NO_MEM = -2
PSF_ERR_CUDA = -3
PSF_ERR_TOO_MANY = -4
NOALLOC_MAX_ITEMS = 64

STATUS_TABLE_FULL = 1
STATUS_RANGE = 2
STATUS_TIMEOUT = 4
STATUS_SUM_RANGE = 8

MAX_PROBE = 4096
MAX_BATCH = 256

_ERRORS = {PSF_ERR_INVALID_ARG: "invalid argument", PSF_ERR_NO_MEM: "insufficient memory",
           PSF_ERR_CUDA: "CUDA error"}


class Config(ctypes.Structure):
    """psf_config."""

    _fields_ = [
        ("log2_capacity", ctypes.c_uint32),
        ("pos_bits_q", ctypes.c_uint32),
        ("dir_bits_d", ctypes.c_uint32),
        ("use_normal", ctypes.c_uint32),
        ("alpha_min", ctypes.c_float),
        ("beta", ctypes.c_float),
        ("cv_max_depth", ctypes.c_uint32),
        ("frac_bits", ctypes.c_uint32),
        ("cache_fp16", ctypes.c_uint32),
        ("blend_mode", ctypes.c_uint32),
        ("key_layout", ctypes.c_uint32),
        ("levels", ctypes.c_uint32),
        ("payload", ctypes.c_uint32),
        ("sh_ridge", ctypes.c_float),
    ]


PAYLOAD_RGB = 0
PAYLOAD_SH = 1  # YCoCg, luminance in two SH bands over the normal


def make_config(log2_capacity: int = 16, pos_bits: int = 4, dir_bits: int = 2, use_normal: bool = True,
                alpha_min: float = 0.1, beta: float = 1.0, cv_max_depth: int = 0xFFFFFFFF,
                frac_bits: int = 24, cache_fp16: bool = False, blend_mode: int = 0, key_layout: int = 0,
                levels: int = 1, payload: int = PAYLOAD_RGB, sh_ridge: float = 0.01) -> Config:
    return Config(log2_capacity, pos_bits, dir_bits, int(bool(use_normal)), alpha_min, beta, cv_max_depth,
                  frac_bits, int(bool(cache_fp16)), blend_mode, key_layout, levels, payload, sh_ridge)


class Stats(ctypes.Structure):
    """psf_stats."""

    _fields_ = [
        ("capacity", ctypes.c_uint64),
        ("live_cells", ctypes.c_uint64),
        ("dropped_vertices", ctypes.c_uint64),
        ("zero_weight_vertices", ctypes.c_uint64),
        ("iterations", ctypes.c_uint64),
        ("status", ctypes.c_uint32),
        ("max_probe", ctypes.c_uint32),
        ("table_bytes", ctypes.c_uint64),
        ("touched_cells", ctypes.c_uint64),
        ("leader_groups", ctypes.c_uint64),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class LaunchConfig(ctypes.Structure):
    """psf_launch_config."""

    _fields_ = [
        ("insert_mode", ctypes.c_uint32),
        ("insert_blocks_per_sm", ctypes.c_uint32),
        ("update_blocks_per_sm", ctypes.c_uint32),
        ("query_blocks_per_sm", ctypes.c_uint32),
        ("vertex_staging", ctypes.c_uint32),
        ("sum_reduction", ctypes.c_uint32),
        ("query_layout", ctypes.c_uint32),
    ]


class BatchItem(ctypes.Structure):
    """psf_batch_item."""

    _fields_ = [
        ("table", ctypes.c_void_p),
        ("d_vertices", ctypes.c_void_p),
        ("d_out_rgb", ctypes.c_void_p),
        ("P", ctypes.c_uint32),
        ("D", ctypes.c_uint32),
        ("d_slots", ctypes.c_void_p),
    ]


class BatchConfig(ctypes.Structure):
    """psf_batch_config."""

    _fields_ = [
        ("insert_mode", ctypes.c_uint32),
        ("blocks_per_sm", ctypes.c_uint32),
        ("barrier_timeout_us", ctypes.c_uint32),
        ("test_phantom_blocks", ctypes.c_uint32),
        ("phase_blocks_per_sm", ctypes.c_uint32 * 3),
    ]


# psf_cell_record as a numpy structured dtype (72 bytes: 68 of fields, padded to 8-byte alignment)
CELL_DTYPE = np.dtype([("key", "<u8"), ("sum", "<i8", (3,)), ("c_new", "<i8"), ("c_old", "<i8"),
                       ("L", "<f4", (3,)), ("L_fp16", "<u2", (3,)), ("pad", "<u2")], align=True)
assert CELL_DTYPE.itemsize == 72
# psf_record (40 bytes): one cell's contribution of one iteration
RECORD_DTYPE = np.dtype([("key", "<u8"), ("sum", "<i8", (3,)), ("c_new", "<i8")])
assert RECORD_DTYPE.itemsize == 40
# psf_sh_cell_record (168 bytes)
SH_CELL_DTYPE = np.dtype([("key", "<u8"), ("sum", "<i8", (16,)), ("c_old", "<i8"), ("coef", "<f4", (6,))], align=True)
assert SH_CELL_DTYPE.itemsize == 168

# every function the header declares, with its ctypes signature
_vp, _u32, _u64, _i = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
SIGNATURES = {
    "psf_abi_version": (_i, []),
    "psf_last_cuda_error": (ctypes.c_char_p, []),
    "psf_table_bytes": (ctypes.c_size_t, [ctypes.POINTER(Config)]),
    "psf_create": (_i, [ctypes.POINTER(Config), _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]),
    "psf_insert": (_i, [_vp, _vp, _u64, _vp]),
    "psf_insert_progressive": (_i, [_vp, _vp, _u32, _u32, _u32, _vp]),
    "psf_update": (_i, [_vp, _vp]),
    "psf_query_cv": (_i, [_vp, _vp, _u32, _u32, _vp, _vp]),
    "psf_step": (_i, [_vp, _vp, _u32, _u32, _vp, _vp]),
    "psf_query_biased": (_i, [_vp, _vp, _u32, _u32, ctypes.c_float, _u32, _u32, _vp, _vp]),
    "psf_reset": (_i, [_vp, _vp]),
    "psf_export": (_i, [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t), _vp]),
    "psf_export_sh": (_i, [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t), _vp]),
    "psf_insert_records": (_i, [_vp, _vp, _u64, _vp]),
    "psf_set_approximant": (_i, [_vp, _vp, _vp, _u64, _vp]),
    "psf_get_stats": (_i, [_vp, ctypes.POINTER(Stats), _vp]),
    "psf_destroy": (_i, [_vp]),
    "psf_set_launch_config": (_i, [_vp, ctypes.POINTER(LaunchConfig)]),
    "psf_batch_create": (_i, [_u32, ctypes.POINTER(BatchConfig), ctypes.POINTER(_vp)]),
    "psf_batch_set": (_i, [_vp, ctypes.POINTER(BatchItem), _u32, _vp]),
    "psf_batch_launch": (_i, [_vp, _vp]),
    "psf_batch_step": (_i, [_vp, ctypes.POINTER(BatchItem), _u32, _vp]),
    "psf_batch_status": (_i, [_vp, ctypes.POINTER(_u32), _vp]),
    "psf_batch_destroy": (_i, [_vp]),
    "psf_batch_step_noalloc": (_i, [ctypes.POINTER(BatchItem), _u32, ctypes.POINTER(BatchConfig), _vp]),
    "psf_get_launch_config": (_i, [_vp, ctypes.POINTER(LaunchConfig)]),
    "psf_insert_slots": (_i, [_vp, _vp, _u32, _u32, _vp, _vp]),
    "psf_query_cv_slots": (_i, [_vp, _vp, _vp, _u32, _u32, _vp, _vp]),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load libpsf.so (built by paper_2005_07547_b300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2005_07547_b300.build` "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(rc: int, what: str) -> int:
    if rc < 0:
        detail = load().psf_last_cuda_error().decode() if rc == PSF_ERR_CUDA else ""
        raise RuntimeError(f"{what} failed: {_ERRORS.get(rc, rc)} {detail}".rstrip())
    return rc
