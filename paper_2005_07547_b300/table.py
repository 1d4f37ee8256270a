"""Python view of one filtering table (one render session) over the C ABI.

PyTorch supplies the device memory (the caching allocator) and the stream; every
step of the computation runs in the CUDA library.
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import _abi


def _stream_handle(stream) -> int:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check_vertices(verts, what: str):
    import torch

    if not isinstance(verts, torch.Tensor) or not verts.is_cuda:
        raise TypeError(f"{what}: vertices must be a CUDA tensor")
    if verts.dtype != torch.float32 or verts.dim() != 2 or verts.shape[1] != 16 or not verts.is_contiguous():
        raise ValueError(f"{what}: vertices must be a contiguous (n, 16) float32 tensor")


class Table:
    """A spatio-directional field table in caller-owned (torch) device memory."""

    def __init__(self, cfg: _abi.Config | None = None, device=None, stream=None, **kw):
        import torch

        lib = _abi.load()
        self.cfg = cfg if cfg is not None else _abi.make_config(**kw)
        self.nbytes = int(lib.psf_table_bytes(ctypes.byref(self.cfg)))
        if self.nbytes == 0:
            raise ValueError("invalid psf configuration")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.mem = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        _abi.check(lib.psf_create(ctypes.byref(self.cfg), self.mem.data_ptr(), self.nbytes,
                                  _stream_handle(stream), ctypes.byref(h)), "psf_create")
        self._h = h

    @property
    def handle(self) -> int:
        return self._h.value

    def insert(self, verts, stream=None) -> None:
        _check_vertices(verts, "insert")
        _abi.check(_abi.load().psf_insert(self._h, verts.data_ptr(), verts.shape[0], _stream_handle(stream)),
                   "psf_insert")

    def insert_progressive(self, verts, P: int, D: int, field: int = 0, stream=None) -> None:
        """Scatter values computed from the approximant at each next vertex (eq. 9; field 0:
        L~_o as in Alg. 1, field 1: L~_{o\\e} as in Alg. 2)."""
        _check_vertices(verts, "insert_progressive")
        if verts.shape[0] != P * D:
            raise ValueError("insert_progressive: vertex count must be P*D")
        _abi.check(_abi.load().psf_insert_progressive(self._h, verts.data_ptr(), P, D, field, _stream_handle(stream)),
                   "psf_insert_progressive")

    def insert_slots(self, verts, P: int, D: int, slots=None, stream=None):
        """psf_insert of D*P depth-major records that also notes, per vertex, the slot its
        query will read (int32 view of uint32; -1 is PSF_NO_SLOT).  Returns the slots."""
        import torch

        _check_vertices(verts, "insert_slots")
        if verts.shape[0] != P * D:
            raise ValueError("insert_slots: vertex count must be P*D")
        if slots is None:
            slots = torch.empty(P * D, dtype=torch.int32, device=verts.device)
        if slots.dtype != torch.int32 or slots.numel() != P * D or not slots.is_contiguous():
            raise ValueError("insert_slots: slots must be a contiguous int32 tensor of P*D")
        _abi.check(_abi.load().psf_insert_slots(self._h, verts.data_ptr(), P, D, slots.data_ptr(),
                                                _stream_handle(stream)), "psf_insert_slots")
        return slots

    def update(self, stream=None) -> int:
        return _abi.check(_abi.load().psf_update(self._h, _stream_handle(stream)), "psf_update")

    def query_cv(self, verts, P: int, D: int, out=None, stream=None):
        import torch

        _check_vertices(verts, "query_cv")
        if verts.shape[0] != P * D:
            raise ValueError("query_cv: vertex count must be P*D")
        if out is None:
            out = torch.empty((P * D, 3), dtype=torch.float32, device=verts.device)
        _abi.check(_abi.load().psf_query_cv(self._h, verts.data_ptr(), P, D, out.data_ptr(),
                                            _stream_handle(stream)), "psf_query_cv")
        return out

    def query_cv_slots(self, verts, slots, P: int, D: int, out=None, stream=None):
        """query_cv reading each vertex's approximant at the slot insert_slots noted."""
        import torch

        _check_vertices(verts, "query_cv_slots")
        if verts.shape[0] != P * D or slots.numel() != P * D or slots.dtype != torch.int32:
            raise ValueError("query_cv_slots: P*D vertices and P*D int32 slots")
        if out is None:
            out = torch.empty((P * D, 3), dtype=torch.float32, device=verts.device)
        _abi.check(_abi.load().psf_query_cv_slots(self._h, verts.data_ptr(), slots.data_ptr(), P, D, out.data_ptr(),
                                                  _stream_handle(stream)), "psf_query_cv_slots")
        return out

    def query_biased(self, verts, P: int, D: int, gamma: float, j_begin: int = 0, j_end: int = 0xFFFFFFFF, out=None,
                     stream=None):
        """gamma * (L - t * C_next) + C on vertices j_begin <= j < j_end (PSTF-B: gamma 0, j 1..2)."""
        import torch

        _check_vertices(verts, "query_biased")
        if verts.shape[0] != P * D:
            raise ValueError("query_biased: vertex count must be P*D")
        if out is None:
            out = torch.empty((P * D, 3), dtype=torch.float32, device=verts.device)
        _abi.check(_abi.load().psf_query_biased(self._h, verts.data_ptr(), P, D, gamma, j_begin, j_end, out.data_ptr(),
                                                _stream_handle(stream)), "psf_query_biased")
        return out

    def step(self, verts, P: int, D: int, out=None, stream=None):
        import torch

        _check_vertices(verts, "step")
        if verts.shape[0] != P * D:
            raise ValueError("step: vertex count must be P*D")
        if out is None:
            out = torch.empty((P * D, 3), dtype=torch.float32, device=verts.device)
        _abi.check(_abi.load().psf_step(self._h, verts.data_ptr(), P, D, out.data_ptr(), _stream_handle(stream)),
                   "psf_step")
        return out

    def insert_records(self, records, stream=None) -> None:
        """Add pre-aggregated cell records (a (n, 5) int64 CUDA tensor laid out as psf_record:
        key, three sums, c_new) to this iteration, as a sharded session's owner does."""
        import torch

        if not isinstance(records, torch.Tensor) or not records.is_cuda or records.dtype != torch.int64 or \
                records.dim() != 2 or records.shape[1] != 5 or not records.is_contiguous():
            raise ValueError("insert_records: records must be a contiguous (n, 5) int64 CUDA tensor")
        _abi.check(_abi.load().psf_insert_records(self._h, records.data_ptr(), records.shape[0], _stream_handle(stream)),
                   "psf_insert_records")

    def set_approximant(self, keys, L, stream=None) -> None:
        """Write the approximant of the given cells (keys: (n,) int64 CUDA tensor holding the
        uint64 keys, L: (n, 3) float32 CUDA tensor)."""
        import torch

        if keys.dtype != torch.int64 or L.dtype != torch.float32 or tuple(L.shape) != (keys.shape[0], 3) or \
                not (keys.is_cuda and L.is_cuda and keys.is_contiguous() and L.is_contiguous()):
            raise ValueError("set_approximant: (n,) int64 keys and (n, 3) float32 values on the device")
        _abi.check(_abi.load().psf_set_approximant(self._h, keys.data_ptr(), L.data_ptr(), keys.shape[0],
                                                   _stream_handle(stream)), "psf_set_approximant")

    def reset(self, stream=None) -> None:
        _abi.check(_abi.load().psf_reset(self._h, _stream_handle(stream)), "psf_reset")

    def export(self, stream=None) -> np.ndarray:
        """All occupied cells in ascending key order (synchronises the stream): psf_cell_record
        rows, or psf_sh_cell_record rows for a table with the SH payload."""
        lib = _abi.load()
        sh = self.cfg.payload == _abi.PAYLOAD_SH
        fn, name, dtype = ((lib.psf_export_sh, "psf_export_sh", _abi.SH_CELL_DTYPE) if sh else
                           (lib.psf_export, "psf_export", _abi.CELL_DTYPE))
        n = ctypes.c_size_t()
        rc = fn(self._h, None, 0, ctypes.byref(n), _stream_handle(stream))
        if rc not in (_abi.PSF_OK, _abi.PSF_ERR_NO_MEM):
            _abi.check(rc, name)
        out = np.zeros(n.value, dtype=dtype)
        if n.value:
            got = ctypes.c_size_t()
            _abi.check(fn(self._h, out.ctypes.data, n.value, ctypes.byref(got), _stream_handle(stream)), name)
            out = out[:got.value]
        return out

    def stats(self, stream=None) -> dict:
        st = _abi.Stats()
        _abi.check(_abi.load().psf_get_stats(self._h, ctypes.byref(st), _stream_handle(stream)), "psf_get_stats")
        return st.as_dict()

    def set_launch(self, insert_mode: int = 0, insert_blocks_per_sm: int = 0, update_blocks_per_sm: int = 0,
                   query_blocks_per_sm: int = 0, vertex_staging: int = 0, sum_reduction: int = 0,
                   query_layout: int = 0) -> None:
        lc = _abi.LaunchConfig(insert_mode, insert_blocks_per_sm, update_blocks_per_sm, query_blocks_per_sm,
                               vertex_staging, sum_reduction, query_layout)
        _abi.check(_abi.load().psf_set_launch_config(self._h, ctypes.byref(lc)), "psf_set_launch_config")

    def get_launch(self) -> dict:
        lc = _abi.LaunchConfig()
        _abi.check(_abi.load().psf_get_launch_config(self._h, ctypes.byref(lc)), "psf_get_launch_config")
        return {name: getattr(lc, name) for name, _ in lc._fields_}

    def close(self, synchronize: bool = True) -> None:
        """Release the table: first wait for the device, unless the caller already knows
        that every kernel enqueued on the table has completed (synchronize=False; then
        nothing here waits on the device)."""
        import torch

        if getattr(self, "_h", None) is not None and self._h.value:
            if synchronize:
                torch.cuda.synchronize(self.device)
            _abi.load().psf_destroy(self._h)
            self._h = ctypes.c_void_p()
        self.mem = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
