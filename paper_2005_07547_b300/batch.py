"""Batched iterations over many tables: one persistent fused kernel per iteration.

The descriptors live in device memory, so `launch()` can be captured in a CUDA
graph once and replayed while `set()` changes which sessions the descriptors
describe (only the copy of the descriptors runs outside the graph).
"""

from __future__ import annotations

import ctypes

from . import _abi
from .table import _check_vertices, _stream_handle


class Batch:
    def __init__(self, max_items: int, insert_mode: int = 0, blocks_per_sm: int = 0, barrier_timeout_us: int = 0,
                 test_phantom_blocks: int = 0, insert_blocks_per_sm: int = 0, update_blocks_per_sm: int = 0,
                 query_blocks_per_sm: int = 0):
        """insert/update/query_blocks_per_sm: how many of the resident blocks per SM work in that
        phase of the fused kernel (0: all of them)."""
        self.max_items = max_items
        self.cfg = _abi.BatchConfig(insert_mode, blocks_per_sm, barrier_timeout_us, test_phantom_blocks,
                                    (ctypes.c_uint32 * 3)(insert_blocks_per_sm, update_blocks_per_sm,
                                                          query_blocks_per_sm))
        h = ctypes.c_void_p()
        _abi.check(_abi.load().psf_batch_create(max_items, ctypes.byref(self.cfg), ctypes.byref(h)), "psf_batch_create")
        self._h = h
        self._keep = []  # tensors the current descriptors point at

    @staticmethod
    def _items(entries):
        """entries: iterable of (Table, vertices (P*D, 16) cuda tensor, out (P*D, 3) cuda tensor, P, D)
        or the same with a sixth element, a (P*D,) int32 cuda tensor: the item's slot cache."""
        import torch

        entries = list(entries)
        arr = (_abi.BatchItem * max(1, len(entries)))()
        keep = []
        for i, entry in enumerate(entries):
            table, verts, out, P, D = entry[:5]
            slots = entry[5] if len(entry) > 5 else None
            if P * D:
                _check_vertices(verts, "batch")
                if verts.shape[0] != P * D or tuple(out.shape) != (P * D, 3) or not out.is_contiguous():
                    raise ValueError("batch: vertices must be (P*D, 16) and outputs (P*D, 3)")
                if slots is not None and (slots.dtype != torch.int32 or slots.numel() != P * D or
                                          not slots.is_contiguous()):
                    raise ValueError("batch: slots must be a contiguous int32 tensor of P*D")
            arr[i] = _abi.BatchItem(table.handle, verts.data_ptr() if P * D else None,
                                    out.data_ptr() if P * D else None, P, D,
                                    slots.data_ptr() if (slots is not None and P * D) else None)
            keep.append((table, verts, out, slots))
        return arr, len(entries), keep

    def set(self, entries, stream=None) -> None:
        arr, n, keep = self._items(entries)
        _abi.check(_abi.load().psf_batch_set(self._h, arr, n, _stream_handle(stream)), "psf_batch_set")
        self._keep = keep

    def launch(self, stream=None) -> None:
        _abi.check(_abi.load().psf_batch_launch(self._h, _stream_handle(stream)), "psf_batch_launch")

    def step(self, entries, stream=None) -> None:
        arr, n, keep = self._items(entries)
        _abi.check(_abi.load().psf_batch_step(self._h, arr, n, _stream_handle(stream)), "psf_batch_step")
        self._keep = keep

    def status(self, stream=None) -> int:
        s = ctypes.c_uint32()
        _abi.check(_abi.load().psf_batch_status(self._h, ctypes.byref(s), _stream_handle(stream)), "psf_batch_status")
        return int(s.value)

    def close(self) -> None:
        import torch

        if getattr(self, "_h", None) is not None and self._h.value:
            torch.cuda.synchronize()
            _abi.load().psf_batch_destroy(self._h)
            self._h = ctypes.c_void_p()
        self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
