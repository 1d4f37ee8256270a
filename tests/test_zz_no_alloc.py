"""psf_batch_step_noalloc: the batched fused iteration for callers that cannot allocate
device memory on their frame path (a pool that owns all device memory, or a loop that
must not call cudaMalloc/cudaFree because they can synchronize the device).

Checked through the C ABI against the allocating entry point (psf_batch_set +
psf_batch_launch) on the same inputs, two calls in a row: identical tables and outputs.
This file is collected last on purpose."""

import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(64, 3), (40, 2), (96, 5), (33, 4), (72, 6)]


def _sessions():
    from synth.scene import config4_q_bits

    out = []
    for k, (w, d) in enumerate(SHAPES):
        h = int(round(9 * w / 16))
        cap = int(math.ceil(math.log2(w * h * d))) + 1
        out.append(dict(width=w, height=h, depth=d, log2_capacity=cap, pos_bits=config4_q_bits(cap, 3), dir_bits=3,
                        alpha_min=0.1, radiance="glossy", seed=9000 + k, camera_step=0.0, camera_x0=0.5,
                        cache_fp16=bool(k % 2)))
    return out


def _tables(psf, sessions):
    return [psf.Table(psf.make_config(log2_capacity=s["log2_capacity"], pos_bits=s["pos_bits"],
                                      dir_bits=s["dir_bits"], alpha_min=s["alpha_min"], cache_fp16=s["cache_fp16"]))
            for s in sessions]


def _items(abi, tables, dev, outs, sessions):
    arr = (abi.BatchItem * len(sessions))()
    for i, s in enumerate(sessions):
        arr[i] = abi.BatchItem(tables[i].handle, dev[i].data_ptr(), outs[i].data_ptr(), s["width"] * s["height"],
                               s["depth"])
    return arr


def _free_bytes():
    import torch

    return min(torch.cuda.mem_get_info()[0] for _ in range(3))


def test_noalloc_matches_batch_step_on_two_calls(psf_mod):
    import torch

    from paper_2005_07547_b300 import _abi
    from synth.scene import iteration_vertices

    lib = _abi.load()
    sessions = _sessions()
    data = [[torch.from_numpy(iteration_vertices(s, it)).cuda() for it in range(2)] for s in sessions]
    t_ref, t_na = _tables(psf_mod, sessions), _tables(psf_mod, sessions)
    o_ref = [torch.zeros((d[0].shape[0], 3), device="cuda") for d in data]
    o_na = [torch.zeros((d[0].shape[0], 3), device="cuda") for d in data]
    ref_batch = psf_mod.Batch(len(sessions))
    cfg = _abi.BatchConfig(0, 0, 0, 0)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        dev = [d[call] for d in data]
        ref_batch.step([(t_ref[i], dev[i], o_ref[i], s["width"] * s["height"], s["depth"])
                        for i, s in enumerate(sessions)])
        items = _items(_abi, t_na, dev, o_na, sessions)
        if call == 1:  # after the first call's one-time set-up nothing is allocated or freed
            torch.cuda.synchronize()
            free_before = _free_bytes()
        assert lib.psf_batch_step_noalloc(items, len(sessions), ctypes.byref(cfg), stream) == _abi.PSF_OK
        torch.cuda.synchronize()
        if call == 1:
            # device-wide free memory: other processes on a shared GPU may move it a little
            assert abs(_free_bytes() - free_before) < (64 << 20)
        for i in range(len(sessions)):
            assert np.array_equal(o_ref[i].cpu().numpy(), o_na[i].cpu().numpy()), (call, i)
            assert t_ref[i].export().tobytes() == t_na[i].export().tobytes(), (call, i)
            assert t_na[i].stats()["status"] == 0
    ref_batch.close()
    for t in t_ref + t_na:
        t.close()


def test_noalloc_rejects_more_items_than_its_array_holds(psf_mod):
    import torch

    from paper_2005_07547_b300 import _abi

    lib = _abi.load()
    s = _sessions()[1]
    t = _tables(psf_mod, [s])[0]
    n = _abi.NOALLOC_MAX_ITEMS + 1
    arr = (_abi.BatchItem * n)()
    for i in range(n):
        arr[i] = _abi.BatchItem(t.handle, None, None, 0, 0)
    rc = lib.psf_batch_step_noalloc(arr, n, None, torch.cuda.current_stream().cuda_stream)
    assert rc == _abi.PSF_ERR_TOO_MANY
    assert b"PSF_NOALLOC_MAX_ITEMS" in lib.psf_last_cuda_error()
    torch.cuda.synchronize()
    assert t.stats()["iterations"] == 0  # nothing was enqueued
    t.close()


def test_noalloc_barrier_timeout_then_a_normal_call(psf_mod):
    """A barrier that waits for blocks that do not exist gives up after its bound (20 ms here):
    every item's table reports PSF_STATUS_TIMEOUT.  The shared array is cleared at the start
    of every call, so the next normal call still matches psf_batch_step."""
    import torch

    from paper_2005_07547_b300 import _abi
    from synth.scene import iteration_vertices

    lib = _abi.load()
    sessions = _sessions()[:3]
    data = [torch.from_numpy(iteration_vertices(s, 0)).cuda() for s in sessions]
    stream = torch.cuda.current_stream().cuda_stream
    stuck = _tables(psf_mod, sessions)
    outs = [torch.zeros((d.shape[0], 3), device="cuda") for d in data]
    phantom = _abi.BatchConfig(0, 0, 20000, 1)
    assert lib.psf_batch_step_noalloc(_items(_abi, stuck, data, outs, sessions), len(sessions),
                                      ctypes.byref(phantom), stream) == _abi.PSF_OK
    torch.cuda.synchronize()
    assert all(t.stats()["status"] & _abi.STATUS_TIMEOUT for t in stuck)
    t_ref, t_na = _tables(psf_mod, sessions), _tables(psf_mod, sessions)
    o_ref = [torch.zeros_like(o) for o in outs]
    o_na = [torch.zeros_like(o) for o in outs]
    ref_batch = psf_mod.Batch(len(sessions))
    ref_batch.step([(t_ref[i], data[i], o_ref[i], s["width"] * s["height"], s["depth"]) for i, s in enumerate(sessions)])
    normal = _abi.BatchConfig(0, 0, 0, 0)
    assert lib.psf_batch_step_noalloc(_items(_abi, t_na, data, o_na, sessions), len(sessions), ctypes.byref(normal),
                                      stream) == _abi.PSF_OK
    torch.cuda.synchronize()
    for i in range(len(sessions)):
        assert np.array_equal(o_ref[i].cpu().numpy(), o_na[i].cpu().numpy()), i
        assert t_ref[i].export().tobytes() == t_na[i].export().tobytes(), i
        assert t_na[i].stats()["status"] == 0
    ref_batch.close()
    for t in stuck + t_ref + t_na:
        t.close()
