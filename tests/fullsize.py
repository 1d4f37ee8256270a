"""Helpers of the full-size parity tests (no method arithmetic here).

Inputs come from the seeded generator in spawned worker processes (spawned, so that no
worker is forked from a process that already uses CUDA), a bounded number of iterations
ahead of the consumer.  Control-variate outputs at full size are compared on every
`stride`-th path (all depths of those paths): the oracle computes each path's outputs on
their own, so a sample of paths is an exact subset of the full comparison.
"""

from __future__ import annotations

import multiprocessing as mp
import os
from collections import deque

import numpy as np


def _gen_named(args):
    name, it = args
    from synth.scene import iteration_vertices, workload

    return iteration_vertices(workload(name), it)


def _gen_session(args):
    s, it = args
    from synth.scene import iteration_vertices

    return iteration_vertices(s, it)


def procs(limit: int = 8) -> int:
    return max(1, min(limit, os.cpu_count() or 1))


def stream(fn, jobs: list, ahead: int | None = None):
    """Results of fn(job) for each job in order, computed by spawned workers at most `ahead`
    jobs ahead of the consumer."""
    ahead = ahead or procs()
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs()) as pool:
        pending = deque()
        it = iter(jobs)
        for job in it:
            pending.append(pool.apply_async(fn, (job,)))
            if len(pending) >= ahead:
                break
        while pending:
            res = pending.popleft().get()
            nxt = next(it, None)
            if nxt is not None:
                pending.append(pool.apply_async(fn, (nxt,)))
            yield res


def named_iterations(name: str, n: int):
    """Iterations 0..n-1 of a named single-session workload."""
    return stream(_gen_named, [(name, it) for it in range(n)])


def session_iterations(sessions: list[dict], it: int) -> list[np.ndarray]:
    """Iteration `it` of every session, in session order."""
    return list(stream(_gen_session, [(s, it) for s in sessions], ahead=2 * procs()))


def sample_paths(v: np.ndarray, P: int, D: int, stride: int) -> tuple[np.ndarray, int]:
    """All depths of every stride-th path, as depth-major records of the sampled paths."""
    vs = np.ascontiguousarray(v.reshape(D, P, 16)[:, ::stride].reshape(-1, 16))
    return vs, vs.shape[0] // D


def sample_out(out, P: int, D: int, stride: int) -> np.ndarray:
    """The same sample of a (P*D, 3) CUDA output tensor, on the host."""
    return out.view(D, P, 3)[:, ::stride].reshape(-1, 3).cpu().numpy()


def oracle_session_check(job: dict) -> dict:
    """One batched session checked against its own oracle (runs in a spawned worker): the
    worker regenerates the session's iterations from their seeds, runs the oracle through
    them, and compares, iteration by iteration, the GPU table after the blend (keys and
    counters exactly, the FP32 approximant and the FP16 copy within their bounds) and the
    GPU control-variate outputs of the sampled paths.  Returns the worst error/bound ratios;
    a mismatch raises AssertionError naming the session and iteration."""
    import oracle
    from parity import TOL_FP16, TOL_FP32, check_after_update, check_cv
    from synth.scene import iteration_vertices, make_scene

    s, gpu, stride = job["session"], job["gpu"], job["stride"]
    fp16 = bool(s["cache_fp16"])
    P, D = s["width"] * s["height"], s["depth"]
    scene = make_scene(s["seed"])
    o = oracle.Oracle(pos_bits=s["pos_bits"], dir_bits=s["dir_bits"], alpha_min=float(np.float32(s["alpha_min"])))
    worst = {"L32": 0.0, "L16": 0.0, "cv": 0.0}
    for it, g in enumerate(gpu):
        v = iteration_vertices(s, it, scene)
        o.insert(v)
        o.update()
        rec = o.export()
        try:
            r32, r16 = check_after_update(g["table"], rec, fp16=fp16)
            vs, Ps = sample_paths(v, P, D, stride)
            rc = check_cv(g["out"], o.query_cv(vs, Ps, D), vs, o.lookup(vs, Ps, D), Ps, D, 1.0, 0xFFFFFFFF, rec["L"],
                          fp16=fp16)
        except AssertionError as e:
            raise AssertionError(f"session {s['name']} iteration {it}: {e}") from None
        worst["L32"] = max(worst["L32"], r32 / TOL_FP32)
        worst["L16"] = max(worst["L16"], (r16 or 0.0) / TOL_FP16)
        worst["cv"] = max(worst["cv"], rc)
    return {"session": s["name"], "cells": len(rec), **worst}


def served_wl(req: dict) -> dict:
    """The generator parameters of a served request at its own size."""
    return dict(width=req["width"], height=req["height"], depth=req["depth"], seed=req["seed"], radiance="glossy",
                camera_step=0.0, camera_x0=0.5)


def _gen_served(args):
    req, it = args
    from synth.scene import iteration_vertices

    return iteration_vertices(served_wl(req), it)


def served_iterations(reqs: list[dict], n: int) -> list[list[np.ndarray]]:
    """n iterations of every request at its own size, in request order."""
    flat = list(stream(_gen_served, [(r, it) for r in reqs for it in range(n)], ahead=2 * procs(16)))
    return [flat[k * n:(k + 1) * n] for k in range(len(reqs))]


def oracle_served_check(job: dict) -> dict:
    """A served session checked against its own oracle over all its iterations (iteration k
    reads input k mod n_inputs, as the server's source does): the GPU table after the last
    blend and the last iteration's sampled control-variate outputs."""
    import oracle
    from parity import TOL_FP16, TOL_FP32, check_after_update, check_cv
    from synth.scene import iteration_vertices, make_scene

    r, stride = job["request"], job["stride"]
    fp16 = bool(r["cache_fp16"])
    P, D = r["width"] * r["height"], r["depth"]
    wl = served_wl(r)
    scene = make_scene(wl["seed"])
    inputs = [iteration_vertices(wl, it, scene) for it in range(job["n_inputs"])]
    o = oracle.Oracle(pos_bits=r["pos_bits"], dir_bits=r["dir_bits"], alpha_min=float(np.float32(r["alpha_min"])))
    for k in range(r["iterations"]):
        o.insert(inputs[k % len(inputs)])
        o.update()
    v = inputs[(r["iterations"] - 1) % len(inputs)]
    rec = o.export()
    try:
        r32, r16 = check_after_update(job["table"], rec, fp16=fp16)
        vs, Ps = sample_paths(v, P, D, stride)
        rc = check_cv(job["out"], o.query_cv(vs, Ps, D), vs, o.lookup(vs, Ps, D), Ps, D, 1.0, 0xFFFFFFFF, rec["L"],
                      fp16=fp16)
    except AssertionError as e:
        raise AssertionError(f"served session {r['name']}: {e}") from None
    return {"session": r["name"], "iterations": r["iterations"], "vertices": P * D, "cells": len(rec),
            "L32": r32 / TOL_FP32, "L16": (r16 or 0.0) / TOL_FP16, "cv": rc}
