"""Benchmark: path vertices filtered per second (insert + update + query per iteration).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl psf|reference]

One step is one whole iteration of the hot path (insert, update, control-variate
query) over one batch of synthetic path vertices shaped like a 1920x1080, 1-spp,
depth-5 path tracer's output (10,368,000 vertices, 2^24-slot table, camera moving
1% of the scene per frame; each step gets a fresh 664 MB batch, larger than the
126 MB L2).  The line is timed with the workload's FP16 query copy of the
approximant; the same steps with the FP32 copy, each cache's error against the FP64
oracle, and the 64-session batched form (one fused persistent launch per iteration
against the plain per-session loop, with its own roofline) are extra keys of the
same line.  Under torchrun every rank runs its own render session on its own GPU
(weak scaling, no collective on the data path); the step time is the maximum over
ranks.

--impl reference times the CPU oracle (test infrastructure: a single-threaded
std::map implementation) on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "path vertices filtered/sec (insert+update+query)"
UNIT = "vertices/s"
DEFAULT_WORKLOAD = "1920x1080_d5"
POOL = 40  # distinct input batches kept resident; longer runs cycle through them
REFERENCE_ITERATIONS = 4  # distinct iterations the reference arm samples its steps from
KERNEL_SOURCES = ["paper_2005_07547_b300/csrc/psf.cu", "paper_2005_07547_b300/csrc/psf_device.cuh"]


# ---------------------------------------------------------------------------
# helpers shared with the tests (host logic only)
# ---------------------------------------------------------------------------

def dist_env() -> tuple[int, int, int]:
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def rank_seed_offset(rank: int) -> int:
    """Each rank renders its own session: iterations are drawn from a disjoint range."""
    return 100000 * rank


def aggregate(per_rank_ms: list[float], vertices_per_step_per_rank: int, steps: int, world: int) -> dict:
    """Whole-job throughput: every rank's vertices over the slowest rank's time."""
    t_ms = max(per_rank_ms)
    total = vertices_per_step_per_rank * steps * world
    return {"ms_per_step": t_ms / steps, "value": total / (t_ms / 1e3)}


def kernel_source_hash(sources=None) -> str:
    h = hashlib.sha256()
    for rel in sources or KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def algorithmic_bytes(V: int, touched: float, cache_fp16: bool, slot_cache: bool = False, payload: int = 0) -> dict:
    """Bytes each kernel must move at minimum (per launch).

    insert: read the 64-B vertex record of every vertex; per touched cell read its
            8-B key and read-modify-write its 32-B accumulator (8 + 64).
    update: per touched cell read + zero the 32-B accumulator, read + write the 16-B
            approximant and the 8-B c_old, write the 8-B FP16 copy (112 or 120).
    query:  read the 64-B record and write the 12-B output of every vertex; per
            touched cell read its key and its approximant (8 + 16, or 8 + 8 for FP16).
    With the slot cache the insert also writes, and the query reads, a 4-B slot per vertex.
    The SH payload (payload 1) has sixteen 64-bit sums and six coefficients per cell: the
    insert read-modify-writes 128 B per touched cell (8 + 256), the update reads and zeroes
    them and reads and writes c_old and the 24-B coefficients (320), the query reads the key
    and the coefficients (8 + 24).
    """
    extra = 4.0 * V if slot_cache else 0.0
    if payload == 1:
        return {"k_insert": 64.0 * V + 264.0 * touched + extra, "k_update": 320.0 * touched,
                "k_query": 76.0 * V + 32.0 * touched + extra}
    return {
        "k_insert": 64.0 * V + 72.0 * touched + extra,
        "k_update": (120.0 if cache_fp16 else 112.0) * touched,
        "k_query": 76.0 * V + (16.0 if cache_fp16 else 24.0) * touched + extra,
    }


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6400.0, "source": "fallback"}


class GroupRates:
    """The bulk-reduction probe's sustained group rate (groups/s) on one table's footprint --
    its slot records and its touched sectors -- memoised per footprint.  The fused kernel
    hands out its warp units in session order, so at any moment its warps add into one or
    two sessions' tables: each session's insert is bound by the rate its own footprint
    allows (a small table stays in L2), not by a probe spread over all tables at once.  A
    launch issues at least 2^22 groups so that the rate is a sustained one."""

    def __init__(self, min_groups: int = 1 << 22):
        self.memo: dict = {}
        self.min_groups = min_groups

    def __call__(self, slot_bytes: int, distinct: float, groups: float) -> float:
        key = (int(slot_bytes), max(1, int(distinct)))
        if key not in self.memo:
            r = atomic_probe_rates(modes=(4,), n_words=key[0] // 8, n_distinct=key[1],
                                   n_groups=max(int(groups), self.min_groups), reps=3)
            self.memo[key] = r["insert_pattern_bulk32_1or"] / 5.0
        return self.memo[key]


def key_layout_of(cfg) -> str:
    """Where the library lays out a configuration's keys: "inline" (inside the 64-byte slot
    records) or "dense" (an 8-byte array beside them, which adds 8 bytes per slot to the table
    size); read from psf_table_bytes, so the library's own rule decides."""
    import ctypes

    from paper_2005_07547_b300 import _abi

    lib = _abi.load()
    inline = _abi.Config()
    ctypes.memmove(ctypes.byref(inline), ctypes.byref(cfg), ctypes.sizeof(cfg))
    inline.key_layout = 2
    return "inline" if lib.psf_table_bytes(ctypes.byref(cfg)) == lib.psf_table_bytes(ctypes.byref(inline)) \
        else "dense"


def load_traffic(kernel: str, staged: bool, setup: dict) -> float | None:
    """DRAM bytes per launch from the committed ncu summary, if it was captured on the same
    kernels (source hash: the file's own, or a capture's own over the sources it lists) and the
    same setup (workload, cache, levels, capacity, knobs); the insert with staged vertex tiles
    is the kernel k_insert_staged."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    for cap in d.get("captures", []):
        if "sources" in cap:  # captured on other kernels (e.g. the fused batched one): its own hash
            if cap.get("source_hash") != kernel_source_hash(cap["sources"]):
                continue
        elif d.get("kernel_source_hash") != kernel_source_hash():
            continue
        if all(cap.get(k) == v for k, v in setup.items()):
            name = kernel + "_staged" if staged and kernel in ("k_insert", "k_query") else kernel
            k = cap.get("kernels", {}).get(name)
            return float(k["bytes_per_launch"]) if k else None
    return None


class _Nvml:
    """Read-only NVML queries through the driver's libnvidia-ml (ctypes)."""

    CLOCK_SM = 1

    def __init__(self):
        import ctypes

        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self._reasons = fn or self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def handle(self, cuda_index: int):
        ct = self.ct
        h = ct.c_void_p()
        try:
            import torch

            p = torch.cuda.get_device_properties(cuda_index)
            bus = f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0".encode()
            if self.lib.nvmlDeviceGetHandleByPciBusId_v2(ct.c_char_p(bus), ct.byref(h)) == 0:
                return h
        except Exception:
            pass
        if self.lib.nvmlDeviceGetHandleByIndex_v2(ct.c_uint(cuda_index), ct.byref(h)) != 0:
            raise RuntimeError("no NVML handle")
        return h

    def sm_mhz(self, h) -> int:
        v = self.ct.c_uint()
        self.lib.nvmlDeviceGetClockInfo(h, self.CLOCK_SM, self.ct.byref(v))
        return int(v.value)

    def max_sm_mhz(self, h) -> int:
        v = self.ct.c_uint()
        self.lib.nvmlDeviceGetMaxClockInfo(h, self.CLOCK_SM, self.ct.byref(v))
        return int(v.value)

    def reasons(self, h) -> int:
        v = self.ct.c_ulonglong()
        self._reasons(h, self.ct.byref(v))
        return int(v.value)

    def power_w(self, h) -> float:
        v = self.ct.c_uint()
        self.lib.nvmlDeviceGetPowerUsage(h, self.ct.byref(v))
        return v.value / 1000.0


class ClockSampler:
    """SM clocks and clock-event (throttle) reasons sampled through NVML every millisecond
    by a background thread while the timed region runs (read-only queries)."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index: int, period_s: float = 0.001):
        self.cuda_index = cuda_index
        self.period = period_s
        self.samples = []
        self.max_mhz = None
        self.error = None
        self._stop = None
        self._thread = None

    def __enter__(self):
        import threading

        try:
            nv = _Nvml()
            h = nv.handle(self.cuda_index)
            self.max_mhz = nv.max_sm_mhz(h)
        except Exception as e:  # no NVML: report unsampled
            self.error = repr(e)
            return self
        self._stop = threading.Event()

        def loop():
            while not self._stop.is_set():
                try:
                    self.samples.append((nv.sm_mhz(h), nv.reasons(h), nv.power_w(h)))
                except Exception as e:
                    self.error = repr(e)
                    return
                self._stop.wait(self.period)

        self._thread = threading.Thread(target=loop, daemon=True)
        self._thread.start()
        return self

    def __exit__(self, *exc):
        if self._thread is not None:
            self._stop.set()
            self._thread.join(timeout=5)

    def summary(self) -> dict:
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unsampled"], "error": self.error}
        reasons = set()
        for _, mask, _ in self.samples:
            for bit, name in self.REASONS.items():
                if mask & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(s[0] for s in self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(reasons), "samples": len(self.samples),
                "power_w_max": max(s[2] for s in self.samples), "source": "NVML (libnvidia-ml), 1 ms"}


def atomic_probe_rates(modes=(0, 1, 2, 3, 4, 5), n_words: int = 1 << 25, reps: int = 3, n_distinct: int = 0,
                       n_groups: int = 0) -> dict:
    """Measured L2 64-bit atomic throughput (ops/s) on this GPU, per probe mode, on a buffer of
    n_words 64-bit words (2^25 words = 256 MB, larger than L2, like a 2^22-slot table).  With
    n_distinct > 0 the sector patterns (modes 2, 4, 5) target that many fixed random sectors;
    n_groups > 0 sets how many groups one launch issues (else 2^24 for the sector patterns,
    2^26 for the others), so that a launch can match a kernel's own count of groups over its
    own distinct sectors (the same reuse of each sector, hence the same share of L2 hits)."""
    import ctypes

    import torch

    from paper_2005_07547_b300 import build as _b

    _b.build()
    lib = ctypes.CDLL(_b.PROBE_LIB)
    lib.atomic_probe.restype = ctypes.c_int
    lib.atomic_probe.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_void_p]
    n_words = max(128, int(n_words) // 128 * 128)  # whole 1-KB blocks (the probe wants a multiple of 4 words)
    buf = torch.zeros(n_words * 8 + (n_words // 128) * 4, dtype=torch.uint8, device="cuda")
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    stream = torch.cuda.current_stream()
    out = {}
    names = {0: "red_random_u64", 1: "atom_random_u64", 2: "insert_pattern_4red_1or", 3: "red_warp_contended_u64",
             4: "insert_pattern_bulk32_1or", 5: "bulk32_only"}
    for mode in modes:
        groups = int(n_groups) if n_groups > 0 else ((1 << 24) if mode in (2, 4, 5) else (1 << 26))
        ops_per_group = 5 if mode in (2, 4, 5) else 1
        args = (buf.data_ptr(), n_words, groups, n_distinct, mode, sms * 8, stream.cuda_stream)
        if lib.atomic_probe(*args) != 0:
            raise RuntimeError("atomic probe failed")
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record(stream)
        for _ in range(reps):
            lib.atomic_probe(*args)
        end.record(stream)
        torch.cuda.synchronize()
        sec = start.elapsed_time(end) / 1e3
        out[names[mode]] = groups * ops_per_group * reps / sec
    del buf
    return out


# ---------------------------------------------------------------------------
# input generation (host, seeded; before any CUDA work)
# ---------------------------------------------------------------------------

def _gen_one(args):
    name, iteration = args
    from synth.scene import iteration_vertices, workload

    return iteration_vertices(workload(name), iteration)


def generate(name: str, iterations: list[int], procs: int) -> list[np.ndarray]:
    if procs <= 1 or len(iterations) == 1:
        return [_gen_one((name, it)) for it in iterations]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(procs, len(iterations))) as pool:
        return pool.map(_gen_one, [(name, it) for it in iterations])


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on a bounded sample
# ---------------------------------------------------------------------------

def run_reference(args) -> None:
    rank, _, _ = dist_env()
    if rank != 0:
        return
    from synth.scene import workload

    w = workload(args.workload)
    # a few distinct iterations (each is a whole image; the steps only sample it), cycled, the
    # sampled window of paths moving on at every cycle
    n_iter = min(args.warmup + args.steps, REFERENCE_ITERATIONS)
    batches = generate(args.workload, list(range(n_iter)), os.cpu_count() or 1)
    # warm-up steps: untimed oracle iterations (bounded)
    import oracle

    P, D = w["width"] * w["height"], w["depth"]
    o = oracle.Oracle(pos_bits=w["pos_bits"], dir_bits=w["dir_bits"], alpha_min=float(np.float32(w["alpha_min"])),
                      levels=args.levels)
    for v in batches[:min(args.warmup, 1)]:
        o.insert(v)
        o.update()
        o.query_cv(v, P, D)
    # each timed step is a bounded sample of that iteration's paths: 1/8 of them for up to 30
    # steps, proportionally fewer for more steps, so the whole run stays within a minute or so
    frac_paths = max(1, (P // 8) * min(30, args.steps) // max(args.steps, 1))
    times = []
    done = 0
    for k in range(args.steps):
        v = batches[(args.warmup + k) % n_iter]
        first = (k // n_iter) * frac_paths % (P - frac_paths + 1)
        sample = v.reshape(D, P, 16)[:, first:first + frac_paths].reshape(-1, 16).copy()
        t0 = time.perf_counter()
        o.insert(sample)
        o.update()
        o.query_cv(sample, frac_paths, D)
        times.append(time.perf_counter() - t0)
        done += sample.shape[0]
    total = sum(times)
    value = done / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "paths": P, "depth": D, "vertices_per_step": frac_paths * D, "levels": args.levels,
                   "sample": f"{frac_paths} consecutive paths of {P} per step, from {n_iter} iterations cycled, "
                             "the window moving on each cycle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} steps x {frac_paths} paths x depth {D} of {w['name']} "
                                   f"(after one whole untimed iteration)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def _oracle_leg(job: dict) -> dict:
    """The oracle's share of the benchmark, run in a spawned process while the GPU arm runs:
    iterations 0..k-1 of the workload (regenerated here from their seeds), the last one timed
    as insert + update + query (the CPU baseline), then the table and the control-variate
    outputs on every `stride`-th path, which the GPU arm's precision report compares with."""
    import oracle
    from synth.scene import iteration_vertices, make_scene, workload

    w = workload(job["name"])
    scene = make_scene(w["seed"])
    P, D = w["width"] * w["height"], w["depth"]
    o = oracle.Oracle(pos_bits=w["pos_bits"], dir_bits=w["dir_bits"], alpha_min=float(np.float32(w["alpha_min"])),
                      levels=job.get("levels", 1))
    k, stride = job["iterations"], job["stride"]
    for it in range(k):
        v = iteration_vertices(w, it, scene)
        if it < k - 1:
            o.insert(v)
            o.update()
            continue
        t0 = time.perf_counter()
        o.insert(v)
        o.update()
        out = o.query_cv(v, P, D)
        dt = time.perf_counter() - t0
    vs = v.reshape(D, P, 16)[:, ::stride].reshape(-1, 16)
    Ps = vs.shape[0] // D
    rec = o.export()
    return {
        "cpu_baseline": {"value": v.shape[0] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"iteration {k - 1} of {w['name']} ({v.shape[0]} vertices, after {k - 1} untimed "
                                   f"iterations), std::map oracle, insert+update+query, single thread, {dt:.1f} s"},
        "key": rec["key"], "c_old": rec["c_old"], "L": rec["L"],
        "out": out.reshape(D, P, 3)[:, ::stride].reshape(-1, 3), "C": o.lookup(vs, Ps, D), "stride": stride,
        "iterations": k,
    }


def _oracle_sessions_worker(args):
    """One host core's share of the batched sessions: generate their first iteration, wait for
    every worker, then run the oracle's insert + update + query on each (timed)."""
    sessions, barrier, out = args
    import oracle
    from synth.scene import iteration_vertices

    data = [iteration_vertices(s, 0) for s in sessions]
    barrier.wait()
    t0 = time.time()
    n = 0
    for s, v in zip(sessions, data):
        o = oracle.Oracle(pos_bits=s["pos_bits"], dir_bits=s["dir_bits"], alpha_min=float(np.float32(s["alpha_min"])))
        o.insert(v)
        o.update()
        o.query_cv(v, s["width"] * s["height"], s["depth"])
        n += v.shape[0]
    out.put((n, t0, time.time()))


def oracle_sessions_aggregate(sessions: list[dict], procs: int) -> dict:
    """The oracle over independent sessions on all host cores (one iteration of every session,
    dealt to `procs` spawned workers largest first, each to the least loaded): vertices over the
    wall time from the common start to the last worker's end."""
    ctx = mp.get_context("spawn")
    shares: list[list[dict]] = [[] for _ in range(max(1, min(procs, len(sessions))))]
    load = [0] * len(shares)
    for s in sorted(sessions, key=lambda s: -s["width"] * s["height"] * s["depth"]):
        k = load.index(min(load))  # longest job first onto the least loaded worker
        shares[k].append(s)
        load[k] += s["width"] * s["height"] * s["depth"]
    barrier = ctx.Barrier(len(shares))
    out = ctx.Queue()
    workers = [ctx.Process(target=_oracle_sessions_worker, args=((sh, barrier, out),)) for sh in shares]
    for w in workers:
        w.start()
    res = [out.get() for _ in workers]
    for w in workers:
        w.join()
    n = sum(r[0] for r in res)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    return {"value": n / wall, "unit": UNIT, "cores": len(shares), "kind": "oracle",
            "sample": f"iteration 0 of all {len(sessions)} sessions ({n} vertices), std::map oracle, insert+update+query, "
                      f"sessions dealt to {len(shares)} processes largest first onto the least loaded, {wall:.1f} s wall"}


def precision_report(psf, make_cfg, dev: list, P: int, D: int, leg: dict, slot_cache: bool) -> dict:
    """Each query cache's error against the FP64 oracle after the oracle leg's iterations: fresh
    tables run the same batches with the benchmark's calls; keys and counters must match
    exactly; the approximant's worst relative error |x - ref| / max(|ref|, 2^-14 max|ref|) and
    the control-variate outputs' worst error over the norm-wise bound (tolerance 1e-5 for the
    FP32 copy, 2e-3 for the FP16 copy) on every stride-th path."""
    import torch

    k, stride = leg["iterations"], leg["stride"]
    ref = leg["L"]
    scale = np.maximum(np.abs(ref), 2.0 ** -14 * float(np.max(np.abs(ref))))
    rep = {"oracle": "FP64 std::map", "iterations": k, "sampled_paths": f"every {stride}th path, all depths"}
    for fp16 in (False, True):
        t = psf.Table(make_cfg(fp16))
        out = torch.empty((P * D, 3), dtype=torch.float32, device="cuda")
        slots = torch.empty(P * D, dtype=torch.int32, device="cuda")
        for it in range(k):
            if slot_cache:
                t.insert_slots(dev[it], P, D, slots=slots)
                t.update()
                t.query_cv_slots(dev[it], slots, P, D, out=out)
            else:
                t.step(dev[it], P, D, out=out)
        g = t.export()
        exact = bool(np.array_equal(g["key"], leg["key"]) and np.array_equal(g["c_old"], leg["c_old"]))
        r = {"keys_and_counters_exact": exact}
        if exact:
            r["L_fp32_max_rel_err"] = float(np.max(np.abs(g["L"].astype(np.float64) - ref) / scale))
            if fp16:
                h = g["L_fp16"].astype(np.uint16).view(np.float16).astype(np.float64)
                r["L_fp16_max_rel_err"] = float(np.max(np.abs(h - ref) / scale))
        vs = dev[k - 1].view(D, P, 16)[:, ::stride].reshape(-1, 16).cpu().numpy().astype(np.float64)
        got = out.view(D, P, 3)[:, ::stride].reshape(-1, 3).cpu().numpy().astype(np.float64)
        Ps = vs.shape[0] // D
        C = leg["C"].reshape(D, Ps, 3)
        Cn = np.zeros_like(C)
        Cn[:-1] = C[1:]
        on = (np.repeat(np.arange(D), Ps) + 1 < D)[:, None]
        fl = 2.0 ** -14 * float(np.max(np.abs(ref)))
        tj = vs[:, [7, 11, 15]]
        norm = np.abs(vs[:, 12:15]) + on * (np.abs(tj) * (np.abs(Cn.reshape(-1, 3)) + fl) + np.abs(C.reshape(-1, 3)) + fl)
        err = np.abs(got - leg["out"])
        tol = 2e-3 if fp16 else 1e-5
        ratio = np.divide(err, norm, out=np.zeros_like(err), where=norm > 0)  # norm 0: both outputs are 0
        assert not np.any(err[norm == 0]), "a zero-norm output differs from the oracle's"
        r["cv_max_rel_err"] = float(np.max(ratio))
        r["cv_err_over_bound"] = float(np.max(ratio) / tol)
        r["tolerance"] = tol
        rep["fp16" if fp16 else "fp32"] = r
        t.close()
    return rep


def time_single(psf, table, dev: list, P: int, D: int, steps: int, warmup: int, slot_cache: bool, local: int,
                world: int) -> dict:
    """Time `steps` whole iterations (insert, update, query) on one table, a different resident
    batch each step, with CUDA events on the launching stream around every kernel."""
    import torch
    import torch.distributed as dist

    V = P * D
    n_iter = len(dev)
    out = torch.empty((V, 3), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    slots = torch.empty(V, dtype=torch.int32, device="cuda") if slot_cache else None

    def insert(v):
        if slots is not None:
            table.insert_slots(v, P, D, slots=slots)
        else:
            table.insert(v)

    def query(v):
        if slots is not None:
            table.query_cv_slots(v, slots, P, D, out=out)
        else:
            table.query_cv(v, P, D, out=out)

    for k in range(warmup):
        insert(dev[k % n_iter])
        table.update()
        query(dev[k % n_iter])
    torch.cuda.synchronize()
    before = table.stats()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        start.record(stream)
        for k in range(steps):
            v = dev[(warmup + k) % n_iter]
            e = ev[k]
            e[0].record(stream)
            insert(v)
            e[1].record(stream)
            table.update()
            e[2].record(stream)
            query(v)
            e[3].record(stream)
        end.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    after = table.stats()
    if after["status"] != 0:
        raise RuntimeError(f"device status {after['status']} during the benchmark")
    kt = {"k_insert": [e[0].elapsed_time(e[1]) for e in ev], "k_update": [e[1].elapsed_time(e[2]) for e in ev],
          "k_query": [e[2].elapsed_time(e[3]) for e in ev]}
    return {"elapsed_ms": start.elapsed_time(end), "kernel_ms": kt, "step_ms": [e[0].elapsed_time(e[3]) for e in ev],
            "touched": (after["touched_cells"] - before["touched_cells"]) / steps,
            "leaders": (after["leader_groups"] - before["leader_groups"]) / steps,
            "live_cells": after["live_cells"], "clocks": clocks.summary()}


def run_psf(args) -> None:
    rank, world, local = dist_env()
    from synth.scene import workload

    w = workload(args.workload)
    P, D = w["width"] * w["height"], w["depth"]
    V = P * D
    off = rank_seed_offset(rank)
    n_iter = min(args.warmup + args.steps, POOL)
    host = generate(args.workload, [off + i for i in range(n_iter)], os.cpu_count() or 1)
    extras = rank == 0 and world == 1 and not args.no_cpu_baseline and args.payload == "rgb"
    sessions_host = None
    if extras and args.batched_extra:
        from synth.scene import session_workloads

        sessions_host = generate_sessions(session_workloads(args.sessions), args.pool)
    leg_proc = None
    if extras:
        # the oracle leg runs beside the GPU arm (spawned before any CUDA call)
        ctx = mp.get_context("spawn")
        leg_pool = ctx.Pool(1)
        leg_proc = leg_pool.apply_async(_oracle_leg, ({"name": args.workload, "iterations": min(3, n_iter),
                                                       "stride": 16, "levels": args.levels},))

    import torch
    import torch.distributed as dist

    import paper_2005_07547_b300 as psf

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    psf.load()
    # coarse levels add few cells (measured live cells over the flat table's: 1.26x at 2
    # levels, 1.35x at 4), so the workload's capacity serves every level count
    log2cap = w["log2_capacity"]
    fp16 = bool(args.fp16 or w["cache_fp16"]) and not args.fp32

    sh = args.payload == "sh"
    if sh:  # the SH payload keeps no FP16 copy; the paper's 5-d key
        fp16 = False

    def make_cfg(cache_fp16, key_layout=None):
        return psf.make_config(log2_capacity=log2cap, pos_bits=w["pos_bits"], dir_bits=w["dir_bits"],
                               alpha_min=w["alpha_min"], cache_fp16=cache_fp16,
                               key_layout=args.key_layout if key_layout is None else key_layout,
                               levels=args.levels, payload=1 if sh else 0, sh_ridge=args.sh_ridge,
                               use_normal=not sh)

    base_knobs = dict(insert_mode=args.insert_mode, vertex_staging=args.staging, sum_reduction=args.sum_reduction,
                      query_layout=args.query_layout, insert_blocks_per_sm=args.insert_blocks,
                      query_blocks_per_sm=args.query_blocks, update_blocks_per_sm=args.update_blocks)
    dev = [torch.from_numpy(v).cuda() for v in host]
    tuned = {}

    def tune(cache_fp16):
        """With --tune the autotuner's pick, timed on this workload's first batches with the
        benchmark's own calls: grid caps, query layout and, unless --key-layout fixes it, where
        the table keeps its keys."""
        if cache_fp16 not in tuned:
            from paper_2005_07547_b300 import autotune

            space = {"insert_blocks_per_sm": (0, 4), "query_blocks_per_sm": (0, 4, 2),
                     "update_blocks_per_sm": (0, 2, 1), "query_layout": (0, 1)}
            if args.key_layout == 0 and not sh:
                space["key_layout"] = (1, 2)
            # 8 timed steps per candidate: the key layouts differ by about 1%, which fewer steps
            # do not resolve from run to run
            res = autotune.tune_table(make_cfg(cache_fp16), dev[:min(6, len(dev))], P, D, space=space, warmup=2,
                                      iters=8, slot_cache=bool(args.slot_cache))
            best = dict(res["best"])
            layout = best.pop("key_layout", args.key_layout)
            tuned[cache_fp16] = {"best": {**base_knobs, **best}, "key_layout": layout, "best_ms": res["best_ms"],
                                 "candidates": len(res["all"]), "space": " x ".join(space)}
        return tuned[cache_fp16]

    def knobs_for(cache_fp16):
        """The launch knobs: the flags' values, or with --tune the autotuner's pick."""
        return dict(tune(cache_fp16)["best"]) if args.tune else dict(base_knobs)

    def cfg_for(cache_fp16):
        """The timed table's configuration: the flag's key layout, or with --tune the tuner's."""
        return make_cfg(cache_fp16, tune(cache_fp16)["key_layout"] if args.tune else None)

    def new_table(cache_fp16):
        t = psf.Table(cfg_for(cache_fp16))
        t.set_launch(**knobs_for(cache_fp16))
        return t

    table = new_table(fp16)
    m = time_single(psf, table, dev, P, D, args.steps, args.warmup, bool(args.slot_cache), local, world)
    table.close()
    elapsed_ms, kt, step_ms, touched, leaders = m["elapsed_ms"], m["kernel_ms"], m["step_ms"], m["touched"], m["leaders"]

    if world > 1:
        t = torch.tensor([elapsed_ms], dtype=torch.float64, device="cuda")
        gathered = [torch.zeros_like(t) for _ in range(world)]
        dist.all_gather(gathered, t)
        per_rank = [float(x.item()) for x in gathered]
    else:
        per_rank = [elapsed_ms]
    agg = aggregate(per_rank, V, args.steps, world)

    other = None
    if extras and not sh:  # the same steps with the other query cache
        t2 = new_table(not fp16)
        m2 = time_single(psf, t2, dev, P, D, args.steps, args.warmup, bool(args.slot_cache), local, 1)
        t2.close()
        other = {"value": V * args.steps / (m2["elapsed_ms"] / 1e3), "ms_per_step": m2["elapsed_ms"] / args.steps,
                 "kernels_avg_ms": {k: sum(x) / len(x) for k, x in m2["kernel_ms"].items()},
                 "p50": float(np.percentile(m2["step_ms"], 50)), "p99": float(np.percentile(m2["step_ms"], 99)),
                 "clocks": m2["clocks"], "launch_knobs": knobs_for(not fp16)}

    # end to end through the public API: pinned host vertices in, host CV outputs back,
    # copies inside the timed region, H2D of step k+1 overlapped with compute of step k
    e2e = None
    if rank == 0:
        t3 = new_table(fp16)
        e2e = run_e2e(psf, t3, host, P, D, args.e2e_steps, bool(args.slot_cache))
        t3.close()

    peaks = load_peaks()
    alg = algorithmic_bytes(V, touched, fp16, bool(args.slot_cache), 1 if sh else 0)
    avg = {k: sum(v) / len(v) for k, v in kt.items()}
    dominant = max(avg, key=avg.get)
    achieved = alg[dominant] / (avg[dominant] / 1e3) / 1e9
    # atomic roofline of the insert: one update of a random 32-byte sector per (warp, key)
    # group plus one bitmap reduction, against the probe's rate for the same pattern on a
    # buffer the size of the table's slot records with the insert's footprint: as many groups
    # per launch as the insert issues, on as many fixed random sectors as it touches cells;
    # mode 4: the sums as one bulk reduction, the default; mode 2: as four 64-bit reductions.
    # The probe at its fixed 2^24 groups (more visits per sector, so more L2 hits) is kept
    # beside it for comparison with earlier lines.
    probe_words = 8 << log2cap
    mode = 4 if args.sum_reduction == 0 else 2
    pname = {4: "insert_pattern_bulk32_1or", 2: "insert_pattern_4red_1or"}[mode]
    run_probe = rank == 0 and not sh
    probe = (atomic_probe_rates(modes=(mode,), n_words=probe_words, n_distinct=max(1, int(touched)),
                                n_groups=max(1, int(leaders)), reps=5) if run_probe else {})
    probe_fixed = (atomic_probe_rates(modes=(mode,), n_words=probe_words, n_distinct=max(1, int(touched)))
                   if run_probe else {})
    peak_groups = probe[pname] / 5.0 if probe else float("nan")
    group_rate = leaders / (avg["k_insert"] / 1e3)
    atomic_roofline = {"kernel": "k_insert", "achieved": group_rate / 1e9, "unit": "G groups/s",
                       "peak": peak_groups / 1e9, "frac": group_rate / peak_groups if probe else None,
                       "leader_groups_per_launch": leaders,
                       "peak_source": f"live probe: random 32-B sector, {'one bulk (TMA) reduction' if mode == 4 else '4 x red.add.u64'} + red.or, "
                                      f"{int(leaders)} groups on {int(touched)} distinct sectors of "
                                      f"{probe_words * 8 / 1e6:.0f} MB (the insert's groups and touched cells of the slot records)",
                       "peak_fixed_2p24_groups": probe_fixed[pname] / 5.0 / 1e9 if probe_fixed else None}
    kernels = {k: {"avg_ms": avg[k], "share": avg[k] / sum(avg.values()),
                   "algorithmic_GBps": alg[k] / (avg[k] / 1e3) / 1e9,
                   "frac_of_hbm": alg[k] / (avg[k] / 1e3) / 1e9 / peaks["hbm_gbs"]} for k in avg}
    # the dominant kernel's binding roof: the larger of its HBM and L2-atomic fractions
    hbm = {"achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
           "peak_source": peaks["source"], "algorithmic_bytes_per_launch": alg[dominant]}
    staged = {"k_insert": bool(args.staging & 1), "k_query": bool(args.staging & 2)}.get(dominant, False)
    setup = {"workload": w["name"], "cache": "fp16" if fp16 else "fp32", "levels": args.levels, "log2_capacity": log2cap,
             "slot_cache": bool(args.slot_cache)}
    if sh:
        setup["payload"] = "sh"
    setup["key_layout"] = key_layout_of(cfg_for(fp16))
    # launch choices other than the defaults the counters were taken with name themselves, so
    # that no committed capture matches them
    for knob in ("insert_mode", "sum_reduction"):
        if getattr(args, knob):
            setup[knob] = getattr(args, knob)
    roofline = {"kernel": dominant, "traffic": load_traffic(dominant, staged, setup), "hbm": hbm}
    binding = hbm
    roofline["bound"] = "hbm"
    if dominant == "k_insert" and atomic_roofline["frac"] is not None:
        roofline["l2_atomic"] = atomic_roofline
        if atomic_roofline["frac"] > hbm["frac"]:
            binding = atomic_roofline
            roofline["bound"] = "l2_atomic"
    for key in ("achieved", "peak", "unit", "frac"):
        roofline[key] = binding[key]
    roofline["peak_note"] = ("of measured" + (" (MEASURED_PEAKS.json hbm_gbs)" if roofline["bound"] == "hbm"
                                              else " (live atomic probe of the same access pattern)"))

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": agg["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": agg["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+i64 fixed point", "data": "synthetic",
        "config": {"workload": w["name"], "paths": P, "depth": D, "vertices_per_step": V,
                   "log2_capacity": log2cap, "levels": args.levels, "cache": "fp16" if fp16 else "fp32",
                   "touched_cells_per_step": touched, "live_cells": m["live_cells"],
                   "camera": f"x = {w['camera_x0']} + {w['camera_step']} * iteration",
                   "l2": f"inputs larger than L2: {n_iter} distinct {V * 64 / 1e6:.0f} MB vertex batches, "
                         "a different one every step",
                   "insert_mode": args.insert_mode, "vertex_staging": args.staging,
                   "sum_reduction": {0: "bulk (TMA) 32-B reduction", 1: "4 x red.add.u64"}[args.sum_reduction],
                   "launch_knobs": knobs_for(fp16),
                   "autotune": ({"space": tuned[fp16]["space"], "candidates": tuned[fp16]["candidates"],
                                 "tuned_ms": tuned[fp16]["best_ms"]} if args.tune else None),
                   "slot_cache": bool(args.slot_cache),
                   "key_layout": {"inline": "keys in the slot records", "dense": "dense key array"}[
                       key_layout_of(cfg_for(fp16))],
                   "payload": ("YCoCg two-band SH over the normal, ridge %g, 5-d key" % args.sh_ridge) if sh else "RGB",
                   "parallelism": f"sessions x{world}"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "mean": float(np.mean(step_ms))},
        "roofline": roofline,
        "kernels": kernels,
        "gpu_launches": 3 * args.steps,
        "clocks": m["clocks"],
        "e2e": e2e,
    }
    if other is not None:
        line["fp32_cache" if fp16 else "fp16_cache"] = other
    if sessions_host is not None:
        line["batched_sessions"] = measure_sessions(args, sessions_host, local)
        line["batched_sessions"]["cpu_baseline"] = oracle_sessions_aggregate(sessions_host["sessions"],
                                                                             min(os.cpu_count() or 1, 32))
    if leg_proc is not None:
        leg = leg_proc.get()
        leg_pool.close()
        leg_pool.join()
        line["cpu_baseline"] = leg["cpu_baseline"]
        line["precision_vs_fp64_oracle"] = precision_report(psf, make_cfg, dev, P, D, leg, bool(args.slot_cache))
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_e2e(psf, table, host: list[np.ndarray], P: int, D: int, steps: int, slot_cache: bool = True) -> dict:
    """Vertices/s through Table.insert(_slots)/update/query_cv(_slots) with host buffers: each
    step copies its batch from pinned host memory and reads the CV outputs back into pinned
    host memory."""
    import torch

    V = P * D
    nb = min(len(host), 3)
    pinned = [torch.from_numpy(host[i]).pin_memory() for i in range(nb)]
    out_host = [torch.empty((V, 3), dtype=torch.float32).pin_memory() for _ in range(2)]
    dev_in = [torch.empty((V, 16), dtype=torch.float32, device="cuda") for _ in range(2)]
    dev_out = [torch.empty((V, 3), dtype=torch.float32, device="cuda") for _ in range(2)]
    slots = torch.empty(V, dtype=torch.int32, device="cuda")  # used on the compute stream only
    compute = torch.cuda.current_stream()
    copy = torch.cuda.Stream()
    ready = [torch.cuda.Event() for _ in range(2)]
    free = [torch.cuda.Event() for _ in range(2)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(compute)
    for s in range(steps + 1):
        b = s % 2
        if s < steps:  # stage step s on the copy stream
            with torch.cuda.stream(copy):
                if s >= 2:
                    copy.wait_event(free[b])
                dev_in[b].copy_(pinned[s % nb], non_blocking=True)
                ready[b].record(copy)
        if s >= 1:  # compute step s - 1
            pb = (s - 1) % 2
            compute.wait_event(ready[pb])
            if slot_cache:
                table.insert_slots(dev_in[pb], P, D, slots=slots)
                table.update()
                table.query_cv_slots(dev_in[pb], slots, P, D, out=dev_out[pb])
            else:
                table.insert(dev_in[pb])
                table.update()
                table.query_cv(dev_in[pb], P, D, out=dev_out[pb])
            out_host[pb].copy_(dev_out[pb], non_blocking=True)
            free[pb].record(compute)
    end.record(compute)
    torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    return {"value": V * steps / (ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": V * 64,
            "d2h_bytes_per_step": V * 12, "steps": steps,
            "note": "pinned host buffers; H2D of step k+1 overlapped with step k on a second stream"}


def _gen_session(args):
    s, iteration = args
    from synth.scene import iteration_vertices

    return iteration_vertices(s, iteration)


def generate_sessions(sessions: list[dict], pool: int) -> dict:
    """Host vertex streams of every session for `pool` iterations (spawned workers, before any
    CUDA call)."""
    jobs = [(s, it) for it in range(pool) for s in sessions]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(os.cpu_count() or 1, 32)) as p:
        flat = p.map(_gen_session, jobs, chunksize=1)
    return {"sessions": sessions, "pool": pool,
            "host": [[flat[it * len(sessions) + k] for it in range(pool)] for k in range(len(sessions))]}


def measure_sessions(args, gen: dict, local: int, tune: bool = True) -> dict:
    """Uneven render sessions: one fused persistent launch per iteration (graph-replayed)
    against the plain per-session loop (three launches per session), eager and
    graph-captured, on the same resident iterations.  The fused kernel's roofline: its
    phases run back to back, so its floor is the sum of each phase's own floor over all
    sessions (insert: per session, the larger of its algorithmic bytes at the measured HBM
    rate and its (warp, key) groups at the bulk-reduction probe's rate on its own footprint,
    since the phase takes the sessions in order; blend and query: their algorithmic bytes at
    the HBM rate), against the measured step."""
    import torch

    import paper_2005_07547_b300 as psf
    from paper_2005_07547_b300 import autotune

    sessions, pool = gen["sessions"], gen["pool"]
    V = sum(s["width"] * s["height"] * s["depth"] for s in sessions)
    dev = [[torch.from_numpy(v).cuda() for v in gen["host"][k]] for k in range(len(sessions))]

    def cfg_of(s, bits=1, key_layout=args.key_layout):
        # the load factor: 2^(ceil(log2 V) + bits) slots (the workload's own sizing is bits = 1);
        # the cell grid q stays the session's, so every choice gives the same cells
        log2cap = int(math.ceil(math.log2(s["width"] * s["height"] * s["depth"]))) + bits
        return psf.make_config(log2_capacity=log2cap, pos_bits=s["pos_bits"], dir_bits=s["dir_bits"],
                               alpha_min=s["alpha_min"], cache_fp16=s["cache_fp16"], key_layout=key_layout)

    outs = [torch.empty((d[0].shape[0], 3), device="cuda") for d in dev]
    # the slot cache (the default): each session's insert notes its vertices' slots and its
    # query reads them, in the fused kernel and in the plain loop alike
    slots = [torch.empty(d[0].shape[0], dtype=torch.int32, device="cuda") if args.slot_cache else None for d in dev]

    def entries(tables, it):
        return [(tables[k], dev[k][it % pool], outs[k], s["width"] * s["height"], s["depth"]) +
                ((slots[k],) if slots[k] is not None else ()) for k, s in enumerate(sessions)]

    def plain_step(table, i, v, P, D):
        if slots[i] is not None:
            table.insert_slots(v, P, D, slots=slots[i])
            table.update()
            table.query_cv_slots(v, slots[i], P, D, out=outs[i])
        else:
            table.step(v, P, D, out=outs[i])

    if tune:
        space = {**autotune.BATCH_SPACE, "capacity_bits": (1, 2)}
        if args.key_layout == 0:
            space["key_layout"] = (1, 2)
        tuned = autotune.tune_batch(
            lambda capacity_bits=1, key_layout=args.key_layout:
                entries([psf.Table(cfg_of(s, capacity_bits, key_layout)) for s in sessions], 0),
            len(sessions), space=space)
        knobs = dict(tuned["best"])
        bits = knobs.pop("capacity_bits")
        layout = knobs.pop("key_layout", args.key_layout)
    else:  # the flags' knobs (fixed launches, e.g. for a profiler capture)
        tuned = {"all": None}
        knobs = {"insert_mode": args.insert_mode, "blocks_per_sm": args.batch_blocks,
                 "update_blocks_per_sm": args.update_blocks, "query_blocks_per_sm": args.query_blocks}
        if args.insert_blocks:
            knobs["insert_blocks_per_sm"] = args.insert_blocks
        bits = args.capacity_bits
        layout = args.key_layout
    tables = [psf.Table(cfg_of(s, bits, layout)) for s in sessions]
    if args.sum_reduction:  # the sessions' sum path (the fused kernel reads it from each table)
        for t in tables:
            t.set_launch(sum_reduction=args.sum_reduction)
    batches = [psf.Batch(len(sessions), **knobs) for _ in range(pool)]
    for it, b in enumerate(batches):
        b.set(entries(tables, it))
    torch.cuda.synchronize()
    graphs = []
    for b in batches:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            b.launch()
        graphs.append(g)

    def timed(step_fn, n_warm, n_steps):
        for k in range(n_warm):
            step_fn(k)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(n_steps + 1)]
        ev[0].record()
        for k in range(n_steps):
            step_fn(n_warm + k)
            ev[k + 1].record()
        torch.cuda.synchronize()
        per = [ev[k].elapsed_time(ev[k + 1]) for k in range(n_steps)]
        return ev[0].elapsed_time(ev[-1]), per

    with ClockSampler(local) as clocks:
        t_batch, per_batch = timed(lambda k: graphs[k % pool].replay(), args.warmup, args.steps)
    status = max(b.status() for b in batches)

    plain_tables = [psf.Table(cfg_of(s, bits, layout)) for s in sessions]
    for t in plain_tables if args.sum_reduction else ():
        t.set_launch(sum_reduction=args.sum_reduction)

    def plain(k):
        for i, s in enumerate(sessions):
            plain_step(plain_tables[i], i, dev[i][k % pool], s["width"] * s["height"], s["depth"])

    t_plain, per_plain = timed(plain, args.warmup, args.steps)
    graph_tables = [psf.Table(cfg_of(s, bits, layout)) for s in sessions]
    for t in graph_tables if args.sum_reduction else ():
        t.set_launch(sum_reduction=args.sum_reduction)
    plain_graphs = []
    for it in range(pool):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for i, s in enumerate(sessions):
                plain_step(graph_tables[i], i, dev[i][it], s["width"] * s["height"], s["depth"])
        plain_graphs.append(g)
    t_pgraph, per_pgraph = timed(lambda k: plain_graphs[k % pool].replay(), args.warmup, args.steps)
    # the batched tables equal the plain ones bit for bit (same iterations, order-free sums)
    same = all(tables[i].export().tobytes() == plain_tables[i].export().tobytes() for i in range(len(sessions)))

    # per-iteration work of every session, counted by the plain tables (the batched kernel
    # does not count (warp, key) groups); every table ran warmup + steps identical iterations
    peaks = load_peaks()
    hbm = peaks["hbm_gbs"] * 1e9
    rates = GroupRates()
    bytes_phase = {"k_insert": 0.0, "k_update": 0.0, "k_query": 0.0}
    insert_floor = groups = touched_all = 0.0
    slot_bytes = 0
    for i, s in enumerate(sessions):
        st = plain_tables[i].stats()
        its = max(1, st["iterations"])
        touched = st["touched_cells"] / its
        g = st["leader_groups"] / its
        groups += g
        touched_all += touched
        sb = 64 << int(plain_tables[i].cfg.log2_capacity)
        slot_bytes += sb
        b = algorithmic_bytes(s["width"] * s["height"] * s["depth"], touched, bool(s["cache_fp16"]), bool(args.slot_cache))
        for k in bytes_phase:
            bytes_phase[k] += b[k]
        insert_floor += max(b["k_insert"] / hbm, g / rates(sb, touched, g))
    floor_s = {"k_insert": insert_floor, "k_update": bytes_phase["k_update"] / hbm,
               "k_query": bytes_phase["k_query"] / hbm}
    step_s = t_batch / args.steps / 1e3
    total_bytes = sum(bytes_phase.values())
    setup = {"workload": f"sessions_{len(sessions)}", "slot_cache": bool(args.slot_cache), "capacity_bits": bits,
             "batch_knobs": knobs}
    if layout:
        setup["key_layout"] = {1: "dense", 2: "inline"}[layout]
    roofline = {"kernel": "k_batch", "bound": "hbm+l2_atomic (phase sum, insert per session)",
                "frac": sum(floor_s.values()) / step_s,
                "traffic": load_traffic("k_batch", False, setup),
                "algorithmic_bytes_per_launch": total_bytes,
                "floor_ms": {k: 1e3 * v for k, v in floor_s.items()},
                "hbm": {"achieved": total_bytes / step_s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": total_bytes / step_s / hbm, "algorithmic_bytes_per_step": total_bytes,
                        "peak_note": "of measured (MEASURED_PEAKS.json hbm_gbs)"},
                "l2_atomic": {"groups_per_step": groups, "touched_per_step": touched_all, "slot_bytes": slot_bytes,
                              "probes": len(rates.memo),
                              "peak_note": "of measured (live bulk-reduction probe per session on its own slot "
                                           "records and touched sectors; the insert floor sums each session's "
                                           "max(bytes at the HBM rate, groups at its probe rate))"}}

    def rate(ms):
        return V * args.steps / (ms / 1e3)

    res = {
        "workload": f"{len(sessions)} sessions, width log-uniform 128..1280, 16:9, depth U{{2..6}}, FP16 cache",
        "value": rate(t_batch), "unit": UNIT, "ms_per_step": t_batch / args.steps, "vertices_per_step": V,
        "steps": args.steps, "warmup": args.warmup, "pool": pool, "batch_knobs": knobs,
        "capacity": f"2^(ceil(log2 V) + {bits}) slots per session ({'autotuned' if tune else 'fixed'} load factor)",
        "key_layout": {0: "auto", 1: "dense key array", 2: "keys in the slot records"}[layout],
        "slot_cache": bool(args.slot_cache),
        "l2": f"inputs larger than L2: {pool} distinct iterations of {V * 64 / 1e9:.1f} GB",
        "latency_ms": {"p50": float(np.percentile(per_batch, 50)), "p99": float(np.percentile(per_batch, 99))},
        "plain_loop": {"value": rate(t_plain), "ms_per_step": t_plain / args.steps, "launches_per_step": 3 * len(sessions),
                       "p50": float(np.percentile(per_plain, 50)), "p99": float(np.percentile(per_plain, 99))},
        "plain_graph": {"value": rate(t_pgraph), "ms_per_step": t_pgraph / args.steps,
                        "p50": float(np.percentile(per_pgraph, 50)), "p99": float(np.percentile(per_pgraph, 99))},
        "speedup_vs_plain_loop": t_plain / t_batch, "speedup_vs_plain_graph": t_pgraph / t_batch,
        "roofline": roofline,
        "identical_to_plain": same, "status": status, "autotune": tuned["all"],
        "gpu_launches": args.steps, "clocks": clocks.summary(),
    }
    for group in (tables, plain_tables, graph_tables):
        for t in group:
            t.close()
    for b in batches:
        b.close()
    return res


def run_sessions(args) -> None:
    """64 uneven render sessions: the fused batched form against the plain per-session loop."""
    rank, world, local = dist_env()
    from synth.scene import session_workloads

    gen = generate_sessions(session_workloads(args.sessions, first_session_seed=4000 + 1000 * rank),
                            max(1, min(args.pool, args.warmup + args.steps)))
    import torch

    torch.cuda.set_device(local)
    r = measure_sessions(args, gen, local, tune=bool(args.tune))
    line = {
        "metric": METRIC + ", 64 batched sessions", "value": r["value"] * world, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64 fixed point", "data": "synthetic",
        "config": {"workload": r["workload"], "vertices_per_step": r["vertices_per_step"], "pool": r["pool"],
                   "batch_knobs": r["batch_knobs"], "capacity": r["capacity"], "key_layout": r["key_layout"],
                   "slot_cache": r["slot_cache"], "l2": r["l2"]},
    }
    line.update({k: r[k] for k in ("latency_ms", "plain_loop", "plain_graph", "speedup_vs_plain_loop",
                                   "speedup_vs_plain_graph", "roofline", "identical_to_plain", "status", "autotune",
                                   "gpu_launches", "clocks")})
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sessions_aggregate(gen["sessions"], min(os.cpu_count() or 1, 32))
    if rank == 0:
        print(json.dumps(line), flush=True)


class TemplateSource:
    """Vertex streams for served requests: each request is mapped to the pre-generated
    template with its depth and the nearest width (log scale); iteration k of a session
    reads template iteration k mod n_iter.  Templates are resident on the device."""

    def __init__(self, templates: dict):
        # templates: {(width, depth): [tensor per iteration]}
        self.templates = templates
        self.widths = {}
        for (w, d) in templates:
            self.widths.setdefault(d, []).append(w)

    def fit(self, req: dict) -> dict:
        """The request resized to its template (the sizes the server will run)."""
        import math

        ws = self.widths[req["depth"]]
        w = min(ws, key=lambda x: abs(math.log(x) - math.log(req["width"])))
        h = int(round(9 * w / 16))
        r = dict(req)
        r["width"], r["height"] = w, h
        v = w * h * req["depth"]
        r["log2_capacity"] = int(math.ceil(math.log2(v))) + 1
        from synth.scene import config4_q_bits

        r["pos_bits"] = config4_q_bits(r["log2_capacity"], r["dir_bits"])
        r["vertices"] = v
        return r

    def __call__(self, req: dict, iteration: int):
        its = self.templates[(req["width"], req["depth"])]
        return its[iteration % len(its)]


def _gen_template(args):
    w, d, it = args
    from synth.scene import iteration_vertices

    h = int(round(9 * w / 16))
    wl = dict(width=w, height=h, depth=d, seed=7000 + 10 * w + d, radiance="glossy", camera_step=0.0,
              camera_x0=0.5)
    return iteration_vertices(wl, it)


TEMPLATE_WIDTHS = (128, 181, 256, 362, 512, 724, 1024, 1280)


def make_templates(depths=(2, 3, 4, 5, 6), widths=TEMPLATE_WIDTHS, iterations=2) -> dict:
    """Real path-vertex streams for a grid of (width, depth), generated on the host."""
    import torch

    jobs = [(w, d, it) for w in widths for d in depths for it in range(iterations)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(os.cpu_count() or 1, 32)) as p:
        res = p.map(_gen_template, jobs, chunksize=1)
    out = {}
    for (w, d, it), v in zip(jobs, res):
        out.setdefault((w, d), []).append(torch.from_numpy(v).cuda())
    return out


def template_stats(src: "TemplateSource", reqs: list[dict]) -> dict:
    """Touched cells and (warp, key) groups of every template iteration the trace reads, keyed
    (width, depth, iteration mod n_iter): both depend only on the batch (its keys and their
    order), not on the table's history or capacity, so one plain table per template counts
    them (untimed, after the served runs)."""
    import paper_2005_07547_b300 as psf
    from paper_2005_07547_b300.serve import table_config

    out = {}
    for (w, d), its in src.templates.items():
        r = next((q for q in reqs if (q["width"], q["depth"]) == (w, d)), None)
        if r is None:
            continue
        t = psf.Table(table_config(r))
        prev = {"touched_cells": 0, "leader_groups": 0}
        for k, v in enumerate(its):
            t.insert(v)
            t.update()
            st = t.stats()
            out[(w, d, k)] = (st["touched_cells"] - prev["touched_cells"], st["leader_groups"] - prev["leader_groups"])
            prev = st
        t.close()
    return out


def served_roofline(tick_log: list, stats: dict, n_iter: int, hbm_bps: float, rate_of,
                    slot_cache: bool) -> dict:
    """Roofline of a served run from its completed ticks.  A tick's floor is the sum over its
    sessions of each session's insert floor -- the larger of its algorithmic bytes at the HBM
    rate and its (warp, key) groups at the bulk-reduction probe's rate on its own footprint,
    rate_of(slot_bytes, touched, groups) -- and its blend and query bytes at the HBM rate.
    It is the same for the fused kernel (which takes the sessions one after the other in each
    phase) and the plain launches.  frac = total floor / total device time of the ticks;
    the caller reports device_busy = device time over the wall time."""
    floor = dev_ms = total_bytes = groups_all = 0.0
    for tick in tick_log:
        dev_ms += tick["ms"]
        for req, it, log2cap in tick["items"]:
            touched, g = stats[(req["width"], req["depth"], it % n_iter)]
            b = algorithmic_bytes(req["width"] * req["height"] * req["depth"], touched, True, slot_cache)
            floor += max(b["k_insert"] / hbm_bps, g / rate_of(64 << log2cap, touched, g)) \
                + (b["k_update"] + b["k_query"]) / hbm_bps
            total_bytes += sum(b.values())
            groups_all += g
    dev_s = dev_ms / 1e3
    return {"frac": floor / dev_s if dev_s > 0 else None, "floor_ms": 1e3 * floor, "device_ms": dev_ms,
            "ticks": len(tick_log), "algorithmic_bytes": total_bytes, "groups": groups_all,
            "hbm_achieved_GBps": total_bytes / dev_s / 1e9 if dev_s > 0 else None}


def run_serving(args) -> None:
    """Poisson arrivals at --rate per second for --duration seconds, 60 GB table budget:
    the continuous-batching server against the plain per-session loop on the same trace."""
    from synth.scene import serving_arrivals

    import torch

    import paper_2005_07547_b300 as psf
    from paper_2005_07547_b300.serve import Server

    rank, world, local = dist_env()
    reqs = serving_arrivals(args.rate, args.duration, seed=5 + rank)
    templates = make_templates()
    torch.cuda.set_device(local)
    psf.load()
    src = TemplateSource(templates)
    reqs = [src.fit(r) for r in reqs]
    reports, logs = {}, {}
    for mode in ("batched", "plain"):
        # keys inside the slot records unless --key-layout says otherwise: the layout the batched
        # tuner picks on the 64-session workload (like the load factor --capacity-bits 1)
        srv = Server(src, budget_bytes=args.budget_gb * 1e9, mode=mode, slot_cache=bool(args.slot_cache),
                     capacity_bits=args.capacity_bits, log_ticks=True, key_layout=args.key_layout or 2)
        with ClockSampler(local) as clocks:
            rep = srv.run(reqs, args.duration)
        rep["clocks"] = clocks.summary()
        logs[mode] = srv.tick_log
        srv.close()
        torch.cuda.synchronize()
        reports[mode] = rep
    # the rooflines (untimed): every template iteration's touched cells and groups, and the
    # bulk-reduction probe on each session footprint the trace ran
    stats = template_stats(src, reqs)
    n_iter = len(next(iter(templates.values())))
    rates = GroupRates()
    hbm = load_peaks()["hbm_gbs"] * 1e9
    for mode, rep in reports.items():
        rl = served_roofline(logs[mode], stats, n_iter, hbm, rates, bool(args.slot_cache))
        rl.update({"kernel": "k_batch" if mode == "batched" else "k_insert + k_update + k_query per session",
                   "bound": "hbm+l2_atomic (sum over each tick's sessions)",
                   "device_busy": rl["device_ms"] / 1e3 / rep["wall_s"] if rep["wall_s"] else None,
                   "peak_note": "of measured (MEASURED_PEAKS.json hbm_gbs; live bulk-reduction probe on each "
                                f"session footprint: {len(rates.memo)} probes)"})
        rep["roofline"] = rl
    b, p = reports["batched"], reports["plain"]
    line = {
        "metric": METRIC + ", served sessions", "value": b["vertices_per_s"] * world, "unit": UNIT, "n_gpus": world,
        "steps": b["ticks"], "warmup": 0, "ms_per_step": 1e3 * b["wall_s"] / max(1, b["ticks"]),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64 fixed point",
        "data": "synthetic",
        "config": {"workload": f"Poisson arrivals {args.rate}/s for {args.duration} s, sessions of 16..128 iterations, "
                               "width log-uniform 128..1280 mapped to the nearest template, depth U{2..6}",
                   "requests": len(reqs), "budget_gb": args.budget_gb, "templates": len(templates),
                   "capacity": f"2^(ceil(log2 V) + {args.capacity_bits}) slots per session",
                   "key_layout": {1: "dense key array", 2: "keys in the slot records"}[args.key_layout or 2]},
        "batched": b, "plain": p, "roofline": b["roofline"],
        "throughput_ratio_batched_over_plain": b["vertices_per_s"] / p["vertices_per_s"] if p["vertices_per_s"] else None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--impl", default="psf", choices=["psf", "reference"])
    ap.add_argument("--fp16", action="store_true", help="FP16 copy of the approximant for the query")
    ap.add_argument("--fp32", action="store_true", help="no FP16 copy: queries read the FP32 approximant")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--insert-mode", type=int, default=0, help="0: warp aggregation of equal keys; 1: none")
    ap.add_argument("--staging", type=int, default=0, help="bit 0: insert, bit 1: query stage vertex records through shared memory (TMA)")
    ap.add_argument("--sessions", type=int, default=64, help="sessions of the batched workload")
    ap.add_argument("--key-layout", type=int, default=0, help="0: auto, 1: dense key array, 2: keys in slot records")
    ap.add_argument("--levels", type=int, default=1, help="hierarchy levels of the table (1: flat)")
    ap.add_argument("--sum-reduction", type=int, default=0, help="0: one bulk (TMA) reduction per group, 1: four red.add")
    ap.add_argument("--slot-cache", type=int, default=1,
                    help="1: the insert notes each vertex's slot and the query reads it there; 0: the query probes")
    ap.add_argument("--pool", type=int, default=4, help="distinct resident iterations per session (batched)")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: Poisson arrival rate per second")
    ap.add_argument("--duration", type=float, default=10.0, help="serving: seconds of arrivals")
    ap.add_argument("--budget-gb", type=float, default=60.0, help="serving: device memory for tables")
    ap.add_argument("--capacity-bits", type=int, default=1,
                    help="serving, and sessions with --tune 0: tables of 2^(ceil(log2 V) + bits) slots")
    ap.add_argument("--tune", type=int, default=1,
                    help="1: pick grid caps and query layout with the autotuner before timing; 0: the flags' knobs")
    ap.add_argument("--batch-blocks", type=int, default=0,
                    help="sessions with --tune 0: resident blocks per SM of the fused kernel (0: occupancy)")
    ap.add_argument("--insert-blocks", type=int, default=0, help="cap on resident insert blocks per SM (0: occupancy)")
    ap.add_argument("--query-blocks", type=int, default=0, help="cap on resident query blocks per SM (0: occupancy)")
    ap.add_argument("--update-blocks", type=int, default=0, help="cap on resident blend blocks per SM (0: occupancy)")
    ap.add_argument("--query-layout", type=int, default=0,
                    help="0: one thread per path; 1: depth-split warp tiles (C_{j+1} by shuffle)")
    ap.add_argument("--payload", default="rgb", choices=["rgb", "sh"],
                    help="cell payload: RGB, or YCoCg with luminance in two SH bands over the normal")
    ap.add_argument("--sh-ridge", type=float, default=0.01, help="SH payload: ridge on band 1")
    ap.add_argument("--batched-extra", type=int, default=1,
                    help="single-session runs at N=1 also measure the 64-session batched form (extra key)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps are required")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "sessions":
        run_sessions(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "atomics":
        import torch

        torch.cuda.set_device(dist_env()[2])
        rates = {"l2_resident_32MB": atomic_probe_rates(n_words=1 << 22),
                 "dram_backed_256MB": atomic_probe_rates(n_words=1 << 25)}
        print(json.dumps({"metric": "L2 64-bit atomic throughput", "unit": "ops/s", "rates": rates}), flush=True)
    else:
        run_psf(args)


if __name__ == "__main__":
    main()
