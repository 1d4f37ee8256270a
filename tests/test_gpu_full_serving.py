"""Full-size serving parity: Poisson arrivals at 200 per second for half a second (about 100
render sessions of 16..128 iterations, width log-uniform 128..1280, 16:9, depth 2..6, each
at its own size with two generated inputs that its iterations alternate), a 60 GB table
budget, the continuous-batching server with its CUDA graph, slot cache and the keys in the
slot records (the benchmark's served configuration).  Every finished session's table and
last outputs equal, bit for bit, those of the same session run alone through plain psf_step
calls on a table with the library's default key layout; four sessions spread over the size range are also
checked against the oracle over all their iterations (spawned workers)."""

import hashlib
import multiprocessing as mp

import numpy as np
import pytest

import fullsize

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

RATE, ARRIVALS_S, N_INPUTS, STRIDE = 200.0, 0.5, 2, 8


def _digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def test_served_sessions_at_full_size_equal_alone_and_oracle(psf_mod, oracle_mod):
    import torch

    from paper_2005_07547_b300.serve import Server, table_config
    from synth.scene import serving_arrivals

    reqs = serving_arrivals(RATE, ARRIVALS_S)
    assert len(reqs) > 50
    # four sessions for the oracle: the lightest of each quarter of the size range
    work = sorted(reqs, key=lambda r: r["vertices"])
    picked = {min(q, key=lambda r: r["vertices"] * r["iterations"])["name"]
              for q in np.array_split(np.array(work, dtype=object), 4)}
    inputs = fullsize.served_iterations(reqs, N_INPUTS)
    dev = {r["name"]: [torch.from_numpy(v).cuda() for v in inputs[k]] for k, r in enumerate(reqs)}
    del inputs

    def source(req, iteration):
        return dev[req["name"]][iteration % N_INPUTS]

    served, keep = {}, {}

    def on_retire(sess):
        r = sess.request
        rec = sess.table.export()
        served[r["name"]] = (_digest(rec), _digest(sess.out.cpu().numpy()), sess.done)
        if r["name"] in picked:
            keep[r["name"]] = {"table": rec, "out": fullsize.sample_out(sess.out, sess.P, sess.D, STRIDE)}

    srv = Server(source, budget_bytes=60e9, mode="batched", use_graph=True, on_retire=on_retire, slot_cache=True,
                 key_layout=2)
    rep = srv.run(reqs, duration_s=ARRIVALS_S, drain=True)
    srv.close()
    print({k: rep[k] for k in ("ticks", "vertices", "vertices_per_s", "sessions_finished", "iteration_latency_ms")})
    admitted = set(served)
    assert rep["sessions_finished"] == len(admitted) > 0 and picked <= admitted
    for r in reqs:
        if r["name"] not in admitted:
            continue
        t = psf_mod.Table(table_config(r))
        P, D = r["width"] * r["height"], r["depth"]
        for k in range(r["iterations"]):
            out = t.step(source(r, k), P, D)
        want = (_digest(t.export()), _digest(out.cpu().numpy()), r["iterations"])
        assert served[r["name"]] == want, r["name"]
        t.close()
    jobs = [{"request": r, "n_inputs": N_INPUTS, "stride": STRIDE, **keep[r["name"]]} for r in reqs if r["name"] in picked]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        for res in pool.map(fullsize.oracle_served_check, jobs, chunksize=1):
            print(res)
    print(f"{len(admitted)} of {len(reqs)} requests served; all equal alone")
