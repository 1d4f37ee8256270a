"""The continuous-batching server: sessions admitted by table memory as others retire,
each session's table and outputs identical alone and in the mix."""

import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _requests():
    from synth.scene import config4_q_bits

    shapes = [(48, 3, 4), (32, 2, 2), (64, 5, 3), (40, 4, 5), (56, 2, 3), (32, 6, 2), (48, 3, 6)]
    out = []
    for k, (w, d, iters) in enumerate(shapes):
        h = int(round(9 * w / 16))
        v = w * h * d
        cap = int(math.ceil(math.log2(v))) + 1
        out.append(dict(name=f"r{k}", arrival_s=0.002 * k, width=w, height=h, depth=d, iterations=iters,
                        log2_capacity=cap, pos_bits=config4_q_bits(cap, 3), dir_bits=3, alpha_min=0.1,
                        cache_fp16=bool(k % 2), seed=500 + k))
    return out


class _Source:
    """Two real iterations per request, generated on the host, resident on the device."""

    def __init__(self, reqs):
        import torch

        from synth.scene import iteration_vertices

        self.data = {}
        for r in reqs:
            wl = dict(width=r["width"], height=r["height"], depth=r["depth"], seed=r["seed"], radiance="glossy",
                      camera_step=0.0, camera_x0=0.5)
            self.data[r["name"]] = [torch.from_numpy(iteration_vertices(wl, it)).cuda() for it in range(2)]

    def __call__(self, req, iteration):
        return self.data[req["name"]][iteration % 2]


@pytest.mark.parametrize("mode,graph,slots", [("batched", True, True), ("batched", False, False), ("plain", False, True),
                                              ("plain", False, False)])
def test_served_sessions_equal_alone(psf_mod, mode, graph, slots):
    import torch

    from paper_2005_07547_b300.serve import Server, table_bytes

    reqs = _requests()
    src = _Source(reqs)
    # a budget of about three tables forces queueing and admission as sessions retire
    budget = sum(sorted(table_bytes(r) for r in reqs)[-3:]) + 1
    results = {}

    def keep(sess):
        results[sess.request["name"]] = (sess.table.export().tobytes(), sess.out.cpu().numpy().copy(), sess.done)

    srv = Server(src, budget_bytes=budget, mode=mode, use_graph=graph, on_retire=keep, slot_cache=slots)
    rep = srv.run(reqs, duration_s=30.0, drain=True)
    srv.close()
    assert rep["sessions_finished"] == len(reqs) and rep["requests_waiting_at_end"] == 0
    assert rep["iteration_latency_ms"]["p99"] is not None
    for r in reqs:
        t = psf_mod.Table(psf_mod.make_config(log2_capacity=r["log2_capacity"], pos_bits=r["pos_bits"],
                                              dir_bits=r["dir_bits"], alpha_min=r["alpha_min"],
                                              cache_fp16=r["cache_fp16"]))
        P, D = r["width"] * r["height"], r["depth"]
        for k in range(r["iterations"]):
            out = t.step(src(r, k), P, D)
        exp, got_out, done = results[r["name"]]
        assert done == r["iterations"]
        assert t.export().tobytes() == exp, r["name"]
        assert np.array_equal(out.cpu().numpy(), got_out), r["name"]
        t.close()
    torch.cuda.synchronize()


def test_admission_respects_the_memory_budget(psf_mod):
    from paper_2005_07547_b300.serve import Server, table_bytes

    reqs = _requests()
    src = _Source(reqs)
    budget = max(table_bytes(r) for r in reqs) + 1  # one table at a time
    peak = []

    class Tracking(Server):
        def _tick(self):
            peak.append((len(self.live), self.used))
            super()._tick()

    srv = Tracking(src, budget_bytes=budget, mode="batched")
    rep = srv.run(reqs, duration_s=30.0, drain=True)
    srv.close()
    assert rep["sessions_finished"] == len(reqs)
    assert all(used <= budget for _, used in peak)
    assert max(n for n, _ in peak) == 1
