"""Full-size, full-length parity: the 1280x720, depth-4 workload (3,686,400 vertices per
iteration, 2^22 slots, FP32 cache) over all 32 of its iterations, in the launch
configuration the benchmark times (the slot-cache insert, the blend, the slot-cache
query on one stream).

Every iteration the whole table is compared with the oracle after the blend (keys and
counters exactly, the approximant within 1e-5 relative), the whole table after the insert
(fixed-point sums and counters exactly) every eighth iteration and at the last, and the
control-variate outputs of every 8th path, all depths.  With equal vertex weights the
blend's square-root factor sqrt(c_new / (c_old + c_new)) falls with the iteration count,
so the 32 iterations take the FP32 blend far down the running average that eq. (10)-(11)
describe (Section "Temporal averaging").
"""

import numpy as np
import pytest

import fullsize
from parity import TOL_FP32, check_after_insert, check_after_update, check_cv

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

NAME, ITERATIONS, STRIDE = "1280x720_d4", 32, 8


def test_1280x720_depth4_all_32_iterations(psf_mod, oracle_mod):
    import torch

    from synth.scene import workload

    w = workload(NAME)
    P, D = w["width"] * w["height"], w["depth"]
    cfg = psf_mod.make_config(log2_capacity=w["log2_capacity"], pos_bits=w["pos_bits"], dir_bits=w["dir_bits"],
                              alpha_min=w["alpha_min"], cache_fp16=False)
    table = psf_mod.Table(cfg)
    ora = oracle_mod.Oracle(pos_bits=w["pos_bits"], dir_bits=w["dir_bits"], alpha_min=float(np.float32(w["alpha_min"])))
    slots = torch.empty(P * D, dtype=torch.int32, device="cuda")
    out = torch.empty((P * D, 3), dtype=torch.float32, device="cuda")
    for it, v in enumerate(fullsize.named_iterations(NAME, ITERATIONS)):
        dv = torch.from_numpy(v).cuda()
        table.insert_slots(dv, P, D, slots=slots)
        st = ora.insert(v)
        if it % 8 == 0 or it == ITERATIONS - 1:
            check_after_insert(table.export(), ora.export())
        table.update()
        ora.update()
        rec = ora.export()
        rel32, _ = check_after_update(table.export(), rec)
        table.query_cv_slots(dv, slots, P, D, out=out)
        vs, Ps = fullsize.sample_paths(v, P, D, STRIDE)
        ratio = check_cv(fullsize.sample_out(out, P, D, STRIDE), ora.query_cv(vs, Ps, D), vs, ora.lookup(vs, Ps, D), Ps,
                         D, float(cfg.beta), cfg.cv_max_depth, rec["L"])
        stats = table.stats()
        assert stats["status"] == st == 0
        assert (stats["dropped_vertices"], stats["zero_weight_vertices"]) == ora.counters()
        assert stats["live_cells"] == len(ora) and stats["iterations"] == it + 1
        print(f"iteration {it}: cells {len(rec)}, approximant err/bound {rel32 / TOL_FP32:.3g}, "
              f"cv err/bound {ratio:.3g}")
        del dv
    table.close()
