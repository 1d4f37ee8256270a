"""Seeded synthetic path-vertex streams (shared input module).

This package produces the inputs that both the CUDA path and the CPU oracle
consume: path vertices shaped like a 1-spp path tracer's output on a small
procedural scene, plus the workload definitions (image size, path depth, table
size, quantisation) they are generated for. It holds none of the filtering
method's arithmetic -- no cell keys, no hashing, no fixed point, no blend and no
control variate -- so sharing it does not couple the oracle to the product.
"""

from .scene import (  # noqa: F401
    FLOATS_PER_VERTEX,
    Scene,
    make_scene,
    trace_paths,
    workload,
    session_workloads,
    serving_arrivals,
    config4_q_bits,
)
