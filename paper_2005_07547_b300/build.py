"""Build the CUDA library libpsf.so in-tree for sm_103a (B300).

    python -m paper_2005_07547_b300.build [--force]

nvcc cross-compiles without a GPU.  The resource usage that ptxas reports
(registers, spills, shared memory) is written to csrc/ptxas.log.
"""

from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libpsf.so")
SOURCES = ["psf.cu", "psf_batch.cu"]
DEPS = SOURCES + ["psf_device.cuh", "psf_table.h"]
# measurement-only library: the L2 atomic-throughput probe (not part of the filtering path)
PROBE_LIB = os.path.join(HERE, "libatomic_probe.so")
PROBE_SOURCES = ["atomic_probe.cu"]

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC", "-shared",
    "-Xptxas", "-v",
]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _stale(lib: str, deps: list[str]) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    paths = [os.path.join(CSRC, f) for f in deps] + [os.path.join(INCLUDE, "psf.h"), __file__]
    return any(os.path.getmtime(d) > t for d in paths)


def _compile(lib: str, sources: list[str], log: str) -> None:
    cmd = [_nvcc(), *NVCC_FLAGS, "-I", INCLUDE, "-I", CSRC,
           *[os.path.join(CSRC, s) for s in sources], "-o", lib + ".tmp"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    with open(os.path.join(CSRC, log), "w") as f:
        f.write(res.stdout + res.stderr)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stderr[-4000:])
    os.replace(lib + ".tmp", lib)


def build(force: bool = False) -> str:
    if force or _stale(LIB, DEPS):
        _compile(LIB, SOURCES, "ptxas.log")
    if force or _stale(PROBE_LIB, PROBE_SOURCES):
        _compile(PROBE_LIB, PROBE_SOURCES, "ptxas_probe.log")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
