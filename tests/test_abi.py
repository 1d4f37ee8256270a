"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
function include/psf.h declares, the binding's struct layouts match the header as a
C compiler lays them out, and host-detected argument errors are reported."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


@pytest.fixture(scope="module")
def lib():
    from paper_2005_07547_b300 import build, _abi

    build.build()
    return _abi.load()


def _declared_functions():
    names = set()
    for fn in os.listdir(INCLUDE):
        if fn.endswith(".h"):
            text = open(os.path.join(INCLUDE, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(psf_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(lib):
    from paper_2005_07547_b300 import _abi

    declared = _declared_functions()
    assert {"psf_create", "psf_insert", "psf_update", "psf_query_cv", "psf_destroy"} <= declared
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (psf_[a-z0-9_]+)$", out, flags=re.M))
    assert declared <= exported, declared - exported
    # the Python binding declares a signature for every one of them
    assert declared <= set(_abi.SIGNATURES), declared - set(_abi.SIGNATURES)
    for name in declared:
        assert getattr(lib, name) is not None


def test_struct_layouts_match_the_header(tmp_path):
    from paper_2005_07547_b300 import _abi

    src = tmp_path / "layout.c"
    src.write_text(r"""
#include <stdio.h>
#include <stddef.h>
#include "psf.h"
int main(void) {
  printf("config %zu %zu %zu %zu\n", sizeof(psf_config), offsetof(psf_config, alpha_min),
         offsetof(psf_config, cv_max_depth), offsetof(psf_config, blend_mode));
  printf("record %zu %zu %zu %zu %zu\n", sizeof(psf_cell_record), offsetof(psf_cell_record, c_new),
         offsetof(psf_cell_record, c_old), offsetof(psf_cell_record, L), offsetof(psf_cell_record, L_fp16));
  printf("stats %zu %zu %zu\n", sizeof(psf_stats), offsetof(psf_stats, status), offsetof(psf_stats, table_bytes));
  printf("shrec %zu %zu %zu\n", sizeof(psf_sh_cell_record), offsetof(psf_sh_cell_record, c_old),
         offsetof(psf_sh_cell_record, coef));
  printf("config2 %zu %zu\n", offsetof(psf_config, payload), offsetof(psf_config, sh_ridge));
  printf("batchcfg %zu %zu\n", sizeof(psf_batch_config), offsetof(psf_batch_config, phase_blocks_per_sm));
  printf("launch %zu %zu\n", sizeof(psf_launch_config), offsetof(psf_launch_config, query_layout));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    lines = dict(l.split(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    C = _abi.Config
    assert lines["config"].split() == [str(x) for x in (ctypes.sizeof(C), C.alpha_min.offset, C.cv_max_depth.offset,
                                                        C.blend_mode.offset)]
    d = _abi.CELL_DTYPE
    assert lines["record"].split() == [str(x) for x in (d.itemsize, d.fields["c_new"][1], d.fields["c_old"][1],
                                                        d.fields["L"][1], d.fields["L_fp16"][1])]
    S = _abi.Stats
    assert lines["stats"].split() == [str(x) for x in (ctypes.sizeof(S), S.status.offset, S.table_bytes.offset)]
    h = _abi.SH_CELL_DTYPE
    assert lines["shrec"].split() == [str(x) for x in (h.itemsize, h.fields["c_old"][1], h.fields["coef"][1])]
    assert lines["config2"].split() == [str(x) for x in (C.payload.offset, C.sh_ridge.offset)]
    B = _abi.BatchConfig
    assert lines["batchcfg"].split() == [str(x) for x in (ctypes.sizeof(B), B.phase_blocks_per_sm.offset)]
    Lc = _abi.LaunchConfig
    assert lines["launch"].split() == [str(x) for x in (ctypes.sizeof(Lc), Lc.query_layout.offset)]


def test_table_bytes_and_config_validation(lib):
    from paper_2005_07547_b300 import _abi

    good = _abi.make_config(log2_capacity=16)
    n16 = lib.psf_table_bytes(ctypes.byref(good))
    # header + 64-byte slot record (key inside, the automatic choice at 2^16 slots) + dirty bits
    assert n16 >= (1 << 16) * 64 + (1 << 16) // 8
    assert n16 % 256 == 0
    fp16 = _abi.make_config(log2_capacity=16, cache_fp16=True)  # plus the FP16 copy and dense keys
    assert lib.psf_table_bytes(ctypes.byref(fp16)) == n16 + (1 << 16) * (8 + 8)
    assert lib.psf_table_bytes(ctypes.byref(_abi.make_config(log2_capacity=17))) > 2 * n16 - 4096
    # a dense key array costs 8 bytes per slot more than keys inside the slot records
    dense = lib.psf_table_bytes(ctypes.byref(_abi.make_config(log2_capacity=16, key_layout=1)))
    assert dense == n16 + (1 << 16) * 8  # the automatic choice keeps a 2^16 table's keys inline
    # the SH payload: 192-byte records and a dense key array
    sh = lib.psf_table_bytes(ctypes.byref(_abi.make_config(log2_capacity=16, payload=1)))
    assert sh == n16 + (1 << 16) * (192 + 8 - 64)
    big = [lib.psf_table_bytes(ctypes.byref(_abi.make_config(log2_capacity=23, key_layout=k))) for k in (0, 1, 2)]
    assert big[0] == big[1] == big[2] + (1 << 23) * 8  # and uses the dense array from 2^23 slots
    for bad in (dict(log2_capacity=3), dict(log2_capacity=31), dict(dir_bits=6), dict(pos_bits=21),
                dict(frac_bits=7), dict(frac_bits=33), dict(alpha_min=1.5), dict(alpha_min=-0.1),
                dict(blend_mode=2), dict(beta=float("nan")), dict(key_layout=3), dict(payload=2),
                dict(payload=1, cache_fp16=True), dict(payload=1, levels=2), dict(payload=1, key_layout=2),
                dict(payload=1, sh_ridge=-1.0), dict(payload=1, sh_ridge=float("inf")),
                dict(payload=1, sh_ridge=float("nan"))):
        assert lib.psf_table_bytes(ctypes.byref(_abi.make_config(**bad))) == 0, bad
    assert lib.psf_table_bytes(None) == 0


def test_host_detected_argument_errors(lib):
    from paper_2005_07547_b300 import _abi

    cfg = _abi.make_config(log2_capacity=8)
    n = lib.psf_table_bytes(ctypes.byref(cfg))
    h = ctypes.c_void_p()
    # these are rejected on the host before any CUDA call
    assert lib.psf_create(ctypes.byref(cfg), None, n, None, ctypes.byref(h)) == _abi.PSF_ERR_INVALID_ARG
    assert lib.psf_create(ctypes.byref(cfg), 0x1000 + 8, n, None, ctypes.byref(h)) == _abi.PSF_ERR_INVALID_ARG
    assert lib.psf_create(ctypes.byref(cfg), 0x100000, n - 256, None, ctypes.byref(h)) == _abi.PSF_ERR_NO_MEM
    bad = _abi.make_config(log2_capacity=2)
    assert lib.psf_create(ctypes.byref(bad), 0x100000, 1 << 20, None, ctypes.byref(h)) == _abi.PSF_ERR_INVALID_ARG
    assert lib.psf_insert(None, None, 0, None) == _abi.PSF_ERR_INVALID_ARG
    assert lib.psf_update(None, None) == _abi.PSF_ERR_INVALID_ARG
    assert lib.psf_query_cv(None, None, 1, 1, None, None) == _abi.PSF_ERR_INVALID_ARG
    assert lib.psf_reset(None, None) == _abi.PSF_ERR_INVALID_ARG
    assert lib.psf_insert_slots(None, None, 1, 1, None, None) == _abi.PSF_ERR_INVALID_ARG
    assert lib.psf_query_cv_slots(None, None, None, 1, 1, None, None) == _abi.PSF_ERR_INVALID_ARG
    assert lib.psf_destroy(None) == _abi.PSF_OK
    assert lib.psf_abi_version() == 7


def test_product_package_does_not_touch_the_oracle():
    """The product path never imports or loads anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_2005_07547_b300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"\boracle\b", text.replace("the oracle", "")), fn
