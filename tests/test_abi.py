"""The C-ABI library builds, loads without a GPU, and exports exactly the
entry points include/gcharm.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    src = open(os.path.join(ROOT, "include", "gcharm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|uint64_t|const char \*)\s*(gc_\w+)\s*\(", src,
                                 re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2008_05712_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = header_symbols()
    for must in ["gc_pool_create", "gc_pool_upload", "gc_submit", "gc_flush",
                 "gc_read_results", "gc_wait", "gc_read_totals", "gc_stats", "gc_strerror"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in header_symbols():
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2008_05712_gb300 import gcharm
    assert gcharm.exported_symbols() == header_symbols()


def test_strerror_without_gpu(lib):
    lib.gc_strerror.restype = ctypes.c_char_p
    lib.gc_strerror.argtypes = [ctypes.c_int]
    assert lib.gc_strerror(0) == b"ok"
    assert b"unknown id" in lib.gc_strerror(-4)


def test_struct_layouts_match_header(tmp_path):
    # compile a probe against the header and compare with the ctypes mirrors
    import subprocess
    from paper_2008_05712_gb300 import gcharm
    probe = tmp_path / "probe.c"
    probe.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "gcharm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(gc_config),
         offsetof(gc_config, cuda_stream), sizeof(gc_task), offsetof(gc_task, target_ids),
         offsetof(gc_task, shift), sizeof(gc_stats_t), offsetof(gc_stats_t, stage_ms_sum),
         sizeof(gc_serve_config), sizeof(gc_serve_report), offsetof(gc_serve_report, wall_s));
  printf("%zu %zu %zu %zu %zu %zu %zu\\n", offsetof(gc_serve_config, keep_pageable),
         offsetof(gc_serve_config, poll_ns), offsetof(gc_serve_report, pinned_bytes),
         offsetof(gc_serve_report, retire_s), sizeof(gc_tuning),
         offsetof(gc_tuning, targets_per_lane), sizeof(gc_nbody_stats_t));
  return 0;
}
""")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)],
                   check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [ctypes.sizeof(gcharm.GcConfig), gcharm.GcConfig.cuda_stream.offset,
            ctypes.sizeof(gcharm.GcTask), gcharm.GcTask.target_ids.offset,
            gcharm.GcTask.shift.offset, ctypes.sizeof(gcharm.GcStats),
            gcharm.GcStats.stage_ms_sum.offset, ctypes.sizeof(gcharm.GcServeConfig),
            ctypes.sizeof(gcharm.GcServeReport), gcharm.GcServeReport.wall_s.offset,
            gcharm.GcServeConfig.keep_pageable.offset, gcharm.GcServeConfig.poll_ns.offset,
            gcharm.GcServeReport.pinned_bytes.offset, gcharm.GcServeReport.retire_s.offset,
            ctypes.sizeof(gcharm.GcTuning), gcharm.GcTuning.targets_per_lane.offset,
            ctypes.sizeof(gcharm.GcNbodyStats)]
    assert got == want


def test_missing_library_fails_loudly(tmp_path):
    from paper_2008_05712_gb300 import gcharm
    saved = gcharm._lib
    gcharm._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            gcharm.load(str(tmp_path / "nope.so"))
    finally:
        gcharm._lib = saved


def test_row_values_on_the_host():
    """gc_row_values (a host function, no GPU needed): the FP64 value s - c of
    each compensated row, component by component, with hand-worked values
    that an FP32 subtraction or swapped halves would get wrong."""
    import numpy as np
    from paper_2008_05712_gb300 import gcharm
    gcharm.load()
    rows = np.array([[1.0, -2.0, 0.5, 3.0, 2.0 ** -30, 0.0, -0.25, 3.0],
                     [0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0]], np.float32)
    v = gcharm.value(rows)
    assert v.dtype == np.float64 and v.shape == (2, 4)
    assert v[0].tolist() == [1.0 - 2.0 ** -30, -2.0, 0.75, 0.0]
    assert v[1].tolist() == [0.0, 0.0, 0.0, 0.0]
    assert gcharm.value(np.zeros((0, 8), np.float32)).shape == (0, 4)


def test_tuning_order_matches_header():
    # the binding's autotuner times are read by index: its order must be the
    # header's (((w * 2 + s) * 3 + t) * 3 + k) * 2 + l - 1 over GC_TUNE_COUNT
    from paper_2008_05712_gb300 import gcharm
    with open(os.path.join(ROOT, "include", "gcharm.h")) as f:
        count = int(re.search(r"#define GC_TUNE_COUNT (\d+)", f.read()).group(1))
    order = gcharm.tune_order()
    assert count == gcharm.GC_TUNE_COUNT == len(order)
    assert len({gcharm.tune_key(t) for t in order}) == count
    for idx, t in enumerate(order):
        w = (8, 16, 32).index(t["wu_max_targets"])
        tp = (64, 128, 256).index(t["tile_pairs"])
        kb = (8, 16, 32).index(t["comp_block"])
        assert idx == (((w * 2 + t["schedule"]) * 3 + tp) * 3 + kb) * 2 + t["targets_per_lane"] - 1
