"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/tpctrack.h declares (no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tpctrack.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tpc_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1712_09416_b300 import build, tpctrack
    build.build()
    return tpctrack.lib()


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ("tpc_track_create", "tpc_track_event", "tpc_track_batch", "tpc_track_submit",
              "tpc_track_poll", "tpc_track_release", "tpc_track_debug_dump",
              "tpc_track_last_error", "tpc_track_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1712_09416_b300 import tpctrack
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert sorted(tpctrack.EXPORTED) == declared_functions()


def test_default_params_without_gpu(lib):
    from paper_1712_09416_b300 import tpctrack
    p = tpctrack.tpc_track_default_params()
    assert p.chi2_hit == 16.0 and p.max_gap == 5 and abs(p.d_max - 0.6) < 1e-7
    assert p.min_tracklet_hits == 10 and abs(p.sin_max - 0.99) < 1e-7


def test_create_rejects_bad_config_before_touching_the_device(lib):
    from paper_1712_09416_b300 import tpctrack
    cfg = tpctrack.tpc_track_config()
    cfg.max_clusters_per_event = 0
    cfg.max_events_in_flight = 1
    cfg.params = tpctrack.tpc_track_default_params()
    ctx = ctypes.c_void_p()
    assert lib.tpc_track_create(ctypes.byref(cfg), ctypes.byref(ctx)) == tpctrack.TPC_EINVAL
    assert not ctx.value
    cfg.max_clusters_per_event = 1000
    cfg.params.chi2_hit = -1.0
    assert lib.tpc_track_create(ctypes.byref(cfg), ctypes.byref(ctx)) == tpctrack.TPC_EINVAL
    assert lib.tpc_track_create(None, ctypes.byref(ctx)) == tpctrack.TPC_EINVAL
    # merger parameters: merge is 0 or 1, a positive cut, an ordered gap window
    cfg.params = tpctrack.tpc_track_default_params()
    assert cfg.params.merge == 0 and cfg.params.merge_chi2 == 30.0
    assert cfg.params.merge_dx_lo == -5.0 and cfg.params.merge_dx_hi == 30.0
    for field, value in (("merge", 2), ("merge_chi2", 0.0), ("merge_dx_lo", 31.0),
                         ("merge_chi2", float("nan"))):
        cfg.params = tpctrack.tpc_track_default_params()
        setattr(cfg.params, field, value)
        assert lib.tpc_track_create(ctypes.byref(cfg), ctypes.byref(ctx)) == tpctrack.TPC_EINVAL, field
        assert not ctx.value


def test_struct_layouts_match_the_header(lib, tmp_path):
    """Every record of tpctrack.h, compiled by gcc: its size and the offset of
    each field equal those of the ctypes mirror in the binding."""
    import shutil
    import subprocess
    from paper_1712_09416_b300 import tpctrack
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    recs = [tpctrack.tpc_geometry, tpctrack.tpc_clusters, tpctrack.tpc_tracks,
            tpctrack.tpc_track_params, tpctrack.tpc_track_config, tpctrack.tpc_track_counters,
            tpctrack.tpc_kernel_time, tpctrack.tpc_track_schedule, tpctrack.tpc_dump_tracklet,
            tpctrack.tpc_async_stats, tpctrack.tpc_chi2_fit]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tpctrack.h"', 'int main(void) {']
    for r in recs:
        n = r.__name__
        lines.append(f'printf("{n} size %zu\\n", sizeof({n}));')
        for f, _ in r._fields_:
            lines.append(f'printf("{n} {f} %zu\\n", offsetof({n}, {f}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(ROOT, "include")
    subprocess.run(["gcc", "-std=c11", "-I", inc, "-o", str(exe), str(src)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        rec, key, val = ln.split()
        got[(rec, key)] = int(val)
    for r in recs:
        n = r.__name__
        assert got[(n, "size")] == ctypes.sizeof(r), n
        for f, _ in r._fields_:
            assert got[(n, f)] == getattr(r, f).offset, (n, f)