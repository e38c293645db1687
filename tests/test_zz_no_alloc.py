"""The allocation-free links entry point against tpc_track_event's links.

tpc_track_links_noalloc serves callers that cannot allocate device memory
(an allocator owned by a host framework, a hard memory budget, or code that
must not trigger the synchronisation of cudaMalloc/cudaFree): its scratch is a
static device array of the library.  This file is collected last so that a
run stopping at the first failure has run every other test before it.
"""
import numpy as np
import pytest

from paper_1712_09416_b300 import synth
from tests import _util

pytestmark = pytest.mark.gpu


def _device(ev):
    import torch
    return (torch.from_numpy(ev.y).cuda(), torch.from_numpy(ev.z).cuda(),
            torch.from_numpy(ev.row.view(np.int16)).cuda(),
            torch.from_numpy(ev.sector.view(np.int16)).cuda())


def test_noalloc_links_equal_tracker_links_twice():
    import torch
    from paper_1712_09416_b300 import build, tpctrack as tp
    build.build()
    ev = synth.one_sector_event()
    g, keep_x = tp.geometry_of(ev)
    params = tp.tpc_track_default_params()
    # links through the existing entry point (context with its own arenas)
    with tp.Tracker(200_000) as t:
        t.event(ev)
        ref_up, ref_dn = tp.dump_links(t.ctx, ev.n)
    dev = _device(ev)
    c, keep = tp.clusters_of(*dev)
    for call in range(2):
        up = torch.full((ev.n,), -7, dtype=torch.int32, device="cuda")
        dn = torch.full((ev.n,), -7, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        rc = tp.tpc_track_links_noalloc(c, g, params, up.data_ptr(), dn.data_ptr(), 0)
        assert rc == tp.TPC_OK, (call, rc)
        assert np.array_equal(up.cpu().numpy(), ref_up), call
        assert np.array_equal(dn.cpu().numpy(), ref_dn), call


def test_noalloc_rejects_more_clusters_than_its_scratch():
    import torch
    from paper_1712_09416_b300 import build, tpctrack as tp
    build.build()
    n = 131073
    y = torch.zeros(n, dtype=torch.float32, device="cuda")
    r = torch.zeros(n, dtype=torch.int16, device="cuda")
    c, keep = tp.clusters_of(y, y, r, r)
    ev = synth.one_sector_event()
    g, keep_x = tp.geometry_of(ev)
    out = torch.zeros(n, dtype=torch.int32, device="cuda")
    rc = tp.tpc_track_links_noalloc(c, g, tp.tpc_track_default_params(), out.data_ptr(),
                                    out.data_ptr(), 0)
    assert rc == tp.TPC_EINVAL


def test_noalloc_at_its_capacity_over_36_sectors(orc):
    """131,072 clusters (the scratch's limit) over 36 sectors with the z split:
    links equal tpc_track_event's on two calls in a row, and the oracle's
    binary64 decision outside its near ties."""
    import torch
    from paper_1712_09416_b300 import build, tpctrack as tp
    build.build()
    full = synth.central_event()
    keep = np.sort(np.random.default_rng(7).choice(full.n, 131072, replace=False))
    ev = synth.Event(full.y[keep], full.z[keep], full.row[keep], full.sector[keep],
                     full.label[keep], full.row_x, full.n_sectors_phi, full.split_z)
    assert ev.n == 131072 and len(np.unique(ev.sector)) == 36
    g, keep_x = tp.geometry_of(ev)
    with tp.Tracker(200_000) as t:
        t.event(ev)
        ref_up, ref_dn = tp.dump_links(t.ctx, ev.n)
    dev = _device(ev)
    c, keep_c = tp.clusters_of(*dev)
    for call in range(2):
        up = torch.full((ev.n,), -7, dtype=torch.int32, device="cuda")
        dn = torch.full((ev.n,), -7, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        rc = tp.tpc_track_links_noalloc(c, g, tp.tpc_track_default_params(), up.data_ptr(),
                                        dn.data_ptr(), 0)
        assert rc == tp.TPC_OK, (call, rc)
        assert np.array_equal(up.cpu().numpy(), ref_up), call
        assert np.array_equal(dn.cpu().numpy(), ref_dn), call
    o = _util.oracle_by_sector(ev, orc)
    diff = np.nonzero((ref_up != o["up"]) | (ref_dn != o["dn"]))[0]
    assert np.all(o["c2_tie"][diff] != 0) and len(diff) <= 1e-3 * max(1, o["n_links"])


def test_noalloc_row_above_4096_is_a_capacity_error():
    """A pad row with more clusters than a row may hold returns TPC_ECAPACITY;
    the next call on the shared scratch is correct again."""
    import torch
    from paper_1712_09416_b300 import build, tpctrack as tp
    build.build()
    n = 5000
    rng = np.random.default_rng(4)
    bad = synth.Event(rng.uniform(-10, 10, n).astype(np.float32),
                      rng.uniform(0, 200, n).astype(np.float32), np.full(n, 40, np.uint16),
                      np.zeros(n, np.uint16), np.full(n, -1, np.int32), synth.default_row_x(), 18, 1)
    g, keep_x = tp.geometry_of(bad)
    c, keep_c = tp.clusters_of(*_device(bad))
    out_u = torch.zeros(n, dtype=torch.int32, device="cuda")
    out_d = torch.zeros(n, dtype=torch.int32, device="cuda")
    rc = tp.tpc_track_links_noalloc(c, g, tp.tpc_track_default_params(), out_u.data_ptr(),
                                    out_d.data_ptr(), 0)
    assert rc == tp.TPC_ECAPACITY
    ev = synth.one_sector_event()
    g1, keep_x1 = tp.geometry_of(ev)
    with tp.Tracker(200_000) as t:
        t.event(ev)
        ref_up, ref_dn = tp.dump_links(t.ctx, ev.n)
    c1, keep_c1 = tp.clusters_of(*_device(ev))
    up = torch.full((ev.n,), -7, dtype=torch.int32, device="cuda")
    dn = torch.full((ev.n,), -7, dtype=torch.int32, device="cuda")
    rc = tp.tpc_track_links_noalloc(c1, g1, tp.tpc_track_default_params(), up.data_ptr(),
                                    dn.data_ptr(), 0)
    assert rc == tp.TPC_OK
    assert np.array_equal(up.cpu().numpy(), ref_up) and np.array_equal(dn.cpu().numpy(), ref_dn)
