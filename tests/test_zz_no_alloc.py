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
