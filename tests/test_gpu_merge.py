"""Sector track merger and global refit on the GPU against the oracle (M0-M5).

The GPU merges its own sector tracks; the oracle merges its own.  Tracks are
compared by hit set; a track is left out of the exact comparison when any of
its source tracks carries a merger near-tie bit or holds a cluster of a
tracklet that differs from the GPU's (which the sector-tracker comparison
allows only at tracklets the oracle flags as near ties).
Parameters of the compared tracks are held to the same bars as the sector
tracks'.  Noiseless helices across phi boundaries (also across phi = 0) and
the membrane come out as one track; batched and served launches give the
same merged tracks as single events.
"""
import math

import numpy as np
import pytest

from paper_1712_09416_b300 import synth
from tests import _parity, _util

pytestmark = pytest.mark.gpu

FIELDS = ("sector", "x", "param", "cov", "chi2", "ndf", "hit_off", "hit_cid")


@pytest.fixture(scope="module")
def tp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1712_09416_b300 import build, tpctrack
    build.build()
    return tpctrack


def merge_params(tp):
    p = tp.tpc_track_default_params()
    p.merge = 1
    return p


@pytest.fixture(scope="module")
def mtrk(tp):
    t = tp.Tracker(2_000_000, max_events_per_launch=4, params=merge_params(tp))
    yield t
    t.close()


def tracklet_taint(tp, ctx, ev, o):
    """Hits of the tracklets of the context's last launch that differ from
    the oracle's: differences are allowed only at tracklets the oracle flags
    as near ties (asserted here), so every tainted hit stems from an oracle
    flag."""
    g = _util.gpu_stages(tp, ctx, ev)
    ex, _ = _parity.check_links(g, o)
    R = len(ev.row_x)
    rep = _parity.compare_tracklets(g["tracklets"], o, R, _parity.chain_exempt(o, ex, R))
    _parity.check_tracklets(rep)
    return rep["taint"]


def merge_taint(o, m, tl_taint):
    """Hits of every oracle output track with a source that carries a merger
    near-tie bit or shares a cluster with a tracklet that differs (tl_taint)."""
    off, cid = o["k_hit_off"], o["k_hit_cid"]
    o_sets = [tuple(cid[off[a]:off[a + 1]].tolist()) for a in range(o["n_tracks"])]
    differs = [bool(set(h) & tl_taint) for h in o_sets]
    taint = set(tl_taint)
    for srcs in m["sources"]:
        if any(m["flags"][g] or differs[g] for g in srcs):
            for g in srcs:
                taint.update(o_sets[g])
    return taint


def check_merged(tp, t, tr, ev, orc, *, o=None, max_diff_frac=2e-3, what="merged tracks"):
    """Merged GPU tracks of the last launch on context t against the oracle's
    merger run on the oracle's own sector tracks."""
    o = orc.track_event(ev) if o is None else o
    m = orc.merge_tracks(ev, o)
    counters = t.counters()
    taint = merge_taint(o, m, tracklet_taint(tp, t.ctx, ev, o))
    rep = _parity.compare_tracks(tr, m, taint)
    n = max(1, rep["n_oracle"])
    assert len(rep["missing"]) + len(rep["extra"]) <= max_diff_frac * n, \
        (len(rep["missing"]), len(rep["extra"]), rep["missing"][:3], rep["extra"][:3])
    assert rep["order_ok"]
    _parity.check_param_bars(rep["param_scaled"], what)
    merged = sum(len(s) > 1 for s in m["sources"])
    assert counters["n_sector_tracks"] == o["n_tracks"]
    assert abs(counters["n_merge_chains"] - merged) <= max_diff_frac * n + 2
    assert counters["n_tracks"] == tr.n_tracks
    longest = max((len(s) for s in m["sources"]), default=0)
    print(f"{what}: {rep['n_oracle']} tracks, {merged} chains (longest {longest} tracks), "
          f"compared {rep['compared_share']:.4f}, plain bars {rep['plain_share']:.4f}")
    return o, m, rep


def test_merged_tracks_match_the_oracle(tp, mtrk, orc):
    ev = synth.batch_events(2, seed0=3000)[1]
    tr = mtrk.event(ev)
    o, m, rep = check_merged(tp, mtrk, tr, ev, orc)
    assert sum(len(s) > 1 for s in m["sources"]) > 1000
    assert rep["compared_share"] > 0.97, rep["compared_share"]


def test_merge_off_gives_the_sector_tracks(tp, mtrk):
    ev = synth.batch_events(2, seed0=3000)[0]
    with tp.Tracker(2_000_000) as t:
        plain = t.event(ev)
        c = t.counters()
    assert c["n_merge_links"] == 0 and c["n_sector_tracks"] == c["n_tracks"]
    merged = mtrk.event(ev)
    assert mtrk.counters()["n_sector_tracks"] == plain.n_tracks
    assert merged.n_tracks <= plain.n_tracks
    # every cluster of a sector track is in exactly one merged track
    assert sorted(merged.hit_cid.tolist()) == sorted(plain.hit_cid.tolist())


@pytest.mark.parametrize("q,pt,tanl,phi0,vz,split", [
    (1.0, 0.5, 0.3, 17.0, 0.0, False), (1.0, 0.3, -0.4, 35.0, 0.0, False),
    (-1.0, 2.0, -0.3, 50.0, 45.0, True)])
def test_noiseless_helices_come_out_whole(tp, mtrk, q, pt, tanl, phi0, vz, split):
    p = synth.Particles(q=np.array([q]), pt=np.array([pt]), tanl=np.array([tanl]),
                        phi0=np.array([math.radians(phi0)]), vx=np.zeros(1), vy=np.zeros(1),
                        vz=np.array([vz]))
    ev = synth.make_event(np.random.default_rng(0), p, n_sectors_phi=18, split_z=split, sigma=0.0,
                          noise_frac=0.0, dtype=np.float32, shuffle=False)
    tr = mtrk.event(ev)
    assert mtrk.counters()["n_sector_tracks"] >= 2
    assert tr.n_tracks == 1
    h0 = tr.hit_cid[0]
    truth = np.array([ev.y[h0], ev.z[h0], ev.true_sinphi[h0], tanl, q / pt])
    err = np.abs(tr.param[0] - truth) / np.maximum(np.abs(truth), 1.0)
    assert err.max() < 2e-4, err  # binary32 coordinates and arithmetic
    assert tr.ndf[0] == 2 * len(tr.hit_cid) - 5


def test_batched_and_served_merges_equal_single_events(tp, mtrk):
    evs = synth.batch_events(n_events=4, seed0=3300)
    alone = [mtrk.event(e) for e in evs]
    got = mtrk.batch(evs)
    for k, (a, b) in enumerate(zip(alone, got)):
        for f in FIELDS:
            assert np.array_equal(getattr(a, f), getattr(b, f)), (k, f)
    s = tp.Tracker(2_000_000, max_events_in_flight=2, max_events_per_launch=2)
    try:
        tp.tpc_track_set_params(s.ctx, merge_params(tp))
        keep, tickets = [], []
        for e in evs:
            g, kx = tp.geometry_of(e)
            c, k = tp.clusters_of(e.y, e.z, e.row, e.sector)
            keep.append((g, kx, c, k))
            tickets.append(tp.tpc_track_submit(s.ctx, c, g, float(e.bz)))
        for k, (a, tk) in enumerate(zip(alone, tickets)):
            b = tp.tpc_track_poll(s.ctx, tk, 60_000_000)
            assert b is not None
            for f in FIELDS:
                assert np.array_equal(getattr(a, f), getattr(b, f)), ("served", k, f)
            tp.tpc_track_release(s.ctx, tk)
    finally:
        s.close()


def test_central_event_merge(tp, orc):
    """The full central event merged on the GPU against the oracle's merger
    (its sector tracks, whole, are compared in the sector-tracker tests)."""
    ev = synth.central_event(seed=2)
    with tp.Tracker(2_000_000, params=merge_params(tp)) as t:
        tr = t.event(ev)
        o, m, rep = check_merged(tp, t, tr, ev, orc, o=_util.oracle_by_sector(ev, orc),
                                 what="central event merged")
        assert t.counters()["n_merge_chains"] > 4000
    assert rep["compared_share"] > 0.95, rep["compared_share"]


def test_empty_tiny_and_one_sector_events_with_merging(tp, mtrk, orc):
    """No clusters, a few noise clusters, a one-wedge event (no partner
    sectors): merging leaves the sector tracks as they are."""
    g, kx = tp.geometry_of(synth.batch_events(1, seed0=3000)[0])
    for n in (0, 1, 7):
        rng = np.random.default_rng(n)
        y = rng.uniform(-10, 10, n).astype(np.float32)
        z = rng.uniform(-100, 100, n).astype(np.float32)
        row = rng.integers(0, 159, n).astype(np.uint16)
        sec = rng.integers(0, 36, n).astype(np.uint16)
        c, keep = tp.clusters_of(y, z, row, sec)
        tr = tp.tpc_track_event(mtrk.ctx, c, g, 0.5)
        assert tr.n_tracks == 0 and mtrk.counters()["n_merge_links"] == 0
    ev = synth.one_sector_event(seed=1)
    tr = mtrk.event(ev)
    c = mtrk.counters()
    assert c["n_merge_links"] == 0 and c["n_tracks"] == c["n_sector_tracks"] == tr.n_tracks
    with tp.Tracker(200_000) as t:
        plain = t.event(ev)
    for f in FIELDS:
        assert np.array_equal(getattr(tr, f), getattr(plain, f)), f


def test_pileup_event_merge(tp, orc):
    """The pile-up event (7.37M clusters; vertices over +-200 cm, so many
    tracks cross the membrane) merged on the GPU against the oracle."""
    ev = synth.pileup_event()
    with tp.Tracker(ev.n + 65536, params=merge_params(tp)) as t:
        tr = t.event(ev)
        o, m, rep = check_merged(tp, t, tr, ev, orc, o=_util.oracle_by_sector(ev, orc),
                                 what="pile-up event merged")
        c = t.counters()
    assert rep["compared_share"] > 0.9, rep["compared_share"]
    merged = sum(len(s) > 1 for s in m["sources"])
    assert merged > 20000
