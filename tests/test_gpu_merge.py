"""Sector track merger and global refit on the GPU against the oracle (M0-M5).

The GPU merges its own sector tracks; the oracle merges its own.  Tracks are
compared by hit set; a track is left out of the exact comparison when any of
its source tracks carries a near-tie bit (tracker or merger) or holds a
cluster of a flagged tracklet, since binary32 may decide those differently.
Parameters of the compared tracks are held to the same bars as the sector
tracks'.  Noiseless helices across phi boundaries (also across phi = 0) and
the membrane come out as one track; batched and served launches give the
same merged tracks as single events.
"""
import math

import numpy as np
import pytest

from paper_1712_09416_b300 import synth
from tests import _parity

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


def merge_taint(o, m, sector_tracks=None):
    """Hits of every oracle output track with a source that carries a merger
    near-tie bit or that differs from the GPU's sector tracks.  sector_tracks
    (the GPU's tracks of the event without merging) gives the sector tracks
    that differ exactly, by hit set (their own parity is tested elsewhere);
    without it every track holding a cluster of a near-tie tracklet counts as
    different (a superset)."""
    off, cid = o["k_hit_off"], o["k_hit_cid"]
    o_sets = [tuple(cid[off[a]:off[a + 1]].tolist()) for a in range(o["n_tracks"])]
    if sector_tracks is None:
        bad_hits = _parity.tainted_hits(o)
        differs = [bool(set(h) & bad_hits) for h in o_sets]
        taint = set(bad_hits)
    else:
        g_sets = {tuple(sector_tracks.hits(j).tolist()) for j in range(sector_tracks.n_tracks)}
        differs = [h not in g_sets for h in o_sets]
        o_set = set(o_sets)
        taint = set()
        for h in g_sets - o_set:  # GPU sector tracks the oracle does not have
            taint.update(h)
    for srcs in m["sources"]:
        if any(m["flags"][g] or differs[g] for g in srcs):
            for g in srcs:
                taint.update(o_sets[g])
    return taint


def check_merged(tr, ev, orc, counters=None, max_diff_frac=2e-3, sector_tracks=None):
    o = orc.track_event(ev)
    m = orc.merge_tracks(ev, o)
    taint = merge_taint(o, m, sector_tracks)
    rep = _parity.compare_tracks(tr, m, taint)
    n = max(1, rep["n_oracle"])
    assert len(rep["missing"]) + len(rep["extra"]) <= max_diff_frac * n, \
        (len(rep["missing"]), len(rep["extra"]), rep["missing"][:3], rep["extra"][:3])
    assert rep["order_ok"]
    _parity.check_param_bars(rep["param_scaled"], "merged tracks", rep["param_sig"])
    merged = sum(len(s) > 1 for s in m["sources"])
    if counters is not None:
        assert counters["n_sector_tracks"] == o["n_tracks"]
        assert abs(counters["n_merge_chains"] - merged) <= max_diff_frac * n + 2
        assert counters["n_tracks"] == tr.n_tracks
    return o, m, rep


def sector_tracks(tp, ev):
    with tp.Tracker(ev.n + 65536) as t:
        return t.event(ev)


def test_merged_tracks_match_the_oracle(tp, mtrk, orc):
    ev = synth.batch_events(2, seed0=3000)[1]
    tr = mtrk.event(ev)
    o, m, rep = check_merged(tr, ev, orc, mtrk.counters())
    assert sum(len(s) > 1 for s in m["sources"]) > 1000
    assert rep["compared"] > 0.85 * rep["n_oracle"]  # the rest touch a near-tie
    # with the exact sector-track differences as the taint
    o, m, rep = check_merged(tr, ev, orc, sector_tracks=sector_tracks(tp, ev))
    assert rep["compared"] > 0.97 * rep["n_oracle"]


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


def check_sector_tracks(st, o, what):
    """The GPU's sector tracks of a whole event against the oracle's: hit sets
    of the tracks sharing no cluster with a near-tie tracklet, order,
    parameters (the merger's inputs, compared at full size)."""
    rep = _parity.compare_tracks(st, o, _parity.tainted_hits(o))
    n = max(1, rep["n_oracle"])
    assert len(rep["missing"]) + len(rep["extra"]) <= 1e-3 * n, \
        (what, len(rep["missing"]), len(rep["extra"]))
    assert rep["order_ok"] and "meta_mismatch" not in rep
    _parity.check_param_bars(rep["param_scaled"], what, rep["param_sig"])


def test_central_event_merge(tp, orc):
    """The full central event merged on the GPU against the oracle (and its
    sector tracks, whole, against the oracle's)."""
    ev = synth.central_event(seed=2)
    with tp.Tracker(2_000_000, params=merge_params(tp)) as t:
        tr = t.event(ev)
        c = t.counters()
    st = sector_tracks(tp, ev)
    o, m, rep = check_merged(tr, ev, orc, c, sector_tracks=st)
    assert c["n_merge_chains"] > 4000
    check_sector_tracks(st, o, "central-event sector tracks")


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


def oracle_by_sector(ev, orc):
    """The oracle's sector tracks of a 36-sector event from one call per
    sector on all host cores (sectors are independent), gathered into the
    record a whole-event call gives (cluster ids of the event)."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    n_sec = ev.n_sectors_phi * (2 if ev.split_z else 1)
    parts = [ev.select_sectors([s]) for s in range(n_sec)]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as pool:
        outs = list(pool.map(orc.track_event, parts))
    o = {}
    for k in ("k_x", "k_p", "k_C", "k_chi2", "k_ndf", "t_flags"):
        o[k] = np.concatenate([r[k] for r in outs])
    o["k_sector"] = np.concatenate([np.full(r["n_tracks"], s, np.int32) for s, r in enumerate(outs)])
    o["k_hit_cid"] = np.concatenate([p.info["parent_index"][r["k_hit_cid"]]
                                     for p, r in zip(parts, outs)]).astype(np.int32)
    o["k_hit_off"] = np.concatenate([[0], np.cumsum(np.concatenate(
        [np.diff(r["k_hit_off"]) for r in outs]))]).astype(np.int32)
    o["t_rowhit"] = np.concatenate([np.where(r["t_rowhit"] >= 0, p.info["parent_index"][r["t_rowhit"]], -1)
                                    for p, r in zip(parts, outs)])
    o["n_tracks"] = len(o["k_sector"])
    return o


def test_pileup_event_merge(tp, orc):
    """The pile-up event (7.37M clusters; vertices over +-200 cm, so many
    tracks cross the membrane) merged on the GPU against the oracle, and its
    sector tracks, whole, against the oracle's."""
    ev = synth.pileup_event()
    with tp.Tracker(ev.n + 65536, params=merge_params(tp)) as t:
        tr = t.event(ev)
        c = t.counters()
    o = oracle_by_sector(ev, orc)
    m = orc.merge_tracks(ev, o)
    st = sector_tracks(tp, ev)
    check_sector_tracks(st, o, "pile-up sector tracks")
    rep = _parity.compare_tracks(tr, m, merge_taint(o, m, st))
    n = max(1, rep["n_oracle"])
    assert len(rep["missing"]) + len(rep["extra"]) <= 2e-3 * n, (len(rep["missing"]), len(rep["extra"]))
    assert rep["order_ok"] and rep["compared"] > 0.9 * n, rep["compared"]
    _parity.check_param_bars(rep["param_scaled"], "merged pile-up tracks", rep["param_sig"])
    assert c["n_sector_tracks"] == o["n_tracks"]
    merged = sum(len(s) > 1 for s in m["sources"])
    assert merged > 20000 and abs(c["n_merge_chains"] - merged) <= 2e-3 * n
