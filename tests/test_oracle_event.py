"""Pins of the oracle's finder and selector (C2-C4, C7, C8) on whole events.

* a hand-derived golden case for the neighbour rule, cleaning and start hits;
* isolated low-noise tracks: every link joins consecutive clusters of one
  particle, and the selector returns exactly one track per particle holding
  all of its clusters (chain plus extension);
* invariants of the cellular automaton and the selector on a dense event;
* Monte-Carlo truth efficiency, fake and clone rates (sanity bars; the paper
  prints no efficiency, so these bars are not paper parity).
"""
import math

import numpy as np
import pytest

from paper_1712_09416_b300 import synth
from tests import _util


def test_golden_neighbours(orc):
    ev, g = _util.golden_event()
    out = orc.track_event(ev)
    exp = g["expected"]
    for name in ("up", "dn", "up_c", "dn_c"):
        for cid, v in exp[name].items():
            assert out[name][int(cid)] == v, (name, cid, out[name][int(cid)], v)
    for cid in exp["no_links_cids"]:
        assert out["up"][cid] == -1 and out["dn"][cid] == -1, cid
    starts = sorted(int(c) for c in np.nonzero((out["up_c"] >= 0) & (out["dn_c"] < 0))[0])
    assert starts == exp["starts"]
    assert out["n_starts"] == len(exp["starts"])
    assert out["n_tracklets"] == len(exp["chains"])
    assert out["t_chain_len"][0] == len(exp["chains"][0])
    assert out["t_start"][0] == exp["chains"][0][0]
    # the case holds exact ties of D and a candidate on a window edge by
    # construction: those hits carry near-tie bits, and no other hit does
    tie = out["c2_tie"]
    assert set(np.nonzero(tie)[0].tolist()) == set(int(c) for c in exp["c2_tie_cids"])


def test_isolated_tracks_links_follow_truth(orc):
    ev = _util.isolated_event()
    out = orc.track_event(ev)
    lab = ev.label
    linked = np.nonzero(out["up"] >= 0)[0]
    assert len(linked) > 0.9 * np.sum((ev.row > 0) & (ev.row < 158))
    for h in linked:
        u, d = out["up"][h], out["dn"][h]
        assert lab[u] == lab[h] == lab[d]
        assert ev.row[u] == ev.row[h] + 1 and ev.row[d] == ev.row[h] - 1


def test_isolated_tracks_one_track_each_with_all_clusters(orc):
    ev = _util.isolated_event()
    out = orc.track_event(ev)
    assert out["n_tracks"] == len(ev.particles)
    seen = set()
    for j in range(out["n_tracks"]):
        hits = _util.track_hits(out, j)
        lab = np.unique(ev.label[hits])
        assert len(lab) == 1
        p = int(lab[0])
        seen.add(p)
        assert set(hits.tolist()) == set(np.nonzero(ev.label == p)[0].tolist())
        # parameters at the innermost hit near truth (sigma = 0.01 cm)
        first = hits[0]
        prm = out["k_p"][j]
        truth = [ev.true_y[first], ev.true_z[first], ev.true_sinphi[first],
                 ev.particles.tanl[p], ev.particles.q[p] / ev.particles.pt[p]]
        cov = _util_cov_diag(orc, out["k_C"][j])
        pulls = (prm - truth) / np.sqrt(cov)
        assert np.all(np.abs(pulls) < 6), pulls
        assert out["k_ndf"][j] == 2 * len(hits) - 5
    assert seen == set(range(len(ev.particles)))


def _util_cov_diag(orc, Ct):
    return np.diag(orc.unpack_cov(Ct))


@pytest.fixture(scope="module")
def dense(orc):
    ev = synth.one_sector_event()
    return ev, orc.track_event(ev)


def test_cleaned_links_are_mutual_and_chains_disjoint(dense):
    ev, out = dense
    up, dn = out["up_c"], out["dn_c"]
    for h in np.nonzero(up >= 0)[0]:
        assert dn[up[h]] == h
    for h in np.nonzero(dn >= 0)[0]:
        assert up[dn[h]] == h
    # every hit is in at most one chain, each chain has exactly one start
    owner = np.full(ev.n, -1)
    starts = np.nonzero((up >= 0) & (dn < 0))[0]
    for s in starts:
        c = s
        while c >= 0:
            assert owner[c] == -1
            owner[c] = s
            c = up[c]
    chained = np.nonzero((up >= 0) | (dn >= 0))[0]
    assert np.all(owner[chained] >= 0)


def test_selector_invariants(orc, dense):
    ev, out = dense
    R = len(ev.row_x)
    all_hits = out["k_hit_cid"]
    assert len(np.unique(all_hits)) == len(all_hits)  # a cluster in at most one track
    keys = []
    for j in range(out["n_tracks"]):
        hits = _util.track_hits(out, j)
        rows = ev.row[hits]
        assert np.all(np.diff(rows.astype(int)) > 0)
        t = out["k_tracklet"][j]
        assert out["t_valid"][t] == 1
        nh = out["t_nhits"][t]
        assert len(hits) >= 10 and 2 * len(hits) >= nh
        key = (int(nh) << 32) | (0xFFFFFFFF - int(out["t_start"][t]))
        assert np.all(out["weight"][hits] == key)
        keys.append((out["k_sector"][j], rows[0], out["t_start"][t]))
        # owned hits are the tracklet's hits whose weight is its key
        th = out["t_rowhit"][t]
        th = th[th >= 0]
        assert set(hits.tolist()) == {c for c in th.tolist() if out["weight"][c] == key}
    assert keys == sorted(keys)
    assert R == 159


def test_weights_are_max_over_valid_tracklets(dense):
    ev, out = dense
    w = np.zeros(ev.n, dtype=np.uint64)
    for t in range(out["n_tracklets"]):
        if not out["t_valid"][t]:
            continue
        key = np.uint64((int(out["t_nhits"][t]) << 32) | (0xFFFFFFFF - int(out["t_start"][t])))
        h = out["t_rowhit"][t]
        h = h[h >= 0]
        w[h] = np.maximum(w[h], key)
    assert np.array_equal(w, out["weight"])


def test_tracklet_hits_and_counts(dense):
    ev, out = dense
    for t in range(out["n_tracklets"]):
        h = out["t_rowhit"][t]
        rows = np.nonzero(h >= 0)[0]
        assert len(rows) == out["t_nhits"][t]
        assert rows[0] == out["t_first_row"][t] and rows[-1] == out["t_last_row"][t]
        assert np.all(ev.row[h[rows]] == rows)
        assert np.all(ev.sector[h[rows]] == out["t_sector"][t])
        assert out["t_ndf"][t] == 2 * len(rows) - 5
        assert out["t_chain_len"][t] >= 3
        assert out["t_x"][t] == pytest.approx(float(ev.row_x[rows[0]]), abs=1e-5)


def test_mc_truth_one_sector(dense):
    ev, out = dense
    s = _util.mc_summary(ev, out)
    assert s["n_reconstructable"] > 100
    assert s["eff_pt02"] >= 0.95, s
    assert s["fake_rate"] < 0.02, s
    assert s["clone_rate"] < 0.05, s


def test_binary32_restatement_differs_only_at_near_ties(orc):
    """The neighbour rule restated in binary32 (the precision of the GPU
    tracker) takes the binary64 decision at every hit without near-tie bits;
    near ties are rare."""
    ev = synth.central_event()
    for sub in (synth.one_sector_event(), ev.select_sectors([3, 30])):
        out = orc.track_event(sub, shadow32=True)
        flip = (out["up32"] != out["up"]) | (out["dn32"] != out["dn"])
        assert not np.any(flip & (out["c2_tie"] == 0))
        assert out["n_c2_ties"] <= 1e-3 * max(1, out["n_links"])


def test_near_tie_bits_mark_what_rounding_can_flip(orc):
    """Moving one coordinate by far less than a binary32 rounding of the slopes
    flips a link only at a hit carrying a near-tie bit: the bits cover the
    pair gap, the D_MAX cut and the window edges."""
    ev, g = _util.golden_event()
    base = orc.track_event(ev)
    rng = np.random.default_rng(5)
    for trial in range(40):
        e = synth.Event(ev.y.copy(), ev.z.copy(), ev.row, ev.sector, ev.label, ev.row_x,
                        ev.n_sectors_phi, ev.split_z)
        k = int(rng.integers(0, ev.n))
        # one binary32 ulp up or down at the hit's coordinate
        e.y[k] = np.nextafter(e.y[k], np.float32(np.inf if trial % 2 else -np.inf))
        out = orc.track_event(e)
        moved = (out["up"] != base["up"]) | (out["dn"] != base["dn"])
        assert not np.any(moved & (base["c2_tie"] == 0) & (out["c2_tie"] == 0)), trial


def test_near_tie_flags_are_rare(dense):
    ev, out = dense
    f = out["t_flags"]
    assert np.count_nonzero(f & ~orc_chain_bit()) <= 0.02 * out["n_tracklets"]
    # chains joining two particles (a chain hit outside the chi2 acceptance)
    assert np.count_nonzero(f & orc_chain_bit()) <= 0.03 * out["n_tracklets"]


def orc_chain_bit():
    from oracle import oracle
    return oracle.TIE_CHAIN


def test_chain_flag_marks_chains_of_two_particles(orc):
    """ORC_TIE_CHAIN: a tracklet whose chain holds clusters of two particles
    that part ways gets the flag; single-particle chains of isolated tracks
    do not."""
    iso = _util.isolated_event()
    out = orc.track_event(iso)
    assert np.count_nonzero(out["t_flags"] & orc.TIE_CHAIN) == 0
    ev = synth.central_event().select_sectors([7])
    out = orc.track_event(ev)
    flagged = np.nonzero(out["t_flags"] & orc.TIE_CHAIN)[0]
    assert len(flagged) > 0
    mixed = 0
    for t in flagged:
        c = [int(out["t_start"][t])]
        while out["up_c"][c[-1]] >= 0:
            c.append(int(out["up_c"][c[-1]]))
        lab = ev.label[c]
        mixed += len(np.unique(lab[lab >= 0])) > 1 or np.any(lab < 0)
    assert mixed >= 0.8 * len(flagged), (mixed, len(flagged))


def test_rejects_invalid_input(orc):
    ev = synth.one_sector_event()
    bad = synth.Event(ev.y.copy(), ev.z, ev.row.copy(), ev.sector, ev.label, ev.row_x,
                      ev.n_sectors_phi, ev.split_z)
    bad.row[5] = 159
    with pytest.raises(RuntimeError):
        orc.track_event(bad)
    bad.row[5] = ev.row[5]
    bad.y[7] = np.nan
    with pytest.raises(RuntimeError):
        orc.track_event(bad)


def test_empty_event(orc):
    e = synth.Event(np.zeros(0, np.float32), np.zeros(0, np.float32), np.zeros(0, np.uint16),
                    np.zeros(0, np.uint16), np.zeros(0, np.int32), synth.default_row_x(), 18, 1)
    out = orc.track_event(e)
    assert out["n_tracks"] == 0 and out["n_tracklets"] == 0


def test_central_event_sectors_mc_truth(orc):
    """A few sectors of the 36-sector central event (about 4% of it)."""
    ev = synth.central_event()
    sub = ev.select_sectors([0, 7, 20, 33])
    out = orc.track_event(sub)
    s = _util.mc_summary(sub, out)
    assert s["eff_pt02"] >= 0.9, s
    assert s["fake_rate"] < 0.05, s
    assert out["n_c2_ties"] <= 1e-3 * out["n_links"]
    # sector independence: one sector alone gives the same tracks as in the subset
    one = ev.select_sectors([7])
    o1 = orc.track_event(one)
    m = out["k_sector"] == 7
    assert o1["n_tracks"] == int(m.sum())
    idx = np.nonzero(m)[0]
    for a, j in enumerate(idx):
        ha = sub.info["parent_index"][_util.track_hits(out, j)]
        hb = one.info["parent_index"][_util.track_hits(o1, a)]
        assert np.array_equal(ha, hb)
        np.testing.assert_array_equal(out["k_p"][j], o1["k_p"][a])


def _drop_rows(ev, particle, rows):
    keep = ~((ev.label == particle) & np.isin(ev.row, rows))
    idx = np.nonzero(keep)[0]
    return synth.Event(ev.y[idx], ev.z[idx], ev.row[idx], ev.sector[idx], ev.label[idx],
                       ev.row_x, ev.n_sectors_phi, ev.split_z, particles=ev.particles,
                       true_y=ev.true_y[idx], true_z=ev.true_z[idx],
                       true_sinphi=ev.true_sinphi[idx])


def _tracks_of(ev, out, particle):
    res = []
    for j in range(out["n_tracks"]):
        h = _util.track_hits(out, j)
        if np.all(ev.label[h] == particle):
            res.append(set(h.tolist()))
    return res


def test_chain_taken_by_a_forward_extension_gets_no_tracklet(orc):
    """C7a: one missing row cuts a track's links into an inner and an outer
    chain; the inner chain's forward extension bridges the gap and takes
    every hit of the outer chain, so the outer chain is dominated (no
    tracklet) and the track comes out once with all its clusters."""
    base = _util.isolated_event()
    full = orc.track_event(base)
    assert full["n_dominated"] == 0
    mid = int(np.median(base.row[base.label == 0]))
    ev = _drop_rows(base, 0, [mid])
    out = orc.track_event(ev)
    assert out["n_dominated"] == 1
    assert out["n_tracklets"] == full["n_tracklets"]
    tr = _tracks_of(ev, out, 0)
    assert len(tr) == 1 and tr[0] == set(np.nonzero(ev.label == 0)[0].tolist())
    # the surviving tracklet of particle 0 starts on its inner chain
    t0 = [t for t in range(out["n_tracklets"]) if ev.label[out["t_start"][t]] == 0]
    assert len(t0) == 1 and ev.row[out["t_start"][t0[0]]] < mid


def test_dominance_removes_tracklets_not_tracks(orc):
    """C7a on a central-event sector: the dominated chains are redundant (their
    clusters end up on emitted tracks nearly always) and the efficiency stays
    that of a sector tracker (pT > 0.2 GeV/c segments of >= 30 clusters found
    with >= 99%); the rule removes about half of the chains' tracklets."""
    ev = synth.central_event().select_sectors([7])
    o = orc.track_event(ev)
    s = _util.mc_summary(ev, o)
    assert s["eff_pt02"] >= 0.99, s
    up_c, dn_c = o["up_c"], o["dn_c"]
    built = set(o["t_start"].tolist())
    on_track = np.zeros(ev.n, bool)
    on_track[o["k_hit_cid"]] = True
    n_dom = n_covered = 0
    for st in np.nonzero((up_c >= 0) & (dn_c < 0))[0]:
        c = [int(st)]
        while up_c[c[-1]] >= 0:
            c.append(int(up_c[c[-1]]))
        if len(c) < 3 or st in built:
            continue
        n_dom += 1
        n_covered += bool(on_track[c].all())
    assert n_dom == o["n_dominated"] and n_dom > 0.4 * (n_dom + o["n_tracklets"])
    assert n_covered >= 0.95 * n_dom, (n_covered, n_dom)


def test_gap_of_max_gap_minus_one_rows_is_bridged(orc):
    """Four consecutive empty rows: the search steps over them (max_gap = 5)."""
    base = _util.isolated_event()
    mid = int(np.median(base.row[base.label == 0]))
    ev = _drop_rows(base, 0, list(range(mid, mid + 4)))
    out = orc.track_event(ev)
    tr = _tracks_of(ev, out, 0)
    assert len(tr) == 1
    assert tr[0] == set(np.nonzero(ev.label == 0)[0].tolist())


def test_gap_of_max_gap_rows_splits_the_track(orc):
    """Five consecutive empty rows end every search: two track segments."""
    base = _util.isolated_event()
    mid = int(np.median(base.row[base.label == 0]))
    ev = _drop_rows(base, 0, list(range(mid, mid + 5)))
    out = orc.track_event(ev)
    tr = _tracks_of(ev, out, 0)
    assert len(tr) == 2
    rows = sorted(sorted(ev.row[list(t)].tolist()) for t in tr)
    assert rows[0][-1] == mid - 1 and rows[1][0] == mid + 5
