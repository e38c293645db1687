"""GPU tracker vs the CPU oracle, stage by stage, through the C ABI.

Every test here runs the CUDA path of libtpctrack.so on the B300 and compares
it element by element with the oracle on the same seeded events (bars in
tests/_parity.py).  Sizes span several look-back tiles and a ragged tail; the
full-size central event is compared on a sample of its sectors (sectors are
independent, so the oracle computes the sampled ones alone).
"""
import numpy as np
import pytest

from paper_1712_09416_b300 import synth
from tests import _parity, _util

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1712_09416_b300 import build, tpctrack
    build.build()
    return tpctrack


@pytest.fixture(scope="module")
def trk(tp):
    t = tp.Tracker(2_000_000, max_events_per_launch=16)
    yield t
    t.close()


# The merger's near-tie width on its match chi2 (1.0) covers the chi2 change
# 2 sqrt(chi2) (m_a + m_b) that deviations of Mahalanobis size m_a, m_b of the
# two sector tracks' states make at the cut (chi2 <= 31): m up to
# 1.0 / (4 sqrt(31)) = 0.045.  The whole-event comparisons report how many
# compared tracks exceed it.
MERGE_TIE_M = 0.045


def run(tp, trk, ev):
    tr = trk.event(ev)
    return dict(_util.gpu_stages(tp, trk.ctx, ev), tracks=tr, counters=trk.counters())


def check_event(tp, trk, ev, orc, *, o=None, max_diff_frac=1e-3, what="event"):
    """Every stage of the GPU run of ev against the oracle (o: the oracle's
    record, computed here when not given).  Returns the GPU record, the
    oracle record and the tracklet and track reports."""
    g = run(tp, trk, ev)
    o = orc.track_event(ev) if o is None else o
    ex, n_link_diff = _parity.check_links(g, o)
    R = len(ev.row_x)
    rep = _parity.compare_tracklets(g["tracklets"], o, R, _parity.chain_exempt(o, ex, R))
    _parity.check_tracklets(rep, max_diff_frac)
    trep = _parity.compare_tracks(g["tracks"], o, rep["taint"])
    assert trep["missing"] == [] and trep["extra"] == [], (trep["missing"][:3], trep["extra"][:3])
    assert trep["order_ok"]
    assert "meta_mismatch" not in trep
    _parity.check_param_bars(trep["param_scaled"], "tracks")
    c = g["counters"]
    assert abs(c["n_links"] - o["n_links"]) <= n_link_diff
    assert c["n_starts"] == len(g["starts"])
    assert abs(c["n_tracklets"] - o["n_tracklets"]) <= len(rep["flagged_diff"])
    print(f"{what}: {o['n_links']} links ({n_link_diff} differ, {o['n_c2_ties']} near ties), "
          f"{rep['n_oracle']} tracklets ({len(rep['flagged_diff'])} flagged ones differ), "
          f"{trep['n_oracle']} tracks, compared {trep['compared_share']:.4f}, "
          f"within the plain bars {trep['plain_share']:.4f}, Mahalanobis deviation max "
          f"{trep['maha'].max() if len(trep['maha']) else 0.0:.2e}, p99.9 "
          f"{np.quantile(trep['maha'], 0.999) if len(trep['maha']) else 0.0:.2e}, above "
          f"{MERGE_TIE_M}: {int((trep['maha'] > MERGE_TIE_M).sum())}")
    return g, o, rep, trep


def test_golden_neighbours_on_gpu(tp, trk):
    ev, gold = _util.golden_event()
    g = run(tp, trk, ev)
    exp = gold["expected"]
    for name in ("up", "dn", "up_c", "dn_c"):
        for cid, v in exp[name].items():
            assert g[name][int(cid)] == v, (name, cid)
    assert g["starts"].tolist() == exp["starts"]


def test_one_sector_event_stage_parity(tp, trk, orc):
    ev = synth.one_sector_event()
    g, o, rep, trep = check_event(tp, trk, ev, orc)
    assert trep["compared"] >= 0.95 * trep["n_oracle"]
    s = _util.mc_summary(ev, g["tracks"])
    assert s["eff_pt02"] >= 0.95 and s["fake_rate"] < 0.02, s


def test_sparse_pp_like_event_stage_parity(tp, trk, orc):
    """A 20-track event over all 36 sectors (the low end of the batched
    workload's multiplicities): every stage against the oracle."""
    rng = np.random.default_rng(3999)
    ev = synth.served_event(rng, 20)
    g, o, rep, trep = check_event(tp, trk, ev, orc)
    assert g["counters"]["n_tracks"] > 0


def test_isolated_tracks(tp, trk, orc):
    ev = _util.isolated_event()
    check_event(tp, trk, ev, orc, max_diff_frac=0.0)


def test_central_event_whole(tp, orc):
    """The full-size central event (1.73M clusters, 36 sectors) on the GPU,
    every stage and every track against the oracle (run sector by sector on
    all host cores: sectors are independent)."""
    ev = synth.central_event()
    with tp.Tracker(ev.n + 65536) as t:
        g, o, rep, trep = check_event(tp, t, ev, orc, o=_util.oracle_by_sector(ev, orc),
                                      what="central event")
    assert trep["compared_share"] >= 0.95, trep["compared_share"]
    assert (trep["maha"] > MERGE_TIE_M).sum() <= np.ceil(1e-3 * len(trep["maha"]))


def test_eight_central_events_in_one_launch_equal_one_alone(tp):
    """The benchmark's timed step: eight copies of the central event side by
    side in one launch (13.9M clusters).  Every event's tracks equal the
    event tracked alone, bit for bit (compared with the oracle in
    test_central_event_whole)."""
    ev = synth.central_event()
    with tp.Tracker(8 * ev.n + 65536, max_events_per_launch=8) as t:
        alone = t.event(ev)
        outs = t.batch([ev] * 8)
        assert t.counters()["n_clusters"] == 8 * ev.n
    assert len(outs) == 8
    for b in outs:
        for f in ("sector", "x", "param", "cov", "chi2", "ndf", "hit_off", "hit_cid"):
            assert np.array_equal(getattr(alone, f), getattr(b, f)), f


def test_pileup_event_whole(tp, orc):
    """Pile-up stress event (50 collisions, vertex z within +-200 cm, about
    7.4M clusters) in one launch, every stage and every track against the
    oracle; the Monte-Carlo efficiency and fake rate of GPU and oracle tracks
    agree up to the tracks that touch a tracklet that differs."""
    ev = synth.pileup_event()
    with tp.Tracker(ev.n + 65536) as t:
        g, o, rep, trep = check_event(tp, t, ev, orc, o=_util.oracle_by_sector(ev, orc),
                                      what="pile-up event")
    assert g["counters"]["n_clusters"] == ev.n
    assert trep["compared_share"] >= 0.90, trep["compared_share"]
    assert (trep["maha"] > MERGE_TIE_M).sum() <= np.ceil(1e-3 * len(trep["maha"]))
    mg = _util.mc_summary(ev, g["tracks"])
    mo = _util.mc_summary(ev, o)
    tol = len(rep["taint"]) + 2
    assert abs(mg["n_reco"] - mo["n_reco"]) <= tol, (mg, mo)
    assert abs(mg["fakes"] - mo["fakes"]) <= tol, (mg, mo)
    assert abs(mg["eff"] - mo["eff"]) * max(1, mg["n_reconstructable"]) <= tol, (mg, mo)
    print("pile-up gpu", mg, "oracle", mo)


def test_batched_launch_against_the_oracle(tp, orc):
    """The 64-event batch of uneven multiplicity (3.7k to 1.66M clusters, 15.45M
    in all) in one launch; eight of its events, from the smallest to the
    largest, every stage and every track against the oracle."""
    evs = synth.batch_events(64)
    sizes = np.array([e.n for e in evs])
    order = np.argsort(sizes)
    pick = sorted(set(order[np.linspace(0, 63, 8).round().astype(int)].tolist()))
    assert int(order[-1]) in pick
    with tp.Tracker(int(sizes.sum()) + 65536, max_events_per_launch=64) as t:
        trs = t.batch(evs)
        for k in pick:
            ev = evs[k]
            g = dict(_util.gpu_stages(tp, t.ctx, ev, event=k), tracks=trs[k])
            o = _util.oracle_by_sector(ev, orc)
            ex, n_link_diff = _parity.check_links(g, o)
            R = len(ev.row_x)
            rep = _parity.compare_tracklets(g["tracklets"], o, R, _parity.chain_exempt(o, ex, R))
            _parity.check_tracklets(rep)
            trep = _parity.compare_tracks(trs[k], o, rep["taint"])
            assert trep["missing"] == [] and trep["extra"] == [], k
            assert trep["order_ok"] and "meta_mismatch" not in trep, k
            _parity.check_param_bars(trep["param_scaled"], f"batch event {k}")
            assert trep["compared_share"] >= 0.95 or trep["n_oracle"] < 100, (k, trep["compared_share"])
            print(f"batch event {k}: {ev.n} clusters, {trep['n_oracle']} tracks, compared "
                  f"{trep['compared_share']:.4f}, plain bars {trep['plain_share']:.4f}")
        # a stage dump outside the launch's events is refused
        with pytest.raises(tp.TpcError):
            tp.dump_starts(t.ctx, event=64)


def test_device_inputs_equal_host_inputs(tp, trk):
    import torch
    ev = synth.one_sector_event(seed=21)
    a = trk.event(ev)
    dev = (torch.from_numpy(ev.y).cuda(), torch.from_numpy(ev.z).cuda(),
           torch.from_numpy(ev.row.view(np.int16)).cuda(),
           torch.from_numpy(ev.sector.view(np.int16)).cuda())
    b = trk.event(ev, device_arrays=dev)
    for f in ("sector", "x", "param", "cov", "chi2", "ndf", "hit_off", "hit_cid"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_repeat_is_bit_identical(tp, trk):
    ev = synth.one_sector_event(seed=33)
    a = trk.event(ev)
    b = trk.event(ev)
    for f in ("sector", "x", "param", "cov", "chi2", "ndf", "hit_off", "hit_cid"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_graph_replay_equals_direct_launches(tp, monkeypatch):
    """The kernel sequence captured as a CUDA graph (default) and launched
    kernel by kernel (TPC_NO_GRAPH=1) give identical results, also when the
    event shape changes between launches and the graph is re-captured."""
    evs = synth.batch_events(n_events=3, seed0=4100)
    monkeypatch.setenv("TPC_NO_GRAPH", "1")
    direct = tp.Tracker(2_000_000)
    monkeypatch.delenv("TPC_NO_GRAPH")
    graph = tp.Tracker(2_000_000)
    try:
        for i in (0, 1, 0, 2, 2, 1):
            a = direct.event(evs[i])
            b = graph.event(evs[i])
            for f in ("sector", "x", "param", "cov", "chi2", "ndf", "hit_off", "hit_cid"):
                assert np.array_equal(getattr(a, f), getattr(b, f)), (i, f)
    finally:
        direct.close()
        graph.close()


def test_schedule_changes_speed_not_results(tp):
    """Every schedule value (grid and block shapes) gives the same tracks;
    out-of-range values are rejected; the autotuner returns a valid schedule
    and leaves the results unchanged."""
    evs = synth.batch_events(n_events=2, seed0=4200)
    with tp.Tracker(2_000_000, max_events_per_launch=2) as t:
        ref = t.batch(evs)
        s0 = tp.tpc_track_get_schedule(t.ctx)
        assert s0["tl_blocks_per_sm"] == s0["tl_max_per_sm"] >= 1 and s0["n_sm"] >= 1
        variants = [dict(nb_threads=64), dict(nb_threads=256), dict(sort_threads=256),
                    dict(bin_blocks_per_sm=1), dict(bin_blocks_per_sm=16),
                    dict(tl_blocks_per_sm=1), dict(tl_blocks_per_sm=max(1, s0["tl_max_per_sm"] // 2)),
                    dict(nb_mode=1)]
        for v in variants:
            tp.tpc_track_set_schedule(t.ctx, **{**s0, **v})
            got = t.batch(evs)
            for a, b in zip(ref, got):
                for f in ("sector", "x", "param", "cov", "chi2", "ndf", "hit_off", "hit_cid"):
                    assert np.array_equal(getattr(a, f), getattr(b, f)), (v, f)
        for bad in (dict(nb_threads=96), dict(sort_threads=128), dict(bin_blocks_per_sm=0),
                    dict(tl_blocks_per_sm=s0["tl_max_per_sm"] + 1), dict(nb_mode=-1)):
            with pytest.raises(tp.TpcError):
                tp.tpc_track_set_schedule(t.ctx, **{**s0, **bad})
        g, keep_x = tp.geometry_of(evs[0])
        cs = [tp.clusters_of(e.y, e.z, e.row, e.sector) for e in evs]
        tuned = tp.tpc_track_autotune(t.ctx, [c for c, _ in cs], g, float(evs[0].bz), reps=1)
        assert tuned["nb_threads"] in (64, 128, 256) and tuned["sort_threads"] in (256, 512)
        assert 1 <= tuned["tl_blocks_per_sm"] <= tuned["tl_max_per_sm"]
        assert tp.tpc_track_get_schedule(t.ctx) == tuned
        got = t.batch(evs)
        for a, b in zip(ref, got):
            for f in ("sector", "x", "param", "cov", "chi2", "ndf", "hit_off", "hit_cid"):
                assert np.array_equal(getattr(a, f), getattr(b, f)), ("tuned", f)


@pytest.mark.parametrize("which", ["central", "batch", "pileup"])
def test_kernel_modes_give_identical_results(tp, which):
    """The row-block neighbour finder (adjacent rows staged in shared memory)
    does the same arithmetic per hit as the thread-per-hit finder: every
    link, tracklet and track is bit-identical, on the central event, a batch
    of events of uneven multiplicity and the pile-up event (rows above the
    staging capacity read from global memory)."""
    if which == "central":
        evs = [synth.central_event()]
    elif which == "batch":
        evs = synth.batch_events(n_events=12, seed0=3000)
    else:
        evs = [synth.pileup_event()]
    cap = sum(e.n for e in evs) + 65536
    with tp.Tracker(cap, max_events_per_launch=len(evs)) as t:
        s0 = tp.tpc_track_get_schedule(t.ctx)
        res = {}
        for mode in (0, 1):
            tp.tpc_track_set_schedule(t.ctx, **{**s0, "nb_mode": mode})
            trs = t.batch(evs)
            dumps = []
            for k, e in enumerate(evs):
                d = tp.dump_tracklets(t.ctx, len(e.row_x), event=k)
                d["up"], d["dn"] = tp.dump_links(t.ctx, e.n, event=k)
                dumps.append(d)
            res[mode] = (trs, dumps, t.counters())
        for k in range(len(evs)):
            a, b = res[0][0][k], res[1][0][k]
            for f in ("sector", "x", "param", "cov", "chi2", "ndf", "hit_off", "hit_cid"):
                assert np.array_equal(getattr(a, f), getattr(b, f)), (which, k, f)
            da, db = res[0][1][k], res[1][1][k]
            for f in da:
                assert np.array_equal(da[f], db[f], equal_nan=True), (which, k, f)
        for c in ("n_valid_tracklets", "n_tracklet_hits", "n_tracks", "n_track_hits"):
            assert res[0][2][c] == res[1][2][c], c


def test_launches_on_several_streams_give_the_same_tracks(tp):
    """Direct launches spread over 3 streams (kernels of consecutive launches
    run concurrently): results come back oldest first and equal those of one
    stream; joining makes the context's stream wait for all of them; a launch
    discards only its own slot's uncollected results; the autotuner keeps
    the stream count in range."""
    import torch
    evs = synth.batch_events(n_events=7, seed0=4300)
    with tp.Tracker(2_000_000) as t1:
        ref = [t1.event(e) for e in evs]
    stream = torch.cuda.Stream()
    t = tp.Tracker(2_000_000, max_events_in_flight=3, cuda_stream=stream.cuda_stream)
    try:
        s0 = tp.tpc_track_get_schedule(t.ctx)
        assert s0["max_streams"] == 3 and s0["streams"] == 1
        with pytest.raises(tp.TpcError):
            tp.tpc_track_set_schedule(t.ctx, **{**s0, "streams": 4})
        tp.tpc_track_set_schedule(t.ctx, **{**s0, "streams": 3})
        g, keep_x = tp.geometry_of(evs[0])
        cs = [tp.clusters_of(e.y, e.z, e.row, e.sector) for e in evs]
        bz = float(evs[0].bz)

        def same(a, b, what):
            for f in ("sector", "x", "param", "cov", "chi2", "ndf", "hit_off", "hit_cid"):
                assert np.array_equal(getattr(a, f), getattr(b, f)), (what, f)
        # three in flight, collected oldest first while the next ones launch
        got = []
        for i, (c, _) in enumerate(cs):
            tp.tpc_track_launch(t.ctx, [c], g, bz)
            if i >= 2:
                got += tp.tpc_track_results(t.ctx, 1)
        got += tp.tpc_track_results(t.ctx, 1) + tp.tpc_track_results(t.ctx, 1)
        for k, (a, b) in enumerate(zip(ref, got)):
            same(a, b, k)
        with pytest.raises(tp.TpcError):
            tp.tpc_track_results(t.ctx, 1)  # nothing pending
        # launches 0..3: launch 3 reuses slot 0 and drops launch 0's results
        for c, _ in cs[:4]:
            tp.tpc_track_launch(t.ctx, [c], g, bz)
        tp.tpc_track_join(t.ctx)
        done = torch.cuda.Event()
        done.record(stream)
        done.synchronize()  # after the join: every launch has finished
        for k in (1, 2, 3):
            same(ref[k], tp.tpc_track_results(t.ctx, 1)[0], ("after join", k))
        # a two-event launch collected into room for one event: refused, and
        # the launch stays pending until collected with room for both
        tp.tpc_track_launch(t.ctx, [cs[1][0], cs[2][0]], g, bz)
        with pytest.raises(tp.TpcError) as err:
            tp.tpc_track_results(t.ctx, 1)
        assert err.value.code == tp.TPC_EINVAL
        two = tp.tpc_track_results(t.ctx, 2)
        same(ref[1], two[0], "two events, first")
        same(ref[2], two[1], "two events, second")
        # batch and single-event calls still work and drop nothing they need
        same(ref[5], t.event(evs[5]), "event")
        tuned = tp.tpc_track_autotune(t.ctx, [cs[6][0]], g, bz, reps=1)
        assert 1 <= tuned["streams"] <= 3
        same(ref[6], t.event(evs[6]), "tuned")
        # launches left in flight on several streams, then the served form on
        # the same context: every slot moves back to its own stream in order
        tp.tpc_track_set_schedule(t.ctx, **{**tuned, "streams": 3})
        for c, _ in cs[:3]:
            tp.tpc_track_launch(t.ctx, [c], g, bz)
        tks = [tp.tpc_track_submit(t.ctx, c, g, bz) for c, _ in cs]
        for k, tk in enumerate(tks):
            same(ref[k], tp.tpc_track_poll(t.ctx, tk, 60_000_000), ("served after launches", k))
            tp.tpc_track_release(t.ctx, tk)
    finally:
        t.close()


def test_served_mix_with_an_invalid_event_and_a_polling_thread(tp):
    """Tickets polled from another thread while events are submitted, up to
    four events per launch: every valid event's tracks equal a single call's,
    and the event with an invalid cluster fails its own ticket only."""
    import threading
    evs = synth.batch_events(n_events=7, seed0=3300)
    bad = 3
    ys = [e.y.copy() for e in evs]
    ys[bad][len(ys[bad]) // 2] = np.nan
    with tp.Tracker(2_000_000) as t:
        alone = {i: t.event(e) for i, e in enumerate(evs) if i != bad}
    s = tp.Tracker(4 * 2_000_000, max_events_in_flight=2, max_events_per_launch=4)
    try:
        keep, tickets, got, errors = [], [None] * len(evs), {}, []

        def poller():
            try:
                for i in range(len(evs)):
                    for _ in range(600000):
                        if tickets[i] is not None:
                            break
                        threading.Event().wait(0.0001)
                    try:
                        got[i] = tp.tpc_track_poll(s.ctx, tickets[i], 60_000_000)
                    except tp.TpcError as e:
                        got[i] = e
                    tp.tpc_track_release(s.ctx, tickets[i])
            except Exception as e:  # surfaced below
                errors.append(e)
        th = threading.Thread(target=poller)
        th.start()
        for i, e in enumerate(evs):
            g, kx = tp.geometry_of(e)
            c, k = tp.clusters_of(ys[i], e.z, e.row, e.sector)
            keep.append((g, kx, c, k))
            tickets[i] = tp.tpc_track_submit(s.ctx, c, g, float(e.bz))
        th.join(120)
        assert not th.is_alive() and not errors, errors
        assert isinstance(got[bad], tp.TpcError) and got[bad].code == tp.TPC_EINVAL
        for i, a in alone.items():
            b = got[i]
            assert b is not None and not isinstance(b, Exception), (i, b)
            for f in ("sector", "x", "param", "cov", "chi2", "ndf", "hit_off", "hit_cid"):
                assert np.array_equal(getattr(a, f), getattr(b, f)), (i, f)
    finally:
        s.close()


def test_batch_equals_single_events(tp, trk):
    evs = synth.batch_events(n_events=6)
    alone = [trk.event(e) for e in evs]
    batch = trk.batch(evs)
    for a, b in zip(alone, batch):
        for f in ("sector", "x", "param", "cov", "chi2", "ndf", "hit_off", "hit_cid"):
            assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_empty_and_tiny_events(tp, trk):
    e0 = synth.Event(np.zeros(0, np.float32), np.zeros(0, np.float32), np.zeros(0, np.uint16),
                     np.zeros(0, np.uint16), np.zeros(0, np.int32), synth.default_row_x(), 18, 1)
    assert trk.event(e0).n_tracks == 0
    e1 = synth.Event(np.array([1.0], np.float32), np.array([2.0], np.float32),
                     np.array([5], np.uint16), np.array([3], np.uint16), np.array([-1], np.int32),
                     synth.default_row_x(), 18, 1)
    assert trk.event(e1).n_tracks == 0
    # noise only: no track survives the selector
    rng = np.random.default_rng(9)
    n = 20000
    en = synth.Event(rng.uniform(-15, 15, n).astype(np.float32),
                     rng.uniform(-250, 250, n).astype(np.float32),
                     rng.integers(0, 159, n).astype(np.uint16), np.zeros(n, np.uint16),
                     np.full(n, -1, np.int32), synth.default_row_x(), 1, 0)
    trk.event(en)


def test_invalid_input_is_rejected(tp, trk):
    ev = synth.one_sector_event()
    for field, bad in (("row", 159), ("sector", 1), ("y", np.nan), ("z", np.inf)):
        e = synth.Event(ev.y.copy(), ev.z.copy(), ev.row.copy(), ev.sector.copy(), ev.label,
                        ev.row_x, ev.n_sectors_phi, ev.split_z)
        getattr(e, field)[17] = bad
        with pytest.raises(tp.TpcError) as ei:
            trk.event(e)
        assert ei.value.code == tp.TPC_EINVAL
    # the context stays usable
    assert trk.event(ev).n_tracks > 0


def test_bounded_wait_gives_up_and_the_context_stays_usable(tp, orc):
    """A look-back tile that never publishes (test hook) makes the tiles after
    it give up after a short poll limit: the launch fails with TPC_ETIMEOUT
    and no result, and the next launch on the same context, with the hook
    off, gives the oracle's tracks."""
    ev = synth.one_sector_event()  # 16,671 clusters: 9 tiles of 2048 sorted hits
    with tp.Tracker(200_000) as t:
        ok = t.event(ev)
        for stall in (0, 3):
            tp.tpc_track_set_debug_waits(t.ctx, 4096, stall)
            with pytest.raises(tp.TpcError) as ei:
                t.event(ev)
            assert ei.value.code == tp.TPC_ETIMEOUT, ei.value
        # the last tile has no successor: no wait, the launch completes
        tp.tpc_track_set_debug_waits(t.ctx, 4096, -1)
        with pytest.raises(tp.TpcError):
            tp.tpc_track_set_debug_waits(t.ctx, -1, -1)
        with pytest.raises(tp.TpcError):
            tp.tpc_track_set_debug_waits(t.ctx, 0, -2)
        tp.tpc_track_set_debug_waits(t.ctx, 0, -1)
        g, o, rep, trep = check_event(tp, t, ev, orc, what="after a timeout")
        for f in ("sector", "x", "param", "cov", "chi2", "ndf", "hit_off", "hit_cid"):
            assert np.array_equal(getattr(ok, f), getattr(g["tracks"], f)), f


def test_row_capacity_overflow_is_reported(tp, trk):
    n = 5000
    rng = np.random.default_rng(4)
    e = synth.Event(rng.uniform(-10, 10, n).astype(np.float32),
                    rng.uniform(0, 200, n).astype(np.float32), np.full(n, 40, np.uint16),
                    np.zeros(n, np.uint16), np.full(n, -1, np.int32), synth.default_row_x(), 18, 1)
    with pytest.raises(tp.TpcError) as ei:
        trk.event(e)
    assert ei.value.code == tp.TPC_ECAPACITY
    assert trk.event(synth.one_sector_event()).n_tracks > 0


def test_too_many_clusters_for_the_context(tp):
    t = tp.Tracker(1000)
    try:
        with pytest.raises(tp.TpcError) as ei:
            t.event(synth.one_sector_event())
        assert ei.value.code == tp.TPC_EINVAL
    finally:
        t.close()


def test_memory_budget_too_small_is_refused_before_allocating(tp):
    """A context whose arenas exceed mem_budget is refused with TPC_ENOMEM
    before any device allocation; the device stays usable."""
    with pytest.raises(tp.TpcError) as ei:
        tp.tpc_track_create(2_000_000, mem_budget=64 << 20)
    assert ei.value.code == tp.TPC_ENOMEM
    with tp.Tracker(200_000) as t:
        assert t.event(synth.one_sector_event(seed=1, n_tracks=20)).n_tracks > 0


def test_tuned_schedule_saved_and_loaded(tp, tmp_path):
    ev = synth.one_sector_event(seed=1)
    with tp.Tracker(200_000, max_events_in_flight=2) as a:
        g, kx = tp.geometry_of(ev)
        c, k = tp.clusters_of(ev.y, ev.z, ev.row, ev.sector)
        tuned = tp.tpc_track_autotune(a.ctx, [c], g, float(ev.bz), reps=1)
        tp.save_schedule(a.ctx, str(tmp_path / "s.json"))
        ref = a.event(ev)
    with tp.Tracker(200_000, max_events_in_flight=2) as b:
        assert tp.load_schedule(b.ctx, str(tmp_path / "s.json")) == tuned
        got = b.event(ev)
    for f in ("sector", "x", "param", "cov", "chi2", "ndf", "hit_off", "hit_cid"):
        assert np.array_equal(getattr(ref, f), getattr(got, f)), f


def test_high_water_marks(tp):
    """The counters' fullest (sector, row) and fullest sector: the first a
    count of the inputs, the second a count of the emitted tracks."""
    ev = synth.batch_events(2, seed0=3000)[1]
    with tp.Tracker(2_000_000) as t:
        tr = t.event(ev)
        c = t.counters()
    R = len(ev.row_x)
    assert c["max_row_hits"] == np.bincount(ev.sector.astype(np.int64) * R + ev.row).max()
    assert c["max_sector_tracks"] == np.bincount(tr.sector).max()
    assert c["max_row_hits"] <= 4096 and c["max_sector_tracks"] <= 4096


def test_served_results_equal_alone(tp):
    evs = synth.batch_events(n_events=8, seed0=3100)
    t = tp.Tracker(2_000_000, max_events_in_flight=2)
    try:
        alone = [t.event(e) for e in evs]
    finally:
        t.close()
    s = tp.Tracker(2_000_000, max_events_in_flight=2)
    try:
        keep = []
        tickets = []
        for e in evs:
            g, kx = tp.geometry_of(e)
            c, k = tp.clusters_of(e.y, e.z, e.row, e.sector)
            keep.append((g, kx, c, k))
            tickets.append(tp.tpc_track_submit(s.ctx, c, g, float(e.bz)))
        for a, tk in zip(alone, tickets):
            b = tp.tpc_track_poll(s.ctx, tk, 60_000_000)
            assert b is not None, "served ticket not done within 60 s"
            for f in ("sector", "x", "param", "cov", "chi2", "ndf", "hit_off", "hit_cid"):
                assert np.array_equal(getattr(a, f), getattr(b, f)), f
            tp.tpc_track_release(s.ctx, tk)
    finally:
        s.close()
