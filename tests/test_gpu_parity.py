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


def run(tp, trk, ev):
    tr = trk.event(ev)
    n = ev.n
    up, dn = tp.dump_links(trk.ctx, n)
    upc, dnc = tp.dump_links(trk.ctx, n, clean=True)
    return {"tracks": tr, "up": up, "dn": dn, "up_c": upc, "dn_c": dnc,
            "starts": tp.dump_starts(trk.ctx),
            "tracklets": tp.dump_tracklets(trk.ctx, len(ev.row_x)),
            "weights": tp.dump_weights(trk.ctx), "counters": trk.counters()}


def check_event(tp, trk, ev, orc, *, max_diff_frac=1e-3):
    g = run(tp, trk, ev)
    o = orc.track_event(ev)
    assert len(_parity.compare_links(g["up"], g["dn"], o["up"], o["dn"])) == 0
    assert len(_parity.compare_links(g["up_c"], g["dn_c"], o["up_c"], o["dn_c"])) == 0
    o_starts = np.sort(np.nonzero((o["up_c"] >= 0) & (o["dn_c"] < 0))[0])
    assert np.array_equal(g["starts"], o_starts)
    rep = _parity.compare_tracklets(g["tracklets"], o, len(ev.row_x))
    assert rep["missing"] == [] and rep["extra"] == []
    assert len(rep["flagged_diff"]) <= max_diff_frac * max(1, rep["n_oracle"]), rep["flagged_diff"]
    assert rep["valid_mismatch"] == [], rep["valid_mismatch"][:10]
    assert rep["hitset_mismatch"] == [], rep["hitset_mismatch"][:10]
    _parity.check_param_bars(rep["param_scaled"], "tracklets")
    trep = _parity.compare_tracks(g["tracks"], o, rep["taint"])
    assert trep["missing"] == [] and trep["extra"] == []
    assert trep["order_ok"]
    assert "meta_mismatch" not in trep
    _parity.check_param_bars(trep["param_scaled"], "tracks")
    c = g["counters"]
    assert c["n_starts"] == o["n_starts"]
    assert c["n_tracklets"] == o["n_tracklets"]
    assert c["n_links"] == o["n_links"]
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


def check_sampled_sectors(tr, ev, orc, sample):
    """GPU tracks of the whole event against the oracle run on single sectors
    (sectors are independent): same untainted hit sets, parameters within
    the bars.  Returns the oracle output per sampled sector."""
    outs = {}
    scaled = []
    for s in sample:
        sub = ev.select_sectors([s])
        o = orc.track_event(sub)
        outs[s] = (sub, o)
        parent = sub.info["parent_index"]
        m = np.nonzero(tr.sector == s)[0]
        # GPU tracks of this sector, hits mapped to the sub-event's cids
        inv = {int(c): i for i, c in enumerate(parent)}
        g_hits = [tuple(inv[int(c)] for c in tr.hits(j)) for j in m]
        o_hits = [tuple(o["k_hit_cid"][o["k_hit_off"][j]:o["k_hit_off"][j + 1]].tolist())
                  for j in range(o["n_tracks"])]
        taint = _parity.tainted_hits(o)
        oc = [h for h in o_hits if not set(h) & taint]
        gc = [h for h in g_hits if not set(h) & taint]
        assert set(oc) <= set(g_hits), s
        assert set(gc) <= set(o_hits), s
        pos = {h: k for k, h in enumerate(g_hits)}
        for h in oc:
            j = m[pos[h]]
            oj = o_hits.index(h)
            _, sc = _parity.param_errors(tr.param[j], o["k_p"][oj])
            scaled.append(sc)
    _parity.check_param_bars(scaled, "sampled-sector tracks")
    return outs


def test_central_event_sampled_sectors(tp, trk, orc):
    """Full-size central event on the GPU; six of its sectors against the oracle."""
    ev = synth.central_event()
    tr = trk.event(ev)
    check_sampled_sectors(tr, ev, orc, [0, 7, 13, 20, 28, 35])


def test_pileup_event_sampled_sectors(tp, orc):
    """Pile-up stress event (50 collisions, vertex z within +-200 cm, about
    7.4M clusters) in one launch; two sectors against the oracle, and the
    Monte-Carlo efficiency and fake rate of the GPU tracks on those sectors
    equal the oracle's up to the tracks that touch near-tie hits."""
    ev = synth.pileup_event()
    with tp.Tracker(ev.n + 65536) as t:
        tr = t.event(ev)
        c = t.counters()
    assert c["n_clusters"] == ev.n and c["n_tracks"] > 0
    sample = [3, 26]
    outs = check_sampled_sectors(tr, ev, orc, sample)
    for s in sample:
        sub, o = outs[s]
        m = np.nonzero(tr.sector == s)[0]
        parent = sub.info["parent_index"]
        inv = np.full(ev.n, -1, np.int64)
        inv[parent] = np.arange(len(parent))
        g_sub = {"n_tracks": len(m), "k_sector": np.full(len(m), s),
                 "k_hit_off": np.concatenate([[0], np.cumsum([len(tr.hits(j)) for j in m])]),
                 "k_hit_cid": np.concatenate([inv[tr.hits(j)] for j in m]) if len(m) else
                 np.zeros(0, np.int64)}
        o_sub = dict(o)
        o_sub["k_sector"] = np.full(o["n_tracks"], s)
        mg = _util.mc_summary(sub, g_sub)
        mo = _util.mc_summary(sub, o_sub)
        tol = len(_parity.tainted_hits(o)) + 2
        assert abs(mg["n_reco"] - mo["n_reco"]) <= tol, (mg, mo)
        assert abs(mg["fakes"] - mo["fakes"]) <= tol, (mg, mo)
        assert abs(mg["eff"] - mo["eff"]) * max(1, mg["n_reconstructable"]) <= tol, (mg, mo)
        print("pile-up sector", s, "gpu", mg, "oracle", mo)


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
                    dict(tl_blocks_per_sm=1), dict(tl_blocks_per_sm=max(1, s0["tl_max_per_sm"] // 2))]
        for v in variants:
            tp.tpc_track_set_schedule(t.ctx, **{**s0, **v})
            got = t.batch(evs)
            for a, b in zip(ref, got):
                for f in ("sector", "x", "param", "cov", "chi2", "ndf", "hit_off", "hit_cid"):
                    assert np.array_equal(getattr(a, f), getattr(b, f)), (v, f)
        for bad in (dict(nb_threads=96), dict(sort_threads=128), dict(bin_blocks_per_sm=0),
                    dict(tl_blocks_per_sm=s0["tl_max_per_sm"] + 1)):
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
