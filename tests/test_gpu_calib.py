"""Event-synchronous parameter updates of the served tracker and the
calibration feedback loop (Sect. 3, items 2-4; Sect. 5.1-5.3), on the GPU.

* Events submitted before tpc_track_set_params are tracked with the old set,
  events after it with the new one, and each ticket reports the set it was
  tracked with; the tracks of both kinds agree with the oracle run with that
  ticket's set.
* A served stream of events smeared with 0.15 cm, tracked assuming 0.1 cm,
  feeds the built-in chi^2 scale fit on its side thread; every finished fit
  is fed back as a new cluster error.  Each fit equals the oracle's fit of the
  same GPU tracks, and the cluster error converges to the smearing (minus
  the hit-cut bias).
"""
import numpy as np
import pytest

from oracle.calib import chi2_scale_fit
from paper_1712_09416_b300 import synth
from tests import _parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1712_09416_b300 import build, tpctrack
    build.build()
    return tpctrack


def events(seed, n, n_tracks, sigma):
    rng = np.random.default_rng(seed)
    return [synth.make_event(rng, synth.draw_particles(rng, n_tracks), n_sectors_phi=synth.N_PHI_FULL,
                             split_z=True, sigma=sigma) for _ in range(n)]


def oracle_params(orc, p):
    """The oracle's parameter record for a library parameter set (binary32
    values carried over exactly)."""
    q = orc.Params()
    q.sigma_y, q.sigma_z = float(p.meas_sigma_y), float(p.meas_sigma_z)
    for f in ("slope_win_y", "slope_win_z", "d_max", "chi2_hit", "max_gap", "min_chain",
              "min_tracklet_hits", "min_track_hits", "sin_max", "edge_margin", "seed_var_s",
              "seed_var_t", "seed_var_q"):
        setattr(q, f, getattr(p, f))
    return q


def check_vs_oracle(tr, ev, orc, params):
    o = orc.track_event(ev, oracle_params(orc, params))
    rep = _parity.compare_tracks(tr, o, _parity.tainted_hits(o))
    assert rep["missing"] == [] and rep["extra"] == []
    assert rep["order_ok"] and "meta_mismatch" not in rep
    _parity.check_param_bars(rep["param_scaled"], "tracks")
    return o


def submit(tp, ctx, ev, keep):
    g, kx = tp.geometry_of(ev)
    c, k = tp.clusters_of(ev.y, ev.z, ev.row, ev.sector)
    keep.append((g, kx, c, k))
    return tp.tpc_track_submit(ctx, c, g, float(ev.bz))


def test_parameter_update_applies_from_its_first_ticket(tp, orc):
    evs = events(4100, 10, 300, 0.1)
    t = tp.Tracker(2_000_000, max_events_in_flight=2)
    try:
        a, v0 = tp.tpc_track_get_params(t.ctx)
        assert v0 == 0
        b = tp.tpc_track_default_params()
        b.min_track_hits, b.chi2_hit, b.meas_sigma_y = 40, 9.0, 0.12
        keep, tickets = [], []
        for e in evs[:5]:
            tickets.append(submit(tp, t.ctx, e, keep))
        first, ver = tp.tpc_track_set_params(t.ctx, b)
        assert (first, ver) == (tickets[-1] + 1, 1)
        bad = tp.tpc_track_default_params()
        bad.sin_max = 1.5
        with pytest.raises(tp.TpcError):
            tp.tpc_track_set_params(t.ctx, bad)  # rejected: the set stays b
        for e in evs[5:]:
            tickets.append(submit(tp, t.ctx, e, keep))
        assert tickets[5] == first
        n_a, n_b, served5 = [], [], None
        for k, (e, tk) in enumerate(zip(evs, tickets)):
            tr = tp.tpc_track_poll(t.ctx, tk, 60_000_000)
            assert tr is not None
            p, v = tp.tpc_track_ticket_params(t.ctx, tk)
            assert v == (0 if k < 5 else 1)
            assert p.min_track_hits == (10 if k < 5 else 40)
            if k in (0, 4, 5, 9):
                check_vs_oracle(tr, e, orc, p)
            (n_a if k < 5 else n_b).append(tr.n_tracks)
            if k == 5:
                served5 = tr
            tp.tpc_track_release(t.ctx, tk)
        assert min(n_a) > max(n_b)  # the stricter set is visible in every event
    finally:
        t.close()
    # a direct call after the same update gives the served ticket's tracks
    d = tp.Tracker(2_000_000)
    try:
        tp.tpc_track_set_params(d.ctx, b)
        tr = d.event(evs[5])
        for f in ("sector", "x", "param", "cov", "chi2", "ndf", "hit_off", "hit_cid"):
            assert np.array_equal(getattr(tr, f), getattr(served5, f)), f
    finally:
        d.close()


def test_calibration_feedback_loop(tp, orc):
    evs = events(4200, 18, 500, 0.15)
    t = tp.Tracker(2_000_000, max_events_in_flight=2)
    cal = tp.Chi2Calib(every_n_events=3, trim=3.0, max_unfinished=2)
    try:
        keep, added, applied = [], [], []
        sigma_of = {0: float(tp.tpc_track_get_params(t.ctx)[0].meas_sigma_y)}

        def feed_back(f):
            s = np.float32(sigma_of[f["params_version"]] * np.sqrt(f["scale2"]))
            p = tp.tpc_track_default_params()
            p.meas_sigma_y = p.meas_sigma_z = float(s)
            first, ver = tp.tpc_track_set_params(t.ctx, p)
            sigma_of[ver] = float(p.meas_sigma_y)
            applied.append((f, first, ver))

        last = None
        for k, e in enumerate(evs):
            tk = submit(tp, t.ctx, e, keep)
            tr = tp.tpc_track_poll(t.ctx, tk, 60_000_000)
            assert tr is not None
            p, ver = tp.tpc_track_ticket_params(t.ctx, tk)
            assert float(p.meas_sigma_y) == sigma_of[ver]
            cal.add(tr.chi2, tr.ndf, ver)
            added.append((tr.chi2.copy(), tr.ndf.copy(), ver))
            if (f := cal.poll(0)) is not None:  # checked at every event, never waited for
                feed_back(f)
            last = (tr, e, p)
            tp.tpc_track_release(t.ctx, tk)
        while (f := cal.poll(-1)) is not None:
            applied.append((f, None, None))
        fits = [a[0] for a in applied]
        assert len(fits) >= 3
        for f in fits:
            sel = added[f["first_event"]: f["last_event"] + 1]
            assert {s[2] for s in sel} == {f["params_version"]}
            o = chi2_scale_fit(np.concatenate([s[0] for s in sel]).astype(np.float64),
                               np.concatenate([s[1] for s in sel]))
            assert f["n_tracks"] == o["n_tracks"] and f["n_kept"] == o["n_kept"]
            assert f["scale2"] == pytest.approx(o["scale2"], rel=1e-12)
        # the first fit sees the full mis-calibration, the last one little of it
        assert 1.35 < np.sqrt(fits[0]["scale2"]) < 1.55, fits[0]
        assert abs(np.sqrt(fits[-1]["scale2"]) - 1.0) < 0.05, fits[-1]
        final = max(sigma_of.items())[1]
        assert 0.138 < final < 0.156, sigma_of
        # the last event, tracked with a fed-back set, agrees with the oracle
        tr, e, p = last
        assert p.meas_sigma_y != np.float32(0.1)
        check_vs_oracle(tr, e, orc, p)
    finally:
        cal.close()
        t.close()
