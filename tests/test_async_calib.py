"""The asynchronous side task (Sect. 3, item 4; Sect. 5.1) and its built-in
accumulate-then-fit task, on the host (no GPU is touched).

* The oracle's chi^2 scale fit is pinned to things other than itself: it
  recovers a known scale from chi^2 draws (law of large numbers), resists a
  fraction of gross outliers that moves the plain ratio, returns the largest
  self-consistent kept set found by brute force over all subsets, scales
  exactly with chi^2, and on oracle tracks of events smeared with 0.15 cm
  while the tracker assumes 0.1 cm it recovers the ratio 1.5 to within the
  hit-cut bias.
* The library's fit (run on its side thread) equals the oracle's on the same
  tracks.
* The runner: jobs run in start order on one thread, start never waits, the
  bound on unfinished jobs is kept, failures become statuses, destroy drops
  what never ran; an event loop with a long fit every n-th event keeps its
  per-event gaps short when the fit runs asynchronously (Fig. 5) and not when
  it runs inline (Fig. 4).
"""
import itertools
import time

import numpy as np
import pytest

from oracle.calib import chi2_scale_fit
from paper_1712_09416_b300 import synth


@pytest.fixture(scope="module")
def tp():
    from paper_1712_09416_b300 import build, tpctrack
    build.build()
    return tpctrack


def chi2_draws(rng, n, scale2, ndf_range=(20, 300)):
    ndf = rng.integers(*ndf_range, n)
    return scale2 * rng.chisquare(ndf), ndf


# --------------------------------------------------------------------------
# oracle pins
# --------------------------------------------------------------------------

def test_recovers_a_known_scale():
    rng = np.random.default_rng(1)
    for scale2 in (0.5, 1.0, 2.25):
        c, d = chi2_draws(rng, 20000, scale2)
        f = chi2_scale_fit(c, d)
        # relative standard error of the ratio: sqrt(2 / sum ndf) ~ 8e-4
        assert abs(f["scale2"] / scale2 - 1) < 5e-3, f
        assert f["n_kept"] == f["n_tracks"] == 20000


def test_gross_outliers_are_trimmed():
    rng = np.random.default_rng(2)
    c, d = chi2_draws(rng, 20000, 1.0)
    bad = rng.random(20000) < 0.05
    c = np.where(bad, 50.0 * d, c)
    f = chi2_scale_fit(c, d)
    assert abs(f["scale2"] - 1) < 0.01, f
    assert f["n_kept"] == int((~bad).sum())
    assert c.sum() / d.sum() > 2.0  # the untrimmed ratio is far off


def test_kept_set_is_the_largest_self_consistent_one():
    """Brute force over all subsets of tiny runs: a kept set K is
    self-consistent if K = {i : chi2_i <= trim * ratio(K) * ndf_i}."""
    rng = np.random.default_rng(3)
    for trial in range(200):
        n = int(rng.integers(1, 9))
        d = rng.integers(1, 6, n).astype(np.float64)
        c = d * rng.lognormal(0.0, 1.2, n)
        trim = float(rng.choice([1.5, 2.0, 3.0]))
        f = chi2_scale_fit(c, d, trim)
        best = None
        for mask in itertools.product([False, True], repeat=n):
            K = np.array(mask)
            if not K.any():
                continue
            r = c[K].sum() / d[K].sum()
            if np.array_equal(c <= trim * r * d, K) and (best is None or K.sum() > best[0].sum()):
                best = (K, r)
        assert best is not None
        assert f["n_kept"] == best[0].sum(), (trial, f, best)
        assert f["scale2"] == pytest.approx(best[1], rel=1e-12)


def test_scale_and_order_invariance():
    rng = np.random.default_rng(4)
    c, d = chi2_draws(rng, 500, 1.3)
    c[:20] *= 30
    f = chi2_scale_fit(c, d)
    g = chi2_scale_fit(7.0 * c, d)
    assert g["scale2"] == pytest.approx(7.0 * f["scale2"], rel=1e-13)
    assert g["n_kept"] == f["n_kept"]
    p = rng.permutation(500)
    h = chi2_scale_fit(c[p], d[p])
    assert h["scale2"] == pytest.approx(f["scale2"], rel=1e-13) and h["n_kept"] == f["n_kept"]


def test_degenerate_runs():
    assert np.isnan(chi2_scale_fit([], [])["scale2"])
    f = chi2_scale_fit([3.0, 5.0], [0, -1])
    assert np.isnan(f["scale2"]) and f["n_tracks"] == 0
    f = chi2_scale_fit([3.0, 4.0, 9.0], [0, 4, 0])  # only ndf > 0 counts
    assert f["scale2"] == 1.0 and f["n_tracks"] == 1


def test_oracle_tracks_recover_the_cluster_error_ratio(orc):
    """Events smeared with sigma_true, tracked by the oracle assuming 0.1 cm:
    sqrt(scale2) estimates sigma_true / 0.1 (slightly low, because the hit
    chi^2 cut of the fit drops the widest residuals)."""
    for sig, lo, hi in ((0.1, 0.97, 1.03), (0.15, 1.40, 1.52)):
        ev = synth.one_sector_event(seed=7, n_tracks=400, sigma=sig)
        o = orc.track_event(ev)
        f = chi2_scale_fit(o["k_chi2"], o["k_ndf"])
        assert f["n_tracks"] > 200
        assert lo < np.sqrt(f["scale2"]) < hi, (sig, f)


# --------------------------------------------------------------------------
# the library's fit and runner
# --------------------------------------------------------------------------

def test_native_fit_equals_the_oracle(tp):
    rng = np.random.default_rng(5)
    cal = tp.Chi2Calib(every_n_events=3, trim=3.0, max_unfinished=64)
    try:
        events = []
        for k in range(12):
            n = int(rng.integers(0, 400))
            c, d = chi2_draws(rng, n, 1.7, (1, 200))
            c[: n // 20] *= 40  # outliers
            d[: n // 50] = 0    # tracks without degrees of freedom
            c32, d32 = c.astype(np.float32), d.astype(np.int32)
            ver = 0 if k < 7 else 1  # a parameter change after event 6
            events.append((c32, d32, ver))
            cal.add(c32, d32, ver)
        fits = []
        while (f := cal.poll(-1)) is not None:
            fits.append(f)
        # events 0-2, 3-5 (version 0); event 6 dropped by the change; 7-9 (version 1)
        assert [(f["first_event"], f["last_event"], f["params_version"]) for f in fits] == \
            [(0, 2, 0), (3, 5, 0), (7, 9, 1)]
        for f in fits:
            sel = events[f["first_event"]: f["last_event"] + 1]
            o = chi2_scale_fit(np.concatenate([e[0] for e in sel]).astype(np.float64),
                               np.concatenate([e[1] for e in sel]))
            assert f["n_events"] == len(sel)
            assert f["n_tracks"] == o["n_tracks"] and f["n_kept"] == o["n_kept"]
            assert f["n_iter"] == o["n_iter"]
            assert f["scale2"] == pytest.approx(o["scale2"], rel=1e-12)
        st = cal.stats()
        assert st["started"] == st["finished"] == 3 and st["queued"] == 0
    finally:
        cal.close()


def test_runner_order_bound_and_failures(tp):
    order = []
    r = tp.AsyncRunner(max_unfinished=2)
    try:
        t1 = r.start(lambda: (time.sleep(0.2), order.append(1), "a")[2])
        t2 = r.start(lambda: (order.append(2), "b")[1])
        assert r.start(lambda: "never") is None  # two unfinished: refused, not queued
        assert r.poll(0) is None                 # the first job is still running
        a = r.poll(-1)
        b = r.poll(-1)
        assert (a[0], a[1], a[2]) == (t1, tp.TPC_OK, "a")
        assert (b[0], b[1], b[2]) == (t2, tp.TPC_OK, "b")
        assert order == [1, 2]
        assert r.poll(-1) is None                # idle: a wait forever returns at once

        def boom():
            raise ValueError("fit failed")
        t3 = r.start(boom)
        tid, st, val = r.poll(-1)
        assert tid == t3 and st == tp.TPC_EINVAL and isinstance(val, ValueError)
        s = r.stats()
        assert s["started"] == 3 and s["finished"] == 3 and s["refused"] == 1
        assert s["max_task_ms"] >= 150
    finally:
        r.close()


def test_init_runs_on_the_thread_and_its_failure_is_returned(tp):
    import threading
    seen = []
    r = tp.AsyncRunner(init=lambda: (seen.append(threading.get_ident()), 0)[1])
    try:
        assert seen and seen[0] != threading.get_ident()
    finally:
        r.close()
    with pytest.raises(tp.TpcError) as e:
        tp.AsyncRunner(init=lambda: tp.TPC_ENOMEM)
    assert e.value.code == tp.TPC_ENOMEM


def test_destroy_drops_queued_jobs_and_unpolled_results(tp):
    r = tp.AsyncRunner(max_unfinished=4)
    r.start(lambda: time.sleep(0.2))
    r.start(lambda: "queued 1")
    r.start(lambda: "queued 2")
    r.close()  # lets the running job finish; the queued ones never run
    assert r._jobs == {} and r._results == {}


def _event_loop(tp, n_events, fit_every, fit_s, asynchronous):
    """Per-event gaps of a loop that spends 1 ms per event and starts a fit of
    fit_s seconds every fit_every events (inline or on the runner)."""
    r = tp.AsyncRunner(max_unfinished=2) if asynchronous else None
    gaps, t_prev, fits = [], time.perf_counter(), 0
    try:
        for k in range(n_events):
            time.sleep(0.001)  # the event's own processing
            if k % fit_every == fit_every - 1:
                if asynchronous:
                    r.start(lambda: time.sleep(fit_s))
                else:
                    time.sleep(fit_s)
                    fits += 1
            if asynchronous and r.poll(0) is not None:
                fits += 1
            now = time.perf_counter()
            gaps.append(now - t_prev)
            t_prev = now
        if asynchronous:
            while r.poll(-1) is not None:
                fits += 1
    finally:
        if r:
            r.close()
    return np.array(gaps), fits


def test_long_fit_does_not_stall_the_event_loop(tp):
    # a fit of 80 ms every 100 events of about 1 ms: shorter than its period
    g_inline, f_inline = _event_loop(tp, 300, 100, 0.08, asynchronous=False)
    g_async, f_async = _event_loop(tp, 300, 100, 0.08, asynchronous=True)
    assert f_inline == f_async == 3
    assert g_inline.max() > 0.08
    assert g_async.max() < 0.04, g_async.max()
