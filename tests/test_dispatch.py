"""Round-robin dispatcher of whole events over tracker instances (paper
Sect. 2: several instances of a component take events in turn).

CPU tests drive the dispatcher of libtpctrack.so through fake instances:
each instance is a host object that "tracks" an event by returning one track
per cluster-count unit it was given, on worker threads of its own, so that
order, round robin, gathering and the re-issue of a failed instance's events
are checked without a GPU.  The GPU test runs two tracker contexts on the one
device and compares every event with a single context's tracks.
"""
import ctypes as C
import threading

import numpy as np
import pytest

from paper_1712_09416_b300 import synth


@pytest.fixture(scope="module")
def tp():
    from paper_1712_09416_b300 import build, tpctrack
    build.build()
    return tpctrack


class FakeInstance:
    """One instance: submit queues the event, a thread 'tracks' it (the
    result records the event size and this instance's id); poll waits for
    it.  fail_at: the poll of this instance's fail_at-th ticket and every
    later call fail with TPC_ECUDA, as a lost device would."""

    def __init__(self, tp, ident, fail_at=None):
        self.tp, self.ident, self.fail_at = tp, ident, fail_at
        self.lock = threading.Lock()
        self.done = {}
        self.next = 1
        self.failed = False
        self.seen = []
        self.bufs = {}

    def submit(self, clusters, geom, bz, ticket_p):
        with self.lock:
            if self.failed:
                return self.tp.TPC_ECUDA
            t = self.next
            self.next += 1
            self.seen.append(int(clusters.contents.n))
        n = int(clusters.contents.n)
        # result: n_tracks = n % 7 + 1 tracks, hit cid i of track j = j, sector = instance id
        k = n % 7 + 1
        arrs = {"sector": np.full(k, self.ident, np.int32), "x": np.zeros(k, np.float32),
                "param": np.zeros(5 * k, np.float32), "cov": np.zeros(15 * k, np.float32),
                "chi2": np.full(k, float(n), np.float32), "ndf": np.zeros(k, np.int32),
                "hit_off": np.arange(k + 1, dtype=np.int32), "hit_cid": np.arange(k, dtype=np.int32)}
        with self.lock:
            self.bufs[t] = arrs
            self.done[t] = threading.Event()
        threading.Timer(0.002, self.done[t].set).start()
        ticket_p[0] = t
        return self.tp.TPC_OK

    def poll(self, ticket, timeout_us, out):
        with self.lock:
            if self.failed or (self.fail_at is not None and ticket >= self.fail_at):
                self.failed = True
                return self.tp.TPC_ECUDA
            ev = self.done.get(ticket)
        if ev is None:
            return self.tp.TPC_EINVAL
        if not ev.wait(None if timeout_us < 0 else timeout_us * 1e-6):
            return self.tp.TPC_EBUSY
        a = self.bufs[ticket]
        o = out.contents
        o.n_tracks = len(a["sector"])
        for f in ("sector", "ndf", "hit_off", "hit_cid"):
            setattr(o, f, a[f].ctypes.data_as(C.POINTER(C.c_int32)))
        for f in ("x", "param", "cov", "chi2"):
            setattr(o, f, a[f].ctypes.data_as(C.POINTER(C.c_float)))
        return self.tp.TPC_OK

    def release(self, ticket):
        with self.lock:
            if ticket not in self.bufs:
                return self.tp.TPC_EINVAL
            del self.bufs[ticket]
        return self.tp.TPC_OK


def make(tp, insts):
    byid = {id(i): i for i in insts}
    ops = (lambda h, c, g, bz, t: byid[h].submit(c, g, bz, t),
           lambda h, t, to, o: byid[h].poll(t, to, o),
           lambda h, t: byid[h].release(t))
    return tp.Dispatcher(ops=ops, instances=[id(i) for i in insts])


def events(tp, sizes):
    ev = synth.one_sector_event()
    g, keep_x = tp.geometry_of(ev)
    cs = [tp.clusters_of(ev.y[:n], ev.z[:n], ev.row[:n], ev.sector[:n]) for n in sizes]
    return g, keep_x, cs


def test_round_robin_order_and_gather(tp):
    insts = [FakeInstance(tp, k) for k in range(3)]
    sizes = [10 + 3 * i for i in range(12)]
    g, kx, cs = events(tp, sizes)
    with make(tp, insts) as d:
        tks = [d.submit(c, g, 0.5) for c, _ in cs]
        assert tks == list(range(1, 13))
        # gathered in submission order, whichever instance ran each event
        for i, t in enumerate(tks):
            tr = d.poll(t)
            assert tr.n_tracks == sizes[i] % 7 + 1 and tr.chi2[0] == sizes[i]
            assert tr.sector[0] == i % 3  # event i went to instance i mod 3
            d.release(t)
        st = d.stats()
        assert st["events"] == [4, 4, 4] and st["healthy"] == [True] * 3 and st["reissued"] == 0
    for k, inst in enumerate(insts):
        assert inst.seen == sizes[k::3]


def test_failed_instance_events_are_reissued(tp):
    """Instance 1 fails at the poll of its second ticket (a rank lost in the
    middle of the stream): it leaves the rotation, every event it held is
    tracked by the others, and no ticket is lost or reordered."""
    insts = [FakeInstance(tp, 0), FakeInstance(tp, 1, fail_at=2), FakeInstance(tp, 2)]
    sizes = [20 + i for i in range(15)]
    g, kx, cs = events(tp, sizes)
    with make(tp, insts) as d:
        tks = [d.submit(c, g, 0.5) for c, _ in cs]
        got = [d.poll(t) for t in tks]
        for i, tr in enumerate(got):
            assert tr.chi2[0] == sizes[i], i
            if i % 3 == 1 and i >= 4:  # held by instance 1 after its first ticket
                assert tr.sector[0] in (0, 2)
        st = d.stats()
        assert st["healthy"] == [True, False, True]
        assert st["reissued"] == 4  # instance 1's tickets 2..5 (events 4, 7, 10, 13)
        # later events skip the failed instance
        c, _ = cs[0]
        t = d.submit(c, g, 0.5)
        assert d.poll(t).sector[0] in (0, 2)


def test_injected_failure_and_no_healthy_instance(tp):
    insts = [FakeInstance(tp, 0), FakeInstance(tp, 1)]
    g, kx, cs = events(tp, [30, 31, 32, 33])
    with make(tp, insts) as d:
        tks = [d.submit(c, g, 0.5) for c, _ in cs]
        d.fail_instance(0)  # host-side fault injection: drain instance 0
        assert [d.poll(t).sector[0] for t in tks] == [1, 1, 1, 1]
        assert d.stats()["reissued"] == 2
        d.fail_instance(1)
        with pytest.raises(tp.TpcError) as ei:
            d.submit(cs[0][0], g, 0.5)
        assert ei.value.code == tp.TPC_ECUDA
        with pytest.raises(tp.TpcError):
            d.fail_instance(5)


def test_invalid_instances_are_refused(tp):
    with pytest.raises(tp.TpcError):
        tp.Dispatcher(ops=(lambda *a: 0, lambda *a: 0, lambda *a: 0), instances=[])


@pytest.mark.gpu
def test_two_contexts_on_one_gpu_give_single_context_tracks(tp):
    """Two tracker contexts on device 0 behind the dispatcher (the layout of
    one context per GPU, on the one GPU available): every event equals a
    single context's tracks, also after one instance is drained mid-stream."""
    import torch
    assert torch.cuda.is_available()
    evs = synth.batch_events(n_events=8, seed0=4400)
    with tp.Tracker(2_000_000) as t:
        ref = [t.event(e) for e in evs]
    g, kx = tp.geometry_of(evs[0])
    cs = [tp.clusters_of(e.y, e.z, e.row, e.sector) for e in evs]
    with tp.Dispatcher([0, 0], 2_000_000, max_events_in_flight=2) as d:
        tks = [d.submit(c, g, float(evs[0].bz)) for c, _ in cs[:5]]
        d.fail_instance(1)
        tks += [d.submit(c, g, float(evs[0].bz)) for c, _ in cs[5:]]
        for k, tk in enumerate(tks):
            b = d.poll(tk, 60_000_000)
            for f in ("sector", "x", "param", "cov", "chi2", "ndf", "hit_off", "hit_cid"):
                assert np.array_equal(getattr(ref[k], f), getattr(b, f)), (k, f)
            d.release(tk)
        st = d.stats()
        assert st["healthy"] == [True, False] and st["events"][0] >= 6
