#!/usr/bin/env python
"""Benchmark of the B300 TPC sector tracker (one JSON line on stdout).

Workload: the central heavy-ion-like event (10,000 primary helices plus 1,000
secondaries plus 5% noise, 36 sectors x 159 pad rows, 0.5 T, seed 2, about
1.73M binary32 clusters).  One step = the whole tracking path (binning,
neighbours, cleaning, start hits, tracklet construction, selection) over one
launch of E such events side by side (E picked from 1-16 by a timed burst),
inputs resident in HBM.  Sixteen device copies of the event are used in turn,
so that the events of one launch are distinct and the inputs of consecutive
steps exceed the 126 MB L2.

Also measured: the same metric end to end through the C ABI with pinned host
buffers (host->device copy of the clusters and device->host copy of the
tracks inside the timed region), per-kernel device times (CUDA events on the
launch stream) for the roofline of the dominant kernel, served (continuous
batching) versus one-event-at-a-time latency under Poisson arrivals, SM
clocks during the timed region, and the CPU oracle on a bounded sample.

--impl reference times the CPU oracle (the plain FP64 statement of the
method) on the same workload and metric, each step a bounded sample of sectors.
Multi-GPU (torchrun): independent replicas, one event stream per GPU, no
collective on the data path; value = clusters of all ranks / slowest rank.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "clusters/s & central-event p50/p99 latency, served vs one-event, 1 B300"
UNIT = "clusters/s"
WORKLOAD = ("central event: 10,000 primaries + 1,000 secondaries + 5% noise, 36 sectors x "
            "159 rows (85-247 cm), |z| < 250 cm, 0.5 T, seed 2")
N_COPIES = 16


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def replica_time(ms_local: float, world: int) -> float:
    """The job's time over replicas: the max over ranks of each rank's time,
    through the initialised process group (a CUDA tensor under nccl, a host
    tensor under gloo)."""
    if world <= 1:
        return ms_local
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, ms_total: float) -> float:
    """Whole-job units per second: every rank's units over the max time."""
    return world * units_per_rank / (ms_total * 1e-3)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# --------------------------------------------------------------------------
# algorithmic bytes per kernel launch (one read or write of each array the
# method needs; reuse of a neighbour's data is not counted)
# --------------------------------------------------------------------------

# Algorithmic bytes per cluster of each step of the method (each stage's
# arrays read or written once, the brute-force pair search not counted; f_a,
# the share of clusters on a tracklet, taken as 0.9): a1 binning 40, a2
# neighbours 14, a3 cleaner 12, a4 start hits 4, a5 tracklet construction 43,
# a6 selector 15; 128 in all.  Each kernel gets the part of its stage that it
# moves: a1 histogram read 12 (k_count), scan 4 (k_rowscan), scatter read 12
# + write 12 (k_scatter); a5 chain links 2 f_a (k_chains), y z 8 and rowhit 4
# per hit forward (k_constructor_fwd), y z 8 per hit and the header 0.7
# backward (k_constructor_bwd), weight init 8 and read-modify-write 16 per
# hit (k_weights); a6 rowhit 4 and weight 8 per hit (k_sel_decide), header
# 0.7 (k_sel_sort), hit cids out 4 per hit (k_sel_write).  Kernels that the
# method's byte model has no part for (the in-row sort, the dominance check)
# get 0.  kernel_bytes() below counts what this implementation's kernels
# move, reported beside them.
F_A = 0.9
STAGE_BYTES = {"a1": 40, "a2": 14, "a3": 12, "a4": 4, "a5": 43, "a6": 15}
PATH_BYTES = sum(STAGE_BYTES.values())
KERNEL_STAGE = {"k_count": "a1", "k_rowscan": "a1", "k_scatter": "a1", "k_rowsort": "a1",
                "k_rowsort_big": "a1", "k_rowsort_big4k": "a1", "k_neighbours": "a2",
                "k_neighbours_crowded": "a2", "k_clean_starts": "a3+a4",
                "k_chains": "a5", "k_constructor_fwd": "a5", "k_dominance": "a5",
                "k_constructor_bwd": "a5", "k_weights": "a5",
                "k_sel_decide": "a6", "k_sel_sort": "a6", "k_sel_write": "a6"}
KERNEL_BYTES = {"k_count": 12, "k_rowscan": 4, "k_scatter": 24, "k_rowsort": 0,
                "k_rowsort_big": 0, "k_rowsort_big4k": 0, "k_neighbours": 14,
                "k_neighbours_crowded": 0, "k_clean_starts": 16,
                "k_chains": 2 * F_A, "k_constructor_fwd": 12 * F_A, "k_dominance": 0,
                "k_constructor_bwd": 8.7 * F_A, "k_weights": 8 + 16 * F_A,
                "k_sel_decide": 12 * F_A, "k_sel_sort": 0.7, "k_sel_write": 4 * F_A}
ROOFLINE_TARGET = 0.40  # share of the HBM roofline asked of the path
EPL_CANDIDATES = (1, 2, 4, 8, 16)  # central events per launch tried for the timed step


def stage_bytes_per_cluster(kernel: str) -> float:
    return KERNEL_BYTES.get(kernel, 0.0)


def stage_rooflines(ktimes: dict, n: int, peak: float) -> dict:
    """Each step of the method (a1 .. a6) as one unit: its algorithmic bytes
    over the summed mean launch times of its kernels."""
    out = {}
    for st, b in STAGE_BYTES.items():
        ks = [k for k, v in KERNEL_STAGE.items() if st in v.split("+") and k in ktimes]
        ms = sum(ktimes[k][0] / ktimes[k][1] for k in ks)
        if ms <= 0:
            continue
        out[st] = {"kernels": ks, "ms": ms, "bytes_per_cluster": b,
                   "achieved_gbs": b * n / (ms * 1e-3) / 1e9,
                   "frac": b * n / (ms * 1e-3) / 1e9 / peak}
    return out


def kernel_bytes(c: dict) -> dict:
    N, RS, B = c["n_clusters"], c["n_rows_total"], c["n_bins"]
    T, Tl, Th = c["n_starts"], c["n_tracklets"], c["n_tracklet_hits"]
    K, Kh = c["n_tracks"], c["n_track_hits"]
    return {
        "k_count": 12 * N + 4 * RS,
        "k_rowscan": 4 * RS + 4 * RS + 32 * RS,
        "k_scatter": 12 * N + 12 * N,
        "k_rowsort": 12 * N + 16 * N + 8 * N + 4 * (B + RS) + 32 * RS,
        "k_rowsort_big": 0,  # its rows' bytes are counted in k_rowsort
        "k_rowsort_big4k": 0,
        "k_neighbours": 8 * N + 4 * N + 4 * B,
        "k_neighbours_crowded": 0,  # its hits' bytes are counted in k_neighbours
        "k_clean_starts": 4 * N + 4 * N + 4 * N + 4 * N + 4 * T,
        "k_chains": 8 * c["n_chain_hits"] + 32 * T,
        # forward passes of every chain, backward passes of the chains kept
        "k_constructor_fwd": 12 * (c["n_chain_hits"] + Th) + 40 * (Tl + c["n_dominated_chains"]),
        "k_dominance": 16 * T + 5 * c["n_chain_hits"],
        "k_constructor_bwd": 16 * Th + 116 * Tl,
        "k_weights": 20 * Th + 32 * Tl,
        "k_sel_decide": 10 * Th + 32 * T,
        "k_sel_sort": 12 * T + 8 * K,
        "k_sel_write": 244 * K + 12 * Kh,
    }


class ClockSampler:
    """nvidia-smi samples every 200 ms (clocks, throttle reasons), each stamped
    with the host time it arrived.  Started before the warm-up; the summary
    covers the samples between two marks (the timed region, extended by a
    hold window of the same steps so that a timed region shorter than the
    sampling period still gets samples)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []  # (host time, line)
        self.t0 = self.t1 = None
        self.t_timed = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def wait_first(self, timeout_s: float = 5.0):
        """Block until the first sample arrived (nvidia-smi takes a moment)."""
        t_end = time.perf_counter() + timeout_s
        while self.proc and not self.lines and time.perf_counter() < t_end:
            time.sleep(0.02)

    def mark(self, which: str):
        now = time.perf_counter()
        if which == "start":
            self.t0 = now
        elif which == "timed_end":
            self.t_timed = now
        else:
            self.t1 = now

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lo = self.t0 if self.t0 is not None else -1e30
        hi = self.t1 if self.t1 is not None else 1e30
        in_timed = 0
        for t, ln in self.lines:
            if not (lo <= t <= hi + 0.25):  # a sample reports the 200 ms before it
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            if self.t_timed is not None and t <= self.t_timed + 0.25:
                in_timed += 1
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        window = {"window_s": (hi - lo) if self.t0 is not None and self.t1 is not None else None,
                  "window": "the timed region and a hold of the same steps after it",
                  "samples_in_timed_region": in_timed}
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "warning": "nvidia-smi gave no sample in the window", **window}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), **window}


def cpu_baseline(ev_full, n_sectors: int = 4) -> dict:
    """The oracle as it stands on the host cores: every sector of the event as
    its own call, one thread per core (the oracle's C code keeps no global
    state and its ctypes calls release the GIL), and single-threaded on a few
    sectors for the per-core figure."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import oracle
    oracle.build()
    sectors = list(range(0, 36, 36 // n_sectors))[:n_sectors]
    sub = ev_full.select_sectors(sectors)
    t0 = time.perf_counter()
    oracle.track_event(sub)
    dt1 = time.perf_counter() - t0
    single = {"value": sub.n / dt1, "unit": UNIT, "cores": 1,
              "sample": f"{n_sectors} of 36 sectors ({sub.n} clusters), {dt1:.1f} s"}
    cores = os.cpu_count() or 1
    parts = [ev_full.select_sectors([s]) for s in range(36)]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as pool:
        list(pool.map(oracle.track_event, parts))
    dtn = time.perf_counter() - t0
    return {"value": ev_full.n / dtn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the whole central event ({ev_full.n} clusters), its 36 sectors as "
                      f"independent calls on {cores} threads, {dtn:.1f} s",
            "single_core": single}


def percentile(v, q):
    v = sorted(v)
    if not v:
        return None
    k = min(len(v) - 1, max(0, int(math.ceil(q / 100.0 * len(v))) - 1))
    return v[k]


SERVED_SLOTS, SERVED_PER_LAUNCH = 4, 2


def served_ctx(tp, host_events, geom, bz, n_per_event, sizes=None):
    """A served context whose pinned result pool is warm: two full bursts of
    the largest events (sizes = their cluster counts, when they differ)."""
    ctx = tp.tpc_track_create(SERVED_PER_LAUNCH * n_per_event + 1024,
                              max_events_in_flight=SERVED_SLOTS,
                              max_events_per_launch=SERVED_PER_LAUNCH)
    order = sorted(range(len(host_events)), key=lambda i: -sizes[i]) if sizes else \
        list(range(len(host_events)))
    for _ in range(2):
        tks = [tp.tpc_track_submit(ctx, host_events[order[i % len(order)]], geom, bz)
               for i in range(SERVED_SLOTS * SERVED_PER_LAUNCH + 4)]
        for t in tks:
            if tp.tpc_track_poll(ctx, t, 60_000_000, copy=False) is None:
                raise TimeoutError("warm-up ticket not done after 60 s")
            tp.tpc_track_release(ctx, t)
    return ctx


def run_one_at_a_time(tp, events, ns, arrivals, geom, bz, n_max):
    """FIFO server, one tpc_track_event call per arrival (waits for it).
    Returns per-event latencies (arrival -> result) and the span."""
    ctx = tp.tpc_track_create(n_max + 65536, max_events_per_launch=1)
    lat = []
    try:
        tp.tpc_track_event(ctx, events[0], geom, bz, copy=False)
        t_start = time.perf_counter()
        for i, a in enumerate(arrivals):
            now = time.perf_counter() - t_start
            if now < a:
                time.sleep(a - now)
            tp.tpc_track_event(ctx, events[i % len(events)], geom, bz, copy=False)
            lat.append(time.perf_counter() - t_start - a)
        span = time.perf_counter() - t_start
    finally:
        tp.tpc_track_destroy(ctx)
    return lat, span


def run_served(tp, events, ns, arrivals, geom, bz, n_max):
    """Served form: submit on arrival, a poller thread collects completions.
    Returns latencies, span and an error string (or None); every wait is
    bounded."""
    n_events = len(arrivals)
    ctx = served_ctx(tp, events, geom, bz, n_max, ns)
    lats = [None] * n_events
    errors = []
    tickets = [None] * n_events
    t_start = time.perf_counter()
    done = threading.Event()

    def poller():
        try:
            for i in range(n_events):
                deadline = time.perf_counter() + 60.0
                while tickets[i] is None:
                    if errors or time.perf_counter() > deadline:
                        raise TimeoutError("ticket never submitted")
                    time.sleep(0.0001)
                if tp.tpc_track_poll(ctx, tickets[i], 60_000_000, copy=False) is None:
                    raise TimeoutError("ticket not done after 60 s")
                lats[i] = time.perf_counter() - t_start - arrivals[i]
                tp.tpc_track_release(ctx, tickets[i])
        except Exception as e:  # reported in the JSON line
            errors.append(repr(e))
        finally:
            done.set()
    th = threading.Thread(target=poller, daemon=True)
    th.start()
    try:
        for i, a in enumerate(arrivals):
            now = time.perf_counter() - t_start
            if now < a:
                time.sleep(a - now)
            tickets[i] = tp.tpc_track_submit(ctx, events[i % len(events)], geom, bz)
    except Exception as e:
        errors.append(repr(e))
    if not done.wait(180.0):
        errors.append("served run did not finish within 180 s")
    span = time.perf_counter() - t_start
    if not errors:
        tp.tpc_track_destroy(ctx)
    return lats, span, (errors[0] if errors else None)


def compare_point(tp, events, ns, arrivals, geom, bz, n_max, rate):
    lat1, span1 = run_one_at_a_time(tp, events, ns, arrivals, geom, bz, n_max)
    lats, spans, err = run_served(tp, events, ns, arrivals, geom, bz, n_max)
    if err:
        return None, err
    n_cl = sum(ns[i % len(ns)] for i in range(len(arrivals)))
    return {"rate_per_s": rate, "events": len(arrivals),
            "one_event": {"p50_ms": percentile(lat1, 50) * 1e3, "p99_ms": percentile(lat1, 99) * 1e3,
                          "clusters_per_s": n_cl / span1},
            "served": {"p50_ms": percentile(lats, 50) * 1e3, "p99_ms": percentile(lats, 99) * 1e3,
                       "clusters_per_s": n_cl / spans}}, None


def at_equal_p99(points, targets_ms=(10.0, 20.0)) -> list:
    """For each p99 target and each server: the highest clusters/s among the
    measured rates whose p99 latency met the target, and that throughput
    interpolated to p99 = target between the last rate that met it and the
    next one (linear in p99), which does not favour the server whose
    measured points happen to lie closer to the target."""
    out = []
    for tgt in targets_ms:
        row = {"p99_target_ms": tgt}
        for side in ("one_event", "served"):
            pts = sorted(points, key=lambda p: p["rate_per_s"])
            ok = [p[side]["clusters_per_s"] for p in pts if p[side]["p99_ms"] <= tgt]
            row[side + "_clusters_per_s"] = max(ok) if ok else None
            interp = None
            for a, b in zip(pts, pts[1:]):
                la, lb = a[side]["p99_ms"], b[side]["p99_ms"]
                if la <= tgt < lb:
                    w = (tgt - la) / (lb - la)
                    interp = a[side]["clusters_per_s"] + w * (b[side]["clusters_per_s"] -
                                                              a[side]["clusters_per_s"])
            if interp is None and ok and pts[-1][side]["p99_ms"] <= tgt:
                interp = pts[-1][side]["clusters_per_s"]  # met at every measured rate
            row[side + "_interp_clusters_per_s"] = interp
        out.append(row)
    return out


def served_summary(served, line) -> dict:
    """Compact record of the served-form comparison (and the headline
    fractions), written as the last key of the bench line."""
    out = {"value": line["value"], "e2e": (line.get("e2e") or {}).get("value"),
           "roofline_frac": line["roofline"]["frac"],
           "path_roofline_frac": line["path_roofline"]["frac"]}
    if not served or "points" not in served:
        out["served"] = None
        return out

    def pick(rows):
        return [{k: (round(v, 4) if isinstance(v, float) and k.endswith("_ms") else
                     (float(f"{v:.4g}") if isinstance(v, float) else v))
                 for k, v in r.items()} for r in rows]
    out["central_events_at_equal_p99"] = pick(served.get("at_equal_p99", []))
    out["central_events_rates"] = len(served["points"])
    st = served.get("stream") or {}
    if "at_equal_p99" in st:
        out["event_stream_at_equal_p99"] = pick(st["at_equal_p99"])
    return out


def served_vs_one(tp, torch, host_events, geom, bz, n_per_event,
                  rate_factors=(0.5, 0.6, 0.7, 0.8, 0.9, 1.0, 1.1, 1.2, 1.3, 1.5, 3.0),
                  n_events=120, seed=4):
    """Poisson arrivals of central events: one-at-a-time FIFO server vs the
    served form (continuous batching over SERVED_SLOTS slots of up to
    SERVED_PER_LAUNCH events).  Rates are set relative to the measured
    one-at-a-time capacity.  Both sides read their results as views of the
    library's pinned buffers (no extra host copy)."""
    import numpy as np
    ctx1 = tp.tpc_track_create(n_per_event + 65536, max_events_per_launch=1)
    try:
        # service time of one event through the C ABI with host inputs
        for e in host_events[:1] * 3:
            tp.tpc_track_event(ctx1, e, geom, bz, copy=False)
        t0 = time.perf_counter()
        for i in range(10):
            tp.tpc_track_event(ctx1, host_events[i % len(host_events)], geom, bz, copy=False)
        service = (time.perf_counter() - t0) / 10
    finally:
        tp.tpc_track_destroy(ctx1)
    cap = 1.0 / service
    out = {"service_ms_one_event": service * 1e3,
           "served_config": {"slots": SERVED_SLOTS, "events_per_launch": SERVED_PER_LAUNCH},
           "points": []}
    rng = np.random.default_rng(seed)
    ns = [n_per_event] * len(host_events)
    for rf in rate_factors:
        lam = rf * cap
        arrivals = np.cumsum(rng.exponential(1.0 / lam, n_events))
        pt, err = compare_point(tp, host_events, ns, arrivals, geom, bz, n_per_event, lam)
        if err:
            out["error"] = err
            return out
        out["points"].append(pt)
    out["at_equal_p99"] = at_equal_p99(out["points"])
    return out


def served_sweep(tp, torch, synth, rates, n_events_of, pool_size=64, seed=4):
    """Config 4: an event stream with Poisson arrivals at the given rates and
    multiplicities min(10000, max(1, round(Exp(1500)))) tracks (arrivals
    cycle through a pool of pool_size such events), one-at-a-time FIFO server
    vs the served form, both with pinned host inputs."""
    import numpy as np
    rng = np.random.default_rng(seed)
    pool = [synth.served_event(rng, synth.served_multiplicity(rng)) for _ in range(pool_size)]
    geom, keep_x = tp.geometry_of(pool[0])
    bz = float(pool[0].bz)
    pinned, cs = [], []
    for e in pool:
        t = [torch.from_numpy(e.y).pin_memory(), torch.from_numpy(e.z).pin_memory(),
             torch.from_numpy(e.row.view(np.int16)).pin_memory(),
             torch.from_numpy(e.sector.view(np.int16)).pin_memory()]
        pinned.append(t)
        cs.append(tp.clusters_of(*t)[0])
    ns = [e.n for e in pool]
    n_max = max(ns)
    out = {"workload": f"pool of {pool_size} events, tracks min(10000, max(1, round(Exp(1500)))), "
                       f"mean {np.mean(ns):.0f} clusters per event",
           "served_config": {"slots": SERVED_SLOTS, "events_per_launch": SERVED_PER_LAUNCH},
           "points": []}
    for lam in rates:
        n_ev = n_events_of(lam)
        arrivals = np.cumsum(rng.exponential(1.0 / lam, n_ev))
        pt, err = compare_point(tp, cs, ns, arrivals, geom, bz, n_max, lam)
        if err:
            out["error"] = err
            return out
        out["points"].append(pt)
    out["at_equal_p99"] = at_equal_p99(out["points"])
    return out


def batched_vs_sequential(tp, torch, synth, stream, n_events=64, reps=3):
    """64 events of uneven multiplicity (20 to 10,000 tracks, log-uniform)
    resident on the device: one launch of all of them (autotuned schedule,
    CUDA graph) against 64 single-event launches one after the other, each
    waited for (launch + results)."""
    import numpy as np
    evs = synth.batch_events(n_events)
    geom, keep_x = tp.geometry_of(evs[0])
    bz = float(evs[0].bz)
    dev = [(torch.from_numpy(e.y).cuda(), torch.from_numpy(e.z).cuda(),
            torch.from_numpy(e.row.view(np.int16)).cuda(),
            torch.from_numpy(e.sector.view(np.int16)).cuda()) for e in evs]
    cs = [tp.clusters_of(*d)[0] for d in dev]
    n_all = sum(e.n for e in evs)
    torch.cuda.synchronize()
    ctx_b = tp.tpc_track_create(n_all + 65536, max_events_per_launch=n_events,
                                cuda_stream=stream.cuda_stream)
    ctx_1 = tp.tpc_track_create(max(e.n for e in evs) + 65536, max_events_per_launch=1,
                                cuda_stream=stream.cuda_stream)
    try:
        sched = tp.tpc_track_autotune(ctx_b, cs, geom, bz, reps=2)
        for _ in range(2):
            tp.tpc_track_launch(ctx_b, cs, geom, bz)
            tp.tpc_track_results(ctx_b, n_events, copy=False)
        t0 = time.perf_counter()
        for _ in range(reps):
            tp.tpc_track_launch(ctx_b, cs, geom, bz)
            tp.tpc_track_results(ctx_b, n_events, copy=False)
        t_batch = (time.perf_counter() - t0) / reps
        n_tracks_b = tp.tpc_track_get_counters(ctx_b)["n_tracks"]
        for c in cs[:4]:
            tp.tpc_track_launch(ctx_1, [c], geom, bz)
            tp.tpc_track_results(ctx_1, 1, copy=False)
        t0 = time.perf_counter()
        n_tracks_s = 0
        for _ in range(reps):
            for c in cs:
                tp.tpc_track_launch(ctx_1, [c], geom, bz)
                tp.tpc_track_results(ctx_1, 1, copy=False)
                n_tracks_s += tp.tpc_track_get_counters(ctx_1)["n_tracks"]
        t_seq = (time.perf_counter() - t0) / reps
        # the same single-event launches spread over 4 streams (concurrent
        # kernels of up to 4 events), every event's results collected
        ctx_4 = tp.tpc_track_create(max(e.n for e in evs) + 65536, max_events_per_launch=1,
                                    max_events_in_flight=4, cuda_stream=stream.cuda_stream)
        tp.tpc_track_set_schedule(ctx_4, **{k: v for k, v in tp.tpc_track_get_schedule(ctx_1).items()
                                            if k in ("bin_blocks_per_sm", "sort_threads",
                                                     "nb_threads", "tl_blocks_per_sm")}, streams=4)

        def pipelined():
            n_tr = 0
            for i, c in enumerate(cs):
                tp.tpc_track_launch(ctx_4, [c], geom, bz)
                if i >= 3:
                    tp.tpc_track_results(ctx_4, 1, copy=False)
                    n_tr += tp.tpc_track_get_counters(ctx_4)["n_tracks"]
            for _ in range(3):
                tp.tpc_track_results(ctx_4, 1, copy=False)
                n_tr += tp.tpc_track_get_counters(ctx_4)["n_tracks"]
            return n_tr
        try:
            pipelined()
            t0 = time.perf_counter()
            for _ in range(reps):
                n_tracks_p = pipelined()
            t_pipe = (time.perf_counter() - t0) / reps
        finally:
            tp.tpc_track_destroy(ctx_4)
    finally:
        tp.tpc_track_destroy(ctx_b)
        tp.tpc_track_destroy(ctx_1)
    return {"workload": f"{n_events} events, 20-10,000 tracks log-uniform, seeds 3000+i",
            "clusters": int(n_all), "tracks": int(n_tracks_b),
            "tracks_sequential": int(n_tracks_s // reps),
            "batch_ms": t_batch * 1e3, "sequential_ms": t_seq * 1e3,
            "clusters_per_s_batch": n_all / t_batch, "clusters_per_s_sequential": n_all / t_seq,
            "speedup": t_seq / t_batch, "schedule": sched,
            "streams4_ms": t_pipe * 1e3, "clusters_per_s_streams4": n_all / t_pipe,
            "tracks_streams4": int(n_tracks_p),
            "timing": "host wall clock around launch + results, inputs resident on the device"}


def pileup_section(tp, torch, synth, stream, reps=3, n_served=4):
    """Config 5: 50 collisions (200-2000 tracks, vertex z within +-200 cm)
    merged into one event, through the batched path (one device-resident
    launch, autotuned) and the served path (host inputs, tickets submitted at
    once), with the Monte-Carlo efficiency, fake and clone rates of the
    tracks."""
    import numpy as np
    ev = synth.pileup_event()
    geom, keep_x = tp.geometry_of(ev)
    bz = float(ev.bz)
    d = (torch.from_numpy(ev.y).cuda(), torch.from_numpy(ev.z).cuda(),
         torch.from_numpy(ev.row.view(np.int16)).cuda(),
         torch.from_numpy(ev.sector.view(np.int16)).cuda())
    c = tp.clusters_of(*d)[0]
    torch.cuda.synchronize()
    out = {"workload": "50 collisions of 200-2000 tracks, vertex z ~ U(-200, 200) cm, seed 5",
           "clusters": int(ev.n)}
    ctx = tp.tpc_track_create(ev.n + 65536, max_events_per_launch=1, cuda_stream=stream.cuda_stream)
    try:
        out["schedule"] = tp.tpc_track_autotune(ctx, [c], geom, bz, reps=2)
        tp.tpc_track_launch(ctx, [c], geom, bz)
        tp.tpc_track_results(ctx, 1, copy=False)
        t0 = time.perf_counter()
        for _ in range(reps):
            tp.tpc_track_launch(ctx, [c], geom, bz)
            outs = tp.tpc_track_results(ctx, 1, copy=False)
        dt = (time.perf_counter() - t0) / reps
        tr = tp.tracks_to_numpy(outs[0])
        out["batched"] = {"ms": dt * 1e3, "clusters_per_s": ev.n / dt,
                          "timing": "host wall clock around launch + results, device inputs"}
        out["tracks"] = int(tr.n_tracks)
        out["mc"] = synth.mc_performance(ev, tr.sector, tr.hit_off, tr.hit_cid)
        out["particles"] = synth.particle_performance(ev, tr.hit_off, tr.hit_cid)
        # the same launch with the sector track merger
        p = tp.tpc_track_default_params()
        p.merge = 1
        tp.tpc_track_set_params(ctx, p)
        tp.tpc_track_launch(ctx, [c], geom, bz)
        tp.tpc_track_results(ctx, 1, copy=False)
        t0 = time.perf_counter()
        for _ in range(reps):
            tp.tpc_track_launch(ctx, [c], geom, bz)
            outs = tp.tpc_track_results(ctx, 1, copy=False)
        dt = (time.perf_counter() - t0) / reps
        tr = tp.tracks_to_numpy(outs[0])
        cm = tp.tpc_track_get_counters(ctx)
        out["merged"] = {"ms": dt * 1e3, "clusters_per_s": ev.n / dt, "tracks": int(tr.n_tracks),
                         "chains": int(cm["n_merge_chains"]),
                         "particles": synth.particle_performance(ev, tr.hit_off, tr.hit_cid)}
    finally:
        tp.tpc_track_destroy(ctx)
    pinned = [torch.from_numpy(ev.y).pin_memory(), torch.from_numpy(ev.z).pin_memory(),
              torch.from_numpy(ev.row.view(np.int16)).pin_memory(),
              torch.from_numpy(ev.sector.view(np.int16)).pin_memory()]
    hc = tp.clusters_of(*pinned)[0]
    sctx = tp.tpc_track_create(ev.n + 1024, max_events_in_flight=2, max_events_per_launch=1)
    try:
        # warm-up: the same burst, so that its pinned result buffers exist
        for t in [tp.tpc_track_submit(sctx, hc, geom, bz) for _ in range(n_served)]:
            if tp.tpc_track_poll(sctx, t, 60_000_000, copy=False) is None:
                raise TimeoutError("pile-up ticket not done after 60 s")
            tp.tpc_track_release(sctx, t)
        t0 = time.perf_counter()
        tks = [tp.tpc_track_submit(sctx, hc, geom, bz) for _ in range(n_served)]
        lat = []
        for t in tks:
            if tp.tpc_track_poll(sctx, t, 60_000_000, copy=False) is None:
                raise TimeoutError("pile-up ticket not done after 60 s")
            lat.append(time.perf_counter() - t0)
            tp.tpc_track_release(sctx, t)
        span = time.perf_counter() - t0
        out["served"] = {"events": n_served, "slots": 2, "clusters_per_s": n_served * ev.n / span,
                         "first_result_ms": lat[0] * 1e3, "last_result_ms": lat[-1] * 1e3,
                         "timing": "host wall clock, pinned host inputs, tickets submitted at once"}
    finally:
        tp.tpc_track_destroy(sctx)
    return out


def calib_loop(tp, ctx, ev, geom, bz, n_cl, n_events, every_n, inline, depth=4):
    """Served stream with the chi^2-scale side task: `depth` events in
    flight; each finished event's tracks are added to the fit; a finished
    fit is fed back with tpc_track_set_params.  inline=True waits for every
    fit where it starts (the task run inside the event loop, Fig. 4);
    inline=False only checks at every event (Sect. 5.1, Fig. 5)."""
    from collections import deque
    cal = tp.Chi2Calib(every_n, 3.0, 2)
    lat, gaps, fits, q = [], [], [], deque()
    p0, v0 = tp.tpc_track_get_params(ctx)
    sigma_of = {v0: float(p0.meas_sigma_y)}
    added = 0

    def feed_back(f):
        fits.append(f)
        s = sigma_of[f["params_version"]] * math.sqrt(f["scale2"])
        p = tp.tpc_track_default_params()
        p.meas_sigma_y = p.meas_sigma_z = s
        _, ver = tp.tpc_track_set_params(ctx, p)
        sigma_of[ver] = float(p.meas_sigma_y)
    try:
        t0 = t_prev = time.perf_counter()
        for i in range(n_events + depth - 1):
            if i < n_events:
                q.append((tp.tpc_track_submit(ctx, ev, geom, bz), time.perf_counter()))
            if len(q) < depth and i < n_events:
                continue
            tk, ts = q.popleft()
            tr = tp.tpc_track_poll(ctx, tk, 60_000_000, copy=False)
            if tr is None:
                raise TimeoutError("ticket not done after 60 s")
            _, ver = tp.tpc_track_ticket_params(ctx, tk)
            cal.add(tr.chi2, tr.ndf, ver)
            added += 1
            tp.tpc_track_release(ctx, tk)
            now = time.perf_counter()
            lat.append(now - ts)
            gaps.append(now - t_prev)
            t_prev = now
            if inline and added % every_n == 0:
                f = cal.poll(-1)
                if f is not None:
                    feed_back(f)
            elif not inline:
                f = cal.poll(0)
                if f is not None:
                    feed_back(f)
        span = time.perf_counter() - t0
        st = cal.stats()
    finally:
        cal.close()
    return {"events": n_events, "fits": len(fits),
            "fit_ms_max": st["max_task_ms"], "fit_ms_mean": st["busy_ms"] / max(1, st["finished"]),
            "tracks_per_fit": fits[0]["n_tracks"] if fits else 0,
            "clusters_per_s": n_events * n_cl / span,
            "latency_p50_ms": percentile(lat, 50) * 1e3, "latency_p99_ms": percentile(lat, 99) * 1e3,
            "latency_max_ms": max(lat) * 1e3, "max_gap_between_events_ms": max(gaps) * 1e3,
            "sigma_after": sigma_of[max(sigma_of)]}


def async_section(tp, torch, host_ev, geom, bz, n_cl, n_events=600, every_n=100):
    """The side task inline vs asynchronous on the same served stream."""
    out = {"workload": f"{n_events} central events served back to back (4 in flight); "
                       f"chi^2-scale fit of the tracks of every {every_n} events, fed back "
                       "as the cluster error"}
    for mode in ("inline", "async"):
        ctx = served_ctx(tp, [host_ev], geom, bz, n_cl)
        try:
            calib_loop(tp, ctx, host_ev, geom, bz, n_cl, 2 * every_n, every_n, mode == "inline")
            out[mode] = calib_loop(tp, ctx, host_ev, geom, bz, n_cl, n_events, every_n,
                                   mode == "inline")
            if mode == "async":  # one event's tracks, for the fit timings below
                tk = tp.tpc_track_submit(ctx, host_ev, geom, bz)
                tr = tp.tpc_track_poll(ctx, tk, 60_000_000)
                tp.tpc_track_release(ctx, tk)
        finally:
            tp.tpc_track_destroy(ctx)
    # the fit alone on the tracks of every_n events: the library's (on its
    # side thread) and the oracle's statement of it, on one core each
    import numpy as np
    from oracle.calib import chi2_scale_fit
    chi2 = np.tile(tr.chi2, every_n)
    ndf = np.tile(tr.ndf, every_n)
    cal = tp.Chi2Calib(1, 3.0, 1)
    try:
        cal.add(chi2, ndf, 0)
        f = cal.poll(-1)
        native_ms = cal.stats()["max_task_ms"]
    finally:
        cal.close()
    t0 = time.perf_counter()
    o = chi2_scale_fit(chi2.astype(np.float64), ndf)
    oracle_ms = (time.perf_counter() - t0) * 1e3
    out["fit"] = {"tracks": int(len(chi2)), "native_ms": native_ms, "oracle_ms": oracle_ms,
                  "same_result": bool(abs(f["scale2"] - o["scale2"]) <= 1e-12 * abs(o["scale2"])
                                      and f["n_kept"] == o["n_kept"])}
    return out


def merge_oracle_baseline(ev) -> dict:
    """The oracle's merger (M1-M5) on the event, on one host core: the
    sector tracks come from 36 per-sector oracle calls on all cores
    (untimed), gathered into one track list in the sector order."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import oracle
    oracle.build()
    import numpy as np
    parts = [ev.select_sectors([s]) for s in range(36)]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as pool:
        outs = list(pool.map(oracle.track_event, parts))
    o = {"n_tracks": 0}
    keys = ("k_sector", "k_x", "k_p", "k_C", "k_chi2", "k_ndf")
    acc = {k: [] for k in keys}
    hits, lens = [], []
    for s, (sub, r) in enumerate(zip(parts, outs)):
        parent = sub.info["parent_index"]
        acc["k_sector"].append(np.full(r["n_tracks"], s, np.int32))
        for k in keys[1:]:
            acc[k].append(r[k])
        hits.append(parent[r["k_hit_cid"]].astype(np.int32))
        lens.append(np.diff(r["k_hit_off"]))
    for k in keys:
        o[k] = np.concatenate(acc[k])
    o["n_tracks"] = len(o["k_sector"])
    o["k_hit_cid"] = np.concatenate(hits)
    o["k_hit_off"] = np.concatenate([[0], np.cumsum(np.concatenate(lens))]).astype(np.int32)
    t0 = time.perf_counter()
    m = oracle.merge_tracks(ev, o)
    dt = time.perf_counter() - t0
    return {"value": ev.n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the merger alone on the central event's {o['n_tracks']} oracle sector "
                      f"tracks -> {m['n_tracks']} tracks, {dt:.1f} s on one core"}


def merge_section(tp, torch, synth, stream, cls, ev, geom, bz, n, base_ms, steps=200, tune=True):
    """The central event with the sector track merger on: step time (timed
    like the headline, autotuned streams), the merger's kernels, and the
    tracks per particle with and without merging."""
    import numpy as np
    p = tp.tpc_track_default_params()
    p.merge = 1
    ctx = tp.tpc_track_create(n + 65536, max_events_per_launch=1, max_events_in_flight=4,
                              cuda_stream=stream.cuda_stream, params=p)
    try:
        sched = tp.tpc_track_autotune(ctx, [cls[0][0]], geom, bz, reps=2) if tune else \
            tp.tpc_track_get_schedule(ctx)
        for i in range(4):
            tp.tpc_track_launch(ctx, [cls[i % len(cls)][0]], geom, bz)
            tp.tpc_track_results(ctx, 1, copy=False)
        c = tp.tpc_track_get_counters(ctx)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(steps):
            tp.tpc_track_launch(ctx, [cls[i % len(cls)][0]], geom, bz)
        tp.tpc_track_join(ctx)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        for _ in range(sched["streams"]):
            tp.tpc_track_results(ctx, 1, copy=False)
        tp.tpc_track_set_profiling(ctx, True)
        for i in range(20):
            tp.tpc_track_launch(ctx, [cls[i % len(cls)][0]], geom, bz)
            tp.tpc_track_results(ctx, 1, copy=False)
        kt = tp.tpc_track_kernel_times(ctx)
        tp.tpc_track_set_profiling(ctx, False)
    finally:
        tp.tpc_track_destroy(ctx)
    mg = {k: v[0] / v[1] for k, v in kt.items() if k.startswith("k_mg_")}
    whole = sum(v[0] / v[1] for v in kt.values())
    perf = {}
    for name, merge in (("without", 0), ("with", 1)):
        q = tp.tpc_track_default_params()
        q.merge = merge
        with tp.Tracker(n + 65536, params=q) as t:
            tr = t.event(ev)
        perf[name] = synth.particle_performance(ev, tr.hit_off, tr.hit_cid)
    # hits of the merged tracks (those spanning more than one sector): the
    # refit reads one 16-byte (x, y, z) record per hit, the gather writes it
    nh = np.diff(tr.hit_off)
    tid = np.repeat(np.arange(tr.n_tracks), nh)
    sec = ev.sector[tr.hit_cid].astype(np.int64)
    spans = np.zeros(tr.n_tracks, bool)
    if len(sec):
        first = np.repeat(sec[tr.hit_off[:-1]], nh)
        np.logical_or.at(spans, tid, sec != first)
    merged_hits = int(nh[spans].sum())
    peak, _ = peaks()
    b_refit = 16 * merged_hits + 2 * 88 * int(c["n_merge_chains"])
    roof = {"k_mg_refit": {"bytes": b_refit, "ms": mg.get("k_mg_refit"),
                           "frac_of_hbm": b_refit / (mg["k_mg_refit"] * 1e-3) / 1e9 / peak,
                           "bound": "latency: one serial Kalman chain per merged track"},
            "k_mg_match": {"bytes": 88 * int(c["n_sector_tracks"]),
                           "ms": mg.get("k_mg_match"),
                           "bound": "latency and ALU: candidate tests from L2 (tracks of one "
                                    "sector ~40 kB)"}}
    return {"workload": "central event with the sector track merger (merge = 1)",
            "roofline": roof, "merged_track_hits": merged_hits,
            "cpu_baseline": merge_oracle_baseline(ev),
            "ms_per_event": ms, "clusters_per_s": n / (ms * 1e-3),
            "ms_per_event_without_merge": base_ms, "schedule": sched,
            "sector_tracks": int(c["n_sector_tracks"]), "tracks": int(c["n_tracks"]),
            "links": int(c["n_merge_links"]), "chains": int(c["n_merge_chains"]),
            "merger_kernels_ms": mg, "merger_share_of_kernel_time": sum(mg.values()) / whole,
            "particles": perf,
            "timing": "CUDA events on the tracker stream over the steps (fork to join); "
                      "kernel times from a separate pass, one stream"}


def traffic_for(kernel: str, counters: dict):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current source of that kernel."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    e = d.get(kernel)
    if not e:
        return None
    srcs = e["source"] if isinstance(e["source"], list) else [e["source"]]
    hs = hashlib.sha256()
    for f in srcs:
        hs.update(open(os.path.join(ROOT, "paper_1712_09416_b300", "csrc", f), "rb").read())
    h = hs.hexdigest()[:16]
    if h != e["source_sha"]:
        return None
    return e["dram_bytes_per_cluster"] * counters["n_clusters"]


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1712_09416_b300 import build, synth, tpctrack as tp
    build.build()
    ev = synth.central_event(seed=2)
    n = ev.n
    geom, keep_x = tp.geometry_of(ev)
    bz = float(ev.bz)
    dev = []
    for _ in range(N_COPIES):
        dev.append((torch.from_numpy(ev.y).cuda(), torch.from_numpy(ev.z).cuda(),
                    torch.from_numpy(ev.row.view(np.int16)).cuda(),
                    torch.from_numpy(ev.sector.view(np.int16)).cuda()))
    cls = [tp.clusters_of(*d) for d in dev]
    torch.cuda.synchronize()
    # a stream of our own: the tracker launches on it and the timing events
    # are recorded on it (torch's default stream is the legacy stream 0, for
    # which the library would create a separate non-blocking stream)
    stream = torch.cuda.Stream()

    def make_ctx(epl):
        # up to eight slots in all: the autotuner may spread consecutive
        # launches over several streams, so that one launch's kernels overlap
        # the next one's (one slot without the autotuner: one stream, and the
        # least device memory for a profiler capture)
        slots = 1 if args.no_autotune else max(2, 8 // epl)
        return tp.tpc_track_create(epl * n + 65536, max_events_per_launch=epl,
                                   max_events_in_flight=slots, cuda_stream=stream.cuda_stream)

    def launch_events(epl, i):
        # launch i takes the device copies i*epl .. i*epl+epl-1 (in turn)
        return [cls[(i * epl + j) % N_COPIES][0] for j in range(epl)]

    # events per launch (the batched form on central events, Sect. 2: many
    # events in flight): each candidate's context is autotuned, then timed on
    # a burst of launches; the fastest is the step of the timed region
    epl_sweep = {}
    if args.no_autotune:
        epl = max(1, args.events_per_launch)
        ctx = make_ctx(epl)
        schedule = tp.tpc_track_get_schedule(ctx)
    else:
        best = None
        for cand in ([args.events_per_launch] if args.events_per_launch > 0 else EPL_CANDIDATES):
            c = make_ctx(cand)
            sch = tp.tpc_track_autotune(c, launch_events(cand, 0), geom, bz, reps=3)
            for i in range(4):
                tp.tpc_track_launch(c, launch_events(cand, i), geom, bz)
                tp.tpc_track_results(c, cand, copy=False)
            k_burst = max(16, 96 // cand)
            torch.cuda.synchronize()
            b0 = torch.cuda.Event(enable_timing=True)
            b1 = torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            for i in range(k_burst):
                tp.tpc_track_launch(c, launch_events(cand, i), geom, bz)
            tp.tpc_track_join(c)
            b1.record(stream)
            torch.cuda.synchronize()
            for _ in range(sch["streams"]):
                tp.tpc_track_results(c, cand, copy=False)
            rate = k_burst * cand * n / (b0.elapsed_time(b1) * 1e-3)
            epl_sweep[cand] = {"clusters_per_s": rate, "streams": sch["streams"],
                               "tl_blocks_per_sm": sch["tl_blocks_per_sm"]}
            if best is None or rate > best[0]:
                if best is not None:
                    tp.tpc_track_destroy(best[1])
                best = (rate, c, cand, sch)
            else:
                tp.tpc_track_destroy(c)
        _, ctx, epl, schedule = best
    n_streams = schedule["streams"]
    n_step = epl * n  # clusters of one step (one launch)

    def step(i):
        tp.tpc_track_launch(ctx, launch_events(epl, i), geom, bz)

    for i in range(args.warmup):
        step(i)
        tp.tpc_track_results(ctx, epl, copy=False)
    counters = tp.tpc_track_get_counters(ctx)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(local)
    clk.__enter__()
    clk.wait_first()
    barrier()
    clk.mark("start")
    e0.record(stream)
    for i in range(args.steps):
        step(i)  # the kernel sequence replays as one CUDA graph per step
    tp.tpc_track_join(ctx)  # the stream waits for the steps on every slot
    e1.record(stream)
    barrier()
    clk.mark("timed_end")
    ms_total = e0.elapsed_time(e1)
    for _ in range(n_streams):  # status of the last step of every slot
        tp.tpc_track_results(ctx, epl, copy=False)
    # hold: the same steps for about three seconds more (untimed), so that
    # the clock record has a dozen samples under the same load even when the
    # timed region is shorter than a few of nvidia-smi's 200 ms periods
    t_hold = time.perf_counter() + 3.0
    i = 0
    while time.perf_counter() < t_hold:
        for _ in range(16):
            step(i)
            i += 1
        tp.tpc_track_join(ctx)
        torch.cuda.synchronize()
        for _ in range(min(16, n_streams)):
            tp.tpc_track_results(ctx, epl, copy=False)
    clk.mark("end")
    clk.__exit__()
    # the same steps on 1..max streams with the tuned grid shapes (outside the
    # timed region): what running consecutive events' kernels together buys
    streams_sweep = {}
    if rank == 0 and not args.no_autotune:
        for k in range(1, schedule["max_streams"] + 1):
            tp.tpc_track_set_schedule(ctx, **{**schedule, "streams": k})
            for i in range(2 * k):
                step(i)
            tp.tpc_track_join(ctx)
            torch.cuda.synchronize()
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            n_sw = min(args.steps, 200)
            for i in range(n_sw):
                step(i)
            tp.tpc_track_join(ctx)
            s1.record(stream)
            torch.cuda.synchronize()
            for _ in range(k):
                tp.tpc_track_results(ctx, epl, copy=False)
            streams_sweep[k] = s0.elapsed_time(s1) / n_sw / epl
        tp.tpc_track_set_schedule(ctx, **schedule)
    # per-kernel device times: the same steps again, kernels launched one by
    # one with a CUDA event after each (outside the timed region)
    tp.tpc_track_set_profiling(ctx, True)
    for i in range(args.steps):
        step(i)
    tp.tpc_track_results(ctx, epl, copy=False)
    ktimes = tp.tpc_track_kernel_times(ctx)
    tp.tpc_track_set_profiling(ctx, False)
    ms_total = replica_time(ms_total, world)
    ms_step = ms_total / args.steps
    value = job_throughput(n_step * args.steps, world, ms_total)
    launches = sum(v[1] for v in ktimes.values())

    # roofline of the dominant kernel: the algorithmic bytes of its step of
    # the method (per cluster, times the clusters of one launch) over its
    # mean launch time; the bytes this implementation's kernels move are
    # reported beside (frac_impl_bytes)
    kb = kernel_bytes(counters)
    peak, peak_src = peaks()
    dom = max(ktimes, key=lambda k: ktimes[k][0])
    dom_ms = ktimes[dom][0] / ktimes[dom][1]
    dom_bytes = stage_bytes_per_cluster(dom) * n_step
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    b_impl = sum(kb.values()) / n_step
    # I/O-only lower bound: the clusters in (12 B) and the tracks out
    io_b = (12 * n_step + 100 * counters["n_tracks"] + 4 * counters["n_track_hits"]) / n_step

    # end to end through the C ABI with pinned host inputs
    pinned = [torch.from_numpy(ev.y).pin_memory(), torch.from_numpy(ev.z).pin_memory(),
              torch.from_numpy(ev.row.view(np.int16)).pin_memory(),
              torch.from_numpy(ev.sector.view(np.int16)).pin_memory()]
    hc, hkeep = tp.clusters_of(*pinned)
    e2e = None
    if not args.no_e2e:
        # bursts of at least 40 events: the served pipeline (4 slots x 2 events)
        # fills and drains once per burst
        k_e2e = max(40, min(args.steps, 80))
        # (a) one event per call (tpc_track_event): copies, launch and result
        # read strictly one after the other
        ctx_h = tp.tpc_track_create(n + 65536, max_events_per_launch=1)
        for _ in range(3):
            tr = tp.tpc_track_event(ctx_h, hc, geom, bz, copy=False)
        barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            tr = tp.tpc_track_event(ctx_h, hc, geom, bz, copy=False)
        barrier()
        seq_s = time.perf_counter() - t0
        n_tr, n_hits = tr.n_tracks, len(tr.hit_cid)
        tp.tpc_track_destroy(ctx_h)
        # (b) the served API (tpc_track_submit / poll) with every event submitted
        # at once: each event's host inputs are copied in and its tracks copied
        # out inside the timed region, overlapped across slots
        ctx_s = served_ctx(tp, [hc], geom, bz, n)
        srv_runs = []
        for _ in range(3):  # three timed bursts; the median is the figure
            barrier()
            t0 = time.perf_counter()
            tks = [tp.tpc_track_submit(ctx_s, hc, geom, bz) for _ in range(k_e2e)]
            for t in tks:
                if tp.tpc_track_poll(ctx_s, t, 60_000_000, copy=False) is None:
                    raise TimeoutError("served ticket not done after 60 s")
                tp.tpc_track_release(ctx_s, t)
            barrier()
            srv_runs.append(time.perf_counter() - t0)
        srv_s = sorted(srv_runs)[1]
        tp.tpc_track_destroy(ctx_s)
        h2d = 12 * n + 4096
        d2h = 256 + n_tr * (4 + 4 + 20 + 60 + 4 + 4 + 4) + 4 * n_hits + 4 * 37
        # the host->device link: pinned copies of the bytes of eight events,
        # best of five; the served figure cannot exceed link / 12 B per cluster
        hbuf = torch.empty(8 * 12 * n, dtype=torch.uint8).pin_memory()
        dbuf = torch.empty(8 * 12 * n, dtype=torch.uint8, device="cuda")
        link = []
        for _ in range(5):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dbuf.copy_(hbuf, non_blocking=True)
            torch.cuda.synchronize()
            link.append(hbuf.numel() / (time.perf_counter() - t0) / 1e9)
        del hbuf, dbuf
        h2d_gbs = max(link)
        e2e = {"value": world * n * k_e2e / srv_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": k_e2e,
               "api": f"tpc_track_submit/poll, {SERVED_SLOTS} slots x {SERVED_PER_LAUNCH} events, "
                      "pinned host inputs, results read from pinned buffers",
               "runs_clusters_per_s": [world * n * k_e2e / x for x in srv_runs],
               "h2d_link_gbs": h2d_gbs,
               "link_bound_clusters_per_s": world * h2d_gbs * 1e9 / 12.0,
               "frac_of_link_bound": (world * n * k_e2e / srv_s) / (world * h2d_gbs * 1e9 / 12.0),
               "one_event_calls": {"value": world * n * k_e2e / seq_s, "unit": UNIT,
                                   "api": "tpc_track_event, one call per event"}}

    served = None
    if not args.no_served and rank == 0:
        try:
            served = served_vs_one(tp, torch, [hc], geom, bz, n)
        except Exception as e:  # reported, the bench line still goes out
            served = {"error": repr(e)}
        try:
            if args.served_sweep == "full":  # rates and lengths of config 4
                rates = (10, 20, 50, 100, 200, 500, 1000, 2000)
                n_of = lambda lam: int(min(2000, 30 * lam))
            else:
                rates = (100, 500, 1000, 2000)
                n_of = lambda lam: int(min(300, 10 * lam))
            served["stream"] = served_sweep(tp, torch, synth, rates, n_of)
        except Exception as e:
            served["stream"] = {"error": repr(e)}

    batched = None
    if not args.no_batched and rank == 0:
        try:
            batched = batched_vs_sequential(tp, torch, synth, stream)
        except Exception as e:  # reported, the bench line still goes out
            batched = {"error": repr(e)}

    pileup = None
    if not args.no_pileup and rank == 0:
        try:
            pileup = pileup_section(tp, torch, synth, stream)
        except Exception as e:  # reported, the bench line still goes out
            pileup = {"error": repr(e)}

    merged = None
    if not args.no_merge and rank == 0:
        try:
            merged = merge_section(tp, torch, synth, stream, cls, ev, geom, bz, n, ms_step / epl,
                                   steps=max(20, min(200, args.steps)), tune=not args.no_autotune)
        except Exception as e:  # reported, the bench line still goes out
            merged = {"error": repr(e)}

    side_task = None
    if not args.no_served and rank == 0:
        try:
            side_task = async_section(tp, torch, hc, geom, bz, n)
        except Exception as e:  # reported, the bench line still goes out
            side_task = {"error": repr(e)}

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        cpu = cpu_baseline(ev)

    tp.tpc_track_destroy(ctx)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "clusters_per_event": n,
                       "events_per_launch": epl, "clusters_per_step": n_step,
                       "events_per_launch_sweep": epl_sweep,
                       "l2": f"inputs rotate over {N_COPIES} device copies "
                             f"({N_COPIES * 12 * n / 1e6:.0f} MB) > 126 MB L2; each event "
                             "also writes ~150 MB of intermediate arrays",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "launch": f"one CUDA graph per step ({len(ktimes)} kernels) over {epl} "
                                 f"central event(s) side by side (events per launch picked "
                                 f"by a timed burst of each of {list(EPL_CANDIDATES)}); "
                                 f"consecutive steps spread over {n_streams} stream(s) so that "
                                 "their kernels run concurrently (autotuned); kernel times from "
                                 "a separate pass with kernels launched one by one on one stream",
                       "schedule": schedule,
                       "tracks_per_event": counters["n_tracks"] / epl,
                       "tracklets_per_event": counters["n_tracklets"] / epl,
                       "fullest_row_hits": counters["max_row_hits"],
                       "fullest_sector_tracks": counters["max_sector_tracks"]},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                         "traffic": traffic_for(dom, counters),
                         "algorithmic_bytes_per_launch": dom_bytes,
                         "algorithmic_bytes_per_cluster": stage_bytes_per_cluster(dom),
                         "stage": KERNEL_STAGE[dom], "launch_ms": dom_ms,
                         "stages": stage_rooflines(ktimes, n_step, peak),
                         "impl_bytes_per_launch": kb[dom],
                         "frac_impl_bytes": kb[dom] / (dom_ms * 1e-3) / 1e9 / peak},
            "path_roofline": {"bytes_per_cluster": PATH_BYTES,
                              "clusters_per_s_at_peak": peak * 1e9 / PATH_BYTES,
                              "frac": value / world / (peak * 1e9 / PATH_BYTES),
                              "target_frac": ROOFLINE_TARGET,
                              "meets_target": value / world / (peak * 1e9 / PATH_BYTES)
                              >= ROOFLINE_TARGET,
                              "impl_bytes_per_cluster": b_impl,
                              "frac_impl_bytes": value / world / (peak * 1e9 / b_impl),
                              "io_bytes_per_cluster": io_b,
                              "io_bound_clusters_per_s": peak * 1e9 / io_b},
            "kernels_ms": {k: v[0] / v[1] for k, v in ktimes.items()},
            "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(),
            "cpu_baseline": cpu, "served": served, "batched": batched, "pileup": pileup,
            "side_task": side_task, "merge": merged,
            "streams_ms_per_event": streams_sweep,
        }
        # last key (a driver that keeps the tail of the line keeps it): served
        # against one event at a time at equal p99, and the roofline fractions
        line["served_summary"] = served_summary(served, line)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


REF_MAX_STEPS = 120


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1712_09416_b300 import synth
    from oracle import oracle
    oracle.build()
    ev = synth.central_event(seed=2)
    sectors = [0, 9, 18, 27]
    sub = ev.select_sectors(sectors)
    for _ in range(args.warmup if args.warmup < 1 else 1):
        oracle.track_event(sub.select_sectors([0]))
    # one sector per step (~0.5 s of one core); at most REF_MAX_STEPS steps so
    # that the arm stays within about a minute whatever --steps asks for
    steps = min(args.steps, REF_MAX_STEPS)
    t0 = time.perf_counter()
    n_total = 0
    for i in range(steps):
        s = sub.select_sectors([sectors[i % len(sectors)]])
        oracle.track_event(s)
        n_total += s.n
    dt = time.perf_counter() - t0
    v = n_total / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": steps, "steps_requested": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "clusters_per_event": ev.n,
                       "sample": "each step tracks one of sectors 0, 9, 18, 27 of the event"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{steps} single sectors of the central event, "
                                       "single-threaded"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-pileup", action="store_true")
    ap.add_argument("--no-merge", action="store_true", help="skip the sector track merger section")
    ap.add_argument("--no-autotune", action="store_true",
                    help="default schedule, one stream (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-input runs (profiling)")
    ap.add_argument("--served-sweep", default="short", choices=["short", "full"],
                    help="event-stream sweep: 4 rates x <=300 events (short) or the 8 rates "
                         "10-2000/s with 30 s or 2000 events each (full)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--events-per-launch", type=int, default=0,
                    help="central events per timed launch (0: pick from %s by a timed burst)"
                         % (EPL_CANDIDATES,))
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        log("warmup raised to 3")
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
