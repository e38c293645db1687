"""Thin ctypes binding of libtpctrack.so (argument marshalling only).

The functions carry the names of the C ABI in ``include/tpctrack.h``; every
step of the tracking path runs in the library's CUDA kernels.  Inputs may be
numpy arrays (host memory) or CUDA torch tensors (device memory); outputs are
copied into numpy arrays.  Loading fails loudly if the library is missing: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtpctrack.so")

TPC_OK, TPC_EINVAL, TPC_ENOMEM, TPC_ECUDA, TPC_ECAPACITY, TPC_ETIMEOUT, TPC_EBUSY = 0, -1, -2, -3, -4, -5, -6
TPC_DUMP_LINKS, TPC_DUMP_CLEAN, TPC_DUMP_STARTS, TPC_DUMP_TRACKLETS, TPC_DUMP_WEIGHTS, TPC_DUMP_SORTED = 1, 2, 3, 4, 5, 6

EXPORTED = ["tpc_track_default_params", "tpc_track_create", "tpc_track_event", "tpc_track_batch",
            "tpc_track_launch", "tpc_track_results", "tpc_track_join", "tpc_track_submit", "tpc_track_poll",
            "tpc_track_release", "tpc_track_get_counters", "tpc_track_stream",
            "tpc_track_set_profiling", "tpc_track_kernel_times",
            "tpc_track_get_schedule", "tpc_track_set_schedule", "tpc_track_autotune",
            "tpc_track_debug_dump", "tpc_track_debug_dump_event", "tpc_track_set_debug_waits",
            "tpc_track_last_error",
            "tpc_track_destroy",
            "tpc_track_links_noalloc", "tpc_track_set_params", "tpc_track_get_params",
            "tpc_track_ticket_params", "tpc_async_create", "tpc_async_start", "tpc_async_poll",
            "tpc_async_get_stats", "tpc_async_destroy", "tpc_chi2_calib_create",
            "tpc_chi2_calib_add", "tpc_chi2_calib_poll", "tpc_chi2_calib_stats",
            "tpc_chi2_calib_destroy", "tpc_dispatch_create", "tpc_dispatch_create_custom",
            "tpc_dispatch_submit", "tpc_dispatch_poll", "tpc_dispatch_release",
            "tpc_dispatch_fail_instance", "tpc_dispatch_stats", "tpc_dispatch_destroy"]


class TpcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tpctrack error {code}: {msg}")
        self.code = code


class tpc_geometry(C.Structure):
    _fields_ = [("n_rows", C.c_int), ("row_x", C.POINTER(C.c_float)), ("n_sectors_phi", C.c_int),
                ("split_z", C.c_int), ("half_angle_rad", C.c_float), ("z_max", C.c_float)]


class tpc_clusters(C.Structure):
    _fields_ = [("n", C.c_int64), ("y", C.c_void_p), ("z", C.c_void_p), ("row", C.c_void_p),
                ("sector", C.c_void_p), ("on_device", C.c_int)]


class tpc_tracks(C.Structure):
    _fields_ = [("n_tracks", C.c_int64), ("sector", C.POINTER(C.c_int32)),
                ("x", C.POINTER(C.c_float)), ("param", C.POINTER(C.c_float)),
                ("cov", C.POINTER(C.c_float)), ("chi2", C.POINTER(C.c_float)),
                ("ndf", C.POINTER(C.c_int32)), ("hit_off", C.POINTER(C.c_int32)),
                ("hit_cid", C.POINTER(C.c_int32))]


class tpc_track_params(C.Structure):
    _fields_ = [("meas_sigma_y", C.c_float), ("meas_sigma_z", C.c_float),
                ("slope_win_y", C.c_float), ("slope_win_z", C.c_float), ("d_max", C.c_float),
                ("chi2_hit", C.c_float), ("max_gap", C.c_int), ("min_chain", C.c_int),
                ("min_tracklet_hits", C.c_int), ("min_track_hits", C.c_int),
                ("sin_max", C.c_float), ("edge_margin", C.c_float), ("seed_var_s", C.c_float),
                ("seed_var_t", C.c_float), ("seed_var_q", C.c_float), ("merge", C.c_int),
                ("merge_chi2", C.c_float), ("merge_dx_lo", C.c_float), ("merge_dx_hi", C.c_float)]


class tpc_track_config(C.Structure):
    _fields_ = [("device", C.c_int), ("mem_budget", C.c_size_t),
                ("max_clusters_per_event", C.c_int64), ("max_events_in_flight", C.c_int),
                ("cuda_stream", C.c_void_p), ("max_rows", C.c_int),
                ("max_events_per_launch", C.c_int), ("params", tpc_track_params)]


class tpc_track_counters(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "n_clusters", "n_rows_total", "n_bins", "n_links", "n_starts", "n_tracklets",
        "n_valid_tracklets", "n_tracklet_hits", "n_tracks", "n_track_hits", "n_chain_hits",
        "n_dominated_chains",
        "n_merge_links", "n_merge_chains", "n_sector_tracks", "max_row_hits", "max_sector_tracks",
        "n_crowded_hits")]


class tpc_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("total_ms", C.c_double), ("launches", C.c_int64)]


class tpc_track_schedule(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("n_sm", "tl_max_per_sm", "bin_blocks_per_sm",
                                       "sort_threads", "nb_threads", "tl_blocks_per_sm",
                                       "max_streams", "streams", "nb_mode")]


class tpc_dump_tracklet(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("start_cid", "sector", "valid", "nhits", "first_row",
                                         "last_row", "ndf", "pad")] + \
        [("x", C.c_float), ("param", C.c_float * 5), ("cov", C.c_float * 15), ("chi2", C.c_float)]


class tpc_async_stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("started", "finished", "refused", "queued", "running",
                                         "unpolled")] + \
        [("busy_ms", C.c_double), ("max_task_ms", C.c_double)]


class tpc_chi2_fit(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("first_event", "last_event", "n_events",
                                          "params_version")] + \
        [("n_tracks", C.c_int64), ("n_kept", C.c_int64), ("n_iter", C.c_int32), ("pad", C.c_int32),
         ("scale2", C.c_double)]


tpc_submit_fn = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(tpc_clusters), C.POINTER(tpc_geometry),
                            C.c_float, C.POINTER(C.c_uint64))
tpc_poll_fn = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_uint64, C.c_int, C.POINTER(tpc_tracks))
tpc_release_fn = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_uint64)


class tpc_instance_ops(C.Structure):
    _fields_ = [("submit", tpc_submit_fn), ("poll", tpc_poll_fn), ("release", tpc_release_fn)]


tpc_async_init_fn = C.CFUNCTYPE(C.c_int, C.c_void_p)
tpc_async_run_fn = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p))
tpc_async_drop_fn = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

_lib = None


def lib():
    """Load libtpctrack.so (it must have been built; see build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_1712_09416_b300.build`")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.tpc_track_create.argtypes = [C.POINTER(tpc_track_config), C.POINTER(P)]
        L.tpc_track_event.argtypes = [P, C.POINTER(tpc_clusters), C.POINTER(tpc_geometry), C.c_float,
                                      C.POINTER(tpc_tracks)]
        L.tpc_track_batch.argtypes = [P, C.c_int, C.POINTER(tpc_clusters), C.POINTER(tpc_geometry),
                                      C.c_float, C.POINTER(tpc_tracks)]
        L.tpc_track_launch.argtypes = [P, C.c_int, C.POINTER(tpc_clusters), C.POINTER(tpc_geometry),
                                       C.c_float]
        L.tpc_track_results.argtypes = [P, C.c_int, C.POINTER(tpc_tracks)]
        L.tpc_track_join.argtypes = [P]
        L.tpc_track_submit.argtypes = [P, C.POINTER(tpc_clusters), C.POINTER(tpc_geometry), C.c_float,
                                       C.POINTER(C.c_uint64)]
        L.tpc_track_poll.argtypes = [P, C.c_uint64, C.c_int, C.POINTER(tpc_tracks)]
        L.tpc_track_release.argtypes = [P, C.c_uint64]
        L.tpc_track_get_counters.argtypes = [P, C.POINTER(tpc_track_counters)]
        L.tpc_track_stream.argtypes = [P]
        L.tpc_track_stream.restype = P
        L.tpc_track_set_profiling.argtypes = [P, C.c_int]
        L.tpc_track_kernel_times.argtypes = [P, C.POINTER(tpc_kernel_time), C.c_int,
                                             C.POINTER(C.c_int)]
        L.tpc_track_get_schedule.argtypes = [P, C.POINTER(tpc_track_schedule)]
        L.tpc_track_set_schedule.argtypes = [P, C.POINTER(tpc_track_schedule)]
        L.tpc_track_autotune.argtypes = [P, C.c_int, C.POINTER(tpc_clusters),
                                         C.POINTER(tpc_geometry), C.c_float, C.c_int,
                                         C.POINTER(tpc_track_schedule)]
        L.tpc_track_debug_dump.argtypes = [P, C.c_int, P, C.c_size_t, C.POINTER(C.c_size_t)]
        L.tpc_track_debug_dump_event.argtypes = [P, C.c_int, C.c_int, P, C.c_size_t,
                                                 C.POINTER(C.c_size_t)]
        L.tpc_track_set_debug_waits.argtypes = [P, C.c_int64, C.c_int32]
        L.tpc_track_last_error.argtypes = [P]
        L.tpc_track_last_error.restype = C.c_char_p
        L.tpc_track_destroy.argtypes = [P]
        L.tpc_track_destroy.restype = None
        L.tpc_track_links_noalloc.argtypes = [C.POINTER(tpc_clusters), C.POINTER(tpc_geometry),
                                              C.POINTER(tpc_track_params), P, P, P]
        L.tpc_track_default_params.argtypes = [C.POINTER(tpc_track_params)]
        L.tpc_track_default_params.restype = None
        L.tpc_track_set_params.argtypes = [P, C.POINTER(tpc_track_params), C.POINTER(C.c_uint64),
                                           C.POINTER(C.c_uint64)]
        L.tpc_track_get_params.argtypes = [P, C.POINTER(tpc_track_params), C.POINTER(C.c_uint64)]
        L.tpc_track_ticket_params.argtypes = [P, C.c_uint64, C.POINTER(tpc_track_params),
                                              C.POINTER(C.c_uint64)]
        L.tpc_async_create.argtypes = [tpc_async_init_fn, tpc_async_run_fn, tpc_async_drop_fn, P,
                                       C.c_int, C.POINTER(P)]
        L.tpc_async_start.argtypes = [P, P, C.POINTER(C.c_uint64)]
        L.tpc_async_poll.argtypes = [P, C.c_int, C.POINTER(C.c_uint64), C.POINTER(P),
                                     C.POINTER(C.c_int)]
        L.tpc_async_get_stats.argtypes = [P, C.POINTER(tpc_async_stats)]
        L.tpc_async_destroy.argtypes = [P]
        L.tpc_async_destroy.restype = None
        L.tpc_chi2_calib_create.argtypes = [C.c_int, C.c_double, C.c_int, C.POINTER(P)]
        L.tpc_chi2_calib_add.argtypes = [P, C.POINTER(tpc_tracks), C.c_uint64]
        L.tpc_chi2_calib_poll.argtypes = [P, C.c_int, C.POINTER(tpc_chi2_fit)]
        L.tpc_chi2_calib_stats.argtypes = [P, C.POINTER(tpc_async_stats)]
        L.tpc_chi2_calib_destroy.argtypes = [P]
        L.tpc_chi2_calib_destroy.restype = None
        L.tpc_dispatch_create.argtypes = [C.POINTER(C.c_int), C.c_int, C.POINTER(tpc_track_config),
                                          C.POINTER(C.c_void_p)]
        L.tpc_dispatch_create_custom.argtypes = [C.POINTER(tpc_instance_ops), C.POINTER(C.c_void_p),
                                                 C.c_int, C.POINTER(C.c_void_p)]
        L.tpc_dispatch_submit.argtypes = [P, C.POINTER(tpc_clusters), C.POINTER(tpc_geometry),
                                          C.c_float, C.POINTER(C.c_uint64)]
        L.tpc_dispatch_poll.argtypes = [P, C.c_uint64, C.c_int, C.POINTER(tpc_tracks)]
        L.tpc_dispatch_release.argtypes = [P, C.c_uint64]
        L.tpc_dispatch_fail_instance.argtypes = [P, C.c_int]
        L.tpc_dispatch_stats.argtypes = [P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                         C.POINTER(C.c_int64)]
        L.tpc_dispatch_destroy.argtypes = [P]
        L.tpc_dispatch_destroy.restype = None
        _lib = L
    return _lib


# --------------------------------------------------------------------------
# marshalling helpers
# --------------------------------------------------------------------------

def geometry_of(ev) -> tuple[tpc_geometry, np.ndarray]:
    """tpc_geometry of an event record (row_x kept alive by the caller)."""
    row_x = np.ascontiguousarray(ev.row_x, dtype=np.float32)
    g = tpc_geometry(len(row_x), row_x.ctypes.data_as(C.POINTER(C.c_float)), int(ev.n_sectors_phi),
                     int(ev.split_z), float(ev.half_angle), float(ev.z_max))
    return g, row_x


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def clusters_of(y, z, row, sector) -> tuple[tpc_clusters, list]:
    """tpc_clusters for numpy (host) or CUDA torch (device) arrays."""
    if _is_torch(y):
        import torch
        keep = [y.contiguous(), z.contiguous(), row.contiguous(), sector.contiguous()]
        assert keep[0].dtype == torch.float32 and keep[1].dtype == torch.float32
        assert keep[2].dtype in (torch.int16, torch.uint16) and keep[3].dtype in (torch.int16, torch.uint16)
        on_dev = 1 if keep[0].is_cuda else 0
        ptrs = [k.data_ptr() for k in keep]
        n = keep[0].numel()
    else:
        keep = [np.ascontiguousarray(y, dtype=np.float32), np.ascontiguousarray(z, dtype=np.float32),
                np.ascontiguousarray(row, dtype=np.uint16), np.ascontiguousarray(sector, dtype=np.uint16)]
        on_dev = 0
        ptrs = [k.ctypes.data for k in keep]
        n = len(keep[0])
    c = tpc_clusters(n, ptrs[0], ptrs[1], ptrs[2], ptrs[3], on_dev)
    return c, keep


@dataclass
class Tracks:
    sector: np.ndarray
    x: np.ndarray
    param: np.ndarray
    cov: np.ndarray
    chi2: np.ndarray
    ndf: np.ndarray
    hit_off: np.ndarray
    hit_cid: np.ndarray

    @property
    def n_tracks(self) -> int:
        return len(self.sector)

    def hits(self, j: int) -> np.ndarray:
        return self.hit_cid[self.hit_off[j]:self.hit_off[j + 1]]


def tracks_to_numpy(t: tpc_tracks, copy: bool = True) -> Tracks:
    """numpy arrays of a result; copy=False gives views of the library's
    buffers, valid until the buffers are released or reused."""
    n = int(t.n_tracks)

    def arr(p, count, dt):
        if count == 0 or not p:
            return np.zeros(count, dtype=dt)
        a = np.ctypeslib.as_array(p, shape=(count,))
        return a.astype(dt, copy=True) if copy else a
    hit_off = arr(t.hit_off, n + 1, np.int32) if n else np.zeros(1, np.int32)
    nh = int(hit_off[-1]) if n else 0
    return Tracks(sector=arr(t.sector, n, np.int32), x=arr(t.x, n, np.float32),
                  param=arr(t.param, 5 * n, np.float32).reshape(n, 5),
                  cov=arr(t.cov, 15 * n, np.float32).reshape(n, 15),
                  chi2=arr(t.chi2, n, np.float32), ndf=arr(t.ndf, n, np.int32), hit_off=hit_off,
                  hit_cid=arr(t.hit_cid, nh, np.int32))


def _check(ctx, rc: int):
    if rc != TPC_OK:
        msg = lib().tpc_track_last_error(ctx).decode() if ctx else ""
        raise TpcError(rc, msg)


# --------------------------------------------------------------------------
# the C ABI, one Python function per entry point
# --------------------------------------------------------------------------

def tpc_track_default_params() -> tpc_track_params:
    p = tpc_track_params()
    lib().tpc_track_default_params(C.byref(p))
    return p


def _config(max_clusters_per_event: int, *, device: int = 0, mem_budget: int = 0,
            max_events_in_flight: int = 1, cuda_stream: int | None = None,
            max_rows: int = 159, max_events_per_launch: int = 64,
            params: tpc_track_params | None = None) -> tpc_track_config:
    cfg = tpc_track_config()
    cfg.device = device
    cfg.mem_budget = mem_budget
    cfg.max_clusters_per_event = int(max_clusters_per_event)
    cfg.max_events_in_flight = max_events_in_flight
    cfg.cuda_stream = cuda_stream
    cfg.max_rows = max_rows
    cfg.max_events_per_launch = max_events_per_launch
    cfg.params = params if params is not None else tpc_track_default_params()
    return cfg


def tpc_track_create(max_clusters_per_event: int, **kw):
    cfg = _config(max_clusters_per_event, **kw)
    ctx = C.c_void_p()
    rc = lib().tpc_track_create(C.byref(cfg), C.byref(ctx))
    if rc != TPC_OK:
        raise TpcError(rc, "tpc_track_create failed")
    return ctx


def tpc_track_event(ctx, clusters: tpc_clusters, geom: tpc_geometry, bz: float, *,
                    copy: bool = True) -> Tracks:
    """Track one event; copy=False returns views of the context's buffers,
    valid until its next call."""
    out = tpc_tracks()
    _check(ctx, lib().tpc_track_event(ctx, C.byref(clusters), C.byref(geom), bz, C.byref(out)))
    return tracks_to_numpy(out, copy)


def tpc_track_batch(ctx, clusters: list[tpc_clusters], geom: tpc_geometry, bz: float, *,
                    copy: bool = True) -> list[Tracks]:
    arr = (tpc_clusters * len(clusters))(*clusters)
    outs = (tpc_tracks * len(clusters))()
    _check(ctx, lib().tpc_track_batch(ctx, len(clusters), arr, C.byref(geom), bz, outs))
    return [tracks_to_numpy(o, copy) for o in outs]


def tpc_track_launch(ctx, clusters: list[tpc_clusters], geom: tpc_geometry, bz: float):
    arr = (tpc_clusters * len(clusters))(*clusters)
    _check(ctx, lib().tpc_track_launch(ctx, len(clusters), arr, C.byref(geom), bz))
    return arr


def tpc_track_results(ctx, n_ev: int, *, copy: bool = True):
    """Tracks of the oldest pending launch, which must have n_ev events or
    fewer (TPC_EINVAL otherwise, the launch staying pending)."""
    outs = (tpc_tracks * n_ev)()
    _check(ctx, lib().tpc_track_results(ctx, n_ev, outs))
    return [tracks_to_numpy(o) for o in outs] if copy else outs


def tpc_track_join(ctx):
    _check(ctx, lib().tpc_track_join(ctx))


def tpc_track_submit(ctx, clusters: tpc_clusters, geom: tpc_geometry, bz: float) -> int:
    t = C.c_uint64()
    _check(ctx, lib().tpc_track_submit(ctx, C.byref(clusters), C.byref(geom), bz, C.byref(t)))
    return t.value


def tpc_track_poll(ctx, ticket: int, timeout_us: int = -1, *, copy: bool = True) -> Tracks | None:
    """Tracks of a finished ticket (None while it runs); copy=False returns
    views of the ticket's buffers, valid until tpc_track_release."""
    out = tpc_tracks()
    rc = lib().tpc_track_poll(ctx, ticket, timeout_us, C.byref(out))
    if rc == TPC_EBUSY:
        return None
    _check(ctx, rc)
    return tracks_to_numpy(out, copy)


def tpc_track_release(ctx, ticket: int):
    _check(ctx, lib().tpc_track_release(ctx, ticket))


def tpc_track_get_counters(ctx) -> dict:
    c = tpc_track_counters()
    _check(ctx, lib().tpc_track_get_counters(ctx, C.byref(c)))
    return {k: int(getattr(c, k)) for k, _ in c._fields_}


def tpc_track_stream(ctx) -> int:
    return lib().tpc_track_stream(ctx) or 0


def tpc_track_set_profiling(ctx, on: bool):
    _check(ctx, lib().tpc_track_set_profiling(ctx, 1 if on else 0))


def tpc_track_kernel_times(ctx) -> dict:
    """{kernel name: (total ms, launches)} recorded since profiling was enabled."""
    arr = (tpc_kernel_time * 64)()
    n = C.c_int()
    _check(ctx, lib().tpc_track_kernel_times(ctx, arr, 64, C.byref(n)))
    return {arr[i].name.decode(): (arr[i].total_ms, int(arr[i].launches)) for i in range(n.value)}


def tpc_track_set_params(ctx, params: tpc_track_params) -> tuple[int, int]:
    """New parameter set from the next submitted event on; returns
    (first ticket tracked with it, its version)."""
    ft, ver = C.c_uint64(), C.c_uint64()
    _check(ctx, lib().tpc_track_set_params(ctx, C.byref(params), C.byref(ft), C.byref(ver)))
    return ft.value, ver.value


def tpc_track_get_params(ctx) -> tuple[tpc_track_params, int]:
    p, ver = tpc_track_params(), C.c_uint64()
    _check(ctx, lib().tpc_track_get_params(ctx, C.byref(p), C.byref(ver)))
    return p, ver.value


def tpc_track_ticket_params(ctx, ticket: int) -> tuple[tpc_track_params, int]:
    p, ver = tpc_track_params(), C.c_uint64()
    _check(ctx, lib().tpc_track_ticket_params(ctx, ticket, C.byref(p), C.byref(ver)))
    return p, ver.value


def _stats_dict(s: tpc_async_stats) -> dict:
    return {k: (float if k.endswith("_ms") else int)(getattr(s, k)) for k, _ in s._fields_}


class AsyncRunner:
    """A tpc_async runner whose jobs are Python callables (for tests and
    host-side tools; the callables run on the runner's thread)."""

    def __init__(self, max_unfinished: int = 1, init=None):
        self._jobs: dict[int, object] = {}
        self._results: dict[int, object] = {}
        self._n = 0
        self._init_py = init

        def _init(_user):
            return int(self._init_py()) if self._init_py else TPC_OK

        def _run(_user, job, result):
            k = int(job)
            fn = self._jobs.pop(k)
            try:
                self._results[k] = fn()
                rc = TPC_OK
            except Exception as e:  # noqa: BLE001 - the job's failure becomes its status
                self._results[k] = e
                rc = TPC_EINVAL
            result[0] = k
            return rc

        def _drop(_user, job, result):
            if job:
                self._jobs.pop(int(job), None)
            if result:
                self._results.pop(int(result), None)
        self._cb = (tpc_async_init_fn(_init), tpc_async_run_fn(_run), tpc_async_drop_fn(_drop))
        h = C.c_void_p()
        rc = lib().tpc_async_create(*self._cb, None, max_unfinished, C.byref(h))
        if rc != TPC_OK:
            raise TpcError(rc, "tpc_async_create")
        self.handle = h

    def start(self, fn) -> int | None:
        """Queue fn (never waits); its task id, or None if the runner is full."""
        self._n += 1
        self._jobs[self._n] = fn
        t = C.c_uint64()
        rc = lib().tpc_async_start(self.handle, C.c_void_p(self._n), C.byref(t))
        if rc == TPC_EBUSY:
            del self._jobs[self._n]
            return None
        if rc != TPC_OK:
            raise TpcError(rc, "tpc_async_start")
        return t.value

    def poll(self, timeout_us: int = 0):
        """(task id, status, value) of the oldest finished job, or None."""
        t, r, st = C.c_uint64(), C.c_void_p(), C.c_int()
        rc = lib().tpc_async_poll(self.handle, timeout_us, C.byref(t), C.byref(r), C.byref(st))
        if rc == TPC_EBUSY:
            return None
        if rc != TPC_OK:
            raise TpcError(rc, "tpc_async_poll")
        return t.value, st.value, self._results.pop(int(r.value), None)

    def stats(self) -> dict:
        s = tpc_async_stats()
        lib().tpc_async_get_stats(self.handle, C.byref(s))
        return _stats_dict(s)

    def close(self):
        if self.handle:
            lib().tpc_async_destroy(self.handle)
            self.handle = None


class Chi2Calib:
    """The built-in accumulate-then-fit side task (tpc_chi2_calib_*)."""

    def __init__(self, every_n_events: int, trim: float = 3.0, max_unfinished: int = 2):
        h = C.c_void_p()
        rc = lib().tpc_chi2_calib_create(every_n_events, trim, max_unfinished, C.byref(h))
        if rc != TPC_OK:
            raise TpcError(rc, "tpc_chi2_calib_create")
        self.handle = h

    def add(self, chi2: np.ndarray, ndf: np.ndarray, params_version: int = 0):
        """Accumulate one event's tracks (chi2 float32, ndf int32)."""
        c = np.ascontiguousarray(chi2, np.float32)
        d = np.ascontiguousarray(ndf, np.int32)
        t = tpc_tracks()
        t.n_tracks = len(c)
        t.chi2 = c.ctypes.data_as(C.POINTER(C.c_float))
        t.ndf = d.ctypes.data_as(C.POINTER(C.c_int32))
        rc = lib().tpc_chi2_calib_add(self.handle, C.byref(t), params_version)
        if rc != TPC_OK:
            raise TpcError(rc, "tpc_chi2_calib_add")

    def poll(self, timeout_us: int = 0) -> dict | None:
        f = tpc_chi2_fit()
        rc = lib().tpc_chi2_calib_poll(self.handle, timeout_us, C.byref(f))
        if rc == TPC_EBUSY:
            return None
        if rc != TPC_OK:
            raise TpcError(rc, "tpc_chi2_calib_poll")
        return {k: (float(getattr(f, k)) if k == "scale2" else int(getattr(f, k)))
                for k, _ in f._fields_ if k != "pad"}

    def stats(self) -> dict:
        s = tpc_async_stats()
        lib().tpc_chi2_calib_stats(self.handle, C.byref(s))
        return _stats_dict(s)

    def close(self):
        if self.handle:
            lib().tpc_chi2_calib_destroy(self.handle)
            self.handle = None


def _schedule_dict(s: tpc_track_schedule) -> dict:
    return {k: int(getattr(s, k)) for k, _ in s._fields_}


def tpc_track_get_schedule(ctx) -> dict:
    s = tpc_track_schedule()
    _check(ctx, lib().tpc_track_get_schedule(ctx, C.byref(s)))
    return _schedule_dict(s)


def tpc_track_set_schedule(ctx, **fields):
    """Change schedule fields by name (the others keep their values)."""
    s = tpc_track_schedule()
    _check(ctx, lib().tpc_track_get_schedule(ctx, C.byref(s)))
    for k, v in fields.items():
        setattr(s, k, int(v))
    _check(ctx, lib().tpc_track_set_schedule(ctx, C.byref(s)))


def save_schedule(ctx, path: str):
    """Write the context's schedule (for instance the autotuner's choice) as JSON."""
    import json
    with open(path, "w") as f:
        json.dump(tpc_track_get_schedule(ctx), f, indent=1)


def load_schedule(ctx, path: str) -> dict:
    """Apply a schedule written by save_schedule (the device fields n_sm,
    tl_max_per_sm and max_streams are read-only and ignored); returns it."""
    import json
    with open(path) as f:
        d = json.load(f)
    tpc_track_set_schedule(ctx, **{k: v for k, v in d.items()
                                   if k not in ("n_sm", "tl_max_per_sm", "max_streams")})
    return tpc_track_get_schedule(ctx)


def tpc_track_autotune(ctx, clusters: list[tpc_clusters], geom: tpc_geometry, bz: float,
                       reps: int = 3) -> dict:
    arr = (tpc_clusters * len(clusters))(*clusters)
    s = tpc_track_schedule()
    _check(ctx, lib().tpc_track_autotune(ctx, len(clusters), arr, C.byref(geom), bz, reps,
                                         C.byref(s)))
    return _schedule_dict(s)


def tpc_track_debug_dump(ctx, stage: int, event: int = 0) -> bytes:
    used = C.c_size_t()
    _check(ctx, lib().tpc_track_debug_dump_event(ctx, stage, event, None, 0, C.byref(used)))
    buf = C.create_string_buffer(max(1, used.value))
    _check(ctx, lib().tpc_track_debug_dump_event(ctx, stage, event, buf, used.value, C.byref(used)))
    return buf.raw[:used.value]


def tpc_track_set_debug_waits(ctx, spin_limit: int, stall_hit_tile: int = -1):
    """Bounded-wait test hook (see the header): poll limit of the look-back
    waits and a hit tile that never publishes, for the launches that follow."""
    _check(ctx, lib().tpc_track_set_debug_waits(ctx, spin_limit, stall_hit_tile))


def tpc_track_links_noalloc(clusters: tpc_clusters, geom: tpc_geometry,
                            params: tpc_track_params, up_cid_ptr: int, dn_cid_ptr: int,
                            stream: int = 0) -> int:
    """Neighbour links by cid into two device int32 arrays, without allocating.
    Returns the status code (the caller checks it)."""
    return lib().tpc_track_links_noalloc(C.byref(clusters), C.byref(geom), C.byref(params),
                                         up_cid_ptr, dn_cid_ptr, stream)


def tpc_track_last_error(ctx) -> str:
    return lib().tpc_track_last_error(ctx).decode()


def tpc_track_destroy(ctx):
    if ctx:
        lib().tpc_track_destroy(ctx)


# --------------------------------------------------------------------------
# decoded debug dumps
# --------------------------------------------------------------------------

def dump_links(ctx, n: int, clean: bool = False, event: int = 0) -> tuple[np.ndarray, np.ndarray]:
    b = np.frombuffer(tpc_track_debug_dump(ctx, TPC_DUMP_CLEAN if clean else TPC_DUMP_LINKS, event),
                      np.int32)
    return b[:n].copy(), b[n:2 * n].copy()


def dump_starts(ctx, event: int = 0) -> np.ndarray:
    return np.frombuffer(tpc_track_debug_dump(ctx, TPC_DUMP_STARTS, event), np.int32).copy()


def dump_weights(ctx, event: int = 0) -> np.ndarray:
    return np.frombuffer(tpc_track_debug_dump(ctx, TPC_DUMP_WEIGHTS, event), np.uint64).copy()


def dump_tracklets(ctx, n_rows: int, event: int = 0) -> dict:
    raw = tpc_track_debug_dump(ctx, TPC_DUMP_TRACKLETS, event)
    count = int(np.frombuffer(raw[:4], np.int32)[0])
    rec = C.sizeof(tpc_dump_tracklet) + 4 * n_rows
    hdr_dt = np.dtype([("start_cid", "<i4"), ("sector", "<i4"), ("valid", "<i4"), ("nhits", "<i4"),
                       ("first_row", "<i4"), ("last_row", "<i4"), ("ndf", "<i4"), ("pad", "<i4"),
                       ("x", "<f4"), ("param", "<f4", 5), ("cov", "<f4", 15), ("chi2", "<f4")])
    full_dt = np.dtype([("h", hdr_dt), ("rowhit", "<i4", n_rows)])
    assert full_dt.itemsize == rec
    a = np.frombuffer(raw[4:4 + count * rec], dtype=full_dt)
    h = a["h"]
    return {"start": h["start_cid"].copy(), "sector": h["sector"].copy(), "valid": h["valid"].copy(),
            "nhits": h["nhits"].copy(), "first_row": h["first_row"].copy(),
            "last_row": h["last_row"].copy(), "ndf": h["ndf"].copy(), "x": h["x"].copy(),
            "p": h["param"].copy(), "C": h["cov"].copy(), "chi2": h["chi2"].copy(),
            "rowhit": a["rowhit"].copy()}


class Dispatcher:
    """Round-robin dispatcher of whole events over tracker instances
    (tpc_dispatch_*): one context per listed device, or caller-made instances
    driven through Python callables (submit, poll, release) with the C
    signatures of tpc_instance_ops."""

    def __init__(self, devices=None, max_clusters_per_event: int = 0, *, ops=None,
                 instances=None, **kw):
        self.d = C.c_void_p()
        self._keep = []
        if ops is not None:
            cops = tpc_instance_ops(tpc_submit_fn(ops[0]), tpc_poll_fn(ops[1]),
                                    tpc_release_fn(ops[2]))
            arr = (C.c_void_p * len(instances))(*instances)
            self._keep += [cops, arr]
            rc = lib().tpc_dispatch_create_custom(C.byref(cops), arr, len(instances),
                                                  C.byref(self.d))
        else:
            cfg = _config(max_clusters_per_event, **kw)
            devs = (C.c_int * len(devices))(*devices)
            rc = lib().tpc_dispatch_create(devs, len(devices), C.byref(cfg), C.byref(self.d))
        if rc != TPC_OK:
            raise TpcError(rc, "tpc_dispatch_create failed")

    def submit(self, clusters: tpc_clusters, geom: tpc_geometry, bz: float) -> int:
        t = C.c_uint64()
        rc = lib().tpc_dispatch_submit(self.d, C.byref(clusters), C.byref(geom), bz, C.byref(t))
        if rc != TPC_OK:
            raise TpcError(rc, "tpc_dispatch_submit failed")
        return t.value

    def poll(self, ticket: int, timeout_us: int = -1, *, copy: bool = True):
        out = tpc_tracks()
        rc = lib().tpc_dispatch_poll(self.d, ticket, timeout_us, C.byref(out))
        if rc == TPC_EBUSY:
            return None
        if rc != TPC_OK:
            raise TpcError(rc, "tpc_dispatch_poll failed")
        return tracks_to_numpy(out, copy)

    def release(self, ticket: int):
        rc = lib().tpc_dispatch_release(self.d, ticket)
        if rc != TPC_OK:
            raise TpcError(rc, "tpc_dispatch_release failed")

    def fail_instance(self, k: int):
        rc = lib().tpc_dispatch_fail_instance(self.d, k)
        if rc != TPC_OK:
            raise TpcError(rc, "tpc_dispatch_fail_instance failed")

    def stats(self) -> dict:
        cap = 1024
        ev = (C.c_int64 * cap)()
        ok = (C.c_int32 * cap)()
        re = C.c_int64()
        n = lib().tpc_dispatch_stats(self.d, cap, ev, ok, C.byref(re))
        if n < 0:
            raise TpcError(n, "tpc_dispatch_stats failed")
        return {"events": list(ev[:n]), "healthy": [bool(x) for x in ok[:n]],
                "reissued": re.value}

    def close(self):
        if self.d:
            lib().tpc_dispatch_destroy(self.d)
            self.d = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Tracker:
    """Convenience owner of one context (closes it on exit)."""

    def __init__(self, max_clusters_per_event: int, **kw):
        self.ctx = tpc_track_create(max_clusters_per_event, **kw)

    def event(self, ev, *, device_arrays=None) -> Tracks:
        g, keep_x = geometry_of(ev)
        arrays = device_arrays if device_arrays is not None else (ev.y, ev.z, ev.row, ev.sector)
        c, keep = clusters_of(*arrays)
        return tpc_track_event(self.ctx, c, g, float(ev.bz))

    def batch(self, evs, *, device_arrays=None) -> list[Tracks]:
        g, keep_x = geometry_of(evs[0])
        cs, keep = [], []
        for i, ev in enumerate(evs):
            arrays = device_arrays[i] if device_arrays is not None else (ev.y, ev.z, ev.row, ev.sector)
            c, k = clusters_of(*arrays)
            cs.append(c)
            keep.append(k)
        return tpc_track_batch(self.ctx, cs, g, float(evs[0].bz))

    def counters(self) -> dict:
        return tpc_track_get_counters(self.ctx)

    def close(self):
        if self.ctx:
            tpc_track_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
