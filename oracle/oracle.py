"""ctypes front end of the plain FP64 CPU oracle (``tpc_oracle.c``).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` import this module.  It shares no code with the
CUDA tracker in the package.

The C file follows the per-sector cellular-automaton track finder and Kalman
track fit named in the paper's Abstract and Sect. 4 (the steps themselves are
readings; each C function states its rule).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

TIE_CHI2_CUT, TIE_CHI2_PAIR, TIE_SIN, TIE_EDGE, TIE_CHAIN = 1, 2, 4, 8, 512
C2_TIE_PAIR, C2_TIE_CUT, C2_TIE_WIN = 1, 2, 4
MTIE_CUT, MTIE_PAIR, MTIE_DX, MTIE_SIN = 16, 32, 64, 128


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (binary64, no contraction of a*b+c)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_track_event.restype = C.c_int
        _lib.orc_transport_packed.restype = C.c_int
        _lib.orc_update_packed.restype = C.c_double
        _lib.orc_fit_fixed.restype = C.c_int
        _lib.orc_rotate_packed.restype = C.c_int
        _lib.orc_merge.restype = C.c_int
    return _lib


class OrcConfig(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "half_angle", "z_max", "bz", "sigma_y", "sigma_z", "chi2_hit", "sin_max", "edge_margin",
        "seed_var_s", "seed_var_t", "seed_var_q", "tie_chi2", "tie_sin", "tie_edge", "tie_d",
        "tie_win")] + \
        [(n, C.c_float) for n in ("slope_win_y", "slope_win_z", "d_max", "pad0")] + \
        [(n, C.c_int32) for n in ("n_rows", "n_sectors_phi", "split_z", "max_gap", "min_chain",
                                  "min_tracklet_hits", "min_track_hits", "pad1")]


_P = C.c_void_p


class OrcResult(C.Structure):
    _fields_ = [("up", _P), ("dn", _P), ("c2_tie", _P), ("up32", _P), ("dn32", _P),
                ("fwd_mark", _P), ("up_c", _P), ("dn_c", _P),
                ("cap_tracklets", C.c_int64),
                ("t_start", _P), ("t_sector", _P), ("t_chain_len", _P), ("t_valid", _P),
                ("t_nhits", _P), ("t_first_row", _P), ("t_last_row", _P), ("t_flags", _P),
                ("t_ndf", _P), ("t_x", _P), ("t_p", _P), ("t_C", _P), ("t_chi2", _P),
                ("t_rowhit", _P), ("weight", _P), ("cap_tracks", C.c_int64),
                ("k_tracklet", _P), ("k_sector", _P), ("k_ndf", _P), ("k_x", _P), ("k_p", _P),
                ("k_C", _P), ("k_chi2", _P), ("k_hit_off", _P), ("k_hit_cid", _P),
                ("n_tracklets", C.c_int64), ("n_tracks", C.c_int64), ("n_track_hits", C.c_int64),
                ("n_links", C.c_int64), ("n_link_flips32", C.c_int64), ("n_c2_ties", C.c_int64),
                ("n_starts", C.c_int64), ("n_dominated", C.c_int64)]


@dataclass
class Params:
    """Tracker parameters (the same defaults as the GPU library's)."""
    sigma_y: float = 0.1
    sigma_z: float = 0.1
    slope_win_y: float = 2.0
    slope_win_z: float = 2.0
    d_max: float = 0.6
    chi2_hit: float = 16.0
    max_gap: int = 5
    min_chain: int = 3
    min_tracklet_hits: int = 10
    min_track_hits: int = 10
    sin_max: float = 0.99
    edge_margin: float = 2.0
    seed_var_s: float = 1.0
    seed_var_t: float = 1.0
    seed_var_q: float = 100.0
    tie_chi2: float = 0.05
    tie_sin: float = 1e-4
    tie_edge: float = 1e-3
    tie_d: float = 1e-4
    tie_win: float = 2e-5


def make_config(params: Params, *, n_rows: int, n_sectors_phi: int, split_z: int,
                half_angle: float, z_max: float, bz: float) -> OrcConfig:
    c = OrcConfig()
    c.half_angle, c.z_max, c.bz = half_angle, z_max, bz
    c.sigma_y, c.sigma_z = params.sigma_y, params.sigma_z
    c.chi2_hit, c.sin_max, c.edge_margin = params.chi2_hit, params.sin_max, params.edge_margin
    c.seed_var_s, c.seed_var_t, c.seed_var_q = params.seed_var_s, params.seed_var_t, params.seed_var_q
    c.tie_chi2, c.tie_sin, c.tie_edge = params.tie_chi2, params.tie_sin, params.tie_edge
    c.tie_d, c.tie_win = params.tie_d, params.tie_win
    c.slope_win_y, c.slope_win_z, c.d_max = params.slope_win_y, params.slope_win_z, params.d_max
    c.n_rows, c.n_sectors_phi, c.split_z = n_rows, n_sectors_phi, int(split_z)
    c.max_gap, c.min_chain = params.max_gap, params.min_chain
    c.min_tracklet_hits, c.min_track_hits = params.min_tracklet_hits, params.min_track_hits
    return c


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def track_event(ev, params: Params | None = None, *, shadow32: bool = False) -> dict:
    """Run C2-C8 on one event; returns every stage's arrays as numpy (cids).

    ``up``/``dn`` are the binary64 neighbour decision and ``c2_tie`` its
    near-tie bits per hit; with shadow32 the binary32 restatement of the same
    rule is returned too (``up32``/``dn32``, diagnostic only)."""
    params = params or Params()
    n = int(ev.n)
    R = len(ev.row_x)
    cfg = make_config(params, n_rows=R, n_sectors_phi=ev.n_sectors_phi, split_z=ev.split_z,
                      half_angle=ev.half_angle, z_max=ev.z_max, bz=ev.bz)
    y = np.ascontiguousarray(ev.y, dtype=np.float32)
    z = np.ascontiguousarray(ev.z, dtype=np.float32)
    row = np.ascontiguousarray(ev.row, dtype=np.uint16)
    sector = np.ascontiguousarray(ev.sector, dtype=np.uint16)
    row_x = np.ascontiguousarray(ev.row_x, dtype=np.float32)
    cap_t = max(16, n // 2)
    cap_k = cap_t
    o = {
        "up": np.empty(n, np.int32), "dn": np.empty(n, np.int32),
        "c2_tie": np.empty(n, np.int32),
        "fwd_mark": np.empty(n, np.int32),
        "up32": np.empty(n, np.int32) if shadow32 else None,
        "dn32": np.empty(n, np.int32) if shadow32 else None,
        "up_c": np.empty(n, np.int32), "dn_c": np.empty(n, np.int32),
        "t_start": np.empty(cap_t, np.int32), "t_sector": np.empty(cap_t, np.int32),
        "t_chain_len": np.empty(cap_t, np.int32), "t_valid": np.empty(cap_t, np.int32),
        "t_nhits": np.empty(cap_t, np.int32), "t_first_row": np.empty(cap_t, np.int32),
        "t_last_row": np.empty(cap_t, np.int32), "t_flags": np.empty(cap_t, np.int32),
        "t_ndf": np.empty(cap_t, np.int32), "t_x": np.empty(cap_t, np.float64),
        "t_p": np.empty((cap_t, 5), np.float64), "t_C": np.empty((cap_t, 15), np.float64),
        "t_chi2": np.empty(cap_t, np.float64), "t_rowhit": np.empty((cap_t, R), np.int32),
        "weight": np.empty(n, np.uint64),
        "k_tracklet": np.empty(cap_k, np.int32), "k_sector": np.empty(cap_k, np.int32),
        "k_ndf": np.empty(cap_k, np.int32), "k_x": np.empty(cap_k, np.float64),
        "k_p": np.empty((cap_k, 5), np.float64), "k_C": np.empty((cap_k, 15), np.float64),
        "k_chi2": np.empty(cap_k, np.float64), "k_hit_off": np.empty(cap_k + 1, np.int32),
        "k_hit_cid": np.empty(max(n, 1), np.int32),
    }
    res = OrcResult()
    for k, a in o.items():
        setattr(res, k, _ptr(a) if a is not None else None)
    res.cap_tracklets, res.cap_tracks = cap_t, cap_k
    rc = lib().orc_track_event(C.byref(cfg), _ptr(row_x), C.c_int64(n), _ptr(y), _ptr(z),
                               _ptr(row), _ptr(sector), C.byref(res))
    if rc != 0:
        raise RuntimeError(f"oracle returned {rc}")
    nt, nk, nh = res.n_tracklets, res.n_tracks, res.n_track_hits
    out = {"status": rc, "n_tracklets": nt, "n_tracks": nk, "n_track_hits": nh,
           "n_links": res.n_links, "n_link_flips32": res.n_link_flips32,
           "n_c2_ties": res.n_c2_ties, "n_dominated": res.n_dominated,
           "n_starts": res.n_starts}
    for k, a in o.items():
        if a is None:
            continue
        if k.startswith("t_"):
            a = a[:nt]
        elif k == "k_hit_off":
            a = a[:nk + 1]
        elif k == "k_hit_cid":
            a = a[:nh]
        elif k.startswith("k_"):
            a = a[:nk]
        out[k] = a
    return out


def transport(x0: float, x1: float, p, Ct, *, bz: float = 0.5, sin_max: float = 0.99):
    """C5 on one state. Returns (rc, p1, C1 packed, J 5x5)."""
    p = np.array(p, dtype=np.float64)
    Ct = np.array(Ct, dtype=np.float64)
    J = np.zeros((5, 5))
    rc = lib().orc_transport_packed(C.c_double(x0), C.c_double(x1), C.c_double(bz),
                                    C.c_double(sin_max), _ptr(p), _ptr(Ct), _ptr(J))
    return rc, p, Ct, J


def update(p, Ct, my: float, mz: float, vy: float, vz: float):
    """C6 on one state. Returns (p1, C1 packed, chi2 increment)."""
    p = np.array(p, dtype=np.float64)
    Ct = np.array(Ct, dtype=np.float64)
    chi2 = lib().orc_update_packed(_ptr(p), _ptr(Ct), C.c_double(my), C.c_double(mz),
                                   C.c_double(vy), C.c_double(vz))
    return p, Ct, chi2


def fit_fixed(row_x, rows, hy, hz, *, n_iter: int = 0, params: Params | None = None,
              bz: float = 0.5, n_rows: int | None = None):
    """C7 passes on a given hit set (no search), then n_iter C9 passes."""
    params = params or Params()
    xr = np.ascontiguousarray(row_x, dtype=np.float64)
    cfg = make_config(params, n_rows=n_rows or len(xr), n_sectors_phi=1, split_z=0,
                      half_angle=np.radians(10.0), z_max=250.0, bz=bz)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    hy = np.ascontiguousarray(hy, dtype=np.float64)
    hz = np.ascontiguousarray(hz, dtype=np.float64)
    p = np.zeros(5)
    Ct = np.zeros(15)
    chi2 = C.c_double()
    ndf = C.c_int32()
    rc = lib().orc_fit_fixed(C.byref(cfg), _ptr(xr), C.c_int(len(rows)), _ptr(rows), _ptr(hy),
                             _ptr(hz), C.c_int(n_iter), _ptr(p), _ptr(Ct), C.byref(chi2),
                             C.byref(ndf))
    return rc, p, Ct, chi2.value, ndf.value


def seed(x0, y0, z0, x1, y1, z1) -> np.ndarray:
    """C7 seed state from the first and last hit of a chain."""
    p = np.zeros(5)
    lib().orc_seed(*[C.c_double(v) for v in (x0, y0, z0, x1, y1, z1)], _ptr(p))
    return p


def unpack_cov(Ct) -> np.ndarray:
    """15 lower-triangle entries (row order) -> symmetric 5x5."""
    M = np.zeros((5, 5))
    k = 0
    for i in range(5):
        for j in range(i + 1):
            M[i, j] = M[j, i] = Ct[k]
            k += 1
    return M


def pack_cov(M) -> np.ndarray:
    return np.array([M[i, j] for i in range(5) for j in range(i + 1)], dtype=np.float64)


# --------------------------------------------------------------------------
# M: sector track merger and global refit (rules M0-M5 in tpc_oracle.c)
# --------------------------------------------------------------------------

@dataclass
class MergeParams:
    """Merger parameters (the same defaults as the GPU library's)."""
    chi2_cut: float = 30.0
    dx_lo: float = -5.0
    dx_hi: float = 30.0
    tie_chi2: float = 1.0
    tie_dx: float = 1e-3


class OrcMergeConfig(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("chi2_cut", "dx_lo", "dx_hi", "tie_chi2", "tie_dx")]


def rotate(d: float, x: float, p, Ct, *, bz: float = 0.5, sin_max: float = 0.99):
    """M0 on one state.  Returns (rc, x1, p1, C1 packed, J 5x5)."""
    xx = C.c_double(x)
    p = np.array(p, dtype=np.float64)
    Ct = np.array(Ct, dtype=np.float64)
    J = np.zeros((5, 5))
    rc = lib().orc_rotate_packed(C.c_double(d), C.c_double(bz), C.c_double(sin_max),
                                 C.byref(xx), _ptr(p), _ptr(Ct), _ptr(J))
    return rc, xx.value, p, Ct, J


def merge_tracks(ev, o: dict, params: Params | None = None, mparams: MergeParams | None = None) -> dict:
    """M1-M5 on the sector tracks o of event ev (from track_event).

    Returns the per-track link arrays and the merged track list: every chain
    head with a successful refit replaces its chain, the other tracks stay as
    they are, in the order of the sector tracks (a merged track takes its
    head's place); hits segment by segment, inner to outer."""
    params = params or Params()
    mparams = mparams or MergeParams()
    R = len(ev.row_x)
    cfg = make_config(params, n_rows=R, n_sectors_phi=ev.n_sectors_phi, split_z=ev.split_z,
                      half_angle=ev.half_angle, z_max=ev.z_max, bz=ev.bz)
    mc = OrcMergeConfig(mparams.chi2_cut, mparams.dx_lo, mparams.dx_hi, mparams.tie_chi2,
                        mparams.tie_dx)
    T = int(o["n_tracks"])
    y = np.ascontiguousarray(ev.y, dtype=np.float32)
    z = np.ascontiguousarray(ev.z, dtype=np.float32)
    row = np.ascontiguousarray(ev.row, dtype=np.uint16)
    row_x = np.ascontiguousarray(ev.row_x, dtype=np.float32)
    sec = np.ascontiguousarray(o["k_sector"], dtype=np.int32)
    tx = np.ascontiguousarray(o["k_x"], dtype=np.float64)
    tp = np.ascontiguousarray(o["k_p"], dtype=np.float64)
    tC = np.ascontiguousarray(o["k_C"], dtype=np.float64)
    off = np.ascontiguousarray(o["k_hit_off"], dtype=np.int32)
    cid = np.ascontiguousarray(o["k_hit_cid"], dtype=np.int32)
    n1 = max(T, 1)
    r = {"link_out": np.empty(n1, np.int32), "flags": np.empty(n1, np.int32),
         "match_chi2": np.empty(n1), "chain_head": np.empty(n1, np.int32),
         "m_x": np.zeros(n1), "m_p": np.zeros((n1, 5)), "m_C": np.zeros((n1, 15)),
         "m_chi2": np.zeros(n1), "m_ndf": np.zeros(n1, np.int32), "m_ok": np.zeros(n1, np.int32),
         "m_len": np.zeros(n1, np.int32)}
    rc = lib().orc_merge(C.byref(cfg), C.byref(mc), _ptr(row_x), _ptr(y), _ptr(z), _ptr(row),
                         C.c_int64(T), _ptr(sec), _ptr(tx), _ptr(tp), _ptr(tC), _ptr(off), _ptr(cid),
                         *[_ptr(r[k]) for k in ("link_out", "flags", "match_chi2", "chain_head",
                                                "m_x", "m_p", "m_C", "m_chi2", "m_ndf", "m_ok",
                                                "m_len")])
    if rc != 0:
        raise RuntimeError(f"oracle merge returned {rc}")
    r = {k: v[:T] for k, v in r.items()}
    # the merged track list
    out_sec, out_x, out_p, out_C, out_chi2, out_ndf, out_hits, out_src = [], [], [], [], [], [], [], []
    for a in range(T):
        h = r["chain_head"][a]
        if h != a:
            continue  # absorbed into an earlier head's chain
        if r["m_ok"][a]:
            segs, b = [], a
            while b >= 0:
                segs.append(b)
                b = r["link_out"][b]
            hits = np.concatenate([cid[off[g]:off[g + 1]] for g in segs])
            out_x.append(r["m_x"][a]); out_p.append(r["m_p"][a]); out_C.append(r["m_C"][a])
            out_chi2.append(r["m_chi2"][a]); out_ndf.append(r["m_ndf"][a])
            out_src.append(segs)
        else:
            hits = cid[off[a]:off[a + 1]]
            out_x.append(tx[a]); out_p.append(tp[a]); out_C.append(tC[a])
            out_chi2.append(o["k_chi2"][a]); out_ndf.append(o["k_ndf"][a])
            out_src.append([a])
        out_sec.append(sec[a])
        out_hits.append(hits)
    hit_off = np.zeros(len(out_hits) + 1, np.int32)
    hit_off[1:] = np.cumsum([len(h) for h in out_hits])
    r.update({"n_tracks": len(out_hits), "k_sector": np.array(out_sec, np.int32),
              "k_x": np.array(out_x, np.float64), "k_p": np.array(out_p, np.float64).reshape(-1, 5),
              "k_C": np.array(out_C, np.float64).reshape(-1, 15),
              "k_chi2": np.array(out_chi2, np.float64), "k_ndf": np.array(out_ndf, np.int32),
              "k_hit_off": hit_off,
              "k_hit_cid": np.concatenate(out_hits).astype(np.int32) if out_hits else np.zeros(0, np.int32),
              "sources": out_src})
    return r
