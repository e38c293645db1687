"""GPU-vs-oracle comparison helpers for the parity tests.

Bars (the tracker computes in binary32, the oracle in binary64):
* links: the kernel's link of every hit equals the oracle's binary64
  decision, except at hits the oracle marks as near ties of that decision
  (the best pair within 1e-4 in D of the next pair or of D_MAX, or a
  candidate within 2e-5 cm of a slope-window edge); links that differ there
  must stay below 0.1% of the links.  Cleaned links and start hits are then
  identical at every hit whose own link and whose partners' links are not
  near ties; a chain through such a hit may differ, and its tracklet is
  treated like a flagged one below;
* tracklet hit sets and validity: identical for every tracklet the oracle
  does not flag as a near-tie (a chi2 within the tie width of the cut or of
  the runner-up, |sin phi| near its bound, a stop bound, or a chain through
  a neighbour near tie); flagged tracklets may differ, and so may the
  dominance of a chain one of whose hits a flagged forward pass took (the
  chain is then built on one side only); those that differ must stay below
  0.1% of all tracklets; the hits of the tracklets that differ (on either
  side) are the taint of the track comparison;
* parameters at the innermost hit: |dy|, |dz| <= 1e-3 cm; |d sin phi|,
  |d tan lambda| <= 1e-4 (relative to values of order one); q/pT within
  1e-4 relative to max(|q/pT|, 2 (GeV/c)^-1): stiff tracks have |q/pT| near
  0, where a purely relative bar has no meaning.  Every compared tracklet
  and track stays within these bars (no budget).  This holds because the
  tracker's backward pass carries a square-root factor of the covariance:
  storing the covariance itself in binary32 moves q/pT of short, curved
  tracks past the bar (tests/test_fp32_covariance_limit.py), and with the
  standard update the worst tracklet of the pile-up event sat at 8x to 67x
  the q/pT bar depending only on how the compiler contracted its binary32
  arithmetic.  The share of tracks within the plain bars (q/pT 1e-4
  relative with no floor) is reported beside these;
* tracks: identical hit lists and order for every track whose tracklet
  shares no hit with a tracklet that differs.
"""
import numpy as np

TOL_YZ = 1e-3
TOL_ANG = 1e-4
TOL_QPT_REL = 1e-4
QPT_FLOOR = 2.0
DIAG = (0, 2, 5, 9, 14)   # variances in the 15-entry lower triangle


def param_errors(gp, op):
    """Per-parameter |GPU - oracle| scaled to the bars (<= 1 passes)."""
    gp = np.asarray(gp, np.float64)
    op = np.asarray(op, np.float64)
    d = np.abs(gp - op)
    s = np.empty_like(d)
    s[..., 0] = d[..., 0] / TOL_YZ
    s[..., 1] = d[..., 1] / TOL_YZ
    s[..., 2] = d[..., 2] / TOL_ANG
    s[..., 3] = d[..., 3] / TOL_ANG
    s[..., 4] = d[..., 4] / (TOL_QPT_REL * np.maximum(np.abs(op[..., 4]), QPT_FLOOR))
    return d, s


def sigma_errors(gp, op, oC, chi2=None, ndf=None):
    """Per-parameter |GPU - oracle| in units of the oracle's standard error,
    scaled by max(1, sqrt(chi2/ndf)) of the oracle's fit when given (the
    usual scale factor of a fit whose chi2 exceeds its degrees of freedom:
    its covariance understates the spread of the parameters)."""
    d = np.abs(np.asarray(gp, np.float64) - np.asarray(op, np.float64))
    var = np.asarray(oC, np.float64)[..., list(DIAG)]
    sd = np.sqrt(np.maximum(var, 1e-300))
    if chi2 is not None and ndf is not None:
        f = np.sqrt(np.maximum(1.0, np.asarray(chi2, np.float64) / np.maximum(np.asarray(ndf), 1)))
        sd = sd * np.asarray(f)[..., None] if np.ndim(f) else sd * f
    return d / sd


def check_param_bars(scaled, what="tracks"):
    """Assert the parameter bars on an (n, 5) array of param_errors scales:
    every row within 1."""
    s = np.asarray(scaled, np.float64).reshape(-1, 5)
    if len(s) == 0:
        return
    worst = s.max(axis=1)
    over = np.nonzero(worst > 1.0)[0]
    assert len(over) == 0, (what, len(over), s.max(axis=0))


def plain_within(gp, op):
    """Rows within the plain bars: |dy|, |dz| <= 1e-3 cm, |d sin phi|,
    |d tan lambda| <= 1e-4, q/pT within 1e-4 relative (no floor)."""
    d = np.abs(np.asarray(gp, np.float64) - np.asarray(op, np.float64)).reshape(-1, 5)
    q = np.abs(np.asarray(op, np.float64).reshape(-1, 5)[:, 4])
    return (d[:, 0] <= TOL_YZ) & (d[:, 1] <= TOL_YZ) & (d[:, 2] <= TOL_ANG) & \
        (d[:, 3] <= TOL_ANG) & (d[:, 4] <= TOL_QPT_REL * q)


def mahalanobis(gp, op, oC):
    """sqrt(d^T C^-1 d) per row, d = GPU - oracle state, C the oracle's
    covariance (15 lower-triangle entries): the size of the binary32
    deviation in units of the track's own statistical error."""
    gp = np.asarray(gp, np.float64).reshape(-1, 5)
    op = np.asarray(op, np.float64).reshape(-1, 5)
    tri = np.asarray(oC, np.float64).reshape(-1, 15)
    C = np.zeros((len(tri), 5, 5))
    k = 0
    for i in range(5):
        for j in range(i + 1):
            C[:, i, j] = C[:, j, i] = tri[:, k]
            k += 1
    d = gp - op
    x = np.linalg.solve(C, d[..., None])[..., 0]
    return np.sqrt(np.maximum(np.einsum("ni,ni->n", d, x), 0.0))


def compare_links(gpu_up, gpu_dn, o_up, o_dn):
    bad = np.nonzero((gpu_up != o_up) | (gpu_dn != o_dn))[0]
    return bad


def c2_exempt(o):
    """Hits whose cleaned links may differ between the binary32 kernel and the
    binary64 oracle: a hit with neighbour near-tie bits, or a hit whose
    oracle partner (up or down) has them.  Elsewhere the raw links of the hit
    and of its partners are identical on both sides, so are the cleaned ones."""
    tie = np.asarray(o["c2_tie"]) != 0
    ex = tie.copy()
    for k in ("up", "dn"):
        a = np.asarray(o[k])
        m = a >= 0
        ex[m] |= tie[a[m]]
    return ex


def check_links(g, o, max_frac=1e-3):
    """Links, cleaned links and start hits of a GPU run g (by cid) against the
    oracle o.  Returns the exempt-hit mask and the number of differing links."""
    tie = np.asarray(o["c2_tie"]) != 0
    bad = compare_links(g["up"], g["dn"], o["up"], o["dn"])
    assert not np.any(~tie[bad]), ("links differ at hits without a near tie", bad[~tie[bad]][:10])
    assert len(bad) <= max_frac * max(1, o["n_links"]), (len(bad), o["n_links"])
    ex = c2_exempt(o)
    badc = compare_links(g["up_c"], g["dn_c"], o["up_c"], o["dn_c"])
    assert not np.any(~ex[badc]), ("cleaned links differ", badc[~ex[badc]][:10])
    o_starts = np.nonzero((np.asarray(o["up_c"]) >= 0) & (np.asarray(o["dn_c"]) < 0))[0]
    sd = np.setxor1d(np.asarray(g["starts"]), o_starts)
    assert not np.any(~ex[sd]), ("start hits differ", sd[~ex[sd]][:10])
    return ex, len(bad)


def chain_exempt(o, ex, n_rows):
    """For every hit: the oracle's chain of cleaned up links from it passes a
    hit of the exempt mask ex (then the GPU's chain from it may differ)."""
    up_c = np.asarray(o["up_c"])
    out = ex.copy()
    cur = up_c.copy()
    for _ in range(n_rows):
        m = cur >= 0
        if not m.any():
            break
        out[m] |= ex[cur[m]]
        cur[m] = up_c[cur[m]]
    return out


def compare_tracklets(gt, ot, n_rows, c2_chain=None):
    """Returns a report dict; keys of tracklets are start cids.  c2_chain
    (from chain_exempt) marks starts whose chains pass a neighbour near tie:
    their tracklets count as flagged, and may be missing or extra.  A chain
    may also be built on one side only when its dominance (all its hits
    taken by forward extension searches) can differ: when one of its hits
    was taken by a forward pass that carries near-tie bits (oracle fwd_mark
    bit 2), or lies on a flagged tracklet that differs."""
    g_index = {int(c): i for i, c in enumerate(gt["start"])}
    o_index = {int(c): i for i, c in enumerate(ot["t_start"])}
    rep = {"n_oracle": len(o_index), "n_gpu": len(g_index), "flagged": 0, "flagged_diff": [],
           "hitset_mismatch": [], "valid_mismatch": [], "param_scaled": [], "param_abs": [],
           "param_sig": [], "taint": set()}
    up_c = np.asarray(ot["up_c"])
    tie_mark = (np.asarray(ot["fwd_mark"]) & 2) != 0 if "fwd_mark" in ot else None

    def c2(c):
        return c2_chain is not None and bool(c2_chain[c])

    def chain_of(c):
        out = [c]
        while up_c[out[-1]] >= 0 and len(out) < n_rows:
            out.append(int(up_c[out[-1]]))
        return out

    def taint_g(gi):
        a = gt["rowhit"][gi]
        rep["taint"].update(a[a >= 0].tolist())

    def taint_o(oi):
        a = ot["t_rowhit"][oi]
        rep["taint"].update(a[a >= 0].tolist())
    for c, oi in o_index.items():
        if c not in g_index:
            continue
        gi = g_index[c]
        same = int(gt["valid"][gi]) == int(ot["t_valid"][oi]) and \
            np.array_equal(gt["rowhit"][gi], ot["t_rowhit"][oi])
        if ot["t_flags"][oi] != 0 or c2(c):
            rep["flagged"] += 1
            if not same:
                rep["flagged_diff"].append(c)
                taint_g(gi)
                taint_o(oi)
            continue
        if int(gt["valid"][gi]) != int(ot["t_valid"][oi]):
            rep["valid_mismatch"].append(c)
            continue
        if not same:
            rep["hitset_mismatch"].append(c)
            continue
        if ot["t_valid"][oi]:
            d, s = param_errors(gt["p"][gi], ot["t_p"][oi])
            rep["param_scaled"].append(s)
            rep["param_abs"].append(d)
            rep["param_sig"].append(sigma_errors(gt["p"][gi], ot["t_p"][oi], ot["t_C"][oi],
                                                 ot["t_chi2"][oi], ot["t_ndf"][oi]))
    differ_hits = set(rep["taint"])

    def explained(c):
        if c2(c):
            return True
        ch = chain_of(c)
        if tie_mark is not None and tie_mark[ch].any():
            return True
        return bool(differ_hits.intersection(ch))
    missing = sorted(set(o_index) - set(g_index))
    extra = sorted(set(g_index) - set(o_index))
    rep["missing"] = [c for c in missing if not explained(c)]
    rep["extra"] = [c for c in extra if not explained(c)]
    for c in missing:
        if explained(c):
            rep["flagged_diff"].append(c)
            taint_o(o_index[c])
    for c in extra:
        if explained(c):
            rep["flagged_diff"].append(c)
            taint_g(g_index[c])
    rep["param_scaled"] = np.array(rep["param_scaled"]).reshape(-1, 5)
    rep["param_abs"] = np.array(rep["param_abs"]).reshape(-1, 5)
    rep["param_sig"] = np.array(rep["param_sig"]).reshape(-1, 5)
    return rep


def check_tracklets(rep, max_diff_frac=1e-3):
    """The tracklet bars on a compare_tracklets report."""
    assert rep["missing"] == [] and rep["extra"] == [], (rep["missing"][:5], rep["extra"][:5])
    assert len(rep["flagged_diff"]) <= max_diff_frac * max(1, rep["n_oracle"]), \
        (len(rep["flagged_diff"]), rep["n_oracle"])
    assert rep["valid_mismatch"] == [], rep["valid_mismatch"][:10]
    assert rep["hitset_mismatch"] == [], rep["hitset_mismatch"][:10]
    check_param_bars(rep["param_scaled"], "tracklets")


def tainted_hits(ot):
    """Clusters of every oracle tracklet flagged as a near-tie (a superset of
    the hits that can differ, for runs whose GPU tracklets are not at hand)."""
    rh = ot["t_rowhit"][ot["t_flags"] != 0]
    return set(rh[rh >= 0].tolist())


def compare_tracks(gtr, ot, taint):
    """Oracle tracks (from track_event) vs GPU Tracks; skips tainted ones."""
    o_tracks = []
    for j in range(ot["n_tracks"]):
        h = ot["k_hit_cid"][ot["k_hit_off"][j]:ot["k_hit_off"][j + 1]]
        o_tracks.append((tuple(h.tolist()), j))
    g_tracks = []
    for j in range(gtr.n_tracks):
        g_tracks.append((tuple(gtr.hits(j).tolist()), j))
    o_set = {h: j for h, j in o_tracks}
    g_set = {h: j for h, j in g_tracks}

    def clean(h):
        return not (set(h) & taint)

    # an oracle track whose tracklet holds a tainted hit it does not own may
    # differ too (the hit's owner differs, so the track may keep it on one
    # side only): test the tracklet's whole hit set when it is known
    def clean_o(h, j):
        if "k_tracklet" in ot and "t_rowhit" in ot:
            rh = ot["t_rowhit"][ot["k_tracklet"][j]]
            return clean(h) and not (set(rh[rh >= 0].tolist()) & taint)
        return clean(h)
    o_clean = [h for h, j in o_tracks if clean_o(h, j)]
    g_clean = [h for h, _ in g_tracks if clean(h)]
    rep = {"n_oracle": len(o_tracks), "n_gpu": len(g_tracks), "compared": 0,
           "missing": [h for h in o_clean if h not in g_set],
           "extra": [h for h in g_clean if h not in o_set], "param_scaled": [], "param_sig": []}
    common = [h for h in o_clean if h in g_set]
    rep["compared"] = len(common)
    # same relative order
    g_pos = [g_set[h] for h in common]
    rep["order_ok"] = all(a < b for a, b in zip(g_pos, g_pos[1:]))
    for h in common:
        gj, oj = g_set[h], o_set[h]
        _, s = param_errors(gtr.param[gj], ot["k_p"][oj])
        rep["param_scaled"].append(s)
        rep["param_sig"].append(sigma_errors(gtr.param[gj], ot["k_p"][oj], ot["k_C"][oj],
                                             ot["k_chi2"][oj], ot["k_ndf"][oj]))
        if gtr.sector[gj] != ot["k_sector"][oj] or gtr.ndf[gj] != ot["k_ndf"][oj]:
            rep.setdefault("meta_mismatch", []).append(h)
    rep["param_scaled"] = np.array(rep["param_scaled"]).reshape(-1, 5)
    rep["param_sig"] = np.array(rep["param_sig"]).reshape(-1, 5)
    if common:
        gp = np.array([gtr.param[g_set[h]] for h in common], np.float64)
        op = np.array([ot["k_p"][o_set[h]] for h in common], np.float64)
        oC = np.array([ot["k_C"][o_set[h]] for h in common], np.float64)
        rep["plain_share"] = float(plain_within(gp, op).mean())
        rep["maha"] = mahalanobis(gp, op, oC)
    else:
        rep["plain_share"] = float("nan")
        rep["maha"] = np.zeros(0)
    rep["compared_share"] = rep["compared"] / max(1, rep["n_oracle"])
    return rep
