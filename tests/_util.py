"""Helpers shared by the tests (event fixtures and MC-truth bookkeeping)."""
import json
import math
import os

import numpy as np

from paper_1712_09416_b300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_event(name="neighbours_small.json"):
    g = json.load(open(os.path.join(GOLDEN, name)))
    h = np.array(g["hits"], dtype=np.float64)
    order = np.argsort(h[:, 0])
    h = h[order]
    assert np.all(h[:, 0] == np.arange(len(h)))
    ev = synth.Event(y=h[:, 3].astype(np.float32), z=h[:, 4].astype(np.float32),
                     row=h[:, 2].astype(np.uint16), sector=h[:, 1].astype(np.uint16),
                     label=np.full(len(h), -1, np.int32),
                     row_x=np.array(g["row_x"], dtype=np.float32),
                     n_sectors_phi=g["n_sectors_phi"], split_z=0)
    return ev, g


def track_hits(out, j, prefix="k_"):
    off = out[prefix + "hit_off"]
    return out[prefix + "hit_cid"][off[j]:off[j + 1]]


def mc_summary(ev, out, min_clusters=30, match_frac=0.9, n_tracks_key="n_tracks"):
    """Efficiency / fake / clone by MC labels, per particle segment in a sector.

    A reco track matches particle P if >= 90% of its hits carry P's label; it
    then matches the segment (P, sector).  A segment is reconstructable if it
    has >= min_clusters clusters.  Clones are extra matches of a segment.
    """
    lab = ev.label
    matched = {}
    fakes = 0
    clones = 0
    sectors = out["k_sector"] if isinstance(out, dict) else out.sector
    for j in range(out[n_tracks_key] if isinstance(out, dict) else out.n_tracks):
        hits = track_hits(out, j) if isinstance(out, dict) else out.hits(j)
        l = lab[hits]
        vals, cnt = np.unique(l, return_counts=True)
        b = np.argmax(cnt)
        if vals[b] >= 0 and cnt[b] >= match_frac * len(hits):
            seg = (int(vals[b]), int(sectors[j]))
            if seg in matched:
                clones += 1
            matched[seg] = matched.get(seg, 0) + 1
        else:
            fakes += 1
    n_reco = out[n_tracks_key] if isinstance(out, dict) else out.n_tracks
    sig = lab >= 0
    key = lab[sig].astype(np.int64) * 64 + ev.sector[sig]
    k, c = np.unique(key, return_counts=True)
    recble = [(int(a // 64), int(a % 64)) for a in k[c >= min_clusters]]
    pt = ev.particles.pt
    res = {"n_reco": n_reco, "n_reconstructable": len(recble), "fakes": fakes, "clones": clones}
    for name, lo in (("eff", 0.0), ("eff_pt02", 0.2)):
        sel = [sg for sg in recble if pt[sg[0]] >= lo]
        res[name] = float(np.mean([sg in matched for sg in sel])) if sel else float("nan")
    res["fake_rate"] = fakes / max(1, n_reco)
    res["clone_rate"] = clones / max(1, n_reco)
    return res


def isolated_event(n_tracks=6, seed=11, sigma=0.01, pt_range=(1.0, 5.0)):
    """A few well separated high-pT tracks in one sector, no noise."""
    rng = np.random.default_rng(seed)
    phis = np.linspace(math.radians(4), math.radians(16), n_tracks)
    p = synth.Particles(q=np.where(np.arange(n_tracks) % 2 == 0, 1.0, -1.0),
                        pt=rng.uniform(*pt_range, n_tracks),
                        tanl=np.linspace(-0.8, 0.8, n_tracks), phi0=phis,
                        vx=np.zeros(n_tracks), vy=np.zeros(n_tracks), vz=np.zeros(n_tracks))
    return synth.make_event(rng, p, n_sectors_phi=1, split_z=False, sigma=sigma,
                            noise_frac=0.0)


def oracle_by_sector(ev, orc, sectors=None, workers=None):
    """The oracle's record of a whole event (or of the given sectors) from one
    call per sector on all host cores: sectors are independent, so this
    equals one call on the whole event (the hit weights aside, whose keys
    hold sector-local cids; they are left out).  Cluster ids are those of ev;
    per-hit arrays of clusters outside the sectors hold -1 (links) or 0."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    n_sec = ev.n_sectors_phi * (2 if ev.split_z else 1)
    sectors = list(range(n_sec)) if sectors is None else list(sectors)
    parts = [ev.select_sectors([s]) for s in sectors]
    with ThreadPoolExecutor(max_workers=workers or os.cpu_count() or 1) as pool:
        outs = list(pool.map(orc.track_event, parts))
    n = ev.n

    def cid_map(p, a):
        a = np.asarray(a)
        return np.where(a >= 0, p.info["parent_index"][np.maximum(a, 0)], -1).astype(np.int32)
    o = {}
    for k in ("up", "dn", "up_c", "dn_c"):
        o[k] = np.full(n, -1, np.int32)
        for p, r in zip(parts, outs):
            o[k][p.info["parent_index"]] = cid_map(p, r[k])
    o["c2_tie"] = np.zeros(n, np.int32)
    o["fwd_mark"] = np.zeros(n, np.int32)
    for p, r in zip(parts, outs):
        o["c2_tie"][p.info["parent_index"]] = r["c2_tie"]
        o["fwd_mark"][p.info["parent_index"]] = r["fwd_mark"]
    for k in ("t_sector", "t_chain_len", "t_valid", "t_nhits", "t_first_row", "t_last_row",
              "t_flags", "t_ndf", "t_x", "t_p", "t_C", "t_chi2", "k_x", "k_p", "k_C", "k_chi2",
              "k_ndf", "k_sector"):
        o[k] = np.concatenate([r[k] for r in outs])
    o["t_start"] = np.concatenate([cid_map(p, r["t_start"]) for p, r in zip(parts, outs)])
    o["t_rowhit"] = np.concatenate([cid_map(p, r["t_rowhit"]) for p, r in zip(parts, outs)])
    base = np.cumsum([0] + [r["n_tracklets"] for r in outs])
    o["k_tracklet"] = np.concatenate([r["k_tracklet"] + b for r, b in zip(outs, base)])
    o["k_hit_cid"] = np.concatenate([cid_map(p, r["k_hit_cid"]) for p, r in zip(parts, outs)])
    o["k_hit_off"] = np.concatenate([[0], np.cumsum(np.concatenate(
        [np.diff(r["k_hit_off"]) for r in outs]))]).astype(np.int32)
    for k in ("n_tracklets", "n_tracks", "n_track_hits", "n_links", "n_c2_ties", "n_starts",
              "n_dominated"):
        o[k] = int(sum(r[k] for r in outs))
    return o


def gpu_stages(tp, ctx, ev, event=0):
    """The stage dumps of one event of the context's last launch, by cid:
    links, cleaned links, start hits, tracklets, hit weights."""
    n = ev.n
    up, dn = tp.dump_links(ctx, n, event=event)
    upc, dnc = tp.dump_links(ctx, n, clean=True, event=event)
    return {"up": up, "dn": dn, "up_c": upc, "dn_c": dnc,
            "starts": tp.dump_starts(ctx, event=event),
            "tracklets": tp.dump_tracklets(ctx, len(ev.row_x), event=event),
            "weights": tp.dump_weights(ctx, event=event)}
