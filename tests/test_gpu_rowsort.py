"""Row-sort tiers against the oracle's neighbour links.

The hits of a pad row are sorted by y-z bin and cid by one warp when the row
holds up to 384 hits, by one block up to 1024 hits (both in k_rowsort), and by
k_rowsort_big up to 2048 and up to 4096 hits.  One sector here carries rows
whose hit counts sit on and around every boundary (and an empty row and a
one-hit row), with straight tracks through the rest so that links exist.
The oracle bins nothing (it tests every hit of the adjacent rows), so a row
sorted wrongly by any tier shows up as a changed link: every hit's up and down
link must equal the oracle's binary64 decision outside its near ties.
"""
import math

import numpy as np
import pytest

from paper_1712_09416_b300 import synth
from tests import _util

pytestmark = pytest.mark.gpu

# pad row -> hits on it (tracks included)
COUNTS = {10: 257, 13: 256, 16: 1, 19: 0, 22: 1023, 25: 1024, 28: 1025, 31: 2047, 34: 2048,
          37: 2049, 40: 3000, 43: 4096, 46: 384, 49: 385}
N_TRACKS = 60
SKIP = {16, 19}  # rows the tracks do not cross


def _event():
    rng = np.random.default_rng(11)
    row_x = synth.default_row_x()
    tan_h = math.tan(synth.HALF_ANGLE)
    # straight tracks from near the beam line: y = a x, z = z0 + b x
    a = rng.uniform(-0.12, 0.12, N_TRACKS)
    b = rng.uniform(0.05, 0.8, N_TRACKS)
    z0 = rng.uniform(0.0, 20.0, N_TRACKS)
    ys, zs, rs, ls = [], [], [], []
    for r, x in enumerate(row_x):
        n = COUNTS.get(r, 24)
        if r not in SKIP:
            ys.append(a * x + rng.normal(0, 0.05, N_TRACKS))
            zs.append(z0 + b * x + rng.normal(0, 0.05, N_TRACKS))
            ls.append(np.arange(N_TRACKS))
            n -= N_TRACKS
        n = max(n, 0)
        w = 0.95 * x * tan_h
        ys.append(rng.uniform(-w, w, n))
        zs.append(rng.uniform(2.0, 240.0, n))
        ls.append(np.full(n, -1))
        rs.append(np.full(n + (0 if r in SKIP else N_TRACKS), r))
    y = np.concatenate(ys).astype(np.float32)
    z = np.concatenate(zs).astype(np.float32)
    row = np.concatenate(rs).astype(np.uint16)
    lab = np.concatenate(ls).astype(np.int32)
    order = rng.permutation(len(y))  # cid = input index, rows interleaved
    return synth.Event(y[order], z[order], row[order], np.zeros(len(y), np.uint16), lab[order],
                       row_x, 18, 1)


def test_row_sort_tiers_give_the_oracles_links(orc):
    from paper_1712_09416_b300 import build, tpctrack as tp
    build.build()
    ev = _event()
    cnt = np.bincount(ev.row, minlength=len(ev.row_x))
    for r, c in COUNTS.items():
        assert cnt[r] == c, (r, cnt[r])
    with tp.Tracker(ev.n + 65536) as t:
        t.event(ev)
        up, dn = tp.dump_links(t.ctx, ev.n)
        assert t.counters()["max_row_hits"] == 4096
    o = _util.oracle_by_sector(ev, orc, sectors=[0])
    diff = np.nonzero((up != o["up"]) | (dn != o["dn"]))[0]
    n_links = int(np.sum(o["up"] >= 0))
    print("links", n_links, "differing", len(diff), "of which on near ties",
          int(np.sum(o["c2_tie"][diff] != 0)))
    assert n_links > 100 * N_TRACKS
    assert np.all(o["c2_tie"][diff] != 0)
    assert len(diff) <= 1e-3 * n_links
    # every boundary row has links to and from it (its sort was used)
    for r in (10, 13, 25, 28, 34, 37, 40, 43, 46, 49):
        on = ev.row == r
        assert np.sum(up[on] >= 0) >= N_TRACKS // 2, r
