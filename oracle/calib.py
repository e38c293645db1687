"""Plain FP64 statement of the accumulate-then-fit side task (the chi^2
scale of a run of tracks).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` import this module.  It shares no code with the
package.

The paper names the kind of task, not its content: a calibration component
that accumulates data at every event and runs a long fit every n-th event
(Sect. 3, item 4; Sect. 5.1).  The fit stated here stands in for it.  Every
track contributes its chi^2 and its number of degrees of freedom ndf (tracks
with ndf <= 0 are skipped).  With Gaussian cluster errors that the tracker
assumes correctly, chi^2 / ndf scatters around 1; when the assumed error is
too small by a factor s, around s^2.  The estimate of s^2:

1. s2 = (sum of chi^2) / (sum of ndf) over all tracks;
2. keep the tracks with chi^2 <= trim * s2 * ndf, and set s2 to the same
   ratio over the kept tracks;
3. repeat 2 until the kept set is the one of the previous round, at most 100
   rounds in all.

Step 2 only ever drops tracks whose ratio lies above trim (> 1) times the
current mean ratio, so s2 never increases and the kept set only shrinks: the
rounds end.
"""
from __future__ import annotations

import numpy as np

MAX_ROUNDS = 100


def chi2_scale_fit(chi2, ndf, trim: float = 3.0) -> dict:
    """The estimate of s^2 above for one run of tracks.

    Returns {"scale2", "n_tracks", "n_kept", "n_iter"}; n_iter counts the
    rounds of step 2 (the round that found the kept set repeated included).
    A run without a track with ndf > 0 gives scale2 = nan."""
    c = np.asarray(chi2, np.float64)
    d = np.asarray(ndf, np.float64)
    use = d > 0
    c, d = c[use], d[use]
    n = len(c)
    if n == 0:
        return {"scale2": float("nan"), "n_tracks": 0, "n_kept": 0, "n_iter": 0}
    s2 = c.sum() / d.sum()
    keep = np.ones(n, bool)
    n_iter = 0
    for n_iter in range(1, MAX_ROUNDS + 1):
        nxt = c <= trim * s2 * d
        if not nxt.any():
            break
        same = bool(np.array_equal(nxt, keep))
        keep = nxt
        s2 = c[keep].sum() / d[keep].sum()
        if same:
            break
    return {"scale2": float(s2), "n_tracks": int(n), "n_kept": int(keep.sum()), "n_iter": int(n_iter)}
