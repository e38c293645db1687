"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a dropped
minus sign, a rotation turned the wrong way, a Jacobian entry lost, a wrong
prior, a path length without the arc), builds it with gcc under a temporary
directory, and checks that the pin written for that part of the oracle
(merger, transport, update, seed) fails on the mutant while it passes on the
oracle.  Nothing here touches the GPU or the package.
"""
import ctypes as C
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1712_09416_b300 import synth

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "tpc_oracle.c")

MUTATIONS = {
    "rotation turned the wrong way": ("    const double s1 = s * cd - c * sd;\n    const double c1 = c * cd + s * sd;",
                                      "    const double s1 = s * cd + c * sd;\n    const double c1 = c * cd - s * sd;"),
    "sign of ds'/dy": ("    Jr[2][0] = -ck * sd;", "    Jr[2][0] = ck * sd;"),
    "dz'/dy dropped": ("    Jr[1][0] = -p[3] * sd / c1;", "    Jr[1][0] = 0.0;"),
    "refit turns the frame backwards": (
        "                const double d = sector_alpha(cfg, sector[a]) - sector_alpha(cfg, sector[chain[g + 1]]);",
        "                const double d = sector_alpha(cfg, sector[chain[g + 1]]) - sector_alpha(cfg, sector[a]);"),
    # the sector tracker's transport, update and seed (pins in test_oracle_transport/_fit)
    "transport: q/pT column of dy lost": (
        "    Jl[0][4] = -kB * dx * dx * (cc + (s0 + s1) * s1 / c1) / (cc * cc);", "    Jl[0][4] = 0.0;"),
    "update: sign of the off-diagonal gain": (
        "    const double I00 = S11 / det, I01 = -S01 / det, I11 = S00 / det;",
        "    const double I00 = S11 / det, I01 = S01 / det, I11 = S00 / det;"),
    "seed: sin(phi) variance with cos^4": (
        "    C[2][2] = cfg->seed_var_s * c2 * c2 * c2;", "    C[2][2] = cfg->seed_var_s * c2 * c2;"),
    "transport: path length without the arc": (
        "    double dS = (h > 0.0) ? ch * asin(h) / h : ch;", "    double dS = ch;"),
    # the neighbour rule (pin: the hand-derived golden case)
    "neighbours: z term of D dropped": (
        "            const double D = (syu - syd) * (syu - syd) + (szu - szd) * (szu - szd);",
        "            const double D = (syu - syd) * (syu - syd);"),
    "neighbours: sign of sy_d": (
        "            const double syd = (H->y[h] - H->y[d]) / (xh - xd);",
        "            const double syd = (H->y[d] - H->y[h]) / (xh - xd);"),
    "neighbours: window edge excluded": (
        "        if (!(fabs(H->y[u] - H->y[h]) <= wyu) || !(fabs(H->z[u] - H->z[h]) <= wzu)) continue;",
        "        if (!(fabs(H->y[u] - H->y[h]) < wyu) || !(fabs(H->z[u] - H->z[h]) < wzu)) continue;"),
    "neighbours: ties to the higher cid(u)": (
        "            if (bu < 0 || D < bestD || (D == bestD && (u < bu || (u == bu && d < bd)))) {\n                if (bu >= 0) second = bestD;",
        "            if (bu < 0 || D < bestD || (D == bestD && (u > bu || (u == bu && d < bd)))) {\n                if (bu >= 0) second = bestD;"),
    "neighbours: pair near-tie bit lost": (
        "    if (bu >= 0 && bestD <= dmax + cfg->tie_d && second - bestD <= cfg->tie_d)",
        "    if (bu >= 0 && bestD <= dmax + cfg->tie_d && second - bestD < 0.0)"),
    "neighbours: window near-tie bit lost": (
        "        if (ay <= wy + tw && az <= wz + tw && (ay > wy - tw || az > wz - tw))",
        "        if (ay <= wy - tw && az <= wz + tw && (ay > wy - tw || az > wz - tw))"),
    "cleaner: up link kept without the partner's down link": (
        "        res->up_c[i] = (u >= 0 && res->dn[u] == (int32_t)i) ? u : -1;",
        "        res->up_c[i] = u;"),
    # the dominance rule (pin: a track cut by one missing row comes out whole, once)
    "dominance: marks also from the tracklet's own chain": (
        "        for (int r = F[i].rk + 1; r <= F[i].last; ++r)",
        "        for (int r = F[i].r0; r <= F[i].last; ++r)"),
    "dominance: one marked hit is enough": (
        "        for (int64_t q = ch_off[i]; q < ch_off[i + 1]; ++q) all = all && marked[ch_hits[q]];",
        "        all = 0; for (int64_t q = ch_off[i]; q < ch_off[i + 1]; ++q) all = all || marked[ch_hits[q]];"),
}


@pytest.fixture
def mutant(orc, tmp_path, monkeypatch):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")

    def build(name):
        old, new = MUTATIONS[name]
        src = open(SRC).read()
        assert src.count(old) == 1, name
        p = tmp_path / "mutant.c"
        p.write_text(src.replace(old, new))
        so = tmp_path / "libmutant.so"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                        str(so), str(p), "-lm"], check=True)
        lib = C.CDLL(str(so))
        for f in ("orc_track_event", "orc_transport_packed", "orc_fit_fixed", "orc_rotate_packed",
                  "orc_merge"):
            getattr(lib, f).restype = C.c_int
        lib.orc_update_packed.restype = C.c_double
        monkeypatch.setattr(orc, "_lib", lib)
        return orc
    return build


def closed_form_ok(orc):
    """The rotation pin: truth in sector A turned into B and carried to a row
    of B lands on the generator's crossing there."""
    p0 = synth.Particles(q=np.array([1.0]), pt=np.array([0.5]), tanl=np.array([0.3]),
                         phi0=np.array([math.radians(17.0)]), vx=np.zeros(1), vy=np.zeros(1),
                         vz=np.zeros(1))
    ev = synth.make_event(np.random.default_rng(0), p0, n_sectors_phi=18, split_z=False, sigma=0.0,
                          noise_frac=0.0, dtype=np.float64, shuffle=False)
    (sa, sb) = sorted(set(ev.sector.tolist()))
    if (sb - sa) % 18 != 1:
        sa, sb = sb, sa
    ma = np.nonzero(ev.sector == sa)[0]
    mb = np.nonzero(ev.sector == sb)[0]
    i, j = ma[np.argmax(ev.row[ma])], mb[np.argmin(ev.row[mb])]
    xr = ev.row_x.astype(np.float64)
    p = np.array([ev.y[i], ev.z[i], ev.true_sinphi[i], 0.3, 2.0])
    rc, x1, p1, _, _ = orc.rotate(math.radians(20.0), xr[ev.row[i]], p, np.zeros(15))
    if rc:
        return False
    rc, p2, _, _ = orc.transport(x1, xr[ev.row[j]], p1, np.zeros(15))
    return rc == 0 and abs(p2[0] - ev.y[j]) < 1e-9 and abs(p2[2] - ev.true_sinphi[j]) < 1e-11


def jacobian_ok(orc):
    """The Jacobian pin: analytic against central differences."""
    x0, X, d = 150.0, 170.0, math.radians(20.0)
    p0 = np.array([3.0, 20.0, 0.2, 0.4, 1.5])
    rc, x1, p1, _, Jr = orc.rotate(d, x0, p0, np.zeros(15))
    rc, p2, _, Jt = orc.transport(x1, X, p1, np.zeros(15))
    J = Jt @ Jr

    def f(p):
        _, x1, p1, _, _ = orc.rotate(d, x0, p, np.zeros(15))
        return orc.transport(x1, X, p1, np.zeros(15))[1]
    for k in range(5):
        h = 1e-6 * max(1.0, abs(p0[k]))
        e = np.zeros(5)
        e[k] = h
        if not np.allclose((f(p0 + e) - f(p0 - e)) / (2 * h), J[:, k], rtol=1e-6, atol=1e-7):
            return False
    return True


def merged_truth_ok(orc):
    """The merger pin: a noiseless helix across a phi boundary comes out as
    one track with the generator's state."""
    p0 = synth.Particles(q=np.array([1.0]), pt=np.array([0.5]), tanl=np.array([0.3]),
                         phi0=np.array([math.radians(17.0)]), vx=np.zeros(1), vy=np.zeros(1),
                         vz=np.zeros(1))
    ev = synth.make_event(np.random.default_rng(0), p0, n_sectors_phi=18, split_z=False, sigma=0.0,
                          noise_frac=0.0, dtype=np.float64, shuffle=False)
    o = orc.track_event(ev)
    m = orc.merge_tracks(ev, o)
    if m["n_tracks"] != 1:
        return False
    h0 = m["k_hit_cid"][0]
    truth = np.array([ev.y[h0], ev.z[h0], ev.true_sinphi[h0], 0.3, 2.0])
    return bool((np.abs(m["k_p"][0] - truth) / np.maximum(np.abs(truth), 1.0)).max() < 2e-5)


def passes(test, *args):
    """Run one of the existing pin tests; True if it passes."""
    try:
        test(*args)
        return True
    except AssertionError:
        return False


def transport_jacobian_ok(orc):
    from tests import test_oracle_transport as t
    return all(passes(t.test_jacobian_matches_finite_differences, orc, seed) for seed in range(12))


def update_ok(orc):
    from tests import test_oracle_transport as t
    return all(passes(t.test_update_equals_information_form, orc, seed) for seed in range(8))


def prior_ok(orc):
    from tests import test_oracle_fit as t
    return all(passes(t.test_zero_field_line_equals_batch_least_squares, orc, s0, tt)
               for s0, tt in ((0.0, 0.0), (0.25, 0.5), (-0.4, -0.9), (0.6, 0.1)))


def dominance_ok(orc):
    from tests import test_oracle_event as t
    return passes(t.test_chain_taken_by_a_forward_extension_gets_no_tracklet, orc) and \
        passes(t.test_isolated_tracks_one_track_each_with_all_clusters, orc) and \
        passes(t.test_dominance_removes_tracklets_not_tracks, orc)


def golden_ok(orc):
    from tests import test_oracle_event as t
    return passes(t.test_golden_neighbours, orc)


def crossings_ok(orc):
    from tests import test_oracle_transport as t
    return passes(t.test_transport_matches_closed_form_crossings, orc, 1.0, 0.35, 0.4,
                  math.radians(10.0))


PINS = {"rotation turned the wrong way": closed_form_ok, "sign of ds'/dy": jacobian_ok,
        "dz'/dy dropped": jacobian_ok, "refit turns the frame backwards": merged_truth_ok,
        "transport: q/pT column of dy lost": transport_jacobian_ok,
        "update: sign of the off-diagonal gain": update_ok,
        "seed: sin(phi) variance with cos^4": prior_ok,
        "transport: path length without the arc": crossings_ok,
        "neighbours: z term of D dropped": golden_ok, "neighbours: sign of sy_d": golden_ok,
        "neighbours: window edge excluded": golden_ok,
        "neighbours: ties to the higher cid(u)": golden_ok,
        "neighbours: pair near-tie bit lost": golden_ok,
        "neighbours: window near-tie bit lost": golden_ok,
        "cleaner: up link kept without the partner's down link": golden_ok,
        "dominance: marks also from the tracklet's own chain": dominance_ok,
        "dominance: one marked hit is enough": dominance_ok}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pin_catches_the_mistake(orc, mutant, name):
    assert PINS[name](orc), "the pin must pass on the oracle itself"
    assert not PINS[name](mutant(name)), f"the pin missed: {name}"


CALIB = os.path.join(os.path.dirname(SRC), "calib.py")
CALIB_MUTATIONS = {
    "mean of the ratios instead of the ratio of the sums": ("    s2 = c.sum() / d.sum()\n    keep",
                                                           "    s2 = (c / d).mean()\n    keep"),
    "trim against the ratio, not ratio x ndf": ("        nxt = c <= trim * s2 * d", "        nxt = c <= trim * s2"),
    "stop after the first round": ("        if same:\n            break", "        break"),
}


@pytest.mark.parametrize("name", sorted(CALIB_MUTATIONS))
def test_fit_pins_catch_the_mistake(tmp_path, name):
    """The chi^2 scale fit's pins (known scale, outliers, brute force) fail on a
    copy of oracle/calib.py with one planted mistake."""
    import importlib.util
    from tests import test_async_calib as t
    old, new = CALIB_MUTATIONS[name]
    src = open(CALIB).read()
    assert src.count(old) == 1, name
    p = tmp_path / "calib_mutant.py"
    p.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("calib_mutant", p)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    pins = (t.test_recovers_a_known_scale, t.test_gross_outliers_are_trimmed,
            t.test_kept_set_is_the_largest_self_consistent_one)
    assert all(passes(f) for f in pins), "the pins must pass on the oracle itself"
    orig = t.chi2_scale_fit
    try:
        t.chi2_scale_fit = mod.chi2_scale_fit
        assert not all(passes(f) for f in pins), f"the pins missed: {name}"
    finally:
        t.chi2_scale_fit = orig
