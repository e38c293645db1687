"""Pins of the oracle's sector track merger and global refit (M0-M5).

* M0 (frame rotation) against the generator's closed-form helix crossings in
  the neighbouring sector's frame (a global-frame formulation), its Jacobian
  against central finite differences, exact round trips and composition.
* M1-M5 on noiseless helices: a particle crossing one or two phi boundaries
  (also across phi = 0) or the z = 0 membrane comes out as one track holding
  every cluster, with the generator's state at its innermost cluster and a
  vanishing chi^2; a particle that stays in one sector is left alone, and so
  are the tracks of particles that do not continue each other.
* On a full event: no merged track joins segments of different particles, and
  the split particles become whole.
"""
import math

import numpy as np
import pytest

from paper_1712_09416_b300 import synth

D20 = math.radians(20.0)


def noiseless(particles, *, split_z=False):
    rng = np.random.default_rng(0)
    return synth.make_event(rng, particles, n_sectors_phi=18, split_z=split_z, sigma=0.0,
                            noise_frac=0.0, dtype=np.float64, shuffle=False)


def one(q, pt, tanl, phi0, vz=0.0):
    return synth.Particles(q=np.array([q]), pt=np.array([pt]), tanl=np.array([tanl]),
                           phi0=np.array([phi0]), vx=np.zeros(1), vy=np.zeros(1), vz=np.array([vz]))


def truth_in(ev, sec):
    m = np.nonzero(ev.sector == sec)[0]
    o = m[np.argsort(ev.row[m])]
    return ev.row_x.astype(np.float64)[ev.row[o]], ev.y[o], ev.z[o], ev.true_sinphi[o]


@pytest.mark.parametrize("q,pt,tanl,phi0", [
    (1.0, 0.5, 0.3, 17.0), (-1.0, 0.5, -0.3, 23.0), (1.0, 0.3, 0.5, 35.0), (-1.0, 0.8, 0.1, 30.0)])
def test_rotation_matches_closed_form_crossings(orc, q, pt, tanl, phi0):
    """A truth state on a row of sector A, turned into the frame of the next
    sector B and transported to a row plane of B, equals the generator's
    crossing of that plane in B."""
    ev = noiseless(one(q, pt, tanl, math.radians(phi0)))
    secs = sorted(set(ev.sector.tolist()))
    assert len(secs) >= 2
    for sa in secs:
        for sb in secs:
            dk = (sb - sa + 9) % 18 - 9  # -1, 0 or +1 around the ring
            if abs(dk) != 1:
                continue
            xa, ya, za, sa_ = truth_in(ev, sa)
            xb, yb, zb, sb_ = truth_in(ev, sb)
            for i in (0, len(xa) // 2, len(xa) - 1):
                for j in (0, len(xb) // 2, len(xb) - 1):
                    p = np.array([ya[i], za[i], sa_[i], tanl, q / pt])
                    rc, x1, p1, _, _ = orc.rotate(dk * D20, xa[i], p, np.zeros(15))
                    assert rc == 0
                    rc, p2, _, _ = orc.transport(x1, xb[j], p1, np.zeros(15))
                    assert rc == 0
                    assert abs(p2[0] - yb[j]) < 1e-9 and abs(p2[1] - zb[j]) < 1e-9
                    assert abs(p2[2] - sb_[j]) < 1e-11
                    assert p2[3] == tanl and p2[4] == q / pt


def test_rotation_jacobian_matches_finite_differences(orc):
    """The state turned by d and carried to a fixed plane of the new frame,
    as a function of the original state: analytic J_transport * J_rotation
    against central differences."""
    x0, X = 150.0, 170.0
    for d in (D20, -D20, 0.3):
        for p0 in ([3.0, 20.0, 0.2, 0.4, 1.5], [-12.0, -40.0, -0.5, -0.8, -3.0],
                   [25.0, 5.0, 0.6, 0.1, 0.2]):
            p0 = np.array(p0)
            rc, x1, p1, _, Jr = orc.rotate(d, x0, p0, np.zeros(15))
            assert rc == 0
            rc, p2, _, Jt = orc.transport(x1, X, p1, np.zeros(15))
            assert rc == 0
            J = Jt @ Jr

            def f(p):
                rc, x1, p1, _, _ = orc.rotate(d, x0, p, np.zeros(15))
                assert rc == 0
                # the plane X is fixed, so moving the point along x' is part of the map
                rc, p2, _, _ = orc.transport(x1, X, p1, np.zeros(15))
                assert rc == 0
                return p2
            for k in range(5):
                h = 1e-6 * max(1.0, abs(p0[k]))
                e = np.zeros(5)
                e[k] = h
                col = (f(p0 + e) - f(p0 - e)) / (2 * h)
                assert np.allclose(col, J[:, k], rtol=1e-6, atol=1e-7), (d, p0, k, col, J[:, k])


def test_rotation_round_trip_and_composition(orc):
    p0 = np.array([7.0, 11.0, 0.3, 0.2, 0.7])
    C0 = np.array([0.01, 0.0, 0.01, 0.001, 0.0, 0.002, 0.0, 0.003, 0.0, 0.01, 0.0, 0.0, 0.0, 0.0, 0.05])
    rc, x1, p1, C1, _ = orc.rotate(0.25, 120.0, p0, C0)
    rc2, x2, p2, C2, _ = orc.rotate(-0.25, x1, p1, C1)
    assert rc == rc2 == 0
    assert abs(x2 - 120.0) < 1e-12 and np.allclose(p2, p0, atol=1e-13)
    assert np.allclose(C2, C0, atol=1e-15)  # the Jacobians are inverse at the same point
    _, xa, pa, _, _ = orc.rotate(0.1, 120.0, p0, C0)
    _, xb, pb, _, _ = orc.rotate(0.15, xa, pa, C0)
    _, xc, pc, _, _ = orc.rotate(0.25, 120.0, p0, C0)
    assert abs(xb - xc) < 1e-12 and np.allclose(pb, pc, atol=1e-13)
    # a turn that makes the track run inward fails
    rc, *_ = orc.rotate(-2.0, 120.0, p0, C0)
    assert rc != 0


def check_whole(orc, ev, q, pt, tanl, n_segments):
    o = orc.track_event(ev)
    assert o["n_tracks"] == n_segments
    m = orc.merge_tracks(ev, o)
    assert m["n_tracks"] == 1
    # every cluster of the sector tracks (all but the last rows of a curler)
    assert sorted(m["k_hit_cid"].tolist()) == sorted(o["k_hit_cid"].tolist())
    assert len(m["k_hit_cid"]) >= ev.n - 3
    h0 = m["k_hit_cid"][0]
    assert m["k_sector"][0] == ev.sector[h0] and m["k_x"][0] == ev.row_x[ev.row[h0]]
    truth = np.array([ev.y[h0], ev.z[h0], ev.true_sinphi[h0], tanl, q / pt])
    err = np.abs(m["k_p"][0] - truth) / np.maximum(np.abs(truth), 1.0)
    assert err.max() < 2e-5, err
    assert m["k_chi2"][0] < 1e-3 and m["k_ndf"][0] == 2 * len(m["k_hit_cid"]) - 5
    return o, m


@pytest.mark.parametrize("q,pt,tanl,phi0,n_seg", [
    (1.0, 0.5, 0.3, 17.0, 2), (-1.0, 0.5, 0.3, 23.0, 2), (1.0, 0.25, 0.1, 8.0, 2),
    (1.0, 0.3, -0.4, 35.0, 3)])  # the last one crosses phi = 0 (sectors 1, 0, 17)
def test_noiseless_helix_across_phi_boundaries_is_one_track(orc, q, pt, tanl, phi0, n_seg):
    ev = noiseless(one(q, pt, tanl, math.radians(phi0)))
    o, m = check_whole(orc, ev, q, pt, tanl, n_seg)
    assert m["m_len"][m["m_ok"] == 1].tolist() == [n_seg]


def test_noiseless_helix_across_the_membrane_is_one_track(orc):
    q, pt, tanl = -1.0, 2.0, -0.3
    ev = noiseless(one(q, pt, tanl, math.radians(50.0), vz=45.0), split_z=True)
    assert set(ev.sector.tolist()) == {2, 20}  # phi sector 2 on both sides of z = 0
    check_whole(orc, ev, q, pt, tanl, 2)


def test_tracks_that_do_not_continue_each_other_stay_apart(orc):
    # one particle per side of a phi boundary, unrelated in curvature and dip
    parts = synth.Particles.concat([one(1.0, 5.0, 0.2, math.radians(18.0)),
                                    one(-1.0, 3.0, -0.5, math.radians(22.0))])
    ev = noiseless(parts)
    o = orc.track_event(ev)
    assert o["n_tracks"] == 2 and len(set(o["k_sector"].tolist())) == 2
    m = orc.merge_tracks(ev, o)
    assert m["n_tracks"] == 2 and (m["link_out"] < 0).all()
    # a single-sector event is left as it is
    ev1 = synth.one_sector_event(seed=1)
    o1 = orc.track_event(ev1)
    m1 = orc.merge_tracks(ev1, o1)
    assert m1["n_tracks"] == o1["n_tracks"] and np.array_equal(m1["k_hit_cid"], o1["k_hit_cid"])
    assert np.array_equal(m1["k_p"], o1["k_p"])


def test_merging_joins_particles_not_strangers(orc):
    """A 36-sector event: no merged track mixes particles, most particles cut
    by a sector boundary come out whole, and the near-tie bits are rare.
    (Sanity bars: the paper gives no merger figures.)"""
    ev = synth.batch_events(2, seed0=3000)[1]
    o = orc.track_event(ev)
    m = orc.merge_tracks(ev, o)
    lab = ev.label

    def major(h):
        l = lab[h]
        l = l[l >= 0]
        return np.bincount(l).argmax() if len(l) else -1
    seg_lab = np.array([major(o["k_hit_cid"][o["k_hit_off"][a]:o["k_hit_off"][a + 1]])
                        for a in range(o["n_tracks"])])
    mixed = sum(len({seg_lab[g] for g in s}) > 1 for s in m["sources"] if len(s) > 1)
    n_merged = sum(len(s) > 1 for s in m["sources"])
    assert n_merged > 1000 and mixed == 0
    # particles with several sector tracks before and after
    before = np.bincount(seg_lab[seg_lab >= 0])
    after_lab = np.array([seg_lab[s[0]] for s in m["sources"]])
    after = np.bincount(after_lab[after_lab >= 0], minlength=len(before))
    split_before = (before > 1).sum()
    split_after = (after > 1).sum()
    assert split_after < 0.1 * split_before, (split_before, split_after)
    assert (m["flags"] != 0).mean() < 0.05
