"""Pins of the oracle's helix transport (C5) and Kalman update (C6).

The transport is checked against the generator's closed-form helix/plane
crossings, computed on the global-frame circle (a different formulation from
the oracle's sector-frame update), and its Jacobian against central finite
differences.  The update is checked against the information form of the same
Bayesian step and against a batch least-squares solution.
"""
import math

import numpy as np
import pytest

from paper_1712_09416_b300 import synth


def _truth_states(ev):
    """Per-row truth (x, y, z, s) of a single-helix event in its most populated sector."""
    sec = np.bincount(ev.sector).argmax()
    m = np.nonzero(ev.sector == sec)[0]
    o = m[np.argsort(ev.row[m])]
    x = ev.row_x.astype(np.float64)[ev.row[o]]
    return x, ev.y[o], ev.z[o], ev.true_sinphi[o], ev.row[o]


@pytest.mark.parametrize("q,pt,tanl,phi0", [
    (1.0, 0.35, 0.4, math.radians(10.0)),
    (-1.0, 0.35, -0.7, math.radians(12.0)),
    (1.0, 2.0, 0.05, math.radians(4.0)),
    (-1.0, 9.0, 0.9, math.radians(17.0)),
    (1.0, 0.8, -0.2, math.radians(14.0)),
])
def test_transport_matches_closed_form_crossings(orc, q, pt, tanl, phi0):
    ev = synth.noiseless_track(q, pt, tanl, phi0, n_sectors_phi=18)
    x, y, z, s, rows = _truth_states(ev)
    assert len(x) > 20
    qpt = q / pt
    # row to row, one large jump outward, and one large jump inward
    pairs = [(i, i + 1) for i in range(len(x) - 1)] + [(0, len(x) - 1), (len(x) - 1, 0),
                                                        (5, len(x) // 2)]
    for a, b in pairs:
        p0 = [y[a], z[a], s[a], tanl, qpt]
        rc, p1, _, _ = orc.transport(x[a], x[b], p0, np.eye(5)[np.tril_indices(5)], bz=0.5)
        assert rc == 0
        assert abs(p1[0] - y[b]) < 1e-10
        assert abs(p1[1] - z[b]) < 1e-10
        assert abs(p1[2] - s[b]) < 1e-12
        assert p1[3] == tanl and p1[4] == qpt


def test_transport_straight_line_at_zero_field(orc):
    s0, t = 0.3, 0.6
    rc, p1, _, _ = orc.transport(100.0, 130.0, [1.0, 2.0, s0, t, 0.7], np.zeros(15), bz=0.0)
    c0 = math.sqrt(1 - s0 * s0)
    assert rc == 0
    assert p1[0] == pytest.approx(1.0 + 30.0 * s0 / c0, abs=1e-12)
    assert p1[1] == pytest.approx(2.0 + t * 30.0 / c0, abs=1e-12)
    assert p1[2] == s0


def test_transport_fails_at_sin_max(orc):
    # q/pT such that s1 = s0 + C_k dx crosses 0.99
    kB = synth.KAPPA * 0.5
    s0, dx = 0.9, 10.0
    qpt = -(0.995 - s0) / (kB * dx)   # C_k = -kB*qpt > 0
    rc, _, _, _ = orc.transport(100.0, 100.0 + dx, [0, 0, s0, 0, qpt], np.zeros(15), bz=0.5)
    assert rc == -1
    qpt = -(0.985 - s0) / (kB * dx)
    rc, _, _, _ = orc.transport(100.0, 100.0 + dx, [0, 0, s0, 0, qpt], np.zeros(15), bz=0.5)
    assert rc == 0


def _num_jac(orc, x0, x1, p, bz):
    J = np.zeros((5, 5))
    for j in range(5):
        h = 1e-6 * max(1.0, abs(p[j]))
        pp = np.array(p, float); pp[j] += h
        pm = np.array(p, float); pm[j] -= h
        _, fp, _, _ = orc.transport(x0, x1, pp, np.zeros(15), bz=bz)
        _, fm, _, _ = orc.transport(x0, x1, pm, np.zeros(15), bz=bz)
        J[:, j] = (fp - fm) / (2 * h)
    return J


@pytest.mark.parametrize("seed", range(12))
def test_jacobian_matches_finite_differences(orc, seed):
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(85, 247)
    dx = rng.choice([-1, 1]) * rng.uniform(0.5, 40.0)
    p = [rng.uniform(-20, 20), rng.uniform(-200, 200), rng.uniform(-0.6, 0.6),
         rng.uniform(-1, 1), rng.choice([0.0, 1e-7, rng.uniform(-8, 8)])]
    bz = 0.5
    rc, _, _, J = orc.transport(x0, x0 + dx, p, np.zeros(15), bz=bz)
    assert rc == 0
    Jn = _num_jac(orc, x0, x0 + dx, p, bz)
    scale = np.maximum(1.0, np.abs(Jn))
    assert np.all(np.abs(J - Jn) / scale < 1e-7), (J, Jn)


def test_covariance_is_propagated_as_J_C_Jt(orc):
    rng = np.random.default_rng(7)
    A = rng.normal(size=(5, 5))
    M = A @ A.T + 0.1 * np.eye(5)
    p = [3.0, -40.0, 0.2, 0.5, 1.3]
    rc, _, Ct1, J = orc.transport(120.0, 131.0, p, orc.pack_cov(M), bz=0.5)
    assert rc == 0
    np.testing.assert_allclose(orc.unpack_cov(Ct1), J @ M @ J.T, rtol=1e-12, atol=1e-12)


def test_transport_round_trip(orc):
    rng = np.random.default_rng(3)
    A = rng.normal(size=(5, 5))
    M = A @ A.T + np.eye(5)
    p = np.array([5.0, 30.0, -0.3, -0.4, -2.5])
    rc, p1, C1, _ = orc.transport(90.0, 200.0, p, orc.pack_cov(M), bz=0.5)
    rc2, p2, C2, _ = orc.transport(200.0, 90.0, p1, C1, bz=0.5)
    assert rc == 0 and rc2 == 0
    np.testing.assert_allclose(p2, p, rtol=0, atol=1e-11)
    np.testing.assert_allclose(orc.unpack_cov(C2), M, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("seed", range(8))
def test_update_equals_information_form(orc, seed):
    rng = np.random.default_rng(100 + seed)
    A = rng.normal(size=(5, 5))
    M = A @ A.T + 0.05 * np.eye(5)
    p = rng.normal(size=5)
    m = rng.normal(size=2)
    vy, vz = 0.01, 0.02
    p1, Ct1, chi2 = orc.update(p, orc.pack_cov(M), m[0], m[1], vy, vz)
    H = np.zeros((2, 5)); H[0, 0] = H[1, 1] = 1.0
    Vi = np.diag([1 / vy, 1 / vz])
    Mi = np.linalg.inv(M)
    Cpost = np.linalg.inv(Mi + H.T @ Vi @ H)
    ppost = Cpost @ (Mi @ p + H.T @ Vi @ m)
    np.testing.assert_allclose(orc.unpack_cov(Ct1), Cpost, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(p1, ppost, rtol=1e-9, atol=1e-12)
    # chi2 increment = minimum of the quadratic objective
    obj = (ppost - p) @ Mi @ (ppost - p) + (m - H @ ppost) @ Vi @ (m - H @ ppost)
    assert chi2 == pytest.approx(obj, rel=1e-9)


def test_sequential_updates_equal_batch_least_squares(orc):
    rng = np.random.default_rng(5)
    A = rng.normal(size=(5, 5))
    M = A @ A.T + 0.5 * np.eye(5)
    p0 = rng.normal(size=5)
    ms = rng.normal(size=(7, 2))
    vy, vz = 0.04, 0.09
    p, Ct, chi2 = p0.copy(), orc.pack_cov(M), 0.0
    for m in ms:
        p, Ct, c = orc.update(p, Ct, m[0], m[1], vy, vz)
        chi2 += c
    H = np.zeros((2, 5)); H[0, 0] = H[1, 1] = 1.0
    Vi = np.diag([1 / vy, 1 / vz])
    Mi = np.linalg.inv(M)
    info = Mi + len(ms) * H.T @ Vi @ H
    pb = np.linalg.solve(info, Mi @ p0 + H.T @ Vi @ ms.sum(axis=0))
    obj = (pb - p0) @ Mi @ (pb - p0) + sum((m - H @ pb) @ Vi @ (m - H @ pb) for m in ms)
    np.testing.assert_allclose(p, pb, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(orc.unpack_cov(Ct), np.linalg.inv(info), rtol=1e-9, atol=1e-12)
    assert chi2 == pytest.approx(obj, rel=1e-9)
