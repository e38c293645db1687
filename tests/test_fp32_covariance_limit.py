"""Why the backward pass carries a square-root factor of the covariance.

Storing the 5x5 covariance itself in binary32 is not enough: for short,
strongly curved tracks the y / sin(phi) block is nearly singular, and
rounding var(y), cov(y, sin phi) and var(sin phi) to binary32 after each
step moves the fitted q/pT by more than 1e-4 relative.  This test re-runs
one such tracklet of the pile-up event (sector 20) with float64 arithmetic
throughout and rounds only what is stored:

* no rounding reproduces the oracle to 1e-8 of the bars (the emulation is
  the oracle's algorithm), and so does the backward pass in Potter's
  square-root form (C = U U^T, two scalar updates per hit);
* rounding the 5-vector alone keeps q/pT within 5% of its bar;
* rounding the covariance alone (exact arithmetic otherwise) already moves
  q/pT beyond its bar;
* rounding everything the tracker stores (forward covariance, backward
  factor U, state) keeps q/pT within 5% of its bar.

So the tracker's backward pass carries U, not C (the forward pass, whose
state only seeds the backward one, keeps C).
"""
import numpy as np
import pytest

from paper_1712_09416_b300 import synth
from tests import _fp32, _parity


@pytest.fixture(scope="module")
def case(orc):
    ev = synth.pileup_event()
    sub = ev.select_sectors([20])
    o = orc.track_event(sub)
    # the tracklet started at cluster 3766336 of the pile-up event (12 hits)
    start = int(np.nonzero(sub.info["parent_index"] == 3766336)[0][0])
    ti = int(np.nonzero(o["t_start"] == start)[0][0])
    assert o["t_valid"][ti] == 1 and o["t_flags"][ti] == 0
    rh = o["t_rowhit"][ti]
    r0 = int(sub.row[start])
    rk = r0 + int(o["t_chain_len"][ti]) - 1
    return sub, o, ti, rh, r0, rk


def _qpt_scaled(sub, o, ti, rh, r0, rk, **kw):
    p = _fp32.fit_known_hits(sub.row_x, sub.y, sub.z, rh, r0, rk, **kw)
    _, s = _parity.param_errors(p, o["t_p"][ti])
    return s


def test_emulation_reproduces_the_oracle(case):
    s = _qpt_scaled(*case)
    assert s.max() < 1e-6, s


def test_binary32_state_storage_is_harmless(case):
    s = _qpt_scaled(*case, round_state=True)
    assert s[4] < 0.05, s


def test_binary32_covariance_storage_exceeds_the_qpt_bar(case):
    s = _qpt_scaled(*case, round_cov=np.ones((5, 5), bool))
    assert s[4] > 1.0, s
    # the y / sin(phi) block alone carries it
    m = np.zeros((5, 5), bool)
    for i, j in ((0, 0), (2, 0), (0, 2), (2, 2)):
        m[i, j] = True
    s_block = _qpt_scaled(*case, round_cov=m)
    assert s_block[4] > 1.0, s_block


def test_factor_form_reproduces_the_oracle(case):
    s = _qpt_scaled(*case, backward_factor=True)
    assert s.max() < 1e-6, s


def test_binary32_factor_storage_stays_within_the_bar(case):
    s = _qpt_scaled(*case, round_cov=np.ones((5, 5), bool), round_state=True,
                    backward_factor=True)
    assert s.max() < 0.05, s
