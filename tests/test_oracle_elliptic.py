"""Pins for the oracle's elliptic functions (A&S 16.4 / 17.6 AGM) against
independent evaluations (scipy's Cephes routines, mpmath) and exact identities."""
import math

import numpy as np
import pytest
import scipy.special as ss

from oracle import elliptic as E


@pytest.mark.parametrize("k", [0.0, 0.1, 0.5, 0.9, 0.99, 0.999999])
def test_K_matches_scipy(k):
    # scipy.special.ellipkm1 takes p = 1 - k^2, formed here without cancellation
    assert E.ellipk(k) == pytest.approx(float(ss.ellipkm1((1 - k) * (1 + k))), rel=1e-14)


def test_K_near_one_with_complement():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    for kp in [1e-3, 1e-6, 1e-9]:
        k = math.sqrt((1 - kp) * (1 + kp))
        ref = float(mpmath.ellipk(1 - mpmath.mpf(kp) ** 2))
        assert E.ellipk(k, kp) == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("k", [0.2, 0.7, 0.95])
def test_sn_cn_dn_match_scipy(k):
    K = E.ellipk(k)
    for u in np.linspace(0.0, 2.0 * K, 9):
        sn, cn, dn = E.ellipj(u, k)
        rs, rc, rd, _ = ss.ellipj(u, k * k)
        assert sn == pytest.approx(rs, abs=1e-13)
        assert cn == pytest.approx(rc, abs=1e-13)
        assert dn == pytest.approx(rd, abs=1e-13)


@pytest.mark.parametrize("kp", [1e-2, 1e-4, 1e-7])
def test_sn_cn_dn_match_mpmath_near_k1(kp):
    # scipy's Cephes ellipj loses ~1e-13 here; 40-digit mpmath is the reference.
    # The AGM's asin steps lose accuracy as k -> 1 (their arguments approach +-1):
    # about 2e-14 absolute for k' = 1e-7, i.e. ~1e-11 relative in c_j at such gaps.
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    k = math.sqrt((1 - kp) * (1 + kp))
    m = 1 - mpmath.mpf(kp) ** 2
    K = E.ellipk(k, kp)
    for u in np.linspace(0.0, 2.0 * K, 9):
        sn, cn, dn = E.ellipj(u, k, kp)
        assert sn == pytest.approx(float(mpmath.ellipfun("sn", u, m=m)), abs=3e-14)
        assert cn == pytest.approx(float(mpmath.ellipfun("cn", u, m=m)), abs=3e-14)
        assert dn == pytest.approx(float(mpmath.ellipfun("dn", u, m=m)), abs=3e-14)


@pytest.mark.parametrize("k", [0.3, 0.99, 1 - 1e-10])
def test_identities_and_quarter_period(k):
    kp = math.sqrt((1 - k) * (1 + k))
    K = E.ellipk(k, kp)
    sn, cn, dn = E.ellipj(K, k, kp)
    assert sn == pytest.approx(1.0, abs=1e-12)
    assert abs(cn) < 1e-7
    assert dn == pytest.approx(kp, rel=1e-6)
    for u in np.linspace(0.1, 0.9, 5) * K:
        sn, cn, dn = E.ellipj(u, k, kp)
        assert sn * sn + cn * cn == pytest.approx(1.0, abs=1e-14)
        assert dn * dn + k * k * sn * sn == pytest.approx(1.0, abs=1e-14)


def test_degenerate_moduli():
    # k = 0: circular functions; k -> 1: hyperbolic ones
    sn, cn, dn = E.ellipj(0.7, 0.0)
    assert (sn, cn, dn) == pytest.approx((math.sin(0.7), math.cos(0.7), 1.0), abs=1e-15)
    sn, cn, dn = E.ellipj(0.7, 1 - 1e-16, 1e-8)
    assert sn == pytest.approx(math.tanh(0.7), abs=1e-12)
    assert cn == pytest.approx(1 / math.cosh(0.7), abs=1e-12)
