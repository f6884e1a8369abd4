"""Host filter construction (C++, through the C ABI) against the oracle."""
import math

import numpy as np
import pytest

import paper_1701_08935_gb300 as Z
from oracle import filter as F

GAPS = [(-1.05, -0.95, 0.95, 1.05), (0.1, 0.3, 2.0, 2.5), (-3.0, -2.999, 4.0, 4.01),
        (-math.inf, 0.5, 1.5, 1.6), (1.0, 1.0001, 1.2, 1.2001)]


@pytest.mark.parametrize("gaps", GAPS)
@pytest.mark.parametrize("r", [(1, 1), (2, 2), (2, 6), (3, 4)])
def test_filter_constants_match_oracle(gaps, r):
    f = Z.Filter(*gaps, *r)
    g = F.ZoloFilter(*gaps, *r)
    I = f.info
    # The oracle's A&S AGM loses accuracy in c_j as l1 -> 0 (cn near its zero): ~1e-13
    # relative for l1 >= 1e-6, up to ~5e-10 at l1 ~ 5e-8.  The product is pinned
    # separately against 40-digit mpmath (test_coefficients_against_mpmath).
    tol = 1e-9 if g.ell1 > 1e-6 else 3e-8
    assert I.ell1 == pytest.approx(g.ell1, rel=1e-12)
    assert I.alpha == pytest.approx(g.alpha, rel=1e-12, abs=1e-12)
    assert I.beta == pytest.approx(g.beta, rel=1e-12, abs=1e-12)
    assert I.gamma == pytest.approx(g.gamma, rel=1e-10)
    assert I.ell2 == pytest.approx(g.ell2, rel=tol)
    # delta0 is a difference of O(1) quantities on both sides: ~1e-16 absolute is all it carries
    assert I.delta0 == pytest.approx(g.delta0, rel=max(1e-7, 30 * tol), abs=2e-15)
    assert np.allclose(f.sigma_hat, g.sigma_hat, rtol=tol, atol=1e-12 * max(1, abs(g.alpha)))
    assert np.allclose(f.w_hat, g.w_hat, rtol=10 * tol, atol=1e-12)
    assert I.const_hat == pytest.approx(g.const_hat, rel=10 * tol, abs=1e-12)
    a, c = g.outer.partial_fractions()
    assert np.allclose(f.a, a, rtol=100 * tol)
    assert np.allclose(f.c, c, rtol=10 * tol)
    assert I.M == pytest.approx(g.M_out, rel=10 * tol)


@pytest.mark.parametrize("ell", [5e-8, 2.5e-5, 0.01, 0.4])
@pytest.mark.parametrize("r", [2, 3, 6])
def test_coefficients_against_mpmath(ell, r):
    """Theorem 1's c_j, M and the extremal error of the product's Zolotarev functions,
    evaluated at 40 digits (the rescaled inner function is exposed through the filter)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    # choose gaps whose Moebius parameter is exactly-ish `ell`: symmetric gaps +-(c, 1/c)
    # give l1 = ((1-c)/(1+c))^2 for this family; solve c from ell
    cc = (1 - ell ** 0.5) / (1 + ell ** 0.5)
    f = Z.Filter(-1 / cc, -cc, cc, 1 / cc, r, 1)
    L = mpmath.mpf(f.info.ell1)
    LP = mpmath.sqrt(1 - L * L)
    KP = mpmath.ellipk(LP ** 2)
    for j in range(1, r + 1):
        ref = L * L * (mpmath.ellipfun("sn", (2 * j - 1) * KP / (2 * r), m=LP ** 2)
                       / mpmath.ellipfun("cn", (2 * j - 1) * KP / (2 * r), m=LP ** 2)) ** 2
        # A&S AGM accuracy near u ~ K'/2 degrades as l -> 0 (see the C++ source)
        tol = 1e-12 if ell >= 1e-4 else (5e-11 if ell >= 1e-6 else 1e-9)
        assert float(f.c_hat[j - 1] / ref - 1) == pytest.approx(0.0, abs=tol)


@pytest.mark.parametrize("gaps", GAPS[:3])
def test_filter_eval_matches_oracle(gaps):
    f = Z.Filter(*gaps, 2, 3)
    g = F.ZoloFilter(*gaps, 2, 3)
    lo, hi = gaps[1] - 3 * (gaps[2] - gaps[1]), gaps[2] + 3 * (gaps[2] - gaps[1])
    x = np.linspace(lo, hi, 5001)
    assert np.max(np.abs(f(x) - g(x))) < 1e-10


def test_automatic_order():
    # smallest r = r1 = r2 with delta0 <= eps (Remark after Algorithm 2)
    gaps = (-1.005, -0.995, 0.995, 1.005)
    f = Z.Filter(*gaps, 0, 0, eps=1e-12)
    r = f.r1
    assert f.r1 == f.r2 and f.info.delta0 <= 1e-12
    assert F.ZoloFilter(*gaps, r - 1, r - 1).delta0 > 1e-12


@pytest.mark.parametrize("bad", [(1.0, 0.5, 2.0, 3.0), (0.0, 1.0, 0.5, 2.0), (0.0, 1.0, 2.0, 2.0),
                                 (math.nan, 1.0, 2.0, 3.0)])
def test_bad_gaps_rejected(bad):
    with pytest.raises(Z.ZoloError) as e:
        Z.Filter(*bad, 2, 2)
    assert e.value.status == Z.EINVAL


def test_inner_function_exact_to_rounding():
    # wide gaps and a high inner order: Zhat(l1) rounds to 1, l2 is clamped below 1
    f = Z.Filter(-2.5, -0.4, 0.4, 2.5, 16, 2)
    assert f.info.ell2 < 1.0 and f.info.delta0 < 1e-15


def test_bad_orders_rejected():
    for r in [(17, 2), (2, 17)]:
        with pytest.raises(Z.ZoloError):
            Z.Filter(0.0, 1.0, 2.0, 3.0, *r)


@pytest.mark.parametrize("gaps", [(-1.1, -0.9, 0.9, 1.1), (0.1, 0.3, 2.0, 2.5), (-math.inf, 0.5, 1.5, 1.6)])
def test_order_table_matches_oracle(gaps):
    t = Z.filter_table(*gaps, 3)
    g = F.delta0_table(*gaps, 3)
    # the oracle's extrema come from a numerical search: ~1e-5 relative at delta0 ~ 1e-10
    assert np.allclose(t, g, rtol=1e-4, atol=1e-15)
    assert np.allclose(t, t.T, rtol=1e-10, atol=1e-15)           # Theorem 2: only r1 r2 matters


def test_order_selection_modes():
    """Orders from eps (Remark after Algorithm 2): r1 fixed -> smallest r2; r2 fixed ->
    smallest r1; both free -> smallest r = r1 = r2, all read off the table."""
    gaps = (-1.1, -0.9, 0.9, 1.1)
    t = Z.filter_table(*gaps, 8)
    eps = 1e-9
    f = Z.Filter(*gaps, 2, 0, eps)
    want = 1 + int(np.argmax(t[1, :] <= eps))
    assert (f.r1, f.r2) == (2, want)
    assert f.info.delta0 <= eps < t[1, want - 2]
    f = Z.Filter(*gaps, 0, 3, eps)
    want = 1 + int(np.argmax(t[:, 2] <= eps))
    assert (f.r1, f.r2) == (want, 3)
    f = Z.Filter(*gaps, 0, 0, eps)
    d = np.diag(t)
    assert f.r1 == f.r2 == 1 + int(np.argmax(d <= eps))
    assert f.info.gap[0] == -1.1 and f.info.gap[3] == 1.1


@pytest.mark.parametrize("kind", ["CITZ", "CIGQ"])
@pytest.mark.parametrize("npoles", [2, 6, 16, 32])
def test_contour_filters_match_oracle(kind, npoles):
    a, b = 0.3, 1.7
    p = Z.ContourFilter(getattr(Z, "FILTER_" + kind), a, b, npoles)
    o = F.ContourFilter(kind, a, b, npoles)
    x = np.linspace(-1.0, 3.0, 401)
    assert np.allclose(p(x), o(x), rtol=1e-12, atol=1e-13)
    assert p.r1 == npoles // 2 and p.r2 == 0 and p.info.kind == getattr(Z, "FILTER_" + kind)
    order = lambda z: np.argsort(z.real + 1e-3 * z.imag)
    assert np.allclose(p.sigma_hat[order(p.sigma_hat)], o.sigma_hat[order(o.sigma_hat)], rtol=1e-14, atol=1e-14)
    assert np.allclose(p.w_hat[order(p.sigma_hat)], o.w_hat[order(o.sigma_hat)], rtol=1e-12, atol=1e-15)


def test_contour_filter_arguments_rejected():
    for args in ((Z.FILTER_CITZ, 1.0, 0.0, 4), (Z.FILTER_CIGQ, 0.0, 1.0, 3), (Z.FILTER_CITZ, 0.0, 1.0, 0),
                 (Z.FILTER_CITZ, 0.0, 1.0, 2 * Z.MAX_R + 2), (7, 0.0, 1.0, 4)):
        with pytest.raises(Z.ZoloError) as e:
            Z.ContourFilter(*args)
        assert e.value.status == Z.EINVAL
