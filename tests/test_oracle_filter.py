"""Pins for the oracle's Zolotarev filter (Theorems 1-3, Propositions 1-2, eq. req)
against closed forms, equioscillation, the modular equation, the paper's worked
values and pointwise identities between independent formulas."""
import math
import os

import numpy as np
import pytest
import scipy.special as ss
from scipy.optimize import brentq

from oracle import elliptic
from oracle import filter as F

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _extrema_points(r, ell):
    """Closed-form equioscillation points x_j = ell / dn((j-1) K'/(2r); ell')."""
    ellp = math.sqrt((1 - ell) * (1 + ell))
    Kp = elliptic.ellipk(ellp, ell)
    return [ell / elliptic.ellipj((j - 1) * Kp / (2 * r), ellp, ell)[2] for j in range(1, 2 * r + 2)]


@pytest.mark.parametrize("ell", [0.1, 0.01, 1e-4])
def test_r1_closed_form(ell):
    z = F.Zolotarev(1, ell)
    assert z.c[0] == pytest.approx(ell, rel=1e-13)
    d = ((1 - math.sqrt(ell)) / (1 + math.sqrt(ell))) ** 2
    assert z.delta == pytest.approx(d, rel=1e-10)
    # l2 = Zhat(l1) = 2 sqrt(l)/(1+l) (Landen transformation)
    assert float(z.scaled(ell)) == pytest.approx(2 * math.sqrt(ell) / (1 + ell), rel=1e-10)


def test_r1_printed_value():
    # value quoted alongside the r = 1 case: delta(2, 0.1) = 0.269874
    assert F.Zolotarev(1, 0.1).delta == pytest.approx(0.269874, abs=5e-7)


@pytest.mark.parametrize("r", [2, 3, 4, 6])
@pytest.mark.parametrize("ell", [0.3, 0.02, 1e-5])
def test_equioscillation(r, ell):
    """1 - Z(x_j) = (-1)^(j+1) delta at the 2r+1 points of Theorem 1's remark."""
    z = F.Zolotarev(r, ell)
    xs = _extrema_points(r, ell)
    assert xs[0] == pytest.approx(ell) and xs[-1] == pytest.approx(1.0)
    for j, x in enumerate(xs, start=1):
        assert 1.0 - float(z(x)) == pytest.approx((-1) ** (j + 1) * z.delta, abs=1e-12 + 1e-9 * z.delta)
    # no sample on [l,1] or [-1,-l] exceeds delta
    t = np.exp(np.linspace(math.log(ell), 0, 50001))
    assert np.max(np.abs(1 - z(t))) <= z.delta * (1 + 1e-9) + 1e-15
    assert np.max(np.abs(-1 - z(-t))) <= z.delta * (1 + 1e-9) + 1e-15


def _modular_delta(r, ell):
    """delta from the degree-2r modular equation K(lt')/K(lt) = K(l')/(2r K(l)),
    lt = (1-delta)/(1+delta); solved by bisection with scipy's K (parameter m = k^2)."""
    # K(k') = ellipkm1(k^2) (scipy's p = 1 - m form), K(k) = ellipk(k^2)
    target = ss.ellipkm1(ell * ell) / (2 * r * ss.ellipk(ell * ell))
    g = lambda lt: ss.ellipkm1(lt * lt) / ss.ellipk(lt * lt) - target
    lt = brentq(g, 1e-12, 1 - 1e-12, xtol=1e-17, rtol=1e-15)
    return (1 - lt) / (1 + lt)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
@pytest.mark.parametrize("ell", [0.5, 0.05])
def test_delta_modular_equation(r, ell):
    z = F.Zolotarev(r, ell)
    assert z.delta == pytest.approx(_modular_delta(r, ell), rel=1e-8)


@pytest.mark.parametrize("r1,r2", [(1, 1), (2, 2), (1, 3), (2, 3), (3, 2)])
@pytest.mark.parametrize("ell1", [0.2, 0.003])
def test_theorem2_composition(r1, r2, ell1):
    """Z_2r2(Zhat_2r1(x; l1); l2) = Z_(2r1)(2r2)(x; l1)  (Theorem 2, eq. Z)."""
    zi = F.Zolotarev(r1, ell1)
    ell2 = float(zi.scaled(ell1))
    zo = F.Zolotarev(r2, ell2)
    zb = F.Zolotarev(2 * r1 * r2, ell1)
    x = np.concatenate([np.exp(np.linspace(math.log(ell1), 0, 301)), [1.7, 5.0]])
    lhs = zo(zi.scaled(x))
    rhs = zb(x)
    assert np.max(np.abs(lhs - rhs)) < 2e-13
    assert np.max(np.abs(zo(zi.scaled(-x)) + rhs)) < 2e-13


@pytest.mark.parametrize("gaps", [(-1.05, -0.95, 0.95, 1.05), (0.1, 0.3, 2.0, 2.5),
                                  (-3.0, -2.999, 4.0, 4.01), (-math.inf, 0.5, 1.5, 1.6)])
def test_mobius_conditions(gaps):
    alpha, beta, gamma, ell1 = F.mobius(*gaps)
    am, ap, bm, bp = gaps
    T = lambda x: F.mobius_eval(x, alpha, beta, gamma)
    assert float(T(ap)) == pytest.approx(1.0, abs=1e-12)
    assert float(T(bm)) == pytest.approx(ell1, abs=1e-12)
    assert float(T(bp)) == pytest.approx(-ell1, abs=1e-12)
    if math.isinf(am):
        assert gamma == pytest.approx(-1.0, abs=1e-12)          # T(-inf) = gamma = -1
    else:
        assert float(T(am)) == pytest.approx(-1.0, abs=1e-10)  # the unused 4th condition
    assert 0 < ell1 < 1
    assert bm < alpha < bp and am < beta < ap                  # reading of eq. req
    assert -1.0 <= gamma <= -ell1


def test_fig4_pole_circle_radius():
    vals = {}
    with open(os.path.join(GOLDEN, "fig4_pole_circle.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                key, *rest = line.split()
                vals[key] = [float(v) for v in rest]
    gaps = vals["gaps"]
    alpha, beta, gamma, _ = F.mobius(*gaps)
    assert round(abs(alpha - beta) / 2, int(vals["digits"][0])) == vals["radius"][0]
    assert abs(alpha + beta) < 1e-12                          # centred at the origin
    # the literal caption gaps give a different circle
    a2, b2, _, _ = F.mobius(-1.1, -0.9, 0.9, 1.1)
    assert abs(abs(a2 - b2) / 2 - 0.994987) < 1e-6


@pytest.mark.parametrize("r", [1, 2, 3, 5, 8])
def test_prop1_cor1_partial_fractions(r):
    z = F.Zolotarev(r, 0.01)
    a, codd = z.partial_fractions()
    x = np.concatenate([np.linspace(-3, 3, 61), [0.0137, 1e-3]])
    pf = z.M * x * sum(aj / (x * x + cj) for aj, cj in zip(a, codd))
    assert np.max(np.abs(pf - z(x))) < 1e-12
    xc = x + 0.3j
    cf = 0.5 * z.M * sum(aj * (1 / (xc + 1j * math.sqrt(cj)) + 1 / (xc - 1j * math.sqrt(cj)))
                         for aj, cj in zip(a, codd))
    prod = z.M * xc * np.prod([xc * xc + z.c[2 * j - 1] for j in range(1, r)], axis=0) \
        / np.prod([xc * xc + z.c[2 * j - 2] for j in range(1, r + 1)], axis=0)
    assert np.max(np.abs(cf - prod)) < 1e-11


@pytest.mark.parametrize("r", [1, 2, 4])
def test_prop2_poles_weights(r):
    alpha, beta, gamma, ell = F.mobius(0.1, 0.3, 2.0, 2.5)
    z = F.Zolotarev(r, ell)
    s, w, const = F.prop2_poles(z, alpha, beta, gamma)
    x = np.concatenate([np.linspace(-4, 6, 57), [0.2, 2.2]]) + 0.0j
    x = np.concatenate([x, x + 0.05j])
    pf = const + sum(wj / (x - sj) + np.conj(wj) / (x - np.conj(sj)) for sj, wj in zip(s, w))
    t = gamma * (x - alpha) / (x - beta)
    ref = z.M * t * np.prod([t * t + z.c[2 * j - 1] for j in range(1, r)], axis=0) \
        / np.prod([t * t + z.c[2 * j - 2] for j in range(1, r + 1)], axis=0)
    assert np.max(np.abs(pf - ref)) < 1e-11 * max(1.0, np.max(np.abs(ref)))
    # all poles on the circle through alpha and beta centred on the real axis (Fig. 4)
    centre, radius = 0.5 * (alpha + beta), 0.5 * abs(alpha - beta)
    assert np.allclose(np.abs(s - centre), radius, rtol=1e-12)
    # one half-plane: sign(Im s) = sign((beta - alpha) gamma)
    assert np.all(np.sign(s.imag) == np.sign((beta - alpha) * gamma))


@pytest.mark.parametrize("r1,r2", [(1, 1), (2, 2), (2, 6), (3, 3)])
def test_filter_endpoints_and_uniform_error(r1, r2):
    gaps = (-1.2, -1.0, 1.0, 1.15)
    f = F.ZoloFilter(*gaps, r1, r2)
    am, ap, bm, bp = gaps
    d0 = f.delta0
    assert float(f(ap)) == pytest.approx(1 - d0, abs=1e-12 + 1e-9 * d0)
    assert float(f(bm)) == pytest.approx(1 - d0, abs=1e-12 + 1e-9 * d0)
    assert float(f(am)) == pytest.approx(d0, abs=1e-12 + 1e-9 * d0)
    assert float(f(bp)) == pytest.approx(d0, abs=1e-12 + 1e-9 * d0)
    inside = np.linspace(ap, bm, 20001)
    outside = np.concatenate([np.linspace(am - 50, am, 20001), np.linspace(bp, bp + 50, 20001),
                              [-1e6, 1e6]])
    assert np.max(np.abs(1 - f(inside))) <= d0 * (1 + 1e-8) + 1e-14
    assert np.max(np.abs(f(outside))) <= d0 * (1 + 1e-8) + 1e-14


@pytest.mark.parametrize("r1,r2", [(1, 2), (2, 2), (2, 3)])
def test_inner_operator_and_outer_combination(r1, r2):
    """G(x) via Proposition 2 equals Zhat(T(x)); Algorithm 2's final combination of the
    2 r2 shifted resolvents of G reproduces R_ab(x) on the real line."""
    f = F.ZoloFilter(0.0, 0.2, 1.0, 1.3, r1, r2)
    x = np.linspace(-2, 3, 401)
    g = f.G_scalar(x)
    assert np.max(np.abs(g - f.inner.scaled(f.T(x)))) < 1e-11
    shifts, omegas = f.outer_shifts()
    rr = 0.5 + sum(om / (g + s) for s, om in zip(shifts, omegas))
    assert np.max(np.abs(rr - f(x))) < 1e-11


@pytest.mark.parametrize("r1,r2", [(1, 1), (2, 2), (2, 3)])
def test_composite_poles_theorem2(r1, r2):
    f = F.ZoloFilter(0.0, 0.2, 1.0, 1.3, r1, r2)
    s, w, c0, big = F.composite_poles(f)
    assert len(s) == 2 * r1 * r2
    x = np.linspace(-2, 3, 301)
    rr = c0 + sum(wj / (x - sj) + np.conj(wj) / (x - np.conj(sj)) for sj, wj in zip(s, w))
    assert np.max(np.abs(rr - f(x))) < 1e-10


def test_six_factorizations_reach_machine_accuracy():
    """Section 2.2 after Fig. 2: with eigengaps 1e-2 around +-1, six factorizations
    (the composite Zolo(6,6)) approximate the rectangle to machine accuracy."""
    f = F.ZoloFilter(-1.005, -0.995, 0.995, 1.005, 6, 6)
    assert f.delta0 < 1e-15
    g = F.ZoloFilter(-1.005, -0.995, 0.995, 1.005, 2, 2)
    assert g.delta0 > 1e-6          # a low order is visibly worse


@pytest.mark.parametrize("r", [1, 2, 3, 5])
@pytest.mark.parametrize("ell", [1e-3, 0.05, 0.3, 0.9])
def test_zolo_c_reflection_identities(r, ell):
    """c_j of Theorem 1 from sn/cn at u_j = j K'/(2r): since sn(K' - u) = cn(u)/dn(u) and
    cn(K' - u) = l sn(u)/dn(u) (modulus l'), c_j c_{2r-j} = l^2 and c_r = l; the c_j increase
    with j (sn/cn increases on (0, K'))."""
    c = F.zolo_c(r, ell)
    assert len(c) == 2 * r - 1
    assert c[r - 1] == pytest.approx(ell, rel=1e-12)
    for j in range(1, 2 * r):
        assert c[j - 1] * c[2 * r - j - 1] == pytest.approx(ell * ell, rel=1e-11)
    assert all(c[i] < c[i + 1] for i in range(len(c) - 1))
    # the product form is odd and positive on (0, 1]
    x = np.linspace(1e-3, 1.0, 50)
    assert np.all(F.zolo_product(x, c) > 0)
    assert np.allclose(F.zolo_product(-x, c), -F.zolo_product(x, c), rtol=0, atol=1e-15)


@pytest.mark.parametrize("npoles", [2, 4, 8, 16])
def test_citz_closed_form(npoles):
    """Trapezoidal rule on the circle through a, b with nodes at 2 pi (j - 1/2)/p: the nodes
    zeta_j = e^{i theta_j} are the roots of zeta^p = -1, and the partial fractions of
    1/(1 + s^p) are sum_j (zeta_j / p) / (zeta_j - s) (residue 1/(p zeta_j^(p-1)) = -zeta_j/p).
    So CITZ(p)(x) = 1 / (1 + ((x - c)/rho)^p) exactly (Section 1.1's trapezoidal filter)."""
    a, b = 0.3, 1.7
    f = F.ContourFilter("CITZ", a, b, npoles)
    x = np.linspace(-2.0, 4.0, 241)
    s = (x - 0.5 * (a + b)) / (0.5 * (b - a))
    assert np.allclose(f(x), 1.0 / (1.0 + s ** npoles), rtol=1e-13, atol=1e-15)
    assert len(f.sigma_hat) == npoles // 2 and np.all(f.sigma_hat.imag > 0)


def test_cigq_pins():
    """Gauss-Legendre contour filter: the integrand at the centre is the constant 1/(2 pi)
    in theta, integrated exactly (R(c) = 1); the rule is symmetric about the centre; with
    many points it converges to the indicator of (a, b) away from the contour and to the
    principal value 1/2 on it (a and b sit at theta = pi, 0, the ends of both half rules)."""
    a, b = -1.0, 3.0
    c, rho = 1.0, 2.0
    f = F.ContourFilter("CIGQ", a, b, 8)
    assert f(np.array([c]))[0] == pytest.approx(1.0, abs=1e-14)
    x = np.linspace(-4, 6, 101)
    assert np.allclose(f(x), f(2 * c - x), atol=1e-14)
    g = F.ContourFilter("CIGQ", a, b, 96)
    inside = np.array([c - 0.5 * rho, c + 0.5 * rho, c + 0.3 * rho])
    outside = np.array([c - 2 * rho, c + 2 * rho, c + 5 * rho])
    assert np.max(np.abs(g(inside) - 1.0)) < 1e-12
    assert np.max(np.abs(g(outside))) < 1e-12
    assert np.allclose(g(np.array([a, b])), 0.5, atol=1e-10)
    # wrong half-weight (pi/2 -> pi) would double R(c)
    assert len(g.sigma_hat) == 48


def test_delta0_table_depends_on_r1_r2_product():
    """Theorem 2: S(x; l1) = Z_{(2r1)(2r2)}(x; l1), so the error delta0 of the Remark after
    Algorithm 2 depends on (r1, r2) only through r1 r2: the table is symmetric and
    delta0(1, 4) = delta0(2, 2) = delta0(4, 1); it decreases along rows and columns."""
    gaps = (-1.1, -0.9, 0.9, 1.1)
    t = F.delta0_table(*gaps, 4)
    assert np.allclose(t, t.T, rtol=1e-6, atol=1e-15)      # (1 - S)/2 carries ~1e-16 absolute
    assert t[0, 3] == pytest.approx(t[1, 1], rel=1e-6)
    assert t[3, 0] == pytest.approx(t[1, 1], rel=1e-6)
    assert np.all(np.diff(t, axis=0) < 0) and np.all(np.diff(t, axis=1) < 0)
    # and the entries are the composite function's error at l1 (the Remark): (1 - S(l1))/2
    f = F.ZoloFilter(*gaps, 2, 3)
    assert t[1, 2] == pytest.approx(0.5 * (1.0 - float(f.S(f.ell1))), rel=1e-12)
