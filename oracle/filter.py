"""Zolotarev-composite rational filter R_ab (oracle).

Test infrastructure only (see ``oracle/__init__``).

Follows Section 2.2 and 2.3 of Li & Yang:
  * Theorem 1 (eq. ZoloFunc, eq. coef): Z_2r(x; l) = M x prod(x^2+c_2j)/prod(x^2+c_2j-1),
    c_j = l^2 sn^2(jK'/2r; l') / cn^2(jK'/2r; l'), l' = sqrt(1-l^2), K' = K(l').
    M is fixed by the equioscillation condition stated with Theorem 1: by oddness of
    Z it reads  min_[l,1] Z + max_[l,1] Z = 2.  The oracle finds the extrema of the
    unscaled product on [l,1] numerically (dense log grid + bounded scalar
    minimisation), i.e. from the definition, not from a closed form.
  * eq. rZ: Zhat = Z / max_[l,1] Z ;  eq. S: S(x;l1) = Z_2r2(Zhat_2r1(x;l1); l2),
    l2 = Zhat_2r1(l1; l1).
  * eq. mo / eq. req: T(x) = gamma (x-alpha)/(x-beta) with T(a-)=-1, T(a+)=1,
    T(b-)=l1, T(b+)=-l1.  l1 comes from cross-ratio invariance of Moebius maps; then
    (gamma, gamma*alpha, beta) solve the three linear equations at a+, b-, b+.
    T(a-) = -1 is left unused and serves as a check.  Reading: the equations fix the
    zero alpha inside (b-,b+) and the pole beta inside (a-,a+); the prose placing alpha
    in (a-,a+) is inconsistent with them.
  * eq. R2: R_ab(x) = (S(T(x); l1) + 1) / 2.
  * Proposition 1 (eq. pa): Z = M x sum_j a_j / (x^2 + c_2j-1) with the printed b_j, a_j.
  * Corollary 1 (eq. paRe): Z = (M/2) sum_j a_j (1/(x + i sqrt c) + 1/(x - i sqrt c)).
  * Proposition 2: Z(T(x)) = M sum_j a_j gamma/(gamma^2+c) + M sum_j (w_j/(x-s_j) + conj),
    s_j = (gamma alpha + i sqrt(c) beta)/(gamma + i sqrt(c)),
    w_j = a_j (s_j - beta) / (2 (gamma + i sqrt(c))).
"""
import math
import numpy as np
from scipy.optimize import minimize_scalar

from . import elliptic


# ----------------------------------------------------------------------------- Theorem 1
def zolo_c(r, ell):
    """c_1..c_{2r-1} of Theorem 1 (eq. coef); returned as a list, c[j-1] = c_j."""
    ellp = math.sqrt((1.0 - ell) * (1.0 + ell))
    Kp = elliptic.ellipk(ellp, ell)
    c = []
    for j in range(1, 2 * r):
        sn, cn, _ = elliptic.ellipj(j * Kp / (2 * r), ellp, ell)
        c.append(ell * ell * sn * sn / (cn * cn))
    return c


def zolo_product(x, c):
    """Unscaled product f(x) = x prod_{j<r}(x^2+c_2j) / prod_{j<=r}(x^2+c_2j-1)."""
    x = np.asarray(x, dtype=np.float64)
    r = (len(c) + 1) // 2
    num = x.copy()
    den = np.ones_like(x)
    for j in range(1, r + 1):
        den = den * (x * x + c[2 * j - 2])
    for j in range(1, r):
        num = num * (x * x + c[2 * j - 1])
    return num / den


def _extrema_on(c, ell):
    """(min f, max f) over [ell, 1] from the definition: log grid + local refinement."""
    xs = np.exp(np.linspace(math.log(ell), 0.0, 20001))
    f = zolo_product(xs, c)
    vals_min = [f[0], f[-1]]
    vals_max = [f[0], f[-1]]
    for i in range(1, len(xs) - 1):
        if f[i] <= f[i - 1] and f[i] <= f[i + 1]:
            res = minimize_scalar(lambda t: float(zolo_product(math.exp(t), c)),
                                  bounds=(math.log(xs[i - 1]), math.log(xs[i + 1])),
                                  method="bounded", options={"xatol": 1e-14})
            vals_min.append(min(float(res.fun), f[i]))
        if f[i] >= f[i - 1] and f[i] >= f[i + 1]:
            res = minimize_scalar(lambda t: -float(zolo_product(math.exp(t), c)),
                                  bounds=(math.log(xs[i - 1]), math.log(xs[i + 1])),
                                  method="bounded", options={"xatol": 1e-14})
            vals_max.append(max(-float(res.fun), f[i]))
    return min(vals_min), max(vals_max)


class Zolotarev:
    """Z_2r(x; ell) of Theorem 1 together with its error delta(2r, ell)."""

    def __init__(self, r, ell):
        if not (r >= 1 and 0.0 < ell < 1.0):
            raise ValueError("need r >= 1 and 0 < ell < 1")
        self.r, self.ell = int(r), float(ell)
        self.c = zolo_c(self.r, self.ell)
        fmin, fmax = _extrema_on(self.c, self.ell)
        # min Z + max Z = 2 on [ell,1]  (equioscillation condition of Theorem 1)
        self.M = 2.0 / (fmin + fmax)
        self.zmax = self.M * fmax            # = 1 + delta
        self.zmin = self.M * fmin            # = 1 - delta
        self.delta = self.zmax - 1.0

    def __call__(self, x):
        return self.M * zolo_product(x, self.c)

    def scaled(self, x):
        """Zhat_2r(x; ell) = Z / max_[ell,1] Z   (eq. rZ)."""
        return self(x) / self.zmax

    # Proposition 1 ----------------------------------------------------------
    def partial_fractions(self):
        """(a_1..a_r, c_1, c_3, ..., c_2r-1) of Proposition 1 (eq. pa)."""
        r, c = self.r, self.c
        codd = [c[2 * j - 2] for j in range(1, r + 1)]      # c_{2j-1}
        ceven = [c[2 * j - 1] for j in range(1, r)]         # c_{2j}
        b = []
        for j in range(1, r):
            p = ceven[j - 1] - codd[j - 1]
            for k in range(1, r):
                if k != j:
                    p *= (ceven[k - 1] - codd[j - 1]) / (codd[k - 1] - codd[j - 1])
            b.append(p)
        a = [b[j - 1] / (codd[r - 1] - codd[j - 1]) for j in range(1, r)]
        a.append(1.0 - sum(a))
        return np.array(a), np.array(codd)


# ----------------------------------------------------------------------------- eq. req
def mobius(a_minus, a_plus, b_minus, b_plus):
    """(alpha, beta, gamma, ell1) of eq. req.  a_minus may be -inf."""
    am, ap, bm, bp = map(float, (a_minus, a_plus, b_minus, b_plus))
    if not (am < ap < bm < bp):
        raise ValueError("need a- < a+ < b- < b+")
    # cross ratio kcr = (b- - a-)(b+ - a+) / ((b- - a+)(b+ - a-)) = ((1+l1)/(1-l1))^2;
    # expanding the products gives kcr - 1 = (a+ - a-)(b+ - b-) / ((b- - a+)(b+ - a-)),
    # so l1 = (sqrt(kcr) - 1)/(sqrt(kcr) + 1) = (kcr - 1)/(sqrt(kcr) + 1)^2 without
    # cancellation for narrow gaps.
    if math.isinf(am):
        km1 = (bp - bm) / (bm - ap)
    else:
        km1 = (ap - am) * (bp - bm) / ((bm - ap) * (bp - am))
    s = math.sqrt(1.0 + km1)
    ell1 = km1 / ((s + 1.0) * (s + 1.0))
    # gamma*x - (gamma*alpha) + T*beta = T*x  at (a+,1), (b-,ell1), (b+,-ell1),
    # written in coordinates shifted by b- (keeps the two close abscissae b-, b+ from
    # cancelling in the 3 x 3 solve)
    rows = [(ap - bm, 1.0), (0.0, ell1), (bp - bm, -ell1)]
    Mx = np.array([[x, -1.0, t] for x, t in rows])
    rhs = np.array([t * x for x, t in rows])
    gamma, p, beta = np.linalg.solve(Mx, rhs)
    return p / gamma + bm, beta + bm, gamma, ell1


def mobius_eval(x, alpha, beta, gamma):
    x = np.asarray(x, dtype=np.float64)
    return gamma * (x - alpha) / (x - beta)


def prop2_poles(zolo, alpha, beta, gamma, rescale=1.0):
    """Poles s_j, weights w_j and the constant of Proposition 2 for M*Z(T(x)).

    Returned weights already include the factor M/rescale (rescale = max Z for the
    scaled function Zhat), i.e.  Z(T(x))/rescale = const + sum_j (w_j/(x-s_j) + conj).
    """
    a, codd = zolo.partial_fractions()
    sq = np.sqrt(codd)
    s = (gamma * alpha + 1j * sq * beta) / (gamma + 1j * sq)
    w = a * (s - beta) / (2.0 * (gamma + 1j * sq))
    Mh = zolo.M / rescale
    const = Mh * float(np.sum(a * gamma / (gamma * gamma + codd)))
    return s, Mh * w, const


# ----------------------------------------------------------------------------- the filter
class ZoloFilter:
    """R_ab(x) = (Z_2r2(Zhat_2r1(T(x); l1); l2) + 1)/2 with all constants of Algorithm 2."""

    def __init__(self, a_minus, a_plus, b_minus, b_plus, r1, r2):
        self.gaps = (float(a_minus), float(a_plus), float(b_minus), float(b_plus))
        self.r1, self.r2 = int(r1), int(r2)
        self.alpha, self.beta, self.gamma, self.ell1 = mobius(*self.gaps)
        self.inner = Zolotarev(self.r1, self.ell1)
        self.ell2 = float(self.inner.scaled(self.ell1))
        self.outer = Zolotarev(self.r2, self.ell2)
        # S(x;l1) attains its largest error at x = l1 (Remark after Algorithm 2)
        s_at_l1 = float(self.outer(self.inner.scaled(self.ell1)))
        self.delta0 = 0.5 * (1.0 - s_at_l1)
        # inner constants (hat quantities, Proposition 2 applied to Zhat)
        self.sigma_hat, self.w_hat, self.const_hat = prop2_poles(
            self.inner, self.alpha, self.beta, self.gamma, rescale=self.inner.zmax)
        # outer constants (Corollary 1)
        self.a_out, self.c_out = self.outer.partial_fractions()
        self.M_out = self.outer.M

    def T(self, x):
        return mobius_eval(x, self.alpha, self.beta, self.gamma)

    def S(self, t):
        return self.outer(self.inner.scaled(t))

    def __call__(self, x):
        return 0.5 * (self.S(self.T(x)) + 1.0)

    def G_scalar(self, x):
        """Zhat(T(x); l1) through the Proposition 2 partial fractions."""
        x = np.asarray(x, dtype=np.complex128)
        out = np.full(x.shape, self.const_hat, dtype=np.complex128)
        for s, w in zip(self.sigma_hat, self.w_hat):
            out += w / (x - s) + np.conj(w) / (x - np.conj(s))
        return out

    def outer_shifts(self):
        """The 2 r2 shifts +- i sqrt(c_2j-1) of eq. solve2 / eq. bcg and their weights.

        R(x) = 1/2 + sum_s omega_s / (G(x) + s)  with omega_s = M a_j / 4 (eq. solve2 and
        Algorithm 2's final combination).
        """
        shifts, omegas = [], []
        for a, c in zip(self.a_out, self.c_out):
            for sgn in (+1.0, -1.0):
                shifts.append(sgn * 1j * math.sqrt(c))
                omegas.append(self.M_out * a / 4.0)
        return np.array(shifts), np.array(omegas)


def composite_poles(flt):
    """Poles/weights of R_ab via Theorem 2: S = Z_{(2r1)(2r2)}(x; l1), then Proposition 2.

    R(x) = 1/2 + const/2 + (1/2) sum_j (w_j/(x-s_j) + conj(w_j)/(x-conj(s_j))).
    Returns (s, w/2, 1/2 + const/2).
    """
    big = Zolotarev(2 * flt.r1 * flt.r2, flt.ell1)
    s, w, const = prop2_poles(big, flt.alpha, flt.beta, flt.gamma, rescale=1.0)
    return s, 0.5 * w, 0.5 + 0.5 * const, big


# ----------------------------------------------------------------------------- order table
def delta0_table(a_minus, a_plus, b_minus, b_plus, rmax):
    """The table the Remark after Algorithm 2 suggests: delta0 = (1 - S(l1; l1))/2 for every
    (r1, r2) in [1, rmax]^2, table[r1 - 1, r2 - 1]."""
    t = np.zeros((rmax, rmax))
    for r1 in range(1, rmax + 1):
        for r2 in range(1, rmax + 1):
            t[r1 - 1, r2 - 1] = ZoloFilter(a_minus, a_plus, b_minus, b_plus, r1, r2).delta0
    return t


# ----------------------------------------------------------------------------- contour filters
class ContourFilter:
    """Rational filters from discretising the contour integral (Section 1.1, eq.
    contourintegral): (1/(2 pi i)) closed integral of dz / (z - x) over the circle with
    centre c = (a+b)/2 and radius rho = (b-a)/2, which is 1 for x inside and 0 outside.
    With z = c + rho e^{i theta}, dz = i rho e^{i theta} d theta, so a rule with nodes
    theta_j and weights h_j (in theta) gives R(x) = sum_j c_j / (z_j - x),
    c_j = h_j rho e^{i theta_j} / (2 pi).

      kind "CITZ": trapezoidal rule, npoles nodes theta_j = 2 pi (j - 1/2)/npoles, h_j = 2 pi / npoles.
      kind "CIGQ": Gauss-Legendre with npoles/2 nodes on each half circle; on the upper one
                   theta = (pi/2)(1 + t), h = (pi/2) omega for the Legendre nodes t, weights omega;
                   the lower half circle is its mirror image (theta -> -theta).

    For the apply, the upper-half nodes are the factored poles sigma_hat with weights
    w_hat = -c_j (c_j / (z_j - x) = w_j / (x - z_j)); each lower node is a conjugate pole
    whose weight is the conjugate, so R(x) = sum_j 2 Re(w_j / (x - sigma_j)), const 0.
    """

    def __init__(self, kind, a, b, npoles):
        if npoles < 2 or npoles % 2:
            raise ValueError("npoles must be even")
        self.kind, self.a, self.b, self.npoles = kind, float(a), float(b), int(npoles)
        self.center, self.rho = 0.5 * (self.a + self.b), 0.5 * (self.b - self.a)
        if kind == "CITZ":
            theta = 2.0 * np.pi * (np.arange(1, npoles + 1) - 0.5) / npoles
            h = np.full(npoles, 2.0 * np.pi / npoles)
        elif kind == "CIGQ":
            t, om = np.polynomial.legendre.leggauss(npoles // 2)
            up = 0.5 * np.pi * (1.0 + t)
            theta = np.concatenate([up, -up])
            h = np.concatenate([0.5 * np.pi * om, 0.5 * np.pi * om])
        else:
            raise ValueError(kind)
        self.z = self.center + self.rho * np.exp(1j * theta)
        self.c = h * self.rho * np.exp(1j * theta) / (2.0 * np.pi)
        upper = self.z.imag > 0
        self.sigma_hat = self.z[upper]
        self.w_hat = -self.c[upper]
        self.const_hat = 0.0
        self.r1 = len(self.sigma_hat)

    def __call__(self, x):
        x = np.asarray(x, dtype=np.float64)
        out = np.zeros(x.shape, dtype=np.complex128)
        for zj, cj in zip(self.z, self.c):
            out += cj / (zj - x)
        return out.real
