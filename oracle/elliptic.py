"""Complete elliptic integral K and Jacobi elliptic functions sn, cn, dn (oracle).

Test infrastructure only (see ``oracle/__init__``).

Theorem 1 (Section 2.2) needs sn(u; l') and cn(u; l') at u = jK'/(2r) with
modulus l' = sqrt(1 - l^2) and K' = K(l').  We follow the arithmetic-geometric
mean (AGM) method of Abramowitz & Stegun 16.4 / 17.6, a published method:

  a0 = 1, b0 = k' (complementary modulus), c0 = k
  a_n = (a_{n-1}+b_{n-1})/2, b_n = sqrt(a_{n-1} b_{n-1}), c_n = (a_{n-1}-b_{n-1})/2
  K(k) = pi / (2 a_N)
  phi_N = 2^N a_N u,  phi_{n-1} = (phi_n + asin(c_n sin(phi_n) / a_n)) / 2
  sn = sin(phi_0), cn = cos(phi_0)
  dn = sqrt(cn^2 + k'^2 sn^2)   (identity dn^2 = 1 - k^2 sn^2; A&S's quotient
                                 cos(phi_0)/cos(phi_1 - phi_0) is 0/0 at u = K)

Both the modulus k and its complement k' are passed in so that k' is never
formed as sqrt(1 - k^2) when k is close to 1 (the Zolotarev case with a tiny
l has k = l' ~ 1 and k' = l exact).  Accuracy (pinned against 40-digit mpmath):
~1e-16 for k' >= 1e-2, degrading to ~2e-14 absolute for k' = 1e-7 because the
asin arguments of the backward recurrence approach +-1.
"""
import math


def _agm_sequence(k, kp):
    a, b, c = [1.0], [kp], [k]
    while abs(c[-1]) > 1e-17 * a[-1] and len(a) < 64:
        an = 0.5 * (a[-1] + b[-1])
        bn = math.sqrt(a[-1] * b[-1])
        cn = 0.5 * (a[-1] - b[-1])
        a.append(an); b.append(bn); c.append(cn)
    return a, b, c


def ellipk(k, kp=None):
    """K(k) = int_0^{pi/2} dtheta / sqrt(1 - k^2 sin^2 theta), modulus k in [0,1)."""
    if kp is None:
        kp = math.sqrt((1.0 - k) * (1.0 + k))
    a, _, _ = _agm_sequence(k, kp)
    return math.pi / (2.0 * a[-1])


def ellipj(u, k, kp=None):
    """(sn, cn, dn)(u; k) for real u and modulus k (A&S 16.4.*)."""
    if kp is None:
        kp = math.sqrt((1.0 - k) * (1.0 + k))
    if k == 0.0:
        return math.sin(u), math.cos(u), 1.0
    a, _, c = _agm_sequence(k, kp)
    n = len(a) - 1
    phi = [0.0] * (n + 1)
    phi[n] = (2.0 ** n) * a[n] * u
    for i in range(n, 0, -1):
        s = c[i] * math.sin(phi[i]) / a[i]
        s = max(-1.0, min(1.0, s))
        phi[i - 1] = 0.5 * (phi[i] + math.asin(s))
    sn = math.sin(phi[0])
    cn = math.cos(phi[0])
    dn = math.sqrt(cn * cn + kp * kp * sn * sn)
    return sn, cn, dn
