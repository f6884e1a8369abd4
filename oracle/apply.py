"""Filtered block Y = R_ab(B^-1 A) X (oracle).

Test infrastructure only (see ``oracle/__init__``).

Three references, from the most to the least independent of the product:
  * ``apply_dense``  (tiny N): generalized eigendecomposition A V = B V diag(lam),
    V^H B V = I, so R(B^-1 A) X = V diag(R(lam)) V^H B X.
  * ``apply_exact``: Theorem 2 gives R_ab(x) = (Z_{(2r1)(2r2)}(T(x); l1) + 1)/2, and
    Proposition 2 writes it as 1/2 + const + sum_j (w_j/(x - s_j) + conj), so
    Y = (1/2+const) X + sum_j ( w_j (A - s_j B)^-1 B X + conj(w_j) (A - conj(s_j) B)^-1 B X )
    with one exact sparse solve per pole and per conjugate pole.
  * ``apply_hybrid``: Algorithm 2 step by step -- the inner operator G of equation
    solve through r1 factored poles, then equation solve2 by GMRES with one Krylov
    basis per column shared by the 2 r2 shifts (shift invariance
    (G + s I) V_m = V_{m+1} (Hbar_m + s Ibar)), per-shift least squares, and the
    combination of Algorithm 2's last line.

Readings (the paper leaves them open): zero initial guess, no restart, classical
Gram-Schmidt applied twice, Euclidean inner product, one step count m for all
columns of the block.  Stop at the first m where, for every column c,
    sum_s |omega_s| res_s / sqrt(l2^2 + |s|^2) <= tol * ||x_c||
(res_s: least-squares residual of shift s), or at m_max.  The left side bounds the
error of the filtered column: the combination's error is sum_s omega_s (G + s)^-1 r_s,
G has real spectrum outside (-l2, l2) (|Zhat| >= l2 on the gap complement) and
s = +-i sqrt(c) is imaginary, so ||(G + s)^-1|| <= 1 / sqrt(l2^2 + |s|^2) in the norm
in which G is normal.
"""
import numpy as np
import scipy.linalg as sla

from . import factor
from .filter import composite_poles


def apply_dense(A, B, X, flt):
    Ad, Bd = A.toarray(), B.toarray()
    lam, V = sla.eigh(Ad, Bd)
    rl = flt(lam)
    return V @ (rl[:, None] * (V.conj().T @ (Bd @ X)))


def apply_exact(A, B, X, flt):
    s, w, c0, _ = composite_poles(flt)
    X = np.asarray(X, dtype=np.complex128)
    BX = B @ X
    Y = c0 * X
    for sj, wj in zip(s, w):
        Y = Y + wj * factor.Solver(A, B, sj).solve(BX)
        Y = Y + np.conj(wj) * factor.Solver(A, B, np.conj(sj)).solve(BX)
    return Y


class InnerOperator:
    """G V = const_hat V + sum_j (w_hat_j K_j^-1 B V + conj(w_hat_j) K_j^-H B V)  (equation solve)."""

    def __init__(self, A, B, flt):
        self.A, self.B, self.flt = A, B, flt
        self.solvers = [factor.Solver(A, B, s) for s in flt.sigma_hat]

    def __call__(self, V):
        BV = self.B @ V
        out = self.flt.const_hat * V
        for sol, w in zip(self.solvers, self.flt.w_hat):
            out = out + w * sol.solve(BV) + np.conj(w) * sol.solve(BV, herm=True)
        return out


def _lsq(Hbar, s, beta):
    """argmin || beta e1 - (Hbar + s Ibar) z ||  and its residual norm."""
    m1, m = Hbar.shape
    Hs = Hbar.astype(np.complex128).copy()
    Hs[np.arange(m), np.arange(m)] += s
    rhs = np.zeros(m1, dtype=np.complex128)
    rhs[0] = beta
    z, _, _, _ = np.linalg.lstsq(Hs, rhs, rcond=None)
    return z, float(np.linalg.norm(rhs - Hs @ z))


def apply_hybrid(A, B, X, flt, tol=1e-12, m_max=100, G=None, return_info=False):
    X = np.asarray(X, dtype=np.complex128)
    n, k = X.shape
    G = G if G is not None else InnerOperator(A, B, flt)
    shifts, omegas = flt.outer_shifts()
    beta = np.linalg.norm(X, axis=0)
    V = [X / beta]
    H = np.zeros((m_max + 1, m_max, k), dtype=np.complex128)
    m = 0
    for i in range(m_max):
        W = G(V[i])
        for _ in range(2):                     # classical Gram-Schmidt, twice
            h = np.array([np.sum(np.conj(V[j]) * W, axis=0) for j in range(i + 1)])
            for j in range(i + 1):
                W = W - V[j] * h[j]
            H[:i + 1, i, :] += h
        hn = np.linalg.norm(W, axis=0)
        H[i + 1, i, :] = hn
        V.append(W / np.where(hn > 0, hn, 1.0))
        m = i + 1
        worst = 0.0
        for c in range(k):
            bound = 0.0
            for s, om in zip(shifts, omegas):
                _, res = _lsq(H[:m + 1, :m, c], s, beta[c])
                bound += abs(om) * res / np.sqrt(flt.ell2 ** 2 + abs(s) ** 2)
            worst = max(worst, bound / beta[c])
        if worst <= tol:
            break
    Y = 0.5 * X
    for c in range(k):
        zeta = np.zeros(m, dtype=np.complex128)
        for s, om in zip(shifts, omegas):
            z, _ = _lsq(H[:m + 1, :m, c], s, beta[c])
            zeta += om * z
        Y[:, c] += np.stack([V[j][:, c] for j in range(m)], axis=1) @ zeta
    if return_info:
        return Y, {"m": m, "H": H[:m + 1, :m, :], "beta": beta, "V": V[:m + 1]}
    return Y


def apply_contour(A, B, X, flt):
    """R(B^-1 A) X for a contour-integral filter: every quadrature point is a factored pole,
    R(B^-1 A) X = sum_j c_j (z_j - B^-1 A)^-1 X = sum_j w_j (A - z_j B)^-1 B X over all points
    (w_j = -c_j), written through the upper-half poles and K^-H for their conjugates."""
    return InnerOperator(A, B, flt)(np.asarray(X, dtype=np.complex128))
