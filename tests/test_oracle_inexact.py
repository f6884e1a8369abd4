"""CPU checks of the two places where the library's arithmetic departs from the paper's
exact inner operator, run on the oracle (which follows the paper exactly):

1. Relaxed inner solves.  Inside shift-invariant GMRES, the shifted solves of step i are
   refined only to eta_i = min(1e-3, max(1e-12, 1e-2 tol / eps_{i-1})), with eps_{i-1} the
   stopping bound after step i - 1.  Here the oracle's exact operator G is perturbed by
   exactly the error such a solve may leave (K_j^-1 r_j, ||r_j|| = eta_i ||B v||). The
   filtered block must still match the exact rational filter to the GMRES tolerance.
2. FP32 projection coefficients.  The Gram-Schmidt coefficients are rounded to complex64
   (update and Hessenberg entries use the same rounded values).  The filtered block must
   match as well.
"""
import numpy as np
import pytest

from oracle import apply as AP
from oracle import eigs as E
from oracle import factor as FA
from oracle import filter as F
import synth


def _case():
    pen = synth.pencil_3d_peierls(9, seed=2, wells=6)
    lam, _ = E.dense_eigs(pen.A, pen.B)
    gaps = (lam[39], lam[40], lam[69], lam[70])
    return pen, F.ZoloFilter(*gaps, 2, 3)


def _colrel(Y, R):
    return float(np.max(np.linalg.norm(Y - R, axis=0) / np.linalg.norm(R, axis=0)))


def _bounds(info, flt, beta):
    """stopping bound of reading 6 after every step 1..m (max over columns, relative)"""
    H = info["H"]
    shifts, omegas = flt.outer_shifts()
    out = []
    for m in range(1, H.shape[1] + 1):
        worst = 0.0
        for c in range(H.shape[2]):
            b = 0.0
            for s, om in zip(shifts, omegas):
                _, res = AP._lsq(H[:m + 1, :m, c], s, beta[c])
                b += abs(om) * res / np.sqrt(flt.ell2 ** 2 + abs(s) ** 2)
            worst = max(worst, b / beta[c])
        out.append(worst)
    return out


class RelaxedOperator:
    """The exact G plus, at call i, the error of shifted solves refined to eta_i."""

    def __init__(self, pen, flt, etas, seed):
        self.G = AP.InnerOperator(pen.A, pen.B, flt)
        self.pen, self.flt, self.etas = pen, flt, etas
        self.rng = np.random.default_rng(seed)
        self.calls = 0

    def __call__(self, V):
        eta = self.etas[min(self.calls, len(self.etas) - 1)]
        self.calls += 1
        out = self.G(V)
        BV = self.pen.B @ V
        for sol, w in zip(self.G.solvers, self.flt.w_hat):
            for herm, coef in ((False, w), (True, np.conj(w))):
                R = self.rng.standard_normal(BV.shape) + 1j * self.rng.standard_normal(BV.shape)
                R *= eta * np.linalg.norm(BV, axis=0) / np.linalg.norm(R, axis=0)
                out = out + coef * sol.solve(R, herm=herm)        # K^-1 r: the solve's error
        return out


@pytest.mark.parametrize("tol", [1e-8, 1e-11])
def test_relaxed_inner_solves_keep_the_filtered_block(tol):
    pen, flt = _case()
    X = synth.random_block(pen.n, 6, 3)
    ref = AP.apply_exact(pen.A, pen.B, X, flt)
    Y0, info = AP.apply_hybrid(pen.A, pen.B, X, flt, tol=tol, m_max=150, return_info=True)
    e_exact = _colrel(Y0, ref)
    # eta_i from the exact run's bound history (the relaxed run's is the same to leading order)
    eps = [1.0] + _bounds(info, flt, info["beta"])
    etas = [min(1e-3, max(1e-12, 1e-2 * tol / e)) for e in eps]
    assert max(etas) >= 1e-3 * 0.999                       # the late steps are relaxed a lot
    G = RelaxedOperator(pen, flt, etas, seed=7)
    Y1 = AP.apply_hybrid(pen.A, pen.B, X, flt, tol=tol, m_max=150, G=G)
    e_relaxed = _colrel(Y1, ref)
    assert e_relaxed <= 10 * tol, (e_relaxed, e_exact)
    # the same perturbation applied at every step, without relaxing, is much worse
    G2 = RelaxedOperator(pen, flt, [1e-3], seed=7)
    Y2 = AP.apply_hybrid(pen.A, pen.B, X, flt, tol=tol, m_max=150, G=G2)
    assert _colrel(Y2, ref) > 10 * e_relaxed


def _hybrid_fp32_coefficients(pen, X, flt, tol, m_max=150):
    """The oracle's shift-invariant GMRES with the Gram-Schmidt coefficients rounded to
    complex64 (FP64 vectors, FP64 update with the rounded coefficients, same stopping rule)."""
    G = AP.InnerOperator(pen.A, pen.B, flt)
    shifts, omegas = flt.outer_shifts()
    n, k = X.shape
    beta = np.linalg.norm(X, axis=0)
    V = [X / beta]
    H = np.zeros((m_max + 1, m_max, k), dtype=np.complex128)
    m = 0
    for i in range(m_max):
        W = G(V[i])
        for _ in range(2):
            h = np.array([np.sum(np.conj(V[j]) * W, axis=0) for j in range(i + 1)])
            h = h.astype(np.complex64).astype(np.complex128)
            for j in range(i + 1):
                W = W - V[j] * h[j]
            H[:i + 1, i, :] += h
        hn = np.linalg.norm(W, axis=0)
        H[i + 1, i, :] = hn
        V.append(W / hn)
        m = i + 1
        worst = 0.0
        for c in range(k):
            b = 0.0
            for s, om in zip(shifts, omegas):
                _, res = AP._lsq(H[:m + 1, :m, c], s, beta[c])
                b += abs(om) * res / np.sqrt(flt.ell2 ** 2 + abs(s) ** 2)
            worst = max(worst, b / beta[c])
        if worst <= tol:
            break
    Y = 0.5 * X
    for c in range(k):
        zeta = np.zeros(m, dtype=np.complex128)
        for s, om in zip(shifts, omegas):
            z, _ = AP._lsq(H[:m + 1, :m, c], s, beta[c])
            zeta += om * z
        Y[:, c] += np.stack([V[j][:, c] for j in range(m)], axis=1) @ zeta
    return Y, m


def test_fp32_projection_coefficients_keep_the_filtered_block():
    pen, flt = _case()
    X = synth.random_block(pen.n, 6, 4)
    ref = AP.apply_exact(pen.A, pen.B, X, flt)
    tol = 1e-11
    Y0, info = AP.apply_hybrid(pen.A, pen.B, X, flt, tol=tol, m_max=150, return_info=True)
    Y1, m1 = _hybrid_fp32_coefficients(pen, X, flt, tol)
    assert _colrel(Y1, ref) <= 10 * tol
    assert abs(m1 - info["m"]) <= 2                       # same number of steps, to within 2
