"""Pins for the oracle's shifted factorisation and solves."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import factor as FA
from oracle import filter as F
from oracle import ordering as O
import synth


def test_lu_nopivot_definition():
    rng = np.random.default_rng(0)
    K = rng.standard_normal((30, 30)) + 1j * rng.standard_normal((30, 30))
    K += 40 * np.eye(30)                     # diagonally dominant: partial pivoting never swaps
    L, U = FA.lu_nopivot(K)
    assert np.allclose(L @ U, K, atol=1e-12)
    assert np.allclose(np.triu(U), U) and np.allclose(np.tril(L), L)
    assert np.allclose(np.diag(L), 1.0)
    P, L2, U2 = sla.lu(K)
    assert np.allclose(P, np.eye(30))
    assert np.allclose(L, L2, atol=1e-12) and np.allclose(U, U2, atol=1e-12)


def test_real_pencil_lu_is_ldlt():
    """Real symmetric pencil: K = A - sigma B is complex symmetric, so U = D L^T."""
    p = synth.pencil_2d_real(8, seed=1)
    t = O.nd_grid(p.dims, 4)
    K = FA.shifted(p.A, p.B, 2.0 + 0.3j).toarray()[np.ix_(t.perm, t.perm)]
    L, U = FA.lu_nopivot(K)
    D = np.diag(np.diag(U))
    assert np.allclose(U, D @ L.T, atol=1e-12)


def test_pole_shift_has_no_zero_pivot_and_solves():
    p = synth.pencil_3d_peierls(5, seed=2, wells=4)
    flt = F.ZoloFilter(-1.0, -0.5, 0.5, 0.6, 2, 2)
    t = O.nd_grid(p.dims, 8)
    for s in flt.sigma_hat:
        K = FA.shifted(p.A, p.B, s).toarray()[np.ix_(t.perm, t.perm)]
        L, U = FA.lu_nopivot(K)
        assert np.min(np.abs(np.diag(U))) > 1e-8 * np.abs(K).max()
        sol = FA.Solver(p.A, p.B, s)
        b = synth.random_block(p.n, 3, 7)
        x = sol.solve(b)
        assert np.linalg.norm(sol.K @ x - b) < 1e-12 * np.linalg.norm(b) * 1e3
        xh = sol.solve(b, herm=True)
        assert np.linalg.norm(sol.K.conj().T @ xh - b) < 1e-12 * np.linalg.norm(b) * 1e3
        # (A - conj(s) B)^-1 = K^-H for Hermitian A, B (equation solve, third equality)
        sol2 = FA.Solver(p.A, p.B, np.conj(s))
        assert np.allclose(sol2.solve(b), xh, atol=1e-10)
