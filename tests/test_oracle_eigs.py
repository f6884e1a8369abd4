"""Pins for the oracle's Algorithm 1: closed-form separable spectra, a gauge-
transformed complex pencil, brute force, Sylvester inertia, residual metrics."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import apply as AP
from oracle import eigs as E
from oracle import filter as F
import synth


def _closed_form_2d(n, w=0.1):
    i = np.arange(1, n + 1)
    kap = 2 - 2 * np.cos(i * math.pi / (n + 1))
    mu = 2.0 / 3.0 + np.cos(i * math.pi / (n + 1)) / 3.0
    # lambda_ij = (kappa_i + kappa_j) / (1 + w mu_i), i the x index
    return np.sort((kap[:, None] + kap[None, :]).ravel() / np.repeat(1 + w * mu, n))


def test_dense_eigs_match_closed_form():
    n = 12
    A = synth.laplacian((n, n))
    B = synth.mass_x((n, n))
    lam, V = E.dense_eigs(A, B)
    assert np.allclose(lam, _closed_form_2d(n), rtol=1e-12, atol=1e-13)
    assert np.allclose(V.conj().T @ (B @ V), np.eye(n * n), atol=1e-12)


def _interval(lam, p, q):
    return (lam[p - 1], lam[p], lam[q - 1], lam[q])   # eigenvalues p+1..q are inside


@pytest.mark.parametrize("r", [(2, 2), (2, 3)])
def test_subspace_iteration_recovers_closed_form(r):
    n = 12
    A = synth.laplacian((n, n))
    B = synth.mass_x((n, n))
    exact = _closed_form_2d(n)
    # choose an interval with clean gaps around it
    gaps = _interval(exact, 20, 36)
    assert gaps[1] - gaps[0] > 1e-3 and gaps[3] - gaps[2] > 1e-3
    flt = F.ZoloFilter(*gaps, *r)
    a, b = 0.5 * (gaps[0] + gaps[1]), 0.5 * (gaps[2] + gaps[3])
    X0 = synth.random_block(n * n, 24, 5, complex_=False)
    lam, X = E.subspace_iteration(A, B, a, b, X0, lambda Q: AP.apply_exact(A, B, Q, flt), n_iter=4)
    assert len(lam) == 16
    assert np.allclose(lam, exact[20:36], rtol=1e-10)
    assert np.max(E.residuals(A, B, lam, X)) < 1e-10
    # e_{Lambda,X} divides by max(|a|,|b|) ||B x|| (~4x smaller than ||A||_inf ||x|| here)
    assert E.relerr(A, B, lam, X, a, b) < 1e-9
    XtBX = X.conj().T @ (B @ X)
    assert np.allclose(XtBX, np.eye(len(lam)), atol=1e-10)


def test_gauge_phase_keeps_spectrum():
    """A constant phase e^{i theta} on every x-link of A and B is the gauge transform
    D = diag(e^{i theta x}) applied to both, so the complex Hermitian pencil
    (D A D^H, D B D^H) has exactly the real pencil's spectrum."""
    n = 6
    dims = (n, n, n)
    A0 = synth.laplacian(dims)
    N = n ** 3
    idx = np.arange(N)
    x = idx % n
    D = sp.diags(np.exp(1j * 0.7 * x))
    A1 = (D @ A0 @ D.conj().T).tocsr()
    B = synth.mass_trilinear(dims)
    l0, _ = E.dense_eigs(A0, B)
    B1 = (D @ B @ D.conj().T).tocsr()
    assert abs(B1 - B).max() > 0.01           # genuinely complex B
    l1, _ = E.dense_eigs(A1, B1)
    assert np.allclose(l0, l1, atol=1e-11)
    # and the 3D separable closed form (kappa_i + kappa_j + kappa_l)/(mu_i mu_j mu_l)
    i = np.arange(1, n + 1)
    kap = 2 - 2 * np.cos(i * math.pi / (n + 1))
    mu = 2.0 / 3.0 + np.cos(i * math.pi / (n + 1)) / 3.0
    cf = np.sort(((kap[:, None, None] + kap[None, :, None] + kap[None, None, :])
                  / (mu[:, None, None] * mu[None, :, None] * mu[None, None, :])).ravel())
    assert np.allclose(l0, cf, rtol=1e-11)


def test_inertia_counts_match_dense():
    p = synth.pencil_3d_peierls(5, seed=2, wells=4)
    lam, _ = E.dense_eigs(p.A, p.B)
    for a, b in [(lam[10] + 1e-6, lam[40] + 1e-6), (-10.0, lam[3] + 1e-6)]:
        assert E.count_in(p.A, p.B, a, b) == int(np.sum((lam > a) & (lam < b)))


def test_residual_metric_flags_a_wrong_pair():
    p = synth.pencil_2d_real(8, seed=1)
    lam, V = E.dense_eigs(p.A, p.B)
    good = E.residuals(p.A, p.B, lam[:5], V[:, :5])
    assert np.max(good) < 1e-13
    bad = E.residuals(p.A, p.B, lam[:5] * (1 + 1e-6), V[:, :5])
    assert np.min(bad) > 1e-8


def test_subspace_iteration_converges_at_the_filter_ratio():
    """Subspace iteration with the exact rational filter (dense application, no GMRES):
    asymptotically the residual of the worst wanted pair shrinks per iteration by
    rho_(k+1) / min_wanted rho, where rho = |R_ab(lambda)| sorted decreasingly and k is
    the subspace dimension (standard subspace-iteration theory).  A weak (1,1) filter keeps
    the ratio near 0.17 so that several iterations stay above rounding."""
    pen = synth.pencil_2d_real(12, seed=1)
    lam, _ = E.dense_eigs(pen.A, pen.B)
    p, q, k = 60, 70, 16
    flt = F.ZoloFilter(lam[p - 1], lam[p], lam[q - 1], lam[q], 1, 1)
    rho = np.abs(flt(lam))
    theory = np.sort(rho)[::-1][k] / np.min(rho[p:q])
    Q = synth.random_block(pen.n, k, 7)
    errs = []
    for _ in range(8):
        th, Q = E.rayleigh_ritz(pen.A, pen.B, AP.apply_dense(pen.A, pen.B, Q, flt), 1e-14)
        res = E.residuals(pen.A, pen.B, th, Q)
        errs.append(max(res[np.argmin(np.abs(th - lam[j]))] for j in range(p, q)))
    measured = (errs[7] / errs[3]) ** 0.25          # geometric mean over iterations 4..8
    assert 0.1 < theory < 0.25                          # the weak-filter regime the test needs
    assert theory / 1.5 <= measured <= theory * 1.5, (measured, theory)


def test_relerr_and_residual_hand_values():
    """e_{Lambda,X} (eq. relerr, Section 3) and the residual metric on a 2 x 2 diagonal pencil
    worked by hand.  A = diag(2, 5), B = diag(1, 4), ||A||_inf = 5; a = -4, b = 3 so that
    max(|a|, |b|) = 4 differs from max(a, b) = 3.
      x1 = (1, 0), lam = 2.1:  A x - lam B x = (-0.1, 0),  ||x|| = 1, ||B x|| = 1
      x2 = (0, 2), lam = 1.3:  A x - lam B x = (0, -0.4),  ||x|| = 2, ||B x|| = 8
    e per column: 0.1 / (4 * 1) = 0.025 and 0.4 / (4 * 8) = 0.0125, max 0.025.
    residual per column: 0.1 / (5 * 1) = 0.02 and 0.4 / (5 * 2) = 0.04.
    A denominator with ||x|| instead of ||B x|| gives 0.05 for x2, one with max(a, b)
    gives 0.0333 for x1, so either mistake fails."""
    A = sp.diags([2.0, 5.0]).tocsr()
    B = sp.diags([1.0, 4.0]).tocsr()
    X = np.array([[1.0, 0.0], [0.0, 2.0]], dtype=np.complex128)
    lam = np.array([2.1, 1.3])
    assert E.relerr(A, B, lam[:1], X[:, :1], -4.0, 3.0) == pytest.approx(0.025, rel=1e-14)
    assert E.relerr(A, B, lam[1:], X[:, 1:], -4.0, 3.0) == pytest.approx(0.0125, rel=1e-14)
    assert E.relerr(A, B, lam, X, -4.0, 3.0) == pytest.approx(0.025, rel=1e-14)
    assert np.allclose(E.residuals(A, B, lam, X), [0.02, 0.04], rtol=1e-14)


def test_relerr_and_residual_complex_hand_values():
    """The same metrics on a complex Hermitian pencil, by hand:
    A = [[2, i], [-i, 2]] (||A||_inf = 3), B = diag(1, 2), x = (1, i), lam = 1:
    A x = (2 + i*i, -i + 2i) = (1, i), B x = (1, 2i), A x - lam B x = (0, -i), norm 1;
    ||x|| = sqrt 2, ||B x|| = sqrt 5.  With (a, b) = (-1, 0.5): e = 1 / sqrt 5,
    residual = 1 / (3 sqrt 2)."""
    A = sp.csr_matrix(np.array([[2.0, 1j], [-1j, 2.0]]))
    B = sp.diags([1.0, 2.0]).tocsr()
    X = np.array([[1.0], [1j]])
    lam = np.array([1.0])
    assert E.relerr(A, B, lam, X, -1.0, 0.5) == pytest.approx(1.0 / math.sqrt(5.0), rel=1e-14)
    assert E.residuals(A, B, lam, X)[0] == pytest.approx(1.0 / (3.0 * math.sqrt(2.0)), rel=1e-14)


def test_lowest_eigenpairs_with_an_unbounded_left_gap():
    """The mode of Section 3.1's Example 1: a- = -inf, a+ = lam_1, b- = lam_20, b+ = lam_21 on
    the Gaussian-well Hamiltonian (8^3, B = I), r = (4, 4), one subspace iteration of 21
    columns with exact poles: the 20 smallest eigenvalues of the dense eigensolver."""
    p = synth.hamiltonian_wells(8, 2)
    lam = np.linalg.eigvalsh(p.A.toarray())
    flt = F.ZoloFilter(-math.inf, lam[0], lam[19], lam[20], 4, 4)
    a, b = lam[0] - 0.5 * (lam[19] - lam[0]), 0.5 * (lam[19] + lam[20])
    X0 = synth.random_block(p.n, 21, 3, complex_=False)
    ev, X = E.subspace_iteration(p.A, p.B, a, b, X0, lambda Q: AP.apply_exact(p.A, p.B, Q, flt), n_iter=1)
    assert len(ev) == 20
    assert np.allclose(ev, lam[:20], rtol=1e-11, atol=0)
    assert np.max(E.residuals(p.A, p.B, ev, X)) < 1e-9
