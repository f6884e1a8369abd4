"""Algorithm 1 (subspace iteration + Rayleigh-Ritz) and eigenpair checks (oracle).

Test infrastructure only (see ``oracle/__init__``).

Algorithm 1 (Section 2.1): Q orthonormal random; repeat { Y = R(B^-1 A) Q;
A~ = Y^H A Y, B~ = Y^H B Y; solve A~ Q~ = Lam~ B~ Q~; Q = Y Q~ }; keep a < Lam~_ii < b.
Readings: the generalized projected problem is solved through the B-Gram matrix
B~ = U diag(mu) U^H, dropping directions with mu < drop * max(mu) (Y is nearly
rank deficient after a sharp filter; when the filtered block carries an error eps,
drop must be at least ~(10 eps)^2 or noise directions survive), then a standard
Hermitian eigenproblem of
W^H A~ W with W = U_kept diag(mu^-1/2).  Selection is strict (a < lam < b),
ascending; eigenvectors are B-normalised.

Accuracy measures: equation relerr  e = max_i ||A x_i - B x_i lam_i|| / ||max(|a|,|b|) B x_i||,
and the residual ||A x - lam B x||_2 / (||A||_inf ||x||_2).  Counts of eigenvalues
in (a,b) use Sylvester's law of inertia: nu(A - bB) - nu(A - aB).
"""
import numpy as np
import scipy.linalg as sla


def rayleigh_ritz(A, B, Y, drop=1e-14):
    At = Y.conj().T @ (A @ Y)
    Bt = Y.conj().T @ (B @ Y)
    At = 0.5 * (At + At.conj().T)
    Bt = 0.5 * (Bt + Bt.conj().T)
    mu, U = np.linalg.eigh(Bt)
    keep = mu > drop * mu.max()
    W = U[:, keep] / np.sqrt(mu[keep])
    Ah = W.conj().T @ At @ W
    lam, Z = np.linalg.eigh(0.5 * (Ah + Ah.conj().T))
    return lam, Y @ (W @ Z)


def subspace_iteration(A, B, a, b, Q0, apply_fn, n_iter=1, drop=1e-14):
    Q = np.asarray(Q0, dtype=np.complex128)
    lam = None
    for _ in range(n_iter):
        Y = apply_fn(Q)
        lam, Q = rayleigh_ritz(A, B, Y, drop)
    sel = (lam > a) & (lam < b)
    return lam[sel], Q[:, sel]


def residuals(A, B, lam, X):
    """||A x - lam B x||_2 / (||A||_inf ||x||_2) per column."""
    Anorm = float(abs(A).sum(axis=1).max())
    R = A @ X - (B @ X) * lam[None, :]
    return np.linalg.norm(R, axis=0) / (Anorm * np.linalg.norm(X, axis=0))


def relerr(A, B, lam, X, a, b):
    """e_{Lambda,X} of equation relerr."""
    BX = B @ X
    R = A @ X - BX * lam[None, :]
    return float(np.max(np.linalg.norm(R, axis=0) / (max(abs(a), abs(b)) * np.linalg.norm(BX, axis=0))))


def dense_eigs(A, B):
    return sla.eigh(A.toarray(), B.toarray())


def inertia_count(A, B, sigma):
    """Number of eigenvalues of (A,B) below sigma = negative inertia of A - sigma B."""
    K = A.toarray() - sigma * B.toarray()
    _, D, _ = sla.ldl(K, hermitian=True)
    ev = np.linalg.eigvalsh(D)
    return int(np.sum(ev < 0))


def count_in(A, B, a, b):
    return inertia_count(A, B, b) - inertia_count(A, B, a)
