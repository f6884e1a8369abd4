"""Shifted matrices K = A - sigma B, their no-pivot LU and solves (oracle).

Test infrastructure only (see ``oracle/__init__``).

Equation mts (Section 2.3) needs solves with K_j = A - sigma_j B and, for the
conjugate poles, with A - conj(sigma_j) B = K_j^H (A, B Hermitian; equation
solve).  K_j is not Hermitian (Im sigma_j != 0), so the factorisation the
product computes is an LU without pivoting on the nested-dissection order
(L unit lower, U upper; for a real pencil K is complex symmetric and U = D L^T).
It exists because i K has definite Hermitian part +-Im(sigma) B, so every leading
principal submatrix is nonsingular.

The oracle gives two independent references:
  * ``lu_nopivot``: the plain right-looking Doolittle elimination of the permuted
    dense matrix (small N), i.e. the unique no-pivot LU by definition;
  * ``Solver``: x = K^-1 b through SuperLU (scipy.sparse.linalg.splu) with its own
    ordering and pivoting -- the solution of K x = b is unique, so any exact solver
    is a valid reference for the product's solves.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def shifted(A, B, sigma):
    return (A.astype(np.complex128) - sigma * B.astype(np.complex128)).tocsc()


def lu_nopivot(K):
    """Dense Doolittle LU without pivoting: K = L U, L unit lower, U upper."""
    U = np.array(K, dtype=np.complex128, copy=True)
    n = U.shape[0]
    L = np.eye(n, dtype=np.complex128)
    for j in range(n):
        piv = U[j, j]
        if piv == 0:
            raise ZeroDivisionError(f"zero pivot at {j}")
        L[j + 1:, j] = U[j + 1:, j] / piv
        U[j + 1:, j:] -= np.outer(L[j + 1:, j], U[j, j:])
        U[j + 1:, j] = 0.0
    return L, U


class Solver:
    """Exact sparse solves with K and K^H (SuperLU)."""

    def __init__(self, A, B, sigma):
        self.K = shifted(A, B, sigma)
        self.lu = spla.splu(self.K)

    def solve(self, b, herm=False):
        return self.lu.solve(np.asarray(b, dtype=np.complex128), trans="H" if herm else "N")
