"""Pins for the oracle's filtered block: three independent definitions agree, and the
Krylov quantities satisfy the Arnoldi and shift-invariance relations."""
import numpy as np
import pytest

from oracle import apply as AP
from oracle import eigs as E
from oracle import filter as F
import synth


def _setup(kind):
    if kind == "real2d":
        p = synth.pencil_2d_real(10, seed=1)
        lam, _ = E.dense_eigs(p.A, p.B)
        gaps = (lam[14], lam[15], lam[29], lam[30])
        X = synth.random_block(p.n, 5, 3, complex_=False)
    else:
        p = synth.pencil_3d_peierls(5, seed=2, wells=4)
        lam, _ = E.dense_eigs(p.A, p.B)
        gaps = (lam[19], lam[20], lam[39], lam[40])
        X = synth.random_block(p.n, 4, 3)
    return p, gaps, X


@pytest.mark.parametrize("kind", ["real2d", "complex3d"])
@pytest.mark.parametrize("r", [(1, 2), (2, 2), (2, 3)])
def test_three_definitions_agree(kind, r):
    p, gaps, X = _setup(kind)
    flt = F.ZoloFilter(*gaps, *r)
    Y1 = AP.apply_dense(p.A, p.B, X, flt)
    Y2 = AP.apply_exact(p.A, p.B, X, flt)
    Y3 = AP.apply_hybrid(p.A, p.B, X, flt, tol=1e-13, m_max=60)
    scale = np.linalg.norm(Y1, axis=0)
    assert np.max(np.linalg.norm(Y1 - Y2, axis=0) / scale) < 1e-11
    assert np.max(np.linalg.norm(Y1 - Y3, axis=0) / scale) < 1e-10


def test_filter_is_projector_on_eigenvectors():
    """R(B^-1 A) x_i = R(lam_i) x_i on generalized eigenvectors."""
    p, gaps, _ = _setup("complex3d")
    flt = F.ZoloFilter(*gaps, 2, 2)
    lam, V = E.dense_eigs(p.A, p.B)
    idx = [0, 20, 30, 39, 40, 100]
    Y = AP.apply_exact(p.A, p.B, V[:, idx], flt)
    assert np.allclose(Y, V[:, idx] * flt(lam[idx])[None, :], atol=1e-11)


def test_arnoldi_and_shift_invariance():
    p, gaps, X = _setup("real2d")
    flt = F.ZoloFilter(*gaps, 2, 2)
    G = AP.InnerOperator(p.A, p.B, flt)
    Y, info = AP.apply_hybrid(p.A, p.B, X, flt, G=G, return_info=True)
    m, H = info["m"], info["H"]
    assert 6 <= m <= 40                     # "6 to 25" GMRES steps (Section 2.3), loosely
    # G V_m = V_{m+1} Hbar and orthonormality of the basis of column 0
    Vm = np.hstack([v[:, :1] for v in info["V"]])
    assert np.allclose(Vm.conj().T @ Vm, np.eye(m + 1), atol=1e-10)
    V = [Vm[:, i:i + 1] for i in range(m + 1)]
    GV = np.hstack([G(V[i]) for i in range(m)])
    assert np.allclose(GV, Vm @ H[:, :, 0], atol=1e-10)
    s = 0.37j
    Hs = H[:, :, 0].copy()
    Hs[np.arange(m), np.arange(m)] += s
    assert np.allclose(GV + s * Vm[:, :m], Vm @ Hs, atol=1e-10)


def test_zero_block_and_single_column():
    p, gaps, X = _setup("real2d")
    flt = F.ZoloFilter(*gaps, 2, 2)
    Y = AP.apply_exact(p.A, p.B, X[:, :1], flt)
    Y3 = AP.apply_hybrid(p.A, p.B, X[:, :1], flt)
    assert np.linalg.norm(Y - Y3) < 1e-10 * np.linalg.norm(Y)
