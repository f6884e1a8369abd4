"""The oracle's pins against planted mistakes.

Each case replaces one oracle function (on the CPU, for the duration of the case) with a
copy carrying one plausible mistake -- a wrong denominator, an index off by one, a swapped
pair, a dropped term or factor, a sign -- and checks that a pin test of the oracle then
fails.  A pin that still passed would not be tying the oracle to the paper."""
import math

import numpy as np
import pytest

from oracle import apply as AP
from oracle import eigs as E
from oracle import elliptic as EL
from oracle import factor as FA
from oracle import filter as F

import test_oracle_apply as T_APPLY
import test_oracle_eigs as T_EIGS
import test_oracle_elliptic as T_ELL
import test_oracle_factor as T_FAC
import test_oracle_filter as T_FLT


def _fails(pin, *args):
    """True when the pin test raises (an assertion, or a crash of the mutated oracle)."""
    try:
        pin(*args)
    except Exception:
        return True
    return False


def test_pins_pass_unmutated():
    """The same pin calls as below, on the oracle as it is: none of them fails."""
    assert not _fails(T_EIGS.test_relerr_and_residual_hand_values)
    assert not _fails(T_ELL.test_sn_cn_dn_match_scipy, 0.7)
    assert not _fails(T_FLT.test_r1_closed_form, 0.1)
    assert not _fails(T_FLT.test_mobius_conditions, (0.1, 0.3, 2.0, 2.5))
    assert not _fails(T_FLT.test_prop2_poles_weights, 2)
    assert not _fails(T_FLT.test_citz_closed_form, 8)
    assert not _fails(T_FAC.test_lu_nopivot_definition)


# ---------------------------------------------------------------- accuracy metrics (eq. relerr)
def test_relerr_with_x_norm_instead_of_bx_norm(monkeypatch):
    def wrong(A, B, lam, X, a, b):
        R = A @ X - (B @ X) * lam[None, :]
        return float(np.max(np.linalg.norm(R, axis=0) / (max(abs(a), abs(b)) * np.linalg.norm(X, axis=0))))
    monkeypatch.setattr(E, "relerr", wrong)
    assert _fails(T_EIGS.test_relerr_and_residual_hand_values)


def test_relerr_with_max_a_b_instead_of_max_abs(monkeypatch):
    def wrong(A, B, lam, X, a, b):
        BX = B @ X
        R = A @ X - BX * lam[None, :]
        return float(np.max(np.linalg.norm(R, axis=0) / (max(a, b) * np.linalg.norm(BX, axis=0))))
    monkeypatch.setattr(E, "relerr", wrong)
    assert _fails(T_EIGS.test_relerr_and_residual_hand_values)


def test_residual_without_the_matrix_norm(monkeypatch):
    def wrong(A, B, lam, X):
        R = A @ X - (B @ X) * lam[None, :]
        return np.linalg.norm(R, axis=0) / np.linalg.norm(X, axis=0)
    monkeypatch.setattr(E, "residuals", wrong)
    assert _fails(T_EIGS.test_relerr_and_residual_hand_values)


# ---------------------------------------------------------------- Jacobi elliptic functions
def test_ellipj_with_sn_and_cn_swapped(monkeypatch):
    good = EL.ellipj

    def wrong(u, k, kp=None):
        sn, cn, dn = good(u, k, kp)
        return cn, sn, dn
    monkeypatch.setattr(EL, "ellipj", wrong)
    assert _fails(T_ELL.test_sn_cn_dn_match_scipy, 0.7)


def test_ellipj_dn_with_the_modulus_for_the_complement(monkeypatch):
    good = EL.ellipj

    def wrong(u, k, kp=None):
        sn, cn, _ = good(u, k, kp)
        return sn, cn, math.sqrt(cn * cn + k * k * sn * sn)
    monkeypatch.setattr(EL, "ellipj", wrong)
    assert _fails(T_ELL.test_sn_cn_dn_match_scipy, 0.7)


# ---------------------------------------------------------------- Theorem 1 coefficients
def test_zolo_c_index_off_by_one(monkeypatch):
    def wrong(r, ell):
        ellp = math.sqrt((1.0 - ell) * (1.0 + ell))
        Kp = EL.ellipk(ellp, ell)
        c = []
        for j in range(1, 2 * r):
            sn, cn, _ = EL.ellipj((j + 1) * Kp / (2 * r), ellp, ell)
            c.append(ell * ell * sn * sn / (cn * cn))
        return c
    monkeypatch.setattr(F, "zolo_c", wrong)
    assert _fails(T_FLT.test_r1_closed_form, 0.1)
    assert _fails(T_FLT.test_zolo_c_reflection_identities, 2, 0.05)


def test_zolo_c_without_the_ell_squared_factor(monkeypatch):
    def wrong(r, ell):
        ellp = math.sqrt((1.0 - ell) * (1.0 + ell))
        Kp = EL.ellipk(ellp, ell)
        c = []
        for j in range(1, 2 * r):
            sn, cn, _ = EL.ellipj(j * Kp / (2 * r), ellp, ell)
            c.append(sn * sn / (cn * cn))
        return c
    monkeypatch.setattr(F, "zolo_c", wrong)
    assert _fails(T_FLT.test_r1_closed_form, 0.1)


def test_zolo_product_with_numerator_and_denominator_coefficients_swapped(monkeypatch):
    def wrong(x, c):
        x = np.asarray(x, dtype=np.float64)
        r = (len(c) + 1) // 2
        num, den = x.copy(), np.ones_like(x)
        for j in range(1, r):
            den = den * (x * x + c[2 * j - 1])
        for j in range(1, r + 1):
            num = num * (x * x + c[2 * j - 2])
        return num / den
    monkeypatch.setattr(F, "zolo_product", wrong)
    assert _fails(T_FLT.test_equioscillation, 3, 0.02)


# ---------------------------------------------------------------- eq. req (Moebius map)
def test_mobius_with_zero_and_pole_swapped(monkeypatch):
    good = F.mobius

    def wrong(*gaps):
        alpha, beta, gamma, ell1 = good(*gaps)
        return beta, alpha, gamma, ell1
    monkeypatch.setattr(F, "mobius", wrong)
    assert _fails(T_FLT.test_mobius_conditions, (0.1, 0.3, 2.0, 2.5))


def test_mobius_ell1_with_a_dropped_square(monkeypatch):
    good = F.mobius

    def wrong(am, ap, bm, bp):
        alpha, beta, gamma, ell1 = good(am, ap, bm, bp)
        km1 = (ap - am) * (bp - bm) / ((bm - ap) * (bp - am))
        s = math.sqrt(1.0 + km1)
        return alpha, beta, gamma, km1 / (s + 1.0)            # (s + 1)^2 -> (s + 1)
    monkeypatch.setattr(F, "mobius", wrong)
    assert _fails(T_FLT.test_mobius_conditions, (0.1, 0.3, 2.0, 2.5))


# ---------------------------------------------------------------- Proposition 2
def test_prop2_weights_without_the_half(monkeypatch):
    good = F.prop2_poles

    def wrong(zolo, alpha, beta, gamma, rescale=1.0):
        s, w, const = good(zolo, alpha, beta, gamma, rescale)
        return s, 2.0 * w, const
    monkeypatch.setattr(F, "prop2_poles", wrong)
    assert _fails(T_FLT.test_prop2_poles_weights, 2)


def test_prop2_poles_conjugated(monkeypatch):
    good = F.prop2_poles

    def wrong(zolo, alpha, beta, gamma, rescale=1.0):
        s, w, const = good(zolo, alpha, beta, gamma, rescale)
        return np.conj(s), w, const
    monkeypatch.setattr(F, "prop2_poles", wrong)
    assert _fails(T_FLT.test_prop2_poles_weights, 2)


# ---------------------------------------------------------------- eq. solve / eq. solve2 (apply)
def test_apply_exact_without_the_conjugate_poles(monkeypatch):
    def wrong(A, B, X, flt):
        s, w, c0, _ = F.composite_poles(flt)
        X = np.asarray(X, dtype=np.complex128)
        BX = B @ X
        Y = c0 * X
        for sj, wj in zip(s, w):
            Y = Y + wj * FA.Solver(A, B, sj).solve(BX)
        return Y
    monkeypatch.setattr(AP, "apply_exact", wrong)
    assert _fails(T_APPLY.test_three_definitions_agree, "real2d", (2, 2))


def test_gmres_least_squares_with_the_shift_on_the_subdiagonal(monkeypatch):
    # (Negating or conjugating every shift would be an equivalent change: the 2 r2 shifts
    # come in pairs +-i sqrt(c) with equal weights, so the sum over them is unchanged.)
    def wrong(Hbar, s, beta):
        m1, m = Hbar.shape
        Hs = Hbar.astype(np.complex128).copy()
        Hs[np.arange(1, m + 1), np.arange(m)] += s          # I-bar placed one row down
        rhs = np.zeros(m1, dtype=np.complex128)
        rhs[0] = beta
        z, _, _, _ = np.linalg.lstsq(Hs, rhs, rcond=None)
        return z, float(np.linalg.norm(rhs - Hs @ z))
    monkeypatch.setattr(AP, "_lsq", wrong)
    assert _fails(T_APPLY.test_three_definitions_agree, "real2d", (2, 2))


def test_outer_weights_doubled(monkeypatch):
    good = F.ZoloFilter.outer_shifts

    def wrong(self):
        s, om = good(self)
        return s, 2.0 * om
    monkeypatch.setattr(F.ZoloFilter, "outer_shifts", wrong)
    assert _fails(T_APPLY.test_three_definitions_agree, "real2d", (2, 2))


# ---------------------------------------------------------------- LU without pivoting
def test_lu_without_the_pivot_division(monkeypatch):
    def wrong(K):
        U = np.array(K, dtype=np.complex128, copy=True)
        n = U.shape[0]
        L = np.eye(n, dtype=np.complex128)
        for j in range(n):
            L[j + 1:, j] = U[j + 1:, j]
            U[j + 1:, j:] -= np.outer(L[j + 1:, j], U[j, j:])
            U[j + 1:, j] = 0.0
        return L, U
    monkeypatch.setattr(FA, "lu_nopivot", wrong)
    assert _fails(T_FAC.test_lu_nopivot_definition)


# ---------------------------------------------------------------- contour rule (eq. contourintegral)
def test_trapezoidal_nodes_without_the_half_step(monkeypatch):
    class Wrong(F.ContourFilter):
        def __init__(self, kind, a, b, npoles):
            super().__init__(kind, a, b, npoles)
            theta = 2.0 * np.pi * np.arange(1, npoles + 1) / npoles     # a node on the real axis
            self.z = self.center + self.rho * np.exp(1j * theta)
            self.c = (2.0 * np.pi / npoles) * self.rho * np.exp(1j * theta) / (2.0 * np.pi)
            upper = self.z.imag > 0
            self.sigma_hat, self.w_hat = self.z[upper], -self.c[upper]
    monkeypatch.setattr(F, "ContourFilter", Wrong)
    assert _fails(T_FLT.test_citz_closed_form, 8)


# ---------------------------------------------------------------- the inner operator G (eq. solve)
def test_inner_operator_with_k_inverse_for_the_conjugate_pole(monkeypatch):
    class Wrong(AP.InnerOperator):
        def __call__(self, V):
            BV = self.B @ V
            out = self.flt.const_hat * V
            for sol, w in zip(self.solvers, self.flt.w_hat):
                out = out + w * sol.solve(BV) + np.conj(w) * sol.solve(BV)     # K^-1 in place of K^-H
            return out
    monkeypatch.setattr(AP, "InnerOperator", Wrong)
    assert _fails(T_APPLY.test_three_definitions_agree, "real2d", (2, 2))


# ---------------------------------------------------------------- Sylvester inertia
def test_inertia_counting_positive_pivots(monkeypatch):
    import scipy.linalg as sla

    def wrong(A, B, sigma):
        K = A.toarray() - sigma * B.toarray()
        _, D, _ = sla.ldl(K, hermitian=True)
        return int(np.sum(np.linalg.eigvalsh(D) > 0))
    monkeypatch.setattr(E, "inertia_count", wrong)
    assert _fails(T_EIGS.test_inertia_counts_match_dense)


# ---------------------------------------------------------------- nested dissection (Section 2.3)
def _nd_grid_variant(split_up=False, separator_first=False):
    """oracle.ordering.nd_grid with one change: the split index rounded up, or the
    separator numbered before its two halves."""
    from oracle import ordering as O

    def nd(dims, leaf_max=32):
        dims = tuple(int(d) for d in dims) + (1,) * (3 - len(dims))
        nx, ny, nz = dims
        perm, first, npiv, parent = [], [], [], []
        count = [0]

        def emit(verts):
            node = len(first)
            first.append(count[0]); npiv.append(len(verts)); parent.append(-1)
            perm.append(verts); count[0] += len(verts)
            return node

        def rec(box):
            ext = [hi - lo for lo, hi in box]
            if ext[0] * ext[1] * ext[2] == 0:
                return None
            if ext[0] * ext[1] * ext[2] <= leaf_max:
                return emit(O._box_vertices(box, nx, ny))
            ax = int(np.argmax(ext))
            lo, hi = box[ax]
            s = lo + (hi - lo + (1 if split_up else 0)) // 2
            lower = list(box); lower[ax] = (lo, s)
            upper = list(box); upper[ax] = (s + 1, hi)
            sep = list(box); sep[ax] = (s, s + 1)
            if separator_first:
                node = emit(O._box_vertices(sep, nx, ny))
                kids = [rec(lower), rec(upper)]
            else:
                kids = [rec(lower), rec(upper)]
                node = emit(O._box_vertices(sep, nx, ny))
            for k in kids:
                if k is not None:
                    parent[k] = node
            return node

        rec([(0, nx), (0, ny), (0, nz)])
        return O.Tree(np.concatenate(perm), first, npiv, parent)
    return nd


def test_nested_dissection_variants_match_the_oracle_when_unchanged():
    from oracle import ordering as O
    a, b = _nd_grid_variant()((7, 5, 3), 4), O.nd_grid((7, 5, 3), 4)
    assert np.array_equal(a.perm, b.perm) and np.array_equal(a.parent, b.parent)


@pytest.mark.parametrize("change", ["split_up", "separator_first"])
def test_nested_dissection_split_or_order_changed(monkeypatch, change):
    from oracle import ordering as O
    import test_oracle_ordering as T_ORD
    monkeypatch.setattr(O, "nd_grid", _nd_grid_variant(**{change: True}))
    assert _fails(T_ORD.test_hand_derived_4x3)
