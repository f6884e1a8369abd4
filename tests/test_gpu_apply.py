"""GPU parity of the filtered block Y = R_ab(B^-1 A) X (the GMRES steps of Algorithm 2) and of
Algorithm 1 against the oracle, through the C ABI."""
import numpy as np
import pytest

import paper_1701_08935_gb300 as Z
from oracle import apply as AP
from oracle import eigs as E
from oracle import filter as F
from gpu_common import case, colrel, dev, host, need_gpu
import synth

pytestmark = pytest.mark.gpu


def _setup(name, r, prec=Z.PREC_FP64, **kw):
    pen, leaf, gaps, lam = case(name)
    flt = Z.Filter(*gaps, *r)
    opts = Z.default_opts(grid=pen.dims, leaf_max=leaf, precision=prec, **kw)
    fac = Z.Factor(pen.A, pen.B, flt, opts=opts)
    return pen, gaps, lam, flt, fac


@pytest.mark.parametrize("name", ["real2d_12", "cplx3d_9", "cplx3d_12", "real2d_40"])
@pytest.mark.parametrize("r", [(2, 2), (2, 6)])
def test_apply_matches_exact_and_hybrid(name, r):
    need_gpu()
    pen, gaps, lam, flt, fac = _setup(name, r)
    X = synth.random_block(pen.n, 37, 4)
    Yd, st = fac.apply(dev(X))
    Y = host(Yd)
    oflt = F.ZoloFilter(*gaps, *r)
    Y2 = AP.apply_exact(pen.A, pen.B, X, oflt)
    assert colrel(Y, Y2) < 1e-9
    Y3, info = AP.apply_hybrid(pen.A, pen.B, X, oflt, return_info=True)
    assert colrel(Y, Y3) < 1e-9
    assert abs(st["n_gmres"] - info["m"]) <= 1
    assert st["gmres_res"] <= 1e-12


@pytest.mark.parametrize("name", ["real2d_12", "cplx3d_12"])
def test_apply_mixed_precision(name):
    need_gpu()
    pen, gaps, lam, flt, fac = _setup(name, (2, 2), Z.PREC_MIXED)
    X = synth.random_block(pen.n, 20, 8)
    Y = host(fac.apply(dev(X))[0])
    Y2 = AP.apply_exact(pen.A, pen.B, X, F.ZoloFilter(*gaps, 2, 2))
    assert colrel(Y, Y2) < 1e-9


@pytest.mark.parametrize("k", [1, 64, 65])
def test_apply_block_widths(k):
    need_gpu()
    pen, gaps, lam, flt, fac = _setup("cplx3d_9", (2, 3))
    X = synth.random_block(pen.n, k, 13)
    Y = host(fac.apply(dev(X))[0])
    assert colrel(Y, AP.apply_exact(pen.A, pen.B, X, F.ZoloFilter(*gaps, 2, 3))) < 1e-9


def test_apply_on_eigenvectors_gives_filter_values():
    """R(B^-1 A) x_i = R(lam_i) x_i (property that holds at any size)."""
    need_gpu()
    pen, gaps, lam, flt, fac = _setup("cplx3d_9", (2, 2))
    lam, V = E.dense_eigs(pen.A, pen.B)
    idx = [0, 39, 40, 55, 69, 70, 300]
    Y = host(fac.apply(dev(V[:, idx]))[0])
    assert np.allclose(Y, V[:, idx] * flt(lam[idx])[None, :], atol=1e-10)


@pytest.mark.parametrize("name,k", [("real2d_40", 32), ("cplx3d_12", 64), ("cplx3d_9", 48)])
@pytest.mark.parametrize("prec", [Z.PREC_FP64, Z.PREC_MIXED])
def test_eigs_match_brute_force(name, k, prec):
    need_gpu()
    pen, gaps, lam, flt, fac = _setup(name, (2, 2), prec, n_iter_max=4)
    a, b = 0.5 * (gaps[0] + gaps[1]), 0.5 * (gaps[2] + gaps[3])
    X0 = synth.random_block(pen.n, k, 21)
    ev, V, res, st, rc = fac.eigs(a, b, k, X0=dev(X0))
    assert rc == Z.OK, st
    inside = lam[(lam > a) & (lam < b)]
    assert len(ev) == len(inside)
    assert np.allclose(ev, inside, rtol=1e-10, atol=1e-12)
    assert np.max(res) <= 1e-10
    Vh = host(V)
    assert np.max(E.residuals(pen.A, pen.B, ev, Vh)) <= 1e-10
    G = Vh.conj().T @ (pen.B @ Vh)
    assert np.allclose(G, np.eye(len(ev)), atol=1e-10)
    assert st["n_iter"] <= 4


def test_eigs_seeded_start_block():
    need_gpu()
    pen, gaps, lam, flt, fac = _setup("real2d_12", (2, 3), n_iter_max=4)
    a, b = 0.5 * (gaps[0] + gaps[1]), 0.5 * (gaps[2] + gaps[3])
    ev, V, res, st, rc = fac.eigs(a, b, 24)
    assert rc == Z.OK
    assert np.allclose(ev, lam[(lam > a) & (lam < b)], rtol=1e-10)
