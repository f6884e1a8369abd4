"""GPU parity of the tcgen05 tensor-core GEMM (3xTF32 split of complex64 operands) inside
the mixed-precision multifrontal factorisation and block solves (Section 2.3), through
the C ABI: forced onto every complex64 launch of small pencils and compared with the
oracle's exact sparse solves, and chosen automatically on a pencil whose top fronts
exceed 256 rows and compared with the FP32-FMA-only path."""
import numpy as np
import pytest

import paper_1701_08935_gb300 as Z
from oracle import apply as AP
from oracle import factor as FA
from oracle import filter as F
from gpu_common import case, colrel, dev, host, need_gpu
import synth

pytestmark = pytest.mark.gpu


def _factor(pen, leaf, gaps, tc, r=(2, 2), **kw):
    flt = Z.Filter(*gaps, *r)
    opts = Z.default_opts(grid=pen.dims, leaf_max=leaf, precision=Z.PREC_MIXED, tensor_core=tc, **kw)
    return flt, Z.Factor(pen.A, pen.B, flt, opts=opts)


@pytest.mark.parametrize("name", ["real2d_40", "cplx3d_9", "cplx3d_12"])
def test_forced_tensor_core_solves(name):
    """K_j^-1 b and K_j^-H b with every complex64 GEMM on the tensor cores, against SuperLU."""
    need_gpu()
    pen, leaf, gaps, _ = case(name)
    flt, fac = _factor(pen, leaf, gaps, Z.TC_ALWAYS)
    for k in (1, 37, 300):
        Bk = synth.random_block(pen.n, k, 5 + k)
        for j, s in enumerate(flt.sigma_hat):
            ref = FA.Solver(pen.A, pen.B, s)
            for herm in (False, True):
                X = host(fac.solve(j, dev(Bk), herm=herm))
                assert colrel(X, ref.solve(Bk, herm=herm)) < 1e-10, (k, j, herm)
    st = fac.stats()
    assert 1 <= st["n_refine_max"] <= 6


@pytest.mark.parametrize("name", ["cplx3d_9", "cplx3d_12"])
def test_forced_tensor_core_inner_operator(name):
    """G X = const X + sum_j (w_j K_j^-1 B X + conj(w_j) K_j^-H B X)  (eq. solve)."""
    need_gpu()
    pen, leaf, gaps, _ = case(name)
    flt, fac = _factor(pen, leaf, gaps, Z.TC_ALWAYS)
    G = AP.InnerOperator(pen.A, pen.B, F.ZoloFilter(*gaps, 2, 2))
    X = synth.random_block(pen.n, 24, 3)
    assert colrel(host(fac.apply_inner(dev(X))), G(X)) < 1e-10


def test_auto_tensor_core_matches_fma_path():
    """On a 20^3 Peierls pencil (top separator fronts of 400+ rows, so the automatic policy
    puts the top levels on the tensor cores) both GEMM engines give the same refined solves,
    with a comparable number of refinement steps (the 3xTF32 factor is about as accurate as
    the FP32 one), and both match SuperLU."""
    need_gpu()
    pen = synth.pencil_3d_peierls(20, seed=2, wells=12)
    gaps = (0.30, 0.31, 0.40, 0.41)
    k = 96
    Bk = synth.random_block(pen.n, k, 21)
    out, nref = {}, {}
    for tc in (Z.TC_AUTO, Z.TC_OFF):
        flt, fac = _factor(pen, 32, gaps, tc)
        out[tc] = [host(fac.solve(j, dev(Bk), herm=h)) for j in range(2) for h in (False, True)]
        nref[tc] = fac.stats()["n_refine_max"]
        sig = flt.sigma_hat
    for a, b in zip(out[Z.TC_AUTO], out[Z.TC_OFF]):
        assert colrel(a, b) < 1e-10
    ref = FA.Solver(pen.A, pen.B, sig[0])
    assert colrel(out[Z.TC_AUTO][0], ref.solve(Bk)) < 1e-10
    assert nref[Z.TC_AUTO] <= nref[Z.TC_OFF] + 2


def test_tensor_core_policy_ignored_in_fp64():
    """complex128 fronts never use the tensor-core kernel: ALWAYS and OFF agree bit for bit
    up to the atomic split-K order (1e-13)."""
    need_gpu()
    pen, leaf, gaps, _ = case("cplx3d_9")
    flt = Z.Filter(*gaps, 2, 2)
    Bk = synth.random_block(pen.n, 16, 2)
    res = []
    for tc in (Z.TC_ALWAYS, Z.TC_OFF):
        opts = Z.default_opts(grid=pen.dims, leaf_max=leaf, precision=Z.PREC_FP64, tensor_core=tc)
        fac = Z.Factor(pen.A, pen.B, flt, opts=opts)
        res.append(host(fac.solve(0, dev(Bk))))
    assert colrel(res[0], res[1]) < 1e-13


@pytest.mark.parametrize("name", ["real2d_40", "cplx3d_12"])
@pytest.mark.parametrize("rtol", [1e-8, 1e-6])
def test_loose_refinement_meets_its_tolerance(name, rtol):
    """Mixed-precision solves refined to a loose tolerance (>= 1e-8: the residuals run in
    double-float arithmetic on the FP32 pipe) meet that tolerance in the FP64 residual
    computed on the host, and agree with SuperLU to what the tolerance allows."""
    need_gpu()
    pen, leaf, gaps, _ = case(name)
    flt, fac = _factor(pen, leaf, gaps, Z.TC_AUTO, refine_tol=rtol)
    Bk = synth.random_block(pen.n, 40, 77)
    for j, s in enumerate(flt.sigma_hat):
        K = (pen.A - s * pen.B).tocsr()
        for herm in (False, True):
            X = host(fac.solve(j, dev(Bk), herm=herm))
            Kh = K.conj().T.tocsr() if herm else K
            R = Bk - Kh @ X
            rel = np.linalg.norm(R, axis=0) / np.linalg.norm(Bk, axis=0)
            assert rel.max() <= rtol * 1.1, (j, herm, rel.max())
