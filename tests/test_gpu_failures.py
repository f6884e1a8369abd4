"""Failure paths on the GPU without any fault: an exactly singular pivot gives
ZOLO_ESINGULAR; step caps give ZOLO_ENOCONV with the context still usable."""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_1701_08935_gb300 as Z
from gpu_common import case, colrel, dev, host, need_gpu
import synth

pytestmark = pytest.mark.gpu


def test_singular_leading_pivot():
    need_gpu()
    n = 40
    A = sp.diags([np.full(n - 1, -0.5), np.arange(1.0, n + 1.0), np.full(n - 1, -0.5)], [-1, 0, 1]).tocsr()
    B = sp.identity(n, format="csr")
    # no grid: one dense front in the natural order, so the first pivot is A[0,0] - s B[0,0] = 0
    with pytest.raises(Z.ZoloError) as e:
        Z.inertia(A, B, [1.0], opts=Z.default_opts())
    assert e.value.status == Z.ESINGULAR
    # the context survives: a regular shift right after works and counts correctly
    lam = np.linalg.eigvalsh(A.toarray())
    c = Z.inertia(A, B, [10.25], opts=Z.default_opts())
    assert int(c[0]) == int(np.sum(lam < 10.25))


def test_gmres_step_cap_reports_noconv():
    need_gpu()
    pen, leaf, gaps, lam = case("cplx3d_9")
    fac = Z.Factor(pen.A, pen.B, Z.Filter(*gaps, 2, 2), opts=Z.default_opts(grid=pen.dims, leaf_max=leaf,
                                                                              gmres_m_max=3))
    X = synth.random_block(pen.n, 8, 2)
    with pytest.raises(Z.ZoloError) as e:
        fac.apply(dev(X))
    assert e.value.status == Z.ENOCONV
    # still usable
    Y = host(fac.matmul("B", dev(X)))
    assert colrel(Y, pen.B @ X) < 1e-14


def test_refinement_cap_reports_noconv():
    need_gpu()
    pen, leaf, gaps, lam = case("real2d_12")
    fac = Z.Factor(pen.A, pen.B, Z.Filter(*gaps, 2, 2),
                   opts=Z.default_opts(grid=pen.dims, leaf_max=leaf, precision=Z.PREC_MIXED, refine_tol=1e-40,
                                       refine_max=1))
    with pytest.raises(Z.ZoloError) as e:
        fac.solve(0, dev(synth.random_block(pen.n, 4, 3)))
    assert e.value.status == Z.ENOCONV


def test_inertia_matches_dense_counts():
    need_gpu()
    pen, leaf, gaps, lam = case("cplx3d_9")
    shifts = [lam[10] + 1e-6, lam[100] - 1e-6, 0.5 * (lam[300] + lam[301])]
    c = Z.inertia(pen.A, pen.B, shifts, opts=Z.default_opts(grid=pen.dims, leaf_max=leaf))
    assert list(c) == [int(np.sum(lam < s)) for s in shifts]
