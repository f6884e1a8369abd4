"""Full-size GPU checks on the 64^3 complex Hermitian benchmark pencil (n = 262144, 206
eigenvalues, r = (2, 6), k = 300, mixed precision): the oracle cannot run at this size, so
the result is checked against properties that hold at any size -- the pair count equals the
difference of two FP64 Sylvester inertia counts, every FP64 residual (recomputed on the
host) is <= 1e-10, the eigenvectors are B-orthonormal, the eigenvalues are distinct, and
R(B^-1 A) x = R(lam) x on sampled pairs (Section 2.1, Algorithm 1).  The run goes through
the benchmark's own modes: GMRES in two column chunks of 150 and split inner extents in the
solve products."""
import numpy as np
import pytest

import paper_1701_08935_gb300 as Z
from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def test_peierls64_properties():
    need_gpu()
    import torch
    import bench
    W = bench.WORKLOADS["peierls64"]
    pen = bench.build_pencil(W["recipe"])
    opts = Z.default_opts(grid=pen.dims, leaf_max=32, precision=Z.PREC_MIXED, n_iter_max=W["n_iter"],
                          tol=bench.TOL, gmres_tol=W["gmres_tol"], gmres_m_max=W["m_max"], gmres_chunk=150)
    sym = Z.Symbolic(pen.A, pen.B, opts)
    iopts = Z.default_opts(grid=pen.dims, leaf_max=32, precision=Z.PREC_FP64)
    am, ap, ca, bm, bp, cb = bench.checked_gaps(Z, pen, sym, iopts, W, Z.PREC_MIXED)
    assert cb - ca == 206
    flt = Z.Filter(am, ap, bm, bp, *W["r"])
    fac = Z.Factor(pen.A, pen.B, flt, sym=sym, opts=opts)
    a, b = 0.5 * (am + ap), 0.5 * (bm + bp)
    ev, V, res, st, rc = fac.eigs(a, b, W["k"])
    assert rc == Z.OK
    chk = bench.check_result(Z, pen, fac, flt, ev, V, res, cb - ca)
    assert chk["ok"], chk
    torch.cuda.empty_cache()
