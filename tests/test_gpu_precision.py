"""The precision form on a 3-D real pencil (3-D 7-point Laplacian + U[0,2] potential,
B = I + 0.1 M1 along x; ~20 eigenvalues between gaps picked as the widest spacing near
indices 100 and 120, filter (2,2), k = 32): complex128 throughout and
mixed precision (complex64 fronts, 3xTF32 / FP32 GEMMs, FP64 refinement) both against the
oracle's dense generalized eigensolver, and against each other."""
import numpy as np
import pytest

import paper_1701_08935_gb300 as Z
from oracle import eigs as E
from gpu_common import dev, host, need_gpu
import synth

pytestmark = pytest.mark.gpu


def _gaps(lam, p_range, q_range):
    """eigengaps at the widest relative spacing near each target index (the 3-D Laplacian's
    near-degenerate clusters would otherwise leave l1 ~ 1 and a weak filter)"""
    rel = np.diff(lam) / np.abs(lam[1:])
    p = p_range[0] + 1 + int(np.argmax(rel[p_range[0]:p_range[1]]))
    q = q_range[0] + 1 + int(np.argmax(rel[q_range[0]:q_range[1]]))
    return lam[p - 1], lam[p], lam[q - 1], lam[q]


@pytest.mark.parametrize("tc", [Z.TC_AUTO, Z.TC_ALWAYS])
def test_precision_form_matches_fp64_and_oracle(tc):
    need_gpu()
    pen = synth.pencil_3d_real(16, seed=3)
    lam, _ = E.dense_eigs(pen.A, pen.B)
    gaps = _gaps(lam, (94, 106), (114, 126))
    a, b = 0.5 * (gaps[0] + gaps[1]), 0.5 * (gaps[2] + gaps[3])
    inside = lam[(lam > a) & (lam < b)]
    X0 = synth.random_block(pen.n, 32, 5)
    out = {}
    for prec in (Z.PREC_FP64, Z.PREC_MIXED):
        flt = Z.Filter(*gaps, 2, 2)
        opts = Z.default_opts(grid=pen.dims, leaf_max=32, precision=prec, tensor_core=tc, n_iter_max=5)
        fac = Z.Factor(pen.A, pen.B, flt, opts=opts)
        ev, V, res, st, rc = fac.eigs(a, b, 32, X0=dev(X0))
        assert rc == Z.OK, (prec, st)
        assert len(ev) == len(inside) and 8 <= len(inside) <= 32
        assert np.max(np.abs(ev - inside) / np.abs(inside)) < 1e-10, prec
        Vh = host(V)
        assert np.max(E.residuals(pen.A, pen.B, ev, Vh)) <= 1e-10
        out[prec] = ev
    assert np.max(np.abs(out[Z.PREC_MIXED] - out[Z.PREC_FP64]) / np.abs(inside)) < 1e-10
