"""GPU parity of spectrum slicing (zolo_eigs_slices; Section 3.2 treats spectrum ranges as
independent problems): the union of the slices' eigenpairs against the oracle's dense
generalized eigensolver, every pair in its own slice, none twice, residuals <= 1e-10."""
import numpy as np
import pytest

import paper_1701_08935_gb300 as Z
from oracle import eigs as E
from gpu_common import host, need_gpu
import synth

pytestmark = pytest.mark.gpu


def _bounds(lam, idx):
    """slice boundaries midway between consecutive eigenvalues at the given indices"""
    return np.array([(lam[i - 1] + lam[i]) / 2 for i in idx])


@pytest.mark.parametrize("prec", [Z.PREC_FP64, Z.PREC_MIXED])
def test_slices_match_dense_eigensolver(prec):
    need_gpu()
    pen = synth.pencil_2d_real(40, seed=1)
    lam, _ = E.dense_eigs(pen.A, pen.B)
    bounds = _bounds(lam, [60, 78, 95, 121])
    opts = Z.default_opts(grid=pen.dims, leaf_max=32, precision=prec, r1=2, r2=3, n_iter_max=6)
    ev, V, res, sl, st, rc = Z.eigs_slices(pen.A, pen.B, bounds, opts=opts)
    assert rc == Z.OK
    ref = lam[(lam > bounds[0]) & (lam < bounds[-1])]
    assert len(ev) == len(ref) == 61
    assert np.max(np.abs(ev - ref) / np.abs(ref)) < 1e-10
    assert np.all(res <= 1e-10)
    for s in range(3):
        e = ev[sl == s]
        assert np.all((e > bounds[s]) & (e < bounds[s + 1]))
        assert len(e) == np.sum((lam > bounds[s]) & (lam < bounds[s + 1]))
    # B-orthonormal within a slice; slices are B-orthogonal to each other up to the accuracy of the pairs
    X = host(V)
    G = X.conj().T @ (pen.B @ X)
    assert np.max(np.abs(G - np.eye(len(ev)))) < 1e-8


def test_slices_on_a_3d_real_pencil():
    need_gpu()
    pen = synth.pencil_3d_real(14, seed=4, vmax=4.0, b_diag=(1.0, 2.0))     # the slicing workload recipe, small
    lam, _ = E.dense_eigs(pen.A, pen.B)
    bounds = _bounds(lam, [20, 45, 70])
    opts = Z.default_opts(grid=pen.dims, leaf_max=32, precision=Z.PREC_MIXED, r1=2, r2=3, n_iter_max=6)
    ev, V, res, sl, st, rc = Z.eigs_slices(pen.A, pen.B, bounds, opts=opts)
    assert rc == Z.OK
    ref = lam[(lam > bounds[0]) & (lam < bounds[-1])]
    assert len(ev) == len(ref)
    assert np.max(np.abs(ev - ref) / np.abs(ref)) < 1e-10
    assert np.all(res <= 1e-10)
