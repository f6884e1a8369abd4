"""Host ordering and symbolic analysis (C++) bit-exact against the oracle."""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_1701_08935_gb300 as Z
from oracle import ordering as O
from paper_1701_08935_gb300 import synth


def _compare(p, leaf):
    sym = Z.Symbolic(p.A, p.B, Z.default_opts(grid=p.dims, leaf_max=leaf))
    got = sym.export()
    t = O.nd_grid(p.dims, leaf)
    S = O.Symbolic(t, O.union_pattern(p.A, p.B))
    assert np.array_equal(got["perm"], t.perm)
    assert np.array_equal(got["first"], t.first)
    assert np.array_equal(got["npiv"], t.npiv)
    assert np.array_equal(got["parent"], t.parent)
    ref_u = np.concatenate([S.U[s] for s in range(t.nnodes)])
    ref_ptr = np.concatenate([[0], np.cumsum([len(u) for u in S.U])])
    assert np.array_equal(got["uptr"], ref_ptr)
    assert np.array_equal(got["urows"], ref_u)
    assert sym.info["nnz_factor"] == S.nnz_factor()
    assert sym.info["nlevels"] == int(S.level.max()) + 1
    return sym


@pytest.mark.parametrize("n,leaf", [(40, 32), (17, 5), (9, 1)])
def test_2d_real_recipe(n, leaf):
    _compare(synth.pencil_2d_real(n, seed=1), leaf)


@pytest.mark.parametrize("n,leaf", [(12, 32), (9, 8), (7, 64)])
def test_3d_complex_recipe_27pt(n, leaf):
    _compare(synth.pencil_3d_peierls(n, seed=2, wells=4), leaf)


def test_3d_nonsquare_grid():
    A = synth.laplacian((10, 7, 5))
    B = synth.mass_x((10, 7, 5))
    p = synth.Pencil(A, B, (10, 7, 5), "box", "")
    _compare(p, 16)


@pytest.mark.slow
def test_full_size_64cubed():
    """The 64^3 27-point recipe (the complex Hermitian workload) at full size."""
    p = synth.pencil_3d_peierls(64, seed=2, wells=32)
    sym = _compare(p, 32)
    assert sym.info["n"] == 64 ** 3


def test_crossing_edge_rejected():
    p = synth.pencil_2d_real(8, seed=1)
    A = p.A.tolil()
    A[0, 63] = -0.1
    A[63, 0] = -0.1
    with pytest.raises(Z.ZoloError) as e:
        Z.Symbolic(A.tocsr(), p.B, Z.default_opts(grid=(8, 8), leaf_max=4))
    assert e.value.status == Z.EINVAL


def test_wrong_grid_dims_rejected():
    p = synth.pencil_2d_real(8, seed=1)
    with pytest.raises(Z.ZoloError):
        Z.Symbolic(p.A, p.B, Z.default_opts(grid=(4, 8), leaf_max=4))


def test_no_grid_single_front():
    p = synth.pencil_2d_real(6, seed=1)
    sym = Z.Symbolic(p.A, p.B, Z.default_opts())
    e = sym.export()
    assert sym.info["nnodes"] == 1 and np.array_equal(e["perm"], np.arange(36))
