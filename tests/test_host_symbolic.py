"""Host ordering and symbolic analysis (C++) bit-exact against the oracle."""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_1701_08935_gb300 as Z
from oracle import ordering as O
import synth


def _compare(p, leaf, graph=False):
    """product vs oracle, geometric ND on p.dims, or graph ND with no geometry given"""
    opts = Z.default_opts(leaf_max=leaf) if graph else Z.default_opts(grid=p.dims, leaf_max=leaf)
    sym = Z.Symbolic(p.A, p.B, opts)
    got = sym.export()
    t = O.nd_graph(O.union_pattern(p.A, p.B), leaf) if graph else O.nd_grid(p.dims, leaf)
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


def test_no_grid_small_pattern_is_one_front():
    p = synth.pencil_2d_real(5, seed=1)
    sym = Z.Symbolic(p.A, p.B, Z.default_opts(leaf_max=32))
    e = sym.export()
    assert sym.info["nnodes"] == 1 and np.array_equal(e["perm"], np.arange(25))


@pytest.mark.parametrize("n,leaf", [(40, 32), (17, 5), (9, 1)])
def test_graph_nd_2d_real_recipe(n, leaf):
    _compare(synth.pencil_2d_real(n, seed=1), leaf, graph=True)


@pytest.mark.parametrize("n,leaf", [(12, 32), (9, 8)])
def test_graph_nd_3d_complex_recipe_27pt(n, leaf):
    _compare(synth.pencil_3d_peierls(n, seed=2, wells=4), leaf, graph=True)


def _pencil_from_pattern(P, name):
    """Hermitian-definite pencil on a given symmetric pattern: A = Laplacian of the graph +
    I, B = I (values do not matter to the ordering)."""
    P = sp.csr_matrix(P, dtype=float)
    P = ((P + P.T) != 0).astype(float)
    P.setdiag(0)
    P.eliminate_zeros()
    deg = np.asarray(P.sum(axis=1)).ravel()
    A = (sp.diags(deg + 1.0) - P).tocsr()
    A.sort_indices()
    B = sp.identity(P.shape[0], format="csr")
    return synth.Pencil(A, B, (P.shape[0],), name, "")


def test_graph_nd_disconnected_and_irregular_patterns():
    rng = np.random.default_rng(5)
    # two grids and an isolated vertex: three components
    g1 = synth.laplacian((7, 6)); g2 = synth.laplacian((5, 5, 3))
    P = sp.block_diag([g1, g2, sp.identity(1)]).tocsr()
    _compare(_pencil_from_pattern(P, "disconnected"), 8, graph=True)
    # random geometric graph in the unit square (no grid structure)
    pts = rng.random((600, 2))
    d = np.sqrt(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1))
    P = sp.csr_matrix((d < 0.07) & (d > 0))
    _compare(_pencil_from_pattern(P, "geometric"), 16, graph=True)
    # a path (1-D chain), and a star: the pseudo-peripheral root is a leaf, so the centre
    # is the separator of 49 isolated leaves
    path = sp.diags([np.ones(199), np.ones(199)], [-1, 1], shape=(200, 200))
    _compare(_pencil_from_pattern(path, "path"), 4, graph=True)
    star = sp.lil_matrix((50, 50)); star[0, 1:] = 1
    sym = _compare(_pencil_from_pattern(star.tocsr(), "star"), 4, graph=True)
    e = sym.export()
    assert sym.info["nnodes"] == 50 and e["perm"][-1] == 0 and np.all(e["npiv"] == 1)
    assert np.all(e["parent"][:-1] == 49) and e["parent"][-1] == -1
