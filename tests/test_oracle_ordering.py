"""Pins for the oracle's nested dissection and front structures: a hand-derived
ordering, the separator property, and brute-force symbolic elimination."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import ordering as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                out[k] = [int(x) for x in v]
    return out


def test_hand_derived_4x3():
    g = _read_golden("nd_4x3_leaf2.txt")
    t = O.nd_grid((4, 3), leaf_max=2)
    assert t.perm.tolist() == g["perm"]
    assert t.first.tolist() == g["first"]
    assert t.npiv.tolist() == g["npiv"]
    assert t.parent.tolist() == g["parent"]


def _stencil_pattern(dims, full):
    """7-point (full=False) or 27-point (full=True) pattern of a grid."""
    dims = tuple(dims) + (1,) * (3 - len(dims))
    nx, ny, nz = dims
    n = nx * ny * nz
    idx = np.arange(n)
    x, y, z = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    rows, cols = [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if not full and abs(dx) + abs(dy) + abs(dz) > 1:
                    continue
                m = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny) & (z + dz >= 0) & (z + dz < nz)
                rows.append(idx[m]); cols.append(idx[m] + dx + nx * (dy + ny * dz))
    r, c = np.concatenate(rows), np.concatenate(cols)
    return sp.csr_matrix((np.ones(len(r)), (r, c)), shape=(n, n))


def _brute_force_structure(P, perm):
    """Boolean Gaussian elimination of the permuted pattern: struct of L by column."""
    Q = P[perm][:, perm].toarray() != 0
    n = Q.shape[0]
    for j in range(n):
        rows = np.nonzero(Q[j + 1:, j])[0] + j + 1
        Q[np.ix_(rows, rows)] = True
    return Q


@pytest.mark.parametrize("dims,full,leaf", [((7, 9), False, 4), ((6, 5), True, 3),
                                            ((5, 4, 6), False, 8), ((4, 5, 4), True, 6),
                                            ((3, 3, 3), True, 1)])
def test_update_rows_equal_brute_force_fill(dims, full, leaf):
    P = _stencil_pattern(dims, full)
    t = O.nd_grid(dims, leaf_max=leaf)
    S = O.Symbolic(t, P)
    Q = _brute_force_structure(P, t.perm)
    total_true = 0
    for s in range(t.nnodes):
        f, e = int(t.first[s]), int(t.first[s] + t.npiv[s])
        true_rows = np.nonzero(Q[e:, f:e].any(axis=1))[0] + e
        assert S.U[s].tolist() == true_rows.tolist()
        total_true += int(np.tril(Q[f:, f:e], -1).sum())
    # dense pivot blocks can only hold more entries than the exact fill
    assert S.nnz_factor() >= total_true


def test_tree_invariants_config_shapes():
    for dims, leaf in [((40, 40), 32), ((12, 10, 9), 32), ((16, 16, 16), 64)]:
        t = O.nd_grid(dims, leaf_max=leaf)
        n = int(np.prod(dims))
        assert sorted(t.perm.tolist()) == list(range(n))
        assert np.all((t.parent == -1) | (t.parent > np.arange(t.nnodes)))
        assert int(np.sum(t.parent == -1)) == 1
        assert np.all(np.diff(t.first) == t.npiv[:-1]) and t.first[0] == 0
        assert int(t.npiv.sum()) == n
        assert int(t.npiv.max()) <= max(leaf, max(dims) ** (len(dims) - 1))


def test_crossing_edge_is_rejected():
    dims = (8, 8)
    P = _stencil_pattern(dims, False).tolil()
    P[0, 63] = 1.0
    P[63, 0] = 1.0
    t = O.nd_grid(dims, leaf_max=4)
    with pytest.raises(ValueError):
        O.Symbolic(t, P.tocsr())


def test_union_pattern_of_config2_recipe_is_27_point():
    p = synth.pencil_3d_peierls(6, seed=2, wells=3)
    P = O.union_pattern(p.A, p.B)
    Q = _stencil_pattern((6, 6, 6), True)
    assert (P != 0).sum() == (Q != 0).sum()
    assert abs((P != 0).astype(int) - (Q != 0).astype(int)).sum() == 0


# ---------------------------------------------------------------- graph nested dissection
def test_graph_nd_hand_derived_path():
    """Path 0-1-...-6, leaf_max 1.  BFS from 0 has 7 levels and the BFS from the far end 6
    has no more, so the root stays 0: separator {3}; the left part 0-1-2 has root 0 and
    separator {1}, the right part 4-5-6 has root 4 and separator {5}.  Completion order:
    0, 2, 1, 4, 6, 5, 3."""
    n = 7
    P = sp.diags([np.ones(n - 1), np.ones(n - 1)], [-1, 1], shape=(n, n)).tocsr()
    t = O.nd_graph(P, leaf_max=1)
    assert t.perm.tolist() == [0, 2, 1, 4, 6, 5, 3]
    assert t.first.tolist() == list(range(7)) and t.npiv.tolist() == [1] * 7
    assert t.parent.tolist() == [2, 2, 6, 5, 5, 6, -1]


@pytest.mark.parametrize("dims,full,leaf", [((7, 9), False, 4), ((6, 5), True, 3),
                                            ((5, 4, 6), False, 8), ((3, 3, 3), True, 1)])
def test_graph_nd_update_rows_equal_brute_force_fill(dims, full, leaf):
    """Graph ND of a stencil pattern (no geometry): the fronts' update rows are exactly the
    fill of a boolean elimination in the same order."""
    P = _stencil_pattern(dims, full)
    t = O.nd_graph(P, leaf_max=leaf)
    S = O.Symbolic(t, P)
    Q = _brute_force_structure(P, t.perm)
    for s in range(t.nnodes):
        f, e = int(t.first[s]), int(t.first[s] + t.npiv[s])
        true_rows = np.nonzero(Q[e:, f:e].any(axis=1))[0] + e
        assert S.U[s].tolist() == true_rows.tolist()


def test_graph_nd_tree_invariants_on_random_graphs():
    rng = np.random.default_rng(11)
    for trial in range(5):
        n = int(rng.integers(50, 400))
        pts = rng.random((n, 2))
        d = np.sqrt(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1))
        P = sp.csr_matrix((d < 1.6 / np.sqrt(n)) & (d > 0)).astype(float)
        t = O.nd_graph(P, leaf_max=int(rng.integers(1, 20)))
        assert sorted(t.perm.tolist()) == list(range(n))
        assert np.all((t.parent == -1) | (t.parent > np.arange(t.nnodes)))
        assert np.all(np.diff(t.first) == t.npiv[:-1]) and t.first[0] == 0
        O.Symbolic(t, P + sp.identity(n))          # separator property: raises if violated
        # a separator is never larger than the set it splits
        sizes = np.zeros(t.nnodes, dtype=int)
        for s in range(t.nnodes):
            sizes[s] += t.npiv[s]
            if t.parent[s] >= 0:
                sizes[t.parent[s]] += sizes[s]
        inner = [s for s in range(t.nnodes) if sizes[s] > t.npiv[s]]
        assert all(t.npiv[s] < sizes[s] for s in inner)
