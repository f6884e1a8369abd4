"""Pins for the oracle's nested dissection and front structures: a hand-derived
ordering, the separator property, and brute-force symbolic elimination."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import ordering as O
from paper_1701_08935_gb300 import synth

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
