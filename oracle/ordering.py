"""Nested-dissection ordering, assembly tree and front structures (oracle).

Test infrastructure only (see ``oracle/__init__``).

The paper factors each A - sigma_j B with the multifrontal method (Section 2.3,
"fast direct solvers"), whose fill is controlled by a nested-dissection
ordering computed once per sparsity pattern.  The paper does not fix the
ordering; this oracle states one rule and the product implements the same rule
so that every index array can be compared bit for bit.

Geometric nested dissection of a grid box [x0,x1) x [y0,y1) x [z0,z1):
  * a box with at most ``leaf_max`` vertices is a leaf: its vertices form one
    front, ordered lexicographically (x fastest, then y, then z);
  * otherwise split the longest axis (ties: x before y before z) at the plane
    lo + d//2 (d = extent); order the lower box, then the upper box, then the
    plane's vertices (lexicographically) as the front that is their parent;
    empty boxes produce no front.
The tree nodes are numbered in that completion (post-)order, so parent > child.

Front structure (standard multifrontal symbolic analysis): with pivots(s) the
contiguous new indices of front s, its update rows are
  U(s) = { new(u) >= end(s) : u adjacent to a pivot of s } U ( U(c) minus pivots(s), c child of s ),
sorted increasingly; the front's rows are pivots(s) followed by U(s).  A pattern
edge that joins two subtrees of the separator tree (a stencil wider than the
nearest neighbours) breaks the dissection; it is reported as an error.
"""
import collections

import numpy as np


class Tree:
    def __init__(self, perm, first, npiv, parent):
        self.perm = np.asarray(perm, dtype=np.int32)          # new -> old
        self.first = np.asarray(first, dtype=np.int32)        # pivot range start per node
        self.npiv = np.asarray(npiv, dtype=np.int32)
        self.parent = np.asarray(parent, dtype=np.int32)      # -1 for a root
        n = len(self.perm)
        self.iperm = np.empty(n, dtype=np.int32)
        self.iperm[self.perm] = np.arange(n, dtype=np.int32)  # old -> new

    @property
    def nnodes(self):
        return len(self.first)


def _box_vertices(box, nx, ny):
    (x0, x1), (y0, y1), (z0, z1) = box
    zz, yy, xx = np.meshgrid(np.arange(z0, z1), np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
    return (xx + nx * (yy + ny * zz)).ravel().astype(np.int32)   # x fastest


def nd_grid(dims, leaf_max=32):
    """Geometric nested dissection of a 1D/2D/3D grid (see module docstring)."""
    dims = tuple(int(d) for d in dims) + (1,) * (3 - len(dims))
    nx, ny, nz = dims
    perm, first, npiv, parent = [], [], [], []
    count = [0]

    def rec(box):
        ext = [hi - lo for lo, hi in box]
        nv = ext[0] * ext[1] * ext[2]
        if nv == 0:
            return None
        if nv <= leaf_max:
            verts = _box_vertices(box, nx, ny)
            node = len(first)
            first.append(count[0]); npiv.append(len(verts)); parent.append(-1)
            perm.append(verts); count[0] += len(verts)
            return node
        ax = int(np.argmax(ext))          # first axis with the largest extent
        lo, hi = box[ax]
        s = lo + (hi - lo) // 2
        lower = list(box); lower[ax] = (lo, s)
        upper = list(box); upper[ax] = (s + 1, hi)
        sep = list(box); sep[ax] = (s, s + 1)
        kids = [rec(lower), rec(upper)]
        verts = _box_vertices(sep, nx, ny)
        node = len(first)
        first.append(count[0]); npiv.append(len(verts)); parent.append(-1)
        perm.append(verts); count[0] += len(verts)
        for k in kids:
            if k is not None:
                parent[k] = node
        return node

    rec([(0, nx), (0, ny), (0, nz)])
    return Tree(np.concatenate(perm), first, npiv, parent)


def nd_graph(pattern, leaf_max=32):
    """Graph nested dissection by level structures (George & Liu), for pencils given
    without grid geometry.  On the symmetric pattern (self-loops ignored), a vertex set S
    is ordered as follows:
      * its connected components (in the subgraph induced by S) are ordered by their
        smallest vertex and become sibling subtrees;
      * a component C with at most ``leaf_max`` vertices is a leaf front (ascending vertex
        index);
      * otherwise a pseudo-peripheral root r is found: start at min(C); BFS gives levels;
        take the vertex of smallest degree in C on the last level (lowest index on ties);
        if its BFS has more levels, it becomes r and the step repeats, else r stays;
      * with the h levels L_0..L_{h-1} of the BFS from r: if h < 3 the component is a leaf
        front; otherwise the middle level L_{h//2} (ascending) is the separator front, whose
        children are the subtrees of L_0..L_{h//2-1} and of L_{h//2+1}..L_{h-1}, ordered first
        (in that order).  Edges join adjacent levels only, so the two parts are disconnected.
    Nodes are numbered in completion order (children before parents); a disconnected
    pattern gives several roots."""
    P = pattern.tocsr()
    n = P.shape[0]
    nbr = []
    for v in range(n):
        cols = P.indices[P.indptr[v]:P.indptr[v + 1]]
        nbr.append(sorted(int(c) for c in set(cols.tolist()) if c != v))
    perm, first, npiv, parent = [], [], [], []
    count = [0]

    def emit(verts):
        node = len(first)
        first.append(count[0]); npiv.append(len(verts)); parent.append(-1)
        perm.append(np.asarray(verts, dtype=np.int32)); count[0] += len(verts)
        return node

    def bfs(inset, root):
        seen = {root}
        levels = [[root]]
        while True:
            nxt = set()
            for v in levels[-1]:
                for u in nbr[v]:
                    if u in inset and u not in seen:
                        nxt.add(u)
            if not nxt:
                return levels
            seen |= nxt
            levels.append(sorted(nxt))

    def components(verts):
        inset = set(verts)
        left = set(verts)
        comps = []
        for v in sorted(verts):
            if v not in left:
                continue
            comp = set()
            stack = [v]
            left.discard(v)
            while stack:
                x = stack.pop()
                comp.add(x)
                for u in nbr[x]:
                    if u in left:
                        left.discard(u)
                        stack.append(u)
            comps.append(sorted(comp))
        return comps

    def rec_set(verts):
        return [rec_connected(c) for c in components(verts)]

    def rec_connected(comp):
        if len(comp) <= leaf_max:
            return emit(comp)
        inset = set(comp)
        r = comp[0]
        levels = bfs(inset, r)
        while True:
            deg = lambda v: sum(1 for u in nbr[v] if u in inset)
            cand = min(levels[-1], key=lambda v: (deg(v), v))
            lv = bfs(inset, cand)
            if len(lv) > len(levels):
                r, levels = cand, lv
            else:
                break
        h = len(levels)
        if h < 3:
            return emit(comp)
        m = h // 2
        part1 = sorted(v for L in levels[:m] for v in L)
        part2 = sorted(v for L in levels[m + 1:] for v in L)
        kids = rec_set(part1) + rec_set(part2)
        node = emit(levels[m])
        for k in kids:
            parent[k] = node
        return node

    rec_set(list(range(n)))
    return Tree(np.concatenate(perm) if perm else np.zeros(0, np.int32), first, npiv, parent)


class Symbolic:
    """Front structures on top of a Tree for a symmetric sparsity pattern."""

    def __init__(self, tree, pattern):
        P = pattern.tocsr()
        n = P.shape[0]
        if len(tree.perm) != n or sorted(tree.perm.tolist()) != list(range(n)):
            raise ValueError("perm is not a permutation of the pattern's vertices")
        self.tree = tree
        nn = tree.nnodes
        children = [[] for _ in range(nn)]
        for s in range(nn):
            if tree.parent[s] >= 0:
                children[tree.parent[s]].append(s)
        node_of = np.empty(n, dtype=np.int32)             # new index -> tree node
        for s in range(nn):
            node_of[tree.first[s]:tree.first[s] + tree.npiv[s]] = s
        self.children = children
        U = [None] * nn
        for s in range(nn):                               # postorder: children first
            f, e = int(tree.first[s]), int(tree.first[s] + tree.npiv[s])
            rows = tree.perm[f:e]
            cols = np.concatenate([P.indices[P.indptr[v]:P.indptr[v + 1]] for v in rows])
            newc = tree.iperm[cols]
            parts = [newc[newc >= e]]
            for c in children[s]:
                parts.append(U[c][U[c] >= e])
            u = np.unique(np.concatenate(parts)).astype(np.int32)
            # separator property: every update row must belong to an ancestor of s
            anc = set()
            p = int(tree.parent[s])
            while p >= 0:
                anc.add(p); p = int(tree.parent[p])
            bad = [int(i) for i in u if int(node_of[i]) not in anc]
            if bad:
                raise ValueError(f"pattern edge crosses the dissection at front {s}")
            U[s] = u
        self.U = U
        self.node_of = node_of
        level = np.zeros(nn, dtype=np.int32)
        for s in range(nn):
            for c in children[s]:
                level[s] = max(level[s], level[c] + 1)
        self.level = level

    def front_rows(self, s):
        t = self.tree
        f = int(t.first[s])
        return np.concatenate([np.arange(f, f + int(t.npiv[s]), dtype=np.int32), self.U[s]])

    def nnz_factor(self):
        """Entries of L (unit diagonal excluded) held by the fronts: sum np*(np-1)/2 + np*nu."""
        t = 0
        for s in range(self.tree.nnodes):
            p = int(self.tree.npiv[s]); u = len(self.U[s])
            t += p * (p - 1) // 2 + p * u
        return t


def union_pattern(A, B):
    """Symmetric sparsity pattern of A + B (values dropped)."""
    P = (abs(A) + abs(B)).tocsr()
    P = ((P + P.T) != 0).astype(np.float64).tocsr()
    P.sort_indices()
    return P
