// Ordering and symbolic analysis (host, once per sparsity pattern).
//
// The multifrontal method (Section 2.3, "fast direct solvers") factors each shifted
// matrix front by front along an assembly tree: the separator tree of a nested
// dissection, by level structures on the pattern's graph when no grid is given (see
// GNDBuilder), else geometric on the grid the pencil lives on:
//   * a box with at most leaf_max vertices is one front (lexicographic, x fastest);
//   * otherwise the longest axis (x before y before z on ties) is split at the plane
//     lo + d/2; the lower box, the upper box and then the plane are ordered, the
//     plane being the front that parents the two boxes' roots; empty boxes vanish.
// Fronts are numbered in that completion order (children before parents).  The
// update rows of front s are the later vertices adjacent to a pivot of s, joined with
// the children's update rows that lie beyond s; its dense front is (pivots, update rows)
// squared.  An edge joining two subtrees (a stencil wider than nearest neighbours)
// breaks the dissection and is rejected.
#include <algorithm>
#include <cmath>
#include <cstring>
#include "zolo_internal.h"

namespace zolo {

namespace {

struct NDBuilder {
    int nx, ny, nz, leaf_max;
    std::vector<int32_t> perm, first, npiv, parent;
    int32_t count = 0;

    void emit_box(int x0, int x1, int y0, int y1, int z0, int z1) {
        for (int z = z0; z < z1; ++z)
            for (int y = y0; y < y1; ++y)
                for (int x = x0; x < x1; ++x) perm.push_back(x + nx * (y + ny * z));
    }
    // returns the node id, or -1 for an empty box
    int rec(int b[3][2]) {
        const int ex = b[0][1] - b[0][0], ey = b[1][1] - b[1][0], ez = b[2][1] - b[2][0];
        const int64_t nv = (int64_t)ex * ey * ez;
        if (nv <= 0) return -1;
        if (nv <= leaf_max) {
            const int node = (int)first.size();
            first.push_back(count);
            emit_box(b[0][0], b[0][1], b[1][0], b[1][1], b[2][0], b[2][1]);
            npiv.push_back((int32_t)nv);
            parent.push_back(-1);
            count += (int32_t)nv;
            return node;
        }
        int ax = 0;
        const int ext[3] = {ex, ey, ez};
        for (int d = 1; d < 3; ++d)
            if (ext[d] > ext[ax]) ax = d;
        const int lo = b[ax][0], hi = b[ax][1];
        const int s = lo + (hi - lo) / 2;
        int lower[3][2], upper[3][2], sep[3][2];
        std::memcpy(lower, b, sizeof(lower));
        std::memcpy(upper, b, sizeof(upper));
        std::memcpy(sep, b, sizeof(sep));
        lower[ax][1] = s;
        upper[ax][0] = s + 1;
        sep[ax][0] = s;
        sep[ax][1] = s + 1;
        const int k0 = rec(lower);
        const int k1 = rec(upper);
        const int node = (int)first.size();
        first.push_back(count);
        const int64_t ns = (int64_t)(sep[0][1] - sep[0][0]) * (sep[1][1] - sep[1][0]) * (sep[2][1] - sep[2][0]);
        emit_box(sep[0][0], sep[0][1], sep[1][0], sep[1][1], sep[2][0], sep[2][1]);
        npiv.push_back((int32_t)ns);
        parent.push_back(-1);
        count += (int32_t)ns;
        if (k0 >= 0) parent[k0] = node;
        if (k1 >= 0) parent[k1] = node;
        return node;
    }
};

// Graph nested dissection by level structures (George & Liu) for pencils without grid
// geometry, on the union pattern of A and B (self-loops ignored).  A vertex set is split
// into its connected components (ordered by smallest vertex, sibling subtrees); a
// component of at most leaf_max vertices is a leaf front (ascending index); otherwise a
// pseudo-peripheral root is found (start at the smallest vertex; repeatedly BFS from the
// last level's vertex of smallest degree in the component, lowest index on ties, while that
// adds levels), and with the BFS levels L_0..L_{h-1} from it the middle level L_{h/2} is
// the separator front (h < 3: leaf), after the subtrees of the levels before it and of the
// levels after it.  Edges only join adjacent levels, so the two parts are disconnected.
struct GNDBuilder {
    int leaf_max = 32;
    std::vector<int64_t> aptr;           // adjacency (sorted, no self-loops)
    std::vector<int32_t> adj;
    std::vector<int32_t> perm, first, npiv, parent;
    int32_t count = 0;
    std::vector<int32_t> in_set, seen;   // stamps: membership of the current set, visits
    int32_t set_stamp = 0, seen_stamp = 0;

    void build_adjacency(const zolo_csr *A, const zolo_csr *B) {
        const int64_t n = A->n;
        aptr.assign(n + 1, 0);
        adj.clear();
        std::vector<int32_t> row;
        for (int64_t v = 0; v < n; ++v) {
            row.clear();
            for (int64_t p = A->row_ptr[v]; p < A->row_ptr[v + 1]; ++p)
                if (A->col_idx[p] != v) row.push_back(A->col_idx[p]);
            for (int64_t p = B->row_ptr[v]; p < B->row_ptr[v + 1]; ++p)
                if (B->col_idx[p] != v) row.push_back(B->col_idx[p]);
            std::sort(row.begin(), row.end());
            row.erase(std::unique(row.begin(), row.end()), row.end());
            adj.insert(adj.end(), row.begin(), row.end());
            aptr[v + 1] = (int64_t)adj.size();
        }
        in_set.assign(n, 0);
        seen.assign(n, 0);
    }
    int emit(const std::vector<int32_t> &verts) {
        const int node = (int)first.size();
        first.push_back(count);
        npiv.push_back((int32_t)verts.size());
        parent.push_back(-1);
        perm.insert(perm.end(), verts.begin(), verts.end());
        count += (int32_t)verts.size();
        return node;
    }
    // BFS levels (each sorted) of the current set from root
    void bfs(int32_t root, std::vector<std::vector<int32_t>> &levels) {
        const int32_t sv = ++seen_stamp, st = set_stamp;
        levels.assign(1, std::vector<int32_t>(1, root));
        seen[root] = sv;
        for (;;) {
            std::vector<int32_t> nxt;
            for (int32_t v : levels.back())
                for (int64_t p = aptr[v]; p < aptr[v + 1]; ++p) {
                    const int32_t u = adj[p];
                    if (in_set[u] == st && seen[u] != sv) {
                        seen[u] = sv;
                        nxt.push_back(u);
                    }
                }
            if (nxt.empty()) return;
            std::sort(nxt.begin(), nxt.end());
            levels.push_back(std::move(nxt));
        }
    }
    int degree_in_set(int32_t v) const {
        int d = 0;
        for (int64_t p = aptr[v]; p < aptr[v + 1]; ++p) d += (in_set[adj[p]] == set_stamp);
        return d;
    }
    // subtrees of a sorted vertex set, one per connected component; returns their roots
    void rec_set(const std::vector<int32_t> &verts, std::vector<int> &roots) {
        const int32_t st = ++set_stamp;
        for (int32_t v : verts) in_set[v] = st;
        const int32_t sv = ++seen_stamp;
        std::vector<std::vector<int32_t>> comps;
        std::vector<int32_t> stack;
        for (int32_t v : verts) {
            if (seen[v] == sv) continue;
            std::vector<int32_t> comp;
            seen[v] = sv;
            stack.assign(1, v);
            while (!stack.empty()) {
                const int32_t x = stack.back();
                stack.pop_back();
                comp.push_back(x);
                for (int64_t p = aptr[x]; p < aptr[x + 1]; ++p) {
                    const int32_t u = adj[p];
                    if (in_set[u] == st && seen[u] != sv) {
                        seen[u] = sv;
                        stack.push_back(u);
                    }
                }
            }
            std::sort(comp.begin(), comp.end());
            comps.push_back(std::move(comp));
        }
        for (auto &c : comps) roots.push_back(rec_connected(c));
    }
    int rec_connected(const std::vector<int32_t> &comp) {
        if ((int64_t)comp.size() <= leaf_max) return emit(comp);
        const int32_t st = ++set_stamp;
        for (int32_t v : comp) in_set[v] = st;
        std::vector<std::vector<int32_t>> levels, lv;
        bfs(comp[0], levels);
        for (;;) {
            int32_t cand = -1;
            int cd = 0;
            for (int32_t v : levels.back()) {          // ascending: the first minimum wins ties
                const int d = degree_in_set(v);
                if (cand < 0 || d < cd) {
                    cand = v;
                    cd = d;
                }
            }
            bfs(cand, lv);
            if (lv.size() > levels.size()) levels.swap(lv);
            else break;
        }
        const int h = (int)levels.size();
        if (h < 3) return emit(comp);
        const int m = h / 2;
        std::vector<int32_t> part1, part2;
        for (int L = 0; L < m; ++L) part1.insert(part1.end(), levels[L].begin(), levels[L].end());
        for (int L = m + 1; L < h; ++L) part2.insert(part2.end(), levels[L].begin(), levels[L].end());
        std::sort(part1.begin(), part1.end());
        std::sort(part2.begin(), part2.end());
        std::vector<int32_t> sep = levels[m];
        std::vector<int> kids;
        rec_set(part1, kids);
        rec_set(part2, kids);
        const int node = emit(sep);
        for (int k : kids) parent[k] = node;
        return node;
    }
};

double sum_sq(double x) { return x * (x + 1.0) * (2.0 * x + 1.0) / 6.0; }   // 0^2 + ... + x^2

}  // namespace

int check_csr(const zolo_csr *M, const char *name, bool &complex_) {
    if (!M) return set_error(ZOLO_EINVAL, std::string(name) + ": null matrix");
    if (M->n <= 0 || M->n > (int64_t)INT32_MAX - 1 || M->nnz < M->n)
        return set_error(ZOLO_EINVAL, std::string(name) + ": bad n / nnz");
    if (!M->row_ptr || !M->col_idx || !M->val) return set_error(ZOLO_EINVAL, std::string(name) + ": null array");
    if (M->dtype != ZOLO_R64 && M->dtype != ZOLO_C128) return set_error(ZOLO_EINVAL, std::string(name) + ": bad dtype");
    complex_ = (M->dtype == ZOLO_C128);
    if (M->row_ptr[0] != 0 || M->row_ptr[M->n] != M->nnz)
        return set_error(ZOLO_EINVAL, std::string(name) + ": row_ptr does not span nnz");
    for (int64_t i = 0; i < M->n; ++i) {
        const int64_t b = M->row_ptr[i], e = M->row_ptr[i + 1];
        if (e < b) return set_error(ZOLO_EINVAL, std::string(name) + ": row_ptr decreasing");
        bool diag = false;
        for (int64_t p = b; p < e; ++p) {
            const int32_t c = M->col_idx[p];
            if (c < 0 || c >= M->n) return set_error(ZOLO_EINVAL, std::string(name) + ": column index out of range");
            if (p > b && c <= M->col_idx[p - 1])
                return set_error(ZOLO_EINVAL, std::string(name) + ": columns not strictly increasing in a row");
            if (c == i) diag = true;
            const double *v = (const double *)M->val + (complex_ ? 2 * p : p);
            if (!std::isfinite(v[0]) || (complex_ && !std::isfinite(v[1])))
                return set_error(ZOLO_EINVAL, std::string(name) + ": non-finite value");
        }
        if (!diag) return set_error(ZOLO_EINVAL, std::string(name) + ": missing diagonal entry");
    }
    return ZOLO_OK;
}

int analyze(const zolo_csr *A, const zolo_csr *B, const zolo_opts &opts, zolo_symbolic_s &S) {
    const int64_t n = A->n;
    if (B->n != n) return set_error(ZOLO_EINVAL, "A and B differ in size");
    S.n = n;
    // ---- ordering
    if (opts.grid[0] > 0) {
        const int nx = opts.grid[0], ny = std::max(1, opts.grid[1]), nz = std::max(1, opts.grid[2]);
        if ((int64_t)nx * ny * nz != n) return set_error(ZOLO_EINVAL, "grid dims do not match n");
        NDBuilder nd;
        nd.nx = nx;
        nd.ny = ny;
        nd.nz = nz;
        nd.leaf_max = opts.leaf_max > 0 ? opts.leaf_max : 32;
        nd.perm.reserve(n);
        int b[3][2] = {{0, nx}, {0, ny}, {0, nz}};
        nd.rec(b);
        S.perm.swap(nd.perm);
        S.first.swap(nd.first);
        S.npiv.swap(nd.npiv);
        S.parent.swap(nd.parent);
    } else {
        GNDBuilder nd;
        nd.leaf_max = opts.leaf_max > 0 ? opts.leaf_max : 32;
        nd.build_adjacency(A, B);
        nd.perm.reserve(n);
        std::vector<int32_t> all(n);
        for (int64_t i = 0; i < n; ++i) all[i] = (int32_t)i;
        std::vector<int> roots;
        nd.rec_set(all, roots);
        S.perm.swap(nd.perm);
        S.first.swap(nd.first);
        S.npiv.swap(nd.npiv);
        S.parent.swap(nd.parent);
    }
    const int32_t nn = (int32_t)S.first.size();
    S.nnodes = nn;
    S.iperm.assign(n, 0);
    for (int64_t t = 0; t < n; ++t) S.iperm[S.perm[t]] = (int32_t)t;
    std::vector<int32_t> node_of(n);
    for (int s = 0; s < nn; ++s)
        for (int t = S.first[s]; t < S.first[s] + S.npiv[s]; ++t) node_of[t] = s;
    S.children.assign(nn, {});
    for (int s = 0; s < nn; ++s)
        if (S.parent[s] >= 0) S.children[S.parent[s]].push_back(s);
    S.lo.assign(nn, 0);
    S.level.assign(nn, 0);
    for (int s = 0; s < nn; ++s) {
        S.lo[s] = s;
        for (int c : S.children[s]) {
            S.lo[s] = std::min(S.lo[s], S.lo[c]);
            S.level[s] = std::max(S.level[s], S.level[c] + 1);
        }
    }
    // ---- update rows
    std::vector<int32_t> mark(n, -1), buf;
    S.uptr.assign(nn + 1, 0);
    S.urows.clear();
    for (int s = 0; s < nn; ++s) {
        const int32_t e = S.first[s] + S.npiv[s];
        buf.clear();
        auto add = [&](int32_t t) {
            if (t >= e && mark[t] != s) {
                mark[t] = s;
                buf.push_back(t);
            }
        };
        for (int32_t t = S.first[s]; t < e; ++t) {
            const int32_t v = S.perm[t];
            for (int64_t p = A->row_ptr[v]; p < A->row_ptr[v + 1]; ++p) add(S.iperm[A->col_idx[p]]);
            for (int64_t p = B->row_ptr[v]; p < B->row_ptr[v + 1]; ++p) add(S.iperm[B->col_idx[p]]);
        }
        for (int c : S.children[s])
            for (int64_t p = S.uptr[c]; p < S.uptr[c + 1]; ++p) add(S.urows[p]);
        std::sort(buf.begin(), buf.end());
        for (int32_t t : buf) {
            const int32_t o = node_of[t];
            if (!(S.lo[o] <= s && s < o))
                return set_error(ZOLO_EINVAL, "pattern edge crosses the nested dissection (stencil wider than "
                                              "nearest neighbours, or wrong grid dims)");
        }
        S.urows.insert(S.urows.end(), buf.begin(), buf.end());
        S.uptr[s + 1] = (int64_t)S.urows.size();
    }
    // ---- levels
    int32_t nl = 0;
    for (int s = 0; s < nn; ++s) nl = std::max(nl, S.level[s] + 1);
    S.nlevels = nl;
    S.level_ptr.assign(nl + 1, 0);
    for (int s = 0; s < nn; ++s) S.level_ptr[S.level[s] + 1]++;
    for (int L = 0; L < nl; ++L) S.level_ptr[L + 1] += S.level_ptr[L];
    S.by_level.assign(nn, 0);
    {
        std::vector<int32_t> fill(S.level_ptr.begin(), S.level_ptr.end() - 1);
        for (int s = 0; s < nn; ++s) S.by_level[fill[S.level[s]]++] = s;
    }
    // ---- info
    zolo_symbolic_info &I = S.info;
    std::memset(&I, 0, sizeof(I));
    I.n = n;
    I.nnodes = nn;
    I.nlevels = nl;
    for (int s = 0; s < nn; ++s) {
        const int64_t p = S.npiv[s], u = S.nu(s), f = p + u;
        I.nnz_factor += p * (p - 1) / 2 + p * u;
        I.front_entries += f * f;
        I.update_rows += u;
        I.max_front = std::max<int32_t>(I.max_front, (int32_t)f);
        I.max_pivots = std::max<int32_t>(I.max_pivots, (int32_t)p);
        // complex multiply-add (8 real flops) per trailing entry per pivot
        I.flops_lu += 8.0 * (sum_sq((double)f - 1.0) - sum_sq((double)(f - p) - 1.0));
    }
    return ZOLO_OK;
}

}  // namespace zolo

int32_t zolo_symbolic_s::pos_in(int s, int32_t t) const {
    if (t >= first[s] && t < first[s] + npiv[s]) return t - first[s];
    auto b = urows.begin() + uptr[s], e = urows.begin() + uptr[s + 1];
    auto it = std::lower_bound(b, e, t);
    if (it == e || *it != t) return -1;
    return npiv[s] + (int32_t)(it - b);
}

extern "C" {

int zolo_analyze(const zolo_csr *A, const zolo_csr *B, const zolo_opts *opts, zolo_symbolic *out) {
    using namespace zolo;
    clear_error();
    if (!out) return set_error(ZOLO_EINVAL, "null output");
    *out = nullptr;
    CsrHost ha, hb;
    int st = csr_host_view(A, ha, &A);
    if (!st) st = csr_host_view(B, hb, &B);
    if (st) return st;
    bool ca, cb;
    st = check_csr(A, "A", ca);
    if (st) return st;
    st = check_csr(B, "B", cb);
    if (st) return st;
    zolo_opts o;
    if (opts) o = *opts; else zolo_opts_default(&o);
    auto *S = new zolo_symbolic_s();
    st = analyze(A, B, o, *S);
    if (st) {
        delete S;
        return st;
    }
    *out = S;
    return ZOLO_OK;
}

int zolo_symbolic_get_info(zolo_symbolic s, zolo_symbolic_info *out) {
    zolo::clear_error();
    if (!s || !out) return zolo::set_error(ZOLO_EINVAL, "null argument");
    *out = s->info;
    return ZOLO_OK;
}

int zolo_symbolic_export(zolo_symbolic s, int32_t *perm, int32_t *first, int32_t *npiv, int32_t *parent,
                         int64_t *uptr, int32_t *urows) {
    zolo::clear_error();
    if (!s) return zolo::set_error(ZOLO_EINVAL, "null handle");
    if (perm) std::copy(s->perm.begin(), s->perm.end(), perm);
    if (first) std::copy(s->first.begin(), s->first.end(), first);
    if (npiv) std::copy(s->npiv.begin(), s->npiv.end(), npiv);
    if (parent) std::copy(s->parent.begin(), s->parent.end(), parent);
    if (uptr) std::copy(s->uptr.begin(), s->uptr.end(), uptr);
    if (urows) std::copy(s->urows.begin(), s->urows.end(), urows);
    return ZOLO_OK;
}

void zolo_symbolic_destroy(zolo_symbolic s) { delete s; }

}  // extern "C"
