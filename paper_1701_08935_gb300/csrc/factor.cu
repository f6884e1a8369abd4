// Multifrontal factorisation of K_j = A - sigma_hat_j B (the factorisation step of Algorithm 2) and the
// block triangular solves with K_j and K_j^H that eq. solve needs, on the device.
//
// Fronts are dense column-major (pivots, update rows)^2 blocks, stored level by level in
// one pool per pole.  A level is factored with a right-looking blocked LU without
// pivoting (panel width NB): per step, the FP64 LU of the diagonal block plus the
// explicit inverses of its triangles, then L21 = A21 U11^-1 and U12 = L11^-1 A12, then
// the Schur update A22 -= L21 U12.  After the last pivot block the lower-right block
// holds the update matrix, which the parent front adds in (extend-add) before its own
// elimination.  The solves walk the same tree: forward (L y = b, or U^H y = b) from
// the leaves, children passing their update vectors to the parent, and backward
// (U x = y, or L^H x = y) from the root, gathering the ancestors' solution rows.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include "factor.h"
#include "df64.cuh"

namespace zolo {

int cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return ZOLO_OK;
    return set_error(e == cudaErrorMemoryAllocation ? ZOLO_ENOMEM : ZOLO_ECUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
}

int dev_alloc(zolo_factor_s *h, size_t bytes, void **out) {
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(ZOLO_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    h->owned.push_back(Buf{p, bytes});
    *out = p;
    return ZOLO_OK;
}

void dev_release(zolo_factor_s *h, Buf &b) {
    if (!b.p) return;
    for (size_t i = 0; i < h->owned.size(); ++i)
        if (h->owned[i].p == b.p) {
            cudaFree(b.p);
            h->owned.erase(h->owned.begin() + i);
            break;
        }
    b = Buf();
}

static void dev_free(zolo_factor_s *h, void *p) {
    if (!p) return;
    for (size_t i = 0; i < h->owned.size(); ++i)
        if (h->owned[i].p == p) {
            cudaFree(p);
            h->owned.erase(h->owned.begin() + i);
            return;
        }
}

namespace {

template <class V> int upload(zolo_factor_s *h, const std::vector<V> &v, V **out) {
    int st = dev_alloc(h, v.size() * sizeof(V), (void **)out);
    if (st) return st;
    if (!v.empty()) return cuda_check(cudaMemcpy(*out, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice), "upload");
    return ZOLO_OK;
}

GJob make_job(int64_t a, int ars, int acs, int64_t b, int brs, int bcs, int64_t c, int crs, int ccs, int m, int n,
              int k, int flags) {
    GJob j;
    std::memset(&j, 0, sizeof(j));
    j.a = a; j.ars = ars; j.acs = acs;
    j.b = b; j.brs = brs; j.bcs = bcs;
    j.c = c; j.crs = crs; j.ccs = ccs;
    j.m = m; j.n = n; j.k = k;
    j.flags = flags;
    j.tm = (m + 63) / 64;
    j.ks = 1;
    return j;
}

// Precision of the launches being planned (complex64 launches may use 128-row tiles)
// and the tensor-core policy (zolo_opts.tensor_core) for complex64 launches.
thread_local bool g_plan_c64 = false;
thread_local int g_plan_tc = ZOLO_TC_AUTO;
// Tile -> job map of the launches being planned (appended by add_gemm when set).
thread_local std::vector<int32_t> *g_plan_tmap = nullptr;
// Smallest inner extent of an accumulating product that add_gemm may split (zolo_opts.split_k_min).
thread_local int g_plan_split_min = 512;
// Instances (grid.z) the launches being planned will run with: they share the waves.
thread_local int g_plan_ninst = 1;
// Complex64 launches whose jobs average at least this many rows go to the tensor cores.
constexpr double TC_MIN_ROWS = 128.0;

// Append a launch of GEMM jobs (empty products dropped) and return its descriptor.
// Tiles of a complex64 launch: the tensor-core kernel (128 x <= 128) when its jobs average
// >= TC_MIN_ROWS rows (every launch with ZOLO_TC_ALWAYS, none with ZOLO_TC_OFF); otherwise
// FP32-FMA tiles: 32 wide when no job has more than 32 columns (32, 64 or 128 rows by the
// average row count), else 128 x 64 when they average >= 256 rows, 32 x 128 when <= 40,
// else 64 x 64.  Complex128 launches take 64 x 64.  With allow_split, a launch with fewer than ~4 waves
// of tiles splits the kk extent of its accumulating jobs (GJ_SUB / GJ_ACC, kk >= g_plan_split_min) over
// several CTAs (atomic adds).
Launch add_gemm(std::vector<GJob> &all, const std::vector<GJob> &jobs_in, bool allow_split = false) {
    Launch L;
    L.off = (int64_t)all.size();
    double msum = 0.0;
    int cnt = 0;
    for (const GJob &j : jobs_in)
        if (j.m > 0 && j.n > 0 && j.k > 0) {
            msum += j.m;
            ++cnt;
        }
    const std::vector<GJob> &jobs = jobs_in;
    const bool big = cnt && msum / cnt >= 256.0;
    L.bm = (g_plan_c64 && big) ? 128 : 64;
    if (g_plan_c64 && cnt && msum / cnt <= 40.0) {       // few pivot rows: 32 x 128 FMA tiles
        L.bm = 32;
        L.bn = 128;
    }
    int nmax = 0;
    for (const GJob &j : jobs_in)
        if (j.m > 0 && j.n > 0 && j.k > 0) nmax = std::max(nmax, j.n);
    if (g_plan_c64 && cnt && nmax <= 32) {                // narrow blocks: 32-wide FMA tiles
        L.bn = 32;
        L.bm = msum / cnt <= 40.0 ? 32 : (msum / cnt <= 96.0 ? 64 : 128);
    }
    // narrow blocks: the tensor-core CTA's fixed cost (tensor-memory allocation, barrier set-up,
    // pipeline fill) outweighs a short inner extent, so those launches need kk >= 256 on average
    double ksum = 0.0;
    for (const GJob &j : jobs_in)
        if (j.m > 0 && j.n > 0 && j.k > 0) ksum += j.k;
    const bool tc_k_ok = nmax > 32 || (cnt && ksum / cnt >= 256.0);
    if (g_plan_c64 && cnt &&
        (g_plan_tc == ZOLO_TC_ALWAYS || (g_plan_tc == ZOLO_TC_AUTO && msum / cnt >= TC_MIN_ROWS && tc_k_ok))) {
        L.bm = 128;
        L.bn = 128;
        L.tc = true;
    }
    const int kmin = std::max(16, g_plan_split_min);
    auto splittable = [&](const GJob &j) { return (j.flags & (GJ_SUB | GJ_ACC)) && j.k >= kmin; };
    auto split_of = [&](const GJob &j, int f) {
        return splittable(j) ? std::max(1, std::min({f, j.k / (kmin / 2), 16})) : 1;
    };
    auto tiles_of = [&](const GJob &j) { return ((j.m + L.bm - 1) / L.bm) * ((j.n + L.bn - 1) / L.bn); };
    int base = 0;
    for (const GJob &j : jobs)
        if (j.m > 0 && j.n > 0 && j.k > 0) base += tiles_of(j);
    int factor = 1;
    if (allow_split && base > 0 && L.tc && base * g_plan_ninst < 8 * 152) {
        // two CTAs per SM: model the launch as waves x (k-stages of 8 of the longest slice +
        // ~8 stages of prologue and epilogue) and take the split that minimises it
        double best = 1e300;
        for (int f = 1; f <= 16; ++f) {
            int64_t t = 0;
            int stages = 0;
            for (const GJob &j : jobs)
                if (j.m > 0 && j.n > 0 && j.k > 0) {
                    const int ks = split_of(j, f);
                    t += (int64_t)tiles_of(j) * ks;
                    stages = std::max(stages, ((j.k + ks - 1) / ks + 7) / 8);
                }
            const double cost = std::ceil((double)t * g_plan_ninst / 304.0) * (stages + 8);
            if (cost < best * (1.0 - 1e-9)) {
                best = cost;
                factor = f;
            }
        }
    } else if (allow_split && base > 0 && base * g_plan_ninst < 4 * 152) {
        factor = (4 * 152 + base * g_plan_ninst - 1) / (base * g_plan_ninst);
    }
    // FMA tiles of skinny accumulating products (inner extent kk well above the row count,
    // e.g. U_pu x_u of the backward solve at deep levels) run long, latency-bound k-loops:
    // split kk into pieces of about twice the tile height however many tiles there are
    auto skinny = [&](const GJob &j) {
        return allow_split && !L.tc && (j.flags & (GJ_SUB | GJ_ACC)) && j.k >= 4 * std::max(j.m, L.bm) && j.k >= 128;
    };
    int tiles = 0;
    if (L.tc) {                            // the tile width the tensor-core kernel derives per job
        L.wmax = 16;
        for (const GJob &j : jobs)
            if (j.m > 0 && j.n > 0 && j.k > 0) {
                const int ntn = (j.n + 127) / 128;
                L.wmax = std::max(L.wmax, ((j.n + ntn - 1) / ntn + 15) / 16 * 16);
            }
    }
    for (GJob j : jobs) {
        if (j.m <= 0 || j.n <= 0 || j.k <= 0) continue;
        j.tm = (j.m + L.bm - 1) / L.bm;
        j.ks = factor > 1 ? split_of(j, factor) : 1;
        if (skinny(j)) j.ks = std::max(j.ks, std::min(16, j.k / (2 * std::max(j.m, L.bm))));
        j.tile0 = tiles;
        const int nt = j.tm * ((j.n + L.bn - 1) / L.bn) * j.ks;
        tiles += nt;
        if (g_plan_tmap) {
            if (L.tmoff < 0) L.tmoff = (int64_t)g_plan_tmap->size();
            g_plan_tmap->insert(g_plan_tmap->end(), nt, (int32_t)L.cnt);
        }
        all.push_back(j);
        L.cnt++;
        L.flops += 8.0 * j.m * j.n * j.k;
        L.bytes += (g_plan_c64 ? 8.0 : 16.0) *
                   ((double)j.m * j.k + (double)j.k * j.n + (double)j.m * j.n * ((j.flags & (GJ_SUB | GJ_ACC)) ? 2 : 1));
    }
    L.ntiles = tiles;
    return L;
}

// Append a launch of row jobs with tile_rows rows per CTA, or (square) 32 x 32 tiles of a
// job's rows x rows block per CTA (matrix extend-add).
Launch add_rows(std::vector<RJob> &all, const std::vector<RJob> &jobs, int tile_rows, bool square = false) {
    Launch L;
    L.off = (int64_t)all.size();
    int tiles = 0;
    for (RJob j : jobs) {
        if (j.rows <= 0) continue;
        j.tile0 = tiles;
        j.tr = (j.rows + tile_rows - 1) / tile_rows;
        const int nt = square ? j.tr * j.tr : j.tr;
        tiles += nt;
        if (g_plan_tmap) {                 // tile -> job map (saves each CTA a binary search)
            if (L.tmoff < 0) L.tmoff = (int64_t)g_plan_tmap->size();
            g_plan_tmap->insert(g_plan_tmap->end(), nt, (int32_t)L.cnt);
        }
        all.push_back(j);
        L.cnt++;
    }
    L.ntiles = tiles;
    return L;
}

RJob rjob(int64_t src, int64_t dst, int64_t map, int rows, int ld_src = 0, int ld_dst = 0) {
    RJob j;
    std::memset(&j, 0, sizeof(j));
    j.src = src; j.dst = dst; j.map = map; j.rows = rows; j.ld_src = ld_src; j.ld_dst = ld_dst;
    return j;
}

int check_hermitian(const zolo_csr *M, const char *name, double &norm_inf) {
    const bool c = (M->dtype == ZOLO_C128);
    const double *v = (const double *)M->val;
    double amax = 0.0;
    norm_inf = 0.0;
    for (int64_t i = 0; i < M->n; ++i) {
        double rs = 0.0;
        for (int64_t p = M->row_ptr[i]; p < M->row_ptr[i + 1]; ++p) {
            const double re = c ? v[2 * p] : v[p], im = c ? v[2 * p + 1] : 0.0;
            const double a = std::hypot(re, im);
            rs += a;
            amax = std::max(amax, a);
        }
        norm_inf = std::max(norm_inf, rs);
    }
    const double tol = 1e-12 * std::max(amax, 1e-300);
    for (int64_t i = 0; i < M->n; ++i) {
        for (int64_t p = M->row_ptr[i]; p < M->row_ptr[i + 1]; ++p) {
            const int32_t j = M->col_idx[p];
            const int32_t *b = M->col_idx + M->row_ptr[j], *e = M->col_idx + M->row_ptr[j + 1];
            const int32_t *it = std::lower_bound(b, e, (int32_t)i);
            if (it == e || *it != i) return set_error(ZOLO_ENOTHERM, std::string(name) + ": pattern not symmetric");
            const int64_t q = M->row_ptr[j] + (it - b);
            const double re1 = c ? v[2 * p] : v[p], im1 = c ? v[2 * p + 1] : 0.0;
            const double re2 = c ? v[2 * q] : v[q], im2 = c ? v[2 * q + 1] : 0.0;
            if (std::fabs(re1 - re2) > tol || std::fabs(im1 + im2) > tol)
                return set_error(ZOLO_ENOTHERM, std::string(name) + " is not Hermitian");
        }
    }
    return ZOLO_OK;
}

int upload_csr(zolo_factor_s *h, const zolo_csr *M, DevCSR &D) {
    D.n = M->n;
    D.nnz = M->nnz;
    std::vector<int64_t> rp(M->row_ptr, M->row_ptr + M->n + 1);
    std::vector<int32_t> ci(M->col_idx, M->col_idx + M->nnz);
    std::vector<c128> v(M->nnz);
    const double *src = (const double *)M->val;
    for (int64_t p = 0; p < M->nnz; ++p)
        v[p] = (M->dtype == ZOLO_C128) ? c128{src[2 * p], src[2 * p + 1]} : c128{src[p], 0.0};
    int st = upload(h, rp, &D.rp);
    if (!st) st = upload(h, ci, &D.ci);
    if (!st) st = upload(h, v, &D.v);
    bool real = true;
    for (int64_t p = 0; p < M->nnz && real; ++p) real = (v[p].im == 0.0);
    if (!st && real) {
        std::vector<double> vr(M->nnz);
        for (int64_t p = 0; p < M->nnz; ++p) vr[p] = v[p].re;
        st = upload(h, vr, &D.vr);
    }
    // double-float copies for the FP32-pipe refinement residual (mixed precision)
    if (!st && h->prec == ZOLO_PREC_MIXED) {
        if (real) {
            std::vector<float2> s2(M->nnz);
            for (int64_t p = 0; p < M->nnz; ++p) df_split(v[p].re, s2[p].x, s2[p].y);
            st = upload(h, s2, &D.vrdf);
        } else {
            std::vector<float4> s4(M->nnz);
            for (int64_t p = 0; p < M->nnz; ++p) {
                df_split(v[p].re, s4[p].x, s4[p].y);
                df_split(v[p].im, s4[p].z, s4[p].w);
            }
            st = upload(h, s4, &D.vdf);
        }
    }
    return st;
}

// Error of an expired wait inside the tensor-core GEMM since the last check (the
// stream has been synchronised by the caller).
int check_tc_status() {
    const int v = gemm_tc_status(true);
    if (v == ZOLO_ETIMEOUT) return set_error(ZOLO_ETIMEOUT, "tensor-core GEMM: an mbarrier wait expired");
    if (v) return set_error(ZOLO_ECUDA, "tensor-core GEMM status unreadable");
    return ZOLO_OK;
}

size_t elem_bytes(int prec) { return prec == ZOLO_PREC_MIXED ? sizeof(c64) : sizeof(c128); }

// ---- layout, assembly maps and the factorisation schedule
int build_factor_plan(zolo_factor_s *h, const zolo_csr *A, const zolo_csr *B) {
    const zolo_symbolic_s &S = h->sym;
    g_plan_c64 = (h->prec == ZOLO_PREC_MIXED);
    g_plan_tc = h->opts.tensor_core;
    std::vector<int32_t> ftm;
    g_plan_tmap = &ftm;
    struct ClearMap {
        ~ClearMap() { g_plan_tmap = nullptr; }
    } clear_map;
    const int nn = S.nnodes;
    h->f_off.assign(nn, 0);
    h->f_inv.assign(nn, 0);
    h->f_wrow.assign(nn, 0);
    h->f_rows.assign(nn, 0);
    h->f_rel.assign(nn, -1);
    h->f_finv.assign(nn, 0);
    int64_t po = 0, io = 0, wo = 0, fo = 0;
    std::vector<int32_t> rows;
    rows.reserve(S.n + S.urows.size());
    for (int idx = 0; idx < nn; ++idx) {
        const int s = S.by_level[idx];
        const int64_t nf = S.nf(s), np = S.npiv[s];
        h->f_off[s] = po;
        po += nf * nf;
        h->f_inv[s] = io;
        io += ((np + NB - 1) / NB) * 2 * NB * NB;
        h->f_wrow[s] = wo;
        wo += nf;
        h->f_finv[s] = fo;
        fo += 2 * np * np;
        h->f_rows[s] = (int64_t)rows.size();
        for (int64_t r = 0; r < np; ++r) rows.push_back(S.perm[S.first[s] + r]);
        for (int64_t p = S.uptr[s]; p < S.uptr[s + 1]; ++p) rows.push_back(S.perm[S.urows[p]]);
    }
    h->pool_elems = po;
    h->inv_elems = io;
    h->wrows = wo;
    h->finv_elems = fo;
    // extend-add maps: child update row -> position in the parent front
    std::vector<int32_t> rel;
    for (int c = 0; c < nn; ++c) {
        const int p = S.parent[c];
        if (p < 0 || S.nu(c) == 0) continue;
        h->f_rel[c] = (int64_t)rel.size();
        for (int64_t q = S.uptr[c]; q < S.uptr[c + 1]; ++q) {
            const int32_t pos = S.pos_in(p, S.urows[q]);
            if (pos < 0) return set_error(ZOLO_EINVAL, "internal: child update row missing from parent front");
            rel.push_back(pos);
        }
    }
    int st = upload(h, rows, &h->d_rows);
    if (!st) st = upload(h, rel, &h->d_rel);
    if (st) return st;
    // assembly maps of the original entries, grouped by level of their front
    std::vector<int32_t> node_of(S.n);
    for (int s = 0; s < nn; ++s)
        for (int t = S.first[s]; t < S.first[s] + S.npiv[s]; ++t) node_of[t] = s;
    const int nl = S.nlevels;
    h->flev.assign(nl, FLevel());
    std::vector<int64_t> asmv;
    auto build_asm = [&](const zolo_csr *M, bool isA) -> int {
        std::vector<std::vector<std::pair<int64_t, int64_t>>> per(nl);
        for (int64_t i = 0; i < M->n; ++i) {
            for (int64_t p = M->row_ptr[i]; p < M->row_ptr[i + 1]; ++p) {
                const int32_t pi = S.iperm[i], pj = S.iperm[M->col_idx[p]];
                const int s = node_of[std::min(pi, pj)];
                const int32_t r = S.pos_in(s, pi), c = S.pos_in(s, pj);
                if (r < 0 || c < 0) return set_error(ZOLO_EINVAL, "internal: entry outside its front");
                per[S.level[s]].push_back({p, h->f_off[s] + r + (int64_t)c * S.nf(s)});
            }
        }
        const int64_t base = (int64_t)asmv.size();
        std::vector<int64_t> src, dst;
        for (int L = 0; L < nl; ++L) {
            (isA ? h->flev[L].asmA_lo : h->flev[L].asmB_lo) = (int64_t)src.size();
            for (auto &e : per[L]) {
                src.push_back(e.first);
                dst.push_back(e.second);
            }
            (isA ? h->flev[L].asmA_hi : h->flev[L].asmB_hi) = (int64_t)src.size();
        }
        (isA ? h->nA_asm : h->nB_asm) = (int64_t)src.size();
        asmv.insert(asmv.end(), src.begin(), src.end());
        asmv.insert(asmv.end(), dst.begin(), dst.end());
        (void)base;
        return ZOLO_OK;
    };
    st = build_asm(A, true);
    if (!st) st = build_asm(B, false);
    if (!st) st = upload(h, asmv, &h->d_asm);
    if (st) return st;
    // schedule
    std::vector<DJob> dj;
    std::vector<GJob> gj;
    std::vector<RJob> ej;
    for (int L = 0; L < nl; ++L) {
        FLevel &F = h->flev[L];
        const int b = S.level_ptr[L], e = S.level_ptr[L + 1];
        const int s0 = S.by_level[b], s1 = S.by_level[e - 1];
        F.pool_lo = h->f_off[s0];
        F.pool_hi = h->f_off[s1] + (int64_t)S.nf(s1) * S.nf(s1);
        // extend-add, one launch per child slot (fronts of one launch have distinct parents)
        size_t maxkids = 0;
        for (int i = b; i < e; ++i) maxkids = std::max(maxkids, S.children[S.by_level[i]].size());
        for (size_t slot = 0; slot < maxkids; ++slot) {
            std::vector<RJob> jobs;
            for (int i = b; i < e; ++i) {
                const int p = S.by_level[i];
                if (slot >= S.children[p].size()) continue;
                const int c = S.children[p][slot];
                const int nu = S.nu(c), np = S.npiv[c], nf = S.nf(c);
                if (nu == 0) continue;
                jobs.push_back(rjob(h->f_off[c] + np + (int64_t)np * nf, h->f_off[p], h->f_rel[c], nu, nf, S.nf(p)));
            }
            F.eadd.push_back(add_rows(ej, jobs, 32, true));
        }
        int maxnp = 0;
        for (int i = b; i < e; ++i) maxnp = std::max(maxnp, S.npiv[S.by_level[i]]);
        for (int t = 0; t * NB < maxnp; ++t) {
            FStep stp;
            std::vector<DJob> dd;
            std::vector<GJob> pL, pU, sc;
            const int kb = t * NB;
            for (int i = b; i < e; ++i) {
                const int s = S.by_level[i];
                const int np = S.npiv[s], nf = S.nf(s);
                if (np <= kb) continue;
                const int nb = std::min(NB, np - kb);
                const int64_t o = h->f_off[s];
                const int64_t iv = h->f_inv[s] + (int64_t)t * 2 * NB * NB;
                DJob d;
                std::memset(&d, 0, sizeof(d));
                d.off = o + kb + (int64_t)kb * nf;
                d.inv = iv;
                d.ld = nf;
                d.nb = nb;
                d.front = s;
                dd.push_back(d);
                const int rest = nf - kb - nb;
                // L21 = A21 Uinv   (A: pool, B: inverse store, C aliases A; n = nb <= BN)
                pL.push_back(make_job(o + kb + nb + (int64_t)kb * nf, 1, nf, iv + NB * NB, 1, NB,
                                      o + kb + nb + (int64_t)kb * nf, 1, nf, rest, nb, nb, 0));
                // U12 = Linv A12   (A: inverse store, B: pool, C aliases B; m = nb <= BM)
                pU.push_back(make_job(iv, 1, NB, o + kb + (int64_t)(kb + nb) * nf, 1, nf,
                                      o + kb + (int64_t)(kb + nb) * nf, 1, nf, nb, rest, nb, 0));
                // A22 -= L21 U12
                sc.push_back(make_job(o + kb + nb + (int64_t)kb * nf, 1, nf, o + kb + (int64_t)(kb + nb) * nf, 1, nf,
                                      o + kb + nb + (int64_t)(kb + nb) * nf, 1, nf, rest, rest, nb, GJ_SUB));
            }
            stp.diag.off = (int64_t)dj.size();
            stp.diag.cnt = (int)dd.size();
            stp.diag.ntiles = (int)dd.size();
            dj.insert(dj.end(), dd.begin(), dd.end());
            stp.panelL = add_gemm(gj, pL);
            stp.panelU = add_gemm(gj, pU);
            stp.schur = add_gemm(gj, sc);
            F.steps.push_back(stp);
        }
        // explicit pivot-block inverses L_pp^-1 and U_pp^-1 (formed row-major np x np), computed by
        // blocked substitution against the identity with the diagonal-block inverses
        F.finv_lo = h->f_finv[s0];
        F.finv_hi = h->f_finv[s1] + 2 * (int64_t)S.npiv[s1] * S.npiv[s1];
        {
            std::vector<RJob> ey;
            for (int i = b; i < e; ++i) {
                const int s = S.by_level[i];
                ey.push_back(rjob(0, h->f_finv[s], 0, S.npiv[s]));
            }
            F.eye = add_rows(ej, ey, 256);
            // then transposed in place to column-major, so that the block solves stream them
            // as contiguous columns (K^-1 and K^-H both)
            Launch tp;
            tp.off = (int64_t)ej.size();
            int tiles = 0;
            for (int i = b; i < e; ++i) {
                const int sn = S.by_level[i];
                const int np = S.npiv[sn];
                if (np <= 0) continue;
                for (int half = 0; half < 2; ++half) {
                    RJob j = rjob(0, h->f_finv[sn] + (int64_t)half * np * np, 0, np);
                    j.tr = (np + 31) / 32;
                    j.tile0 = tiles;
                    const int nt = j.tr * (j.tr + 1) / 2;
                    tiles += nt;
                    if (tp.tmoff < 0) tp.tmoff = (int64_t)ftm.size();
                    ftm.insert(ftm.end(), nt, (int32_t)tp.cnt);
                    ej.push_back(j);
                    tp.cnt++;
                }
            }
            tp.ntiles = tiles;
            F.tpose = tp;
        }
        for (int t = 0; t * NB < maxnp; ++t) {                      // L: forward, rows below
            std::vector<GJob> ap, up;
            const int kb = t * NB;
            for (int i = b; i < e; ++i) {
                const int s = S.by_level[i];
                const int np = S.npiv[s], nf = S.nf(s);
                if (np <= kb) continue;
                const int nb = std::min(NB, np - kb);
                const int64_t X = h->f_finv[s], iv = h->f_inv[s] + (int64_t)t * 2 * NB * NB, o = h->f_off[s];
                ap.push_back(make_job(iv, 1, NB, X + (int64_t)kb * np, np, 1, X + (int64_t)kb * np, np, 1, nb, kb + nb,
                                      nb, 0));
                up.push_back(make_job(o + kb + nb + (int64_t)kb * nf, 1, nf, X + (int64_t)kb * np, np, 1,
                                      X + (int64_t)(kb + nb) * np, np, 1, np - kb - nb, kb + nb, nb, GJ_SUB));
            }
            F.linv.push_back(add_gemm(gj, ap));
            F.linv.push_back(add_gemm(gj, up));
        }
        const int maxblk = (maxnp + NB - 1) / NB;
        for (int t = 0; t < maxblk; ++t) {                           // U: backward, rows above
            std::vector<GJob> ap, up;
            for (int i = b; i < e; ++i) {
                const int s = S.by_level[i];
                const int np = S.npiv[s], nf = S.nf(s);
                const int nblk = (np + NB - 1) / NB;
                if (nblk <= t) continue;
                const int bi = nblk - 1 - t, kb = bi * NB, nb = std::min(NB, np - kb);
                const int64_t X = h->f_finv[s] + (int64_t)np * np;
                const int64_t iv = h->f_inv[s] + (int64_t)bi * 2 * NB * NB + NB * NB, o = h->f_off[s];
                ap.push_back(make_job(iv, 1, NB, X + (int64_t)kb * np + kb, np, 1, X + (int64_t)kb * np + kb, np, 1, nb,
                                      np - kb, nb, 0));
                up.push_back(make_job(o + (int64_t)kb * nf, 1, nf, X + (int64_t)kb * np + kb, np, 1, X + kb, np, 1, kb,
                                      np - kb, nb, GJ_SUB));
            }
            F.uinv.push_back(add_gemm(gj, ap));
            F.uinv.push_back(add_gemm(gj, up));
        }
    }
    st = upload(h, dj, &h->d_djobs);
    if (!st) st = upload(h, gj, &h->d_fjobs);
    if (!st) st = upload(h, ftm, &h->d_ftmap);
    if (!st) st = upload(h, ej, &h->d_ejobs);
    h->n_djobs = (int64_t)dj.size();
    if (!st) st = dev_alloc(h, std::max<int64_t>(1, h->n_djobs) * h->r1 * sizeof(double), (void **)&h->d_minpiv);
    if (!st) st = dev_alloc(h, sizeof(int), (void **)&h->d_err);
    return st;
}

template <class T> int run_factor(zolo_factor_s *h, cudaStream_t st) {
    const int np_ = h->r1;
    const size_t eb = sizeof(cx<T>);
    int rc = cuda_check(cudaMemsetAsync(h->d_err, 0, sizeof(int), st), "memset err");
    if (!rc && h->count_neg) rc = cuda_check(cudaMemsetAsync(h->d_negcnt, 0, h->r1 * sizeof(int), st), "memset neg");
    if (rc) return rc;
    const int64_t *asrcA = h->d_asm, *adstA = h->d_asm + h->nA_asm;
    const int64_t *asrcB = h->d_asm + 2 * h->nA_asm, *adstB = asrcB + h->nB_asm;
    for (int p0 = 0; p0 < np_; p0 += MAX_INST) {
        const int ni = std::min(MAX_INST, np_ - p0);
        cx<T> *pool[MAX_INST], *inv[MAX_INST], *finv[MAX_INST];
        for (int z = 0; z < ni; ++z) {
            pool[z] = (cx<T> *)h->pool[p0 + z];
            inv[z] = (cx<T> *)h->inv[p0 + z];
            finv[z] = (cx<T> *)h->finv[p0 + z];
        }
        for (const FLevel &F : h->flev) {
            for (int z = 0; z < ni; ++z) {
                rc = cuda_check(cudaMemsetAsync(pool[z] + F.pool_lo, 0, (F.pool_hi - F.pool_lo) * eb, st), "memset front");
                if (rc) return rc;
            }
            AsmArgs<T> aa;
            std::memset(&aa, 0, sizeof(aa));
            for (int z = 0; z < ni; ++z) aa.pool[z] = pool[z];
            aa.val = h->A.v;
            aa.src = asrcA + F.asmA_lo;
            aa.dst = adstA + F.asmA_lo;
            aa.count = F.asmA_hi - F.asmA_lo;
            for (int z = 0; z < ni; ++z) aa.scale[z] = c128{1.0, 0.0};
            launch_assemble<T>(aa, ni, st);
            aa.val = h->B.v;
            aa.src = asrcB + F.asmB_lo;
            aa.dst = adstB + F.asmB_lo;
            aa.count = F.asmB_hi - F.asmB_lo;
            for (int z = 0; z < ni; ++z)
                aa.scale[z] = c128{-h->fi.sigma_hat[2 * (p0 + z)], -h->fi.sigma_hat[2 * (p0 + z) + 1]};
            launch_assemble<T>(aa, ni, st);
            for (const Launch &E : F.eadd) {
                EaddArgs<T> ea;
                std::memset(&ea, 0, sizeof(ea));
                ea.jobs = h->d_ejobs + E.off;
                ea.tmap = E.tmoff >= 0 ? h->d_ftmap + E.tmoff : nullptr;
                ea.njobs = E.cnt;
                ea.ntiles = E.ntiles;
                ea.rel = h->d_rel;
                for (int z = 0; z < ni; ++z) ea.pool[z] = pool[z];
                launch_extend_add<T>(ea, ni, st);
            }
            for (const FStep &S : F.steps) {
                DiagArgs<T> da;
                std::memset(&da, 0, sizeof(da));
                da.jobs = h->d_djobs + S.diag.off;
                da.njobs = S.diag.cnt;
                da.err = h->d_err;
                da.minpiv = h->d_minpiv + S.diag.off * np_ + (int64_t)p0 * S.diag.cnt;
                da.negcnt = h->count_neg ? h->d_negcnt + p0 : nullptr;
                for (int z = 0; z < ni; ++z) {
                    da.pool[z] = pool[z];
                    da.inv[z] = inv[z];
                }
                launch_diag_lu<T>(da, ni, st);
                auto gemm = [&](const Launch &L, int abase, int bbase) {
                    if (!L.cnt) return;
                    GemmArgs<T> g;
                    std::memset(&g, 0, sizeof(g));
                    g.bm = L.bm;
                    g.bn = L.bn;
                    g.wmax = L.wmax;
                    g.real = h->real_fac ? 1 : 0;
                    for (int z = 0; z < ni; ++z) {
                        g.jobs[z] = h->d_fjobs + L.off;
                        g.tmap[z] = L.tmoff >= 0 ? h->d_ftmap + L.tmoff : nullptr;
                        g.njobs[z] = L.cnt;
                        g.ntiles[z] = L.ntiles;
                        g.A[z] = abase ? inv[z] : pool[z];
                        g.B[z] = bbase ? inv[z] : pool[z];
                        g.C[z] = pool[z];
                    }
                    launch_gemm<T>(g, ni, st, L.flops * ni, L.bytes * ni);
                };
                gemm(S.panelL, 0, 1);   // L21 = A21 Uinv
                gemm(S.panelU, 1, 0);   // U12 = Linv A12
                gemm(S.schur, 0, 0);    // A22 -= L21 U12
            }
            // pivot-block inverses of this level's fronts (the solves use them; an inertia
            // count needs the pivots only)
            if (h->count_neg) continue;
            for (int z = 0; z < ni; ++z) {
                rc = cuda_check(cudaMemsetAsync(finv[z] + F.finv_lo, 0, (F.finv_hi - F.finv_lo) * eb, st), "memset inv");
                if (rc) return rc;
            }
            EyeArgs<T> ey;
            std::memset(&ey, 0, sizeof(ey));
            ey.jobs = h->d_ejobs + F.eye.off;
            ey.tmap = F.eye.tmoff >= 0 ? h->d_ftmap + F.eye.tmoff : nullptr;
            ey.njobs = F.eye.cnt;
            ey.ntiles = F.eye.ntiles;
            for (int z = 0; z < ni; ++z) ey.P[z] = finv[z];
            launch_eye<T>(ey, ni, st);
            auto igemm = [&](const Launch &L, bool a_pool) {
                if (!L.cnt) return;
                GemmArgs<T> g;
                std::memset(&g, 0, sizeof(g));
                g.bm = L.bm;
                g.bn = L.bn;
                g.wmax = L.wmax;
                for (int z = 0; z < ni; ++z) {
                    g.jobs[z] = h->d_fjobs + L.off;
                    g.tmap[z] = L.tmoff >= 0 ? h->d_ftmap + L.tmoff : nullptr;
                    g.njobs[z] = L.cnt;
                    g.ntiles[z] = L.ntiles;
                    g.A[z] = a_pool ? pool[z] : inv[z];
                    g.B[z] = finv[z];
                    g.C[z] = finv[z];
                }
                launch_gemm<T>(g, ni, st, L.flops * ni, L.bytes * ni);
            };
            for (size_t q = 0; q + 1 < F.linv.size(); q += 2) {
                igemm(F.linv[q], false);
                igemm(F.linv[q + 1], true);
            }
            for (size_t q = 0; q + 1 < F.uinv.size(); q += 2) {
                igemm(F.uinv[q], false);
                igemm(F.uinv[q + 1], true);
            }
            EyeArgs<T> tp;                                  // row-major -> column-major
            std::memset(&tp, 0, sizeof(tp));
            tp.jobs = h->d_ejobs + F.tpose.off;
            tp.tmap = F.tpose.tmoff >= 0 ? h->d_ftmap + F.tpose.tmoff : nullptr;
            tp.njobs = F.tpose.cnt;
            tp.ntiles = F.tpose.ntiles;
            for (int z = 0; z < ni; ++z) tp.P[z] = finv[z];
            launch_transpose_sq<T>(tp, ni, st);
        }
    }
    return cuda_check(cudaGetLastError(), "factor launch");
}

}  // namespace

// Pre-split solve operands (mixed precision): L_pp^-1, U_pp^-1, L_up and U_pu of every front
// whose operand has >= 128 rows and an inner extent >= 64 -- the products the tensor-core
// kernel takes -- get a copy as TF32 planes (16 bytes per element against 8, see PJob).  The
// copies are optional: when they would take more than half of the free device memory, or the
// allocation fails, the solves convert A on the fly as before.
static int setup_presplit(zolo_factor_s *h) {
    const zolo_symbolic_s &S = h->sym;
    const int nn = S.nnodes;
    h->f_ps.assign(4 * (size_t)nn, -1);
    std::vector<PJob> pj;
    int64_t fl = 0, blk = 0;
    auto add = [&](int s, int kind, int64_t a, int acs, int m, int k, int base) {
        if (m < 128 || k < 64) return;
        PJob j;
        std::memset(&j, 0, sizeof(j));
        j.a = a;
        j.ps = fl;
        j.blk0 = blk;
        j.acs = acs;
        j.m = m;
        j.k = k;
        j.base = base;
        const int64_t nb = (int64_t)((m + 127) / 128) * ((k + 7) / 8);
        h->f_ps[4 * (size_t)s + kind] = fl;
        fl += nb * 4096;
        blk += nb;
        pj.push_back(j);
    };
    for (int s = 0; s < nn; ++s) {
        const int np = S.npiv[s], nu = S.nu(s), nf = S.nf(s);
        const int64_t X = h->f_finv[s], o = h->f_off[s];
        add(s, 0, X, np, np, np, 1);                            // L_pp^-1 (column-major)
        add(s, 1, X + (int64_t)np * np, np, np, np, 1);         // U_pp^-1
        add(s, 2, o + np, nf, nu, np, 0);                       // L_up
        add(s, 3, o + (int64_t)np * nf, nf, np, nu, 0);         // U_pu
    }
    auto disable = [&]() {
        h->f_ps.assign(4 * (size_t)nn, -1);
        h->n_psjobs = 0;
        h->ps_floats = h->ps_blocks = 0;
    };
    if (pj.empty()) {
        disable();
        return ZOLO_OK;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        disable();
        return ZOLO_OK;
    }
    const double need = (double)fl * 4.0 * h->r1 + (double)pj.size() * sizeof(PJob);
    if (need > 0.5 * (double)free_b || blk > 0x7fffffffLL) {
        disable();
        return ZOLO_OK;
    }
    for (int j = 0; j < h->r1; ++j) {
        if (dev_alloc(h, (size_t)fl * sizeof(float), &h->presplit[j])) {
            for (int q = 0; q < j; ++q) {
                dev_free(h, h->presplit[q]);
                h->presplit[q] = nullptr;
            }
            clear_error();
            disable();
            return ZOLO_OK;
        }
    }
    int rc = dev_alloc(h, pj.size() * sizeof(PJob), (void **)&h->d_psjobs);
    if (!rc) rc = cuda_check(cudaMemcpy(h->d_psjobs, pj.data(), pj.size() * sizeof(PJob), cudaMemcpyHostToDevice),
                             "presplit jobs");
    if (rc) return rc;
    h->n_psjobs = (int)pj.size();
    h->ps_floats = fl;
    h->ps_blocks = blk;
    return ZOLO_OK;
}

// the pre-split planes of the current factors (after every factorisation)
static void build_presplit(zolo_factor_s *h, cudaStream_t st) {
    if (h->n_psjobs == 0) return;
    for (int p0 = 0; p0 < h->r1; p0 += MAX_INST) {
        const int ni = std::min(MAX_INST, h->r1 - p0);
        PresplitArgs a;
        std::memset(&a, 0, sizeof(a));
        a.jobs = h->d_psjobs;
        a.njobs = h->n_psjobs;
        for (int z = 0; z < ni; ++z) {
            a.pool[z] = (const c64 *)h->pool[p0 + z];
            a.finv[z] = (const c64 *)h->finv[p0 + z];
            a.out[z] = (float *)h->presplit[p0 + z];
        }
        launch_presplit(a, h->ps_blocks, ni, st);
    }
}

int factor_numeric(zolo_factor_s *h, cudaStream_t st) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    h->stats.solve_cols = 0;                       // per-factorisation counters
    h->stats.n_refine_max = 0;
    int rc = (h->prec == ZOLO_PREC_MIXED) ? run_factor<float>(h, st) : run_factor<double>(h, st);
    if (!rc && h->prec == ZOLO_PREC_MIXED) build_presplit(h, st);
    cudaEventRecord(e1, st);
    if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "factor");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    h->stats.t_factor_ms = ms;
    int err = 0;
    rc = cuda_check(cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost), "err copy");
    if (rc) return rc;
    std::vector<double> mp(std::max<int64_t>(1, h->n_djobs) * h->r1);
    rc = cuda_check(cudaMemcpy(mp.data(), h->d_minpiv, mp.size() * sizeof(double), cudaMemcpyDeviceToHost), "minpiv");
    if (rc) return rc;
    double m = 1e300;
    for (int64_t i = 0; i < h->n_djobs * h->r1; ++i) m = std::min(m, mp[i]);
    h->stats.min_pivot = m;
    if (err) return set_error(ZOLO_ESINGULAR, "zero or non-finite pivot in a front");
    return check_tc_status();
}

// a non-Hermitian solve job of front s whose operand `kind` (PJob order) is pre-split
static GJob presplit_job(const zolo_factor_s *h, int s, int kind, GJob j) {
    const size_t i = 4 * (size_t)s + kind;
    if (i < h->f_ps.size() && h->f_ps[i] >= 0) {
        j.flags |= GJ_PRESPLIT;
        j.ps = h->f_ps[i];
    }
    return j;
}

// ---- solve schedule for a block width k
int ensure_solve_schedule(zolo_factor_s *h, int64_t k) {
    if (h->k_sched == k) return ZOLO_OK;
    const zolo_symbolic_s &S = h->sym;
    g_plan_c64 = (h->prec == ZOLO_PREC_MIXED);
    g_plan_tc = h->opts.tensor_core;
    g_plan_split_min = h->opts.split_k_min > 0 ? h->opts.split_k_min : 512;
    // a real pencil's real blocks run one instance per pole, otherwise K^-1 and K^-H per pole
    g_plan_ninst = std::min(MAX_INST, (pencil_is_real(h) && h->opts.real_block) ? h->r1 : 2 * h->r1);
    struct ResetNinst {
        ~ResetNinst() { g_plan_ninst = 1; }
    } reset_ninst;
    std::vector<int32_t> stm;
    g_plan_tmap = &stm;
    struct ClearMap {
        ~ClearMap() { g_plan_tmap = nullptr; }
    } clear_map;
    std::vector<GJob> gj;
    std::vector<RJob> rj;
    h->fwd.clear();
    h->bwd.clear();
    const int K = (int)k;
    const int nl = S.nlevels;
    auto gemm_op = [&](std::vector<GJob> &n, std::vector<GJob> &hh, int ab, int bb, int cb) {
        SOp o;
        o.kind = SOP_GEMM;
        o.abase = ab;
        o.bbase = bb;
        o.cbase = cb;
        o.L = add_gemm(gj, n, true);
        o.LH = add_gemm(gj, hh, true);
        return o;
    };
    // Per front s (np pivots, nu update rows, W_s = its nf x k workspace rows, Y_s = its np
    // rows of the pivot-row block, Linv/Uinv = explicit pivot-block inverses):
    //   forward  K:   Y_s = Linv W_p,         W_u -= L_up Y_s         (children add W_u upwards)
    //            K^H: Y_s = Uinv^H W_p,       W_u -= U_pu^H Y_s
    //   backward K:   Y_s -= U_pu x_u,        x_p = Uinv Y_s
    //            K^H: Y_s -= L_up^H x_u,      x_p = Linv^H Y_s
    for (int L = 0; L < nl; ++L) {                 // forward: leaves to root
        const int b = S.level_ptr[L], e = S.level_ptr[L + 1];
        std::vector<RJob> g;
        for (int i = b; i < e; ++i) {
            const int s = S.by_level[i];
            g.push_back(rjob(0, h->f_wrow[s] * k, h->f_rows[s], S.npiv[s]));
        }
        SOp og;
        og.kind = SOP_GATHER_IN;
        og.L = add_rows(rj, g, rows_per_tile(k));
        h->fwd.push_back(og);
        size_t maxkids = 0;
        for (int i = b; i < e; ++i) maxkids = std::max(maxkids, S.children[S.by_level[i]].size());
        for (size_t slot = 0; slot < maxkids; ++slot) {
            std::vector<RJob> ea;
            for (int i = b; i < e; ++i) {
                const int p = S.by_level[i];
                if (slot >= S.children[p].size()) continue;
                const int c = S.children[p][slot];
                if (S.nu(c) == 0) continue;
                ea.push_back(rjob((h->f_wrow[c] + S.npiv[c]) * k, h->f_wrow[p] * k, h->f_rel[c], S.nu(c)));
            }
            SOp oe;
            oe.kind = SOP_EADD;
            oe.L = add_rows(rj, ea, rows_per_tile(k));
            h->fwd.push_back(oe);
        }
        std::vector<GJob> yN, yH, uN, uH;
        for (int i = b; i < e; ++i) {
            const int s = S.by_level[i];
            const int np = S.npiv[s], nu = S.nu(s), nf = S.nf(s);
            const int64_t X = h->f_finv[s], o = h->f_off[s];
            const int64_t wp = h->f_wrow[s] * k, wu = (h->f_wrow[s] + np) * k, y = (int64_t)S.first[s] * k;
            // Y starts zeroed (the whole pivot-row block is cleared per solve): accumulate
            // Linv and Uinv are stored column-major (transposed in place after they are formed)
            yN.push_back(presplit_job(h, s, 0, make_job(X, 1, np, wp, K, 1, y, K, 1, np, K, np, GJ_ACC)));  // Linv
            yH.push_back(make_job(X + (int64_t)np * np, np, 1, wp, K, 1, y, K, 1, np, K, np,
                                  GJ_ACC | GJ_CONJA));                                                   // Uinv^H
            uN.push_back(presplit_job(h, s, 2, make_job(o + np, 1, nf, y, K, 1, wu, K, 1, nu, K, np, GJ_SUB)));  // L_up
            uH.push_back(make_job(o + (int64_t)np * nf, nf, 1, y, K, 1, wu, K, 1, nu, K, np, GJ_SUB | GJ_CONJA));
        }
        h->fwd.push_back(gemm_op(yN, yH, BK_INVFULL, BK_W, BK_YP));
        h->fwd.push_back(gemm_op(uN, uH, BK_POOL, BK_YP, BK_W));
    }
    for (int L = nl - 1; L >= 0; --L) {           // backward: root to leaves
        const int b = S.level_ptr[L], e = S.level_ptr[L + 1];
        std::vector<RJob> g, sc, zr;
        std::vector<GJob> aN, aH, xN, xH;
        for (int i = b; i < e; ++i) {
            const int s = S.by_level[i];
            const int np = S.npiv[s], nu = S.nu(s), nf = S.nf(s);
            const int64_t X = h->f_finv[s], o = h->f_off[s];
            const int64_t wp = h->f_wrow[s] * k, wu = (h->f_wrow[s] + np) * k, y = (int64_t)S.first[s] * k;
            if (nu > 0) g.push_back(rjob(0, wu, h->f_rows[s] + np, nu));
            aN.push_back(presplit_job(h, s, 3, make_job(o + (int64_t)np * nf, 1, nf, wu, K, 1, y, K, 1, np, K, nu,
                                                        GJ_SUB)));                                        // U_pu
            aH.push_back(make_job(o + np, nf, 1, wu, K, 1, y, K, 1, np, K, nu, GJ_SUB | GJ_CONJA));      // L_up^H
            // W_p is cleared first (ROW_ZERO), then accumulated into
            xN.push_back(presplit_job(h, s, 1, make_job(X + (int64_t)np * np, 1, np, y, K, 1, wp, K, 1, np, K, np,
                                                        GJ_ACC)));                                        // Uinv
            xH.push_back(make_job(X, np, 1, y, K, 1, wp, K, 1, np, K, np, GJ_ACC | GJ_CONJA));           // Linv^H
            sc.push_back(rjob(wp, 0, h->f_rows[s], np));
            zr.push_back(rjob(0, wp, 0, np));
        }
        SOp og;
        og.kind = SOP_GATHER_OUT;
        og.L = add_rows(rj, g, rows_per_tile(k));
        h->bwd.push_back(og);
        h->bwd.push_back(gemm_op(aN, aH, BK_POOL, BK_W, BK_YP));
        SOp oz;
        oz.kind = SOP_ZERO;
        oz.L = add_rows(rj, zr, rows_per_tile(k));
        h->bwd.push_back(oz);
        h->bwd.push_back(gemm_op(xN, xH, BK_INVFULL, BK_YP, BK_W));
        SOp os;
        os.kind = SOP_SCATTER_OUT;
        os.L = add_rows(rj, sc, rows_per_tile(k));
        h->bwd.push_back(os);
    }
    // device copies: [GJob... | RJob...]
    if (h->sched_buf.p) {
        dev_free(h, h->sched_buf.p);
        h->sched_buf = Buf();
    }
    const size_t gb = gj.size() * sizeof(GJob), rb = rj.size() * sizeof(RJob), tb = stm.size() * sizeof(int32_t);
    void *p = nullptr;
    int rc = dev_alloc(h, gb + rb + tb + 16, &p);
    if (rc) return rc;
    h->sched_buf = Buf{p, gb + rb + tb + 16};
    h->d_sjobs = (GJob *)p;
    h->d_rjobs = (RJob *)((char *)p + gb);
    h->d_stmap = (int32_t *)((char *)p + gb + rb);
    if (gb) rc = cuda_check(cudaMemcpy(h->d_sjobs, gj.data(), gb, cudaMemcpyHostToDevice), "sched");
    if (!rc && rb) rc = cuda_check(cudaMemcpy(h->d_rjobs, rj.data(), rb, cudaMemcpyHostToDevice), "sched");
    if (!rc && tb) rc = cuda_check(cudaMemcpy(h->d_stmap, stm.data(), tb, cudaMemcpyHostToDevice), "sched");
    if (rc) return rc;
    // workspaces: one front workspace and one pivot-row block per batched instance used
    if (h->w_buf.p) {
        dev_free(h, h->w_buf.p);
        h->w_buf = Buf();
    }
    const int ninst = std::min(MAX_INST, 2 * h->r1);
    const size_t per = (size_t)h->wrows * k * elem_bytes(h->prec);
    const size_t pery = (size_t)h->n * k * elem_bytes(h->prec);
    rc = dev_alloc(h, (per + pery) * ninst, &p);
    if (rc) return rc;
    h->w_buf = Buf{p, (per + pery) * ninst};
    for (int z = 0; z < MAX_INST; ++z) {
        h->W[z] = z < ninst ? (char *)p + z * per : nullptr;
        h->Yp[z] = z < ninst ? (char *)p + ninst * per + z * pery : nullptr;
    }
    h->k_sched = k;
    return ZOLO_OK;
}

namespace {

template <class T>
int run_solve(zolo_factor_s *h, int ninst, const int *pole, const int *herm, int64_t k, const c128 *const *Xin,
              int64_t ldin, c128 *const *Xout, int64_t ldout, cudaStream_t st) {
    const size_t per = (size_t)h->wrows * k * sizeof(cx<T>);
    const size_t pery = (size_t)h->n * k * sizeof(cx<T>);
    for (int z = 0; z < ninst; ++z) {
        int rc = cuda_check(cudaMemsetAsync(h->W[z], 0, per, st), "memset W");
        if (!rc) rc = cuda_check(cudaMemsetAsync(h->Yp[z], 0, pery, st), "memset Y");
        if (rc) return rc;
    }
    auto run = [&](const std::vector<SOp> &ops) {
        for (const SOp &o : ops) {
            if (o.kind == SOP_GEMM) {
                GemmArgs<T> g;
                std::memset(&g, 0, sizeof(g));
                double fl = 0.0;
                g.bm = o.L.bm;
                g.bn = o.L.bn;
                g.wmax = std::max(o.L.wmax, o.LH.wmax);
                auto base = [&](int kind, int z) -> cx<T> * {
                    switch (kind) {
                        case BK_POOL: return (cx<T> *)h->pool[pole[z]];
                        case BK_INVBLK: return (cx<T> *)h->inv[pole[z]];
                        case BK_INVFULL: return (cx<T> *)h->finv[pole[z]];
                        case BK_YP: return (cx<T> *)h->Yp[z];
                        default: return (cx<T> *)h->W[z];
                    }
                };
                double by = 0.0;
                for (int z = 0; z < ninst; ++z) {
                    const Launch &L = herm[z] ? o.LH : o.L;
                    by += L.bytes;
                    g.jobs[z] = h->d_sjobs + L.off;
                    g.tmap[z] = L.tmoff >= 0 ? h->d_stmap + L.tmoff : nullptr;
                    g.njobs[z] = L.cnt;
                    g.ntiles[z] = L.ntiles;
                    g.A[z] = base(o.abase, z);
                    g.B[z] = base(o.bbase, z);
                    g.C[z] = base(o.cbase, z);
                    g.ps[z] = (const float *)h->presplit[pole[z]];
                    fl += L.flops;
                }
                launch_gemm<T>(g, ninst, st, fl, by);
            } else {
                RowArgs<T> r;
                std::memset(&r, 0, sizeof(r));
                r.jobs = h->d_rjobs + o.L.off;
                r.tmap = o.L.tmoff >= 0 ? h->d_stmap + o.L.tmoff : nullptr;
                r.njobs = o.L.cnt;
                r.ntiles = o.L.ntiles;
                r.map = (o.kind == SOP_EADD) ? h->d_rel : h->d_rows;
                r.k = (int)k;
                r.rpt = rows_per_tile(k);
                r.ldw = k;
                r.mode = (o.kind == SOP_EADD) ? ROW_EADD
                         : (o.kind == SOP_SCATTER_OUT ? ROW_SCATTER : (o.kind == SOP_ZERO ? ROW_ZERO : ROW_GATHER));
                r.ldx = (o.kind == SOP_GATHER_IN) ? ldin : ldout;
                for (int z = 0; z < ninst; ++z) {
                    r.W[z] = (cx<T> *)h->W[z];
                    r.X[z] = (o.kind == SOP_GATHER_IN) ? const_cast<c128 *>(Xin[z]) : Xout[z];
                }
                launch_rows<T>(r, ninst, st);
            }
        }
    };
    run(h->fwd);
    run(h->bwd);
    return cuda_check(cudaGetLastError(), "solve launch");
}

}  // namespace

int solve_batch(zolo_factor_s *h, int ninst, const int *pole, const int *herm, int64_t k, const c128 *const *Xin,
                int64_t ldin, c128 *const *Xout, int64_t ldout, cudaStream_t st) {
    if (ninst > MAX_INST || ninst > 2 * h->r1) return set_error(ZOLO_EINVAL, "internal: too many instances");
    int rc = ensure_solve_schedule(h, k);
    if (rc) return rc;
    h->stats.solve_cols += (int64_t)ninst * k;
    return (h->prec == ZOLO_PREC_MIXED) ? run_solve<float>(h, ninst, pole, herm, k, Xin, ldin, Xout, ldout, st)
                                        : run_solve<double>(h, ninst, pole, herm, k, Xin, ldin, Xout, ldout, st);
}

int ensure_scratch(zolo_factor_s *h, int64_t k, int blocks, c128 **out) {
    const size_t need = (size_t)blocks * h->n * k * sizeof(c128);
    if (h->scratch.bytes < need) {
        if (h->scratch.p) dev_free(h, h->scratch.p);
        h->scratch = Buf();
        void *p = nullptr;
        int rc = dev_alloc(h, need, &p);
        if (rc) return rc;
        h->scratch = Buf{p, need};
    }
    *out = (c128 *)h->scratch.p;
    return ZOLO_OK;
}

int ensure_colpart(zolo_factor_s *h, int64_t k, double **out) {
    const size_t need = (size_t)COLNORM_PARTS * std::max<int64_t>(k, 1) * sizeof(double);
    if (h->colpart.bytes < need) {
        dev_release(h, h->colpart);
        void *p = nullptr;
        int rc = dev_alloc(h, need, &p);
        if (rc) return rc;
        h->colpart = Buf{p, need};
    }
    *out = (double *)h->colpart.p;
    return ZOLO_OK;
}

int colnorm2(zolo_factor_s *h, int64_t k, const c128 *X, int64_t ldx, double *out, cudaStream_t st, bool imag_only) {
    double *part = nullptr;
    int rc = ensure_colpart(h, k, &part);
    if (rc) return rc;
    launch_colnorm2(h->n, k, X, ldx, out, part, st, imag_only);
    return ZOLO_OK;
}

int block_is_real(zolo_factor_s *h, int64_t k, const c128 *X, int64_t ldx, cudaStream_t st, bool *real) {
    *real = false;
    if (h->norms_k < k) {
        if (h->d_norms) dev_free(h, h->d_norms);
        int rc = dev_alloc(h, 2 * MAX_INST * k * sizeof(double), (void **)&h->d_norms);
        if (rc) return rc;
        h->norms_k = k;
    }
    int rc = colnorm2(h, k, X, ldx, h->d_norms, st, true);
    if (rc) return rc;
    std::vector<double> im(k);
    rc = cuda_check(cudaMemcpyAsync(im.data(), h->d_norms, k * sizeof(double), cudaMemcpyDeviceToHost, st), "imag");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "imag");
    if (rc) return rc;
    bool r = true;
    for (double v : im) r = r && (v == 0.0);
    *real = r;
    return ZOLO_OK;
}

int solve_refined(zolo_factor_s *h, int ninst, const int *pole, const int *herm, int64_t k, const c128 *const *Xin,
                  int64_t ldin, c128 *const *Xout, int64_t ldout, cudaStream_t st, int *n_refine) {
    if (n_refine) *n_refine = 0;
    int rc = solve_batch(h, ninst, pole, herm, k, Xin, ldin, Xout, ldout, st);
    if (rc || h->prec != ZOLO_PREC_MIXED) return rc;
    // FP64 iterative refinement: r = b - K x (K = A - sigma B, or K^H = A - conj(sigma) B),
    // dx = K~^-1 r with the complex64 factors, x += dx, until ||r_c|| <= tol ||b_c|| for
    // every column of every instance.
    return refine_loop(h, ninst, pole, herm, k, Xin, ldin, Xout, ldout, st, n_refine);
}

int refine_loop(zolo_factor_s *h, int ninst, const int *pole, const int *herm, int64_t k, const c128 *const *Xin,
                int64_t ldin, c128 *const *Xout, int64_t ldout, cudaStream_t st, int *n_refine) {
    const size_t blk = (size_t)h->n * k;
    const size_t need = 2 * (size_t)ninst * blk * sizeof(c128);
    if (h->rscratch.bytes < need) {
        if (h->rscratch.p) dev_free(h, h->rscratch.p);
        h->rscratch = Buf();
        void *p = nullptr;
        int rc = dev_alloc(h, need, &p);
        if (rc) return rc;
        h->rscratch = Buf{p, need};
    }
    if (h->norms_k < k) {
        if (h->d_norms) dev_free(h, h->d_norms);
        int rc = dev_alloc(h, 2 * MAX_INST * k * sizeof(double), (void **)&h->d_norms);
        if (rc) return rc;
        h->norms_k = k;
    }
    c128 *R = (c128 *)h->rscratch.p, *DX = R + ninst * blk;
    std::vector<double> hb(ninst * k), hr(ninst * k);
    for (int z = 0; z < ninst; ++z) {
        int rc = colnorm2(h, k, Xin[z], ldin, h->d_norms + z * k, st);
        if (rc) return rc;
    }
    int rc = cuda_check(cudaMemcpyAsync(hb.data(), h->d_norms, ninst * k * sizeof(double), cudaMemcpyDeviceToHost, st),
                        "norms");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "norms");
    if (rc) return rc;
    const double tol = std::max(h->opts.refine_tol > 0 ? h->opts.refine_tol : 1e-12, h->refine_tol_now);
    const int itmax = h->opts.refine_max > 0 ? h->opts.refine_max : 8;
    double prev = 0.0;
    for (int it = 0;; ++it) {
        ResidArgs ra;
        std::memset(&ra, 0, sizeof(ra));
        ra.ninst = ninst;
        ra.k = (int)k;
        ra.ldb = ldin;
        ra.ldx = ldout;
        ra.ldr = k;
        for (int z = 0; z < ninst; ++z) {
            const c128 sg{h->fi.sigma_hat[2 * pole[z]], h->fi.sigma_hat[2 * pole[z] + 1]};
            ra.Bz[z] = Xin[z];
            ra.Xz[z] = Xout[z];
            ra.Rz[z] = R + z * blk;
            ra.s[z] = herm[z] ? conj(sg) : sg;          // K^H = A - conj(sigma) B
        }
        // A tolerance >= 1e-8 leaves a margin of 1e6 over the double-float rounding (~1e-14
        // of sum |K||x|): those residuals run on the FP32 pipe, tighter ones in FP64.
        const bool use_df = tol >= 1e-8 && (h->A.vdf || h->A.vrdf) && (h->B.vdf || h->B.vrdf);
        if (use_df) {
            ResidDfArgs rd;
            std::memset(&rd, 0, sizeof(rd));
            rd.ninst = ninst;
            rd.k = (int)k;
            rd.ldb = ldin;
            rd.ldr = k;
            for (int z = 0; z < ninst; ++z) {
                float4 *xs = (float4 *)(DX + z * blk);           // DX is free until the next solve
                launch_split_df(h->n, k, Xout[z], ldout, xs, st);
                rd.Bz[z] = Xin[z];
                rd.Xs[z] = xs;
                rd.Rz[z] = R + z * blk;
                df_split(ra.s[z].re, rd.s[z].x, rd.s[z].y);
                df_split(ra.s[z].im, rd.s[z].z, rd.s[z].w);
            }
            launch_refine_resid_df(h->A, h->B, rd, st);
        } else {
            launch_refine_resid(h->A, h->B, ra, st);
        }
        for (int z = 0; z < ninst && !rc; ++z) rc = colnorm2(h, k, R + z * blk, k, h->d_norms + z * k, st);
        if (rc) return rc;
        rc = cuda_check(cudaMemcpyAsync(hr.data(), h->d_norms, ninst * k * sizeof(double), cudaMemcpyDeviceToHost, st),
                        "norms");
        if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "norms");
        if (!rc) rc = check_tc_status();
        if (rc) return rc;
        double worst = 0.0;
        for (int64_t i = 0; i < ninst * k; ++i) worst = std::max(worst, std::sqrt(hr[i] / std::max(hb[i], 1e-300)));
        if (h->opts.verbose) std::fprintf(stderr, "[zolo] refine step %d: max ||b - K x|| / ||b|| = %.3e\n", it, worst);
        if (worst <= tol) break;
        // stagnation below 1e-10 is the FP64 rounding floor of the residual itself: accept
        if (it > 0 && worst > 0.5 * prev && worst < 1e-10) break;
        if (it >= itmax) return set_error(ZOLO_ENOCONV, "refinement of a shifted solve did not converge (" +
                                                            std::to_string(worst) + ")");
        prev = worst;
        const c128 *rin[MAX_INST];
        c128 *dout[MAX_INST];
        for (int z = 0; z < ninst; ++z) {
            rin[z] = R + z * blk;
            dout[z] = DX + z * blk;
        }
        rc = solve_batch(h, ninst, pole, herm, k, rin, k, dout, k, st);
        if (rc) return rc;
        for (int z = 0; z < ninst; ++z) {
            LinArgs a;
            std::memset(&a, 0, sizeof(a));
            a.n = h->n;
            a.k = k;
            a.ldy = ldout;
            a.Y = Xout[z];
            a.nterm = 2;
            a.coef[0] = c128{1.0, 0.0};
            a.X[0] = Xout[z];
            a.ldx[0] = ldout;
            a.coef[1] = c128{1.0, 0.0};
            a.X[1] = DX + z * blk;
            a.ldx[1] = k;
            launch_lincomb(a, st);
        }
        if (n_refine) (*n_refine)++;
    }
    return ZOLO_OK;
}

int apply_inner(zolo_factor_s *h, int64_t k, const c128 *X, int64_t ldx, c128 *Y, int64_t ldy, cudaStream_t st,
                const float2 *Xs) {
    // GX = const_hat X + sum_j ( w_hat_j K_j^-1 B X + conj(w_hat_j) K_j^-H B X )   (eq. solve)
    // With real A, B and X (h->realx), K_j^-H B X = conj(K_j^-1 B X), so
    // GX = const_hat X + 2 Re sum_j w_hat_j K_j^-1 B X: one solve per pole.
    const int r1 = h->r1;
    const bool rx = h->realx;
    const int nsol = rx ? r1 : 2 * r1;                  // solve instances
    const int nblk = 1 + nsol;
    c128 *scr = nullptr;
    int rc = ensure_scratch(h, k, nblk, &scr);
    if (rc) return rc;
    c128 *BX = scr;
    if (Xs && (h->B.vrdf || h->B.vdf))
        launch_spmm_df(h->B, k, Xs, BX, st);
    else
        launch_spmm(h->B, k, X, ldx, BX, k, c128{1.0, 0.0}, false, st);
    for (int p0 = 0; p0 < nsol; p0 += MAX_INST) {
        const int ni = std::min(MAX_INST, nsol - p0);
        int pole[MAX_INST], herm[MAX_INST];
        const c128 *in[MAX_INST];
        c128 *out[MAX_INST];
        for (int z = 0; z < ni; ++z) {
            const int q = p0 + z;
            pole[z] = rx ? q : q / 2;
            herm[z] = rx ? 0 : q % 2;
            in[z] = BX;
            out[z] = scr + (size_t)(1 + q) * h->n * k;
        }
        int nref = 0;
        rc = solve_refined(h, ni, pole, herm, k, in, k, out, k, st, &nref);
        if (rc) return rc;
        h->stats.n_refine_max = std::max(h->stats.n_refine_max, nref);
    }
    LinArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = h->n;
    a.k = k;
    a.ldy = ldy;
    a.Y = Y;
    a.real_out = rx ? 1 : 0;
    a.nterm = 0;
    a.coef[a.nterm] = c128{h->fi.const_hat, 0.0};
    a.X[a.nterm] = X;
    a.ldx[a.nterm++] = ldx;
    // the linear combination kernel takes at most LIN_MAX terms: accumulate in passes
    for (int q = 0; q < nsol; ++q) {
        const int j = rx ? q : q / 2, hh = rx ? 0 : q % 2;
        const c128 w{h->fi.w_hat[2 * j], h->fi.w_hat[2 * j + 1]};
        if (a.nterm == LIN_MAX) {
            launch_lincomb(a, st);
            a.nterm = 0;
            a.coef[a.nterm] = c128{1.0, 0.0};
            a.X[a.nterm] = Y;
            a.ldx[a.nterm++] = ldy;
        }
        a.coef[a.nterm] = rx ? c128{2.0 * w.re, 2.0 * w.im} : (hh ? conj(w) : w);
        a.X[a.nterm] = scr + (size_t)(1 + q) * h->n * k;
        a.ldx[a.nterm++] = k;
    }
    launch_lincomb(a, st);
    return cuda_check(cudaGetLastError(), "apply_inner");
}

}  // namespace zolo

// ============================================================== ABI
using namespace zolo;

extern "C" {

}  // extern "C"

namespace zolo {
// Upload the pencil and factor A - sigma_j B for the given poles (sigma as re, im pairs).
static int factor_create(const zolo_csr *A, const zolo_csr *B, const zolo_filter_info &fi, zolo_symbolic sym,
                         const zolo_opts *opts, cudaStream_t stream, bool count_neg, zolo_factor_s **out) {
    *out = nullptr;
    CsrHost ha, hb;
    int rc = csr_host_view(A, ha, &A);
    if (!rc) rc = csr_host_view(B, hb, &B);
    if (rc) return rc;
    bool ca, cb;
    rc = check_csr(A, "A", ca);
    if (!rc) rc = check_csr(B, "B", cb);
    if (rc) return rc;
    if (A->n != B->n) return set_error(ZOLO_EINVAL, "A and B differ in size");
    if (opts && (opts->tensor_core < ZOLO_TC_AUTO || opts->tensor_core > ZOLO_TC_ALWAYS))
        return set_error(ZOLO_EINVAL, "tensor_core must be ZOLO_TC_AUTO, ZOLO_TC_OFF or ZOLO_TC_ALWAYS");
    auto *h = new zolo_factor_s();
    if (opts) h->opts = *opts; else zolo_opts_default(&h->opts);
    h->prec = h->opts.precision == ZOLO_PREC_MIXED ? ZOLO_PREC_MIXED : ZOLO_PREC_FP64;
    h->n = A->n;
    h->cplx = ca || cb;
    h->fi = fi;
    h->r1 = fi.r1;
    h->count_neg = count_neg;
    std::memset(&h->stats, 0, sizeof(h->stats));
    cudaGetDevice(&h->device);
    double nb_inf = 0.0;
    rc = check_hermitian(A, "A", h->normA_inf);
    if (!rc) rc = check_hermitian(B, "B", nb_inf);
    if (rc) {
        delete h;
        return rc;
    }
    if (sym) {
        h->sym = *sym;
        if (h->sym.n != A->n) {
            delete h;
            return set_error(ZOLO_EINVAL, "symbolic analysis is for another size");
        }
    } else {
        rc = analyze(A, B, h->opts, h->sym);
        if (rc) {
            delete h;
            return rc;
        }
    }
    rc = upload_csr(h, A, h->A);
    if (!rc) rc = upload_csr(h, B, h->B);
    if (!rc) rc = build_factor_plan(h, A, B);
    if (!rc && count_neg) rc = dev_alloc(h, h->r1 * sizeof(int), (void **)&h->d_negcnt);
    // a real pencil at real shifts (inertia counts) factors real matrices: one FMA per product
    h->real_fac = count_neg && h->prec == ZOLO_PREC_FP64 && h->A.vr && h->B.vr;
    for (int j = 0; j < h->r1; ++j) h->real_fac = h->real_fac && fi.sigma_hat[2 * j + 1] == 0.0;
    const size_t eb = elem_bytes(h->prec);
    for (int j = 0; !rc && j < h->r1; ++j) {
        rc = dev_alloc(h, h->pool_elems * eb, &h->pool[j]);
        if (!rc) rc = dev_alloc(h, std::max<int64_t>(1, h->inv_elems) * eb, &h->inv[j]);
        if (!rc) rc = dev_alloc(h, (count_neg ? 1 : std::max<int64_t>(1, h->finv_elems)) * eb, &h->finv[j]);
    }
    if (!rc && h->prec == ZOLO_PREC_MIXED && !count_neg) rc = setup_presplit(h);
    h->stats.flops_factor = h->sym.info.flops_lu * h->r1;
    h->stats.flops_solve = 16.0 * (double)h->sym.info.nnz_factor;     // fwd + bwd, complex, per column
    if (!rc) rc = factor_numeric(h, stream);
    if (rc) {
        zolo_factor_destroy(h);
        return rc;
    }
    *out = h;
    return ZOLO_OK;
}
}  // namespace zolo

extern "C" {

int zolo_factor(const zolo_csr *A, const zolo_csr *B, zolo_filter f, zolo_symbolic sym, const zolo_opts *opts,
                void *stream, zolo_factor_h *out) {
    clear_error();
    if (!out || !f) return set_error(ZOLO_EINVAL, "null argument");
    return factor_create(A, B, f->info, sym, opts, (cudaStream_t)stream, false, out);
}

int zolo_inertia(const zolo_csr *A, const zolo_csr *B, zolo_symbolic sym, const zolo_opts *opts, int32_t nshift,
                 const double *sigma, int64_t *count, void *stream) {
    clear_error();
    if (!sigma || !count || nshift < 1) return set_error(ZOLO_EINVAL, "bad argument");
    CsrHost ha, hb;                                 // one host copy for every batch of shifts
    int rc0 = csr_host_view(A, ha, &A);
    if (!rc0) rc0 = csr_host_view(B, hb, &B);
    if (rc0) return rc0;
    for (int i = 0; i < nshift; ++i)
        if (!std::isfinite(sigma[i])) return set_error(ZOLO_EINVAL, "non-finite shift");
    // Always complex128 fronts: the no-pivot LDL^H of an indefinite A - sigma B keeps the
    // signs of its pivots only with FP64 arithmetic (complex64 counts are unreliable).
    zolo_opts o;
    if (opts) o = *opts; else zolo_opts_default(&o);
    o.precision = ZOLO_PREC_FP64;
    zolo_symbolic_s local;
    const zolo_symbolic_s *S = sym;
    if (!S) {
        int rc = analyze(A, B, o, local);
        if (rc) return rc;
        S = &local;
    }
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    const double per_shift = (double)S->info.front_entries * sizeof(c128);
    int batch = (int)std::max(1.0, std::min((double)std::min(nshift, ZOLO_MAX_R),
                                             0.7 * (double)fr / std::max(per_shift, 1.0)));
    for (int i0 = 0; i0 < nshift; i0 += batch) {
        const int nb = std::min(batch, nshift - i0);
        zolo_filter_info fi;
        std::memset(&fi, 0, sizeof(fi));
        fi.r1 = nb;
        for (int i = 0; i < nb; ++i) fi.sigma_hat[2 * i] = sigma[i0 + i];
        zolo_factor_s *h = nullptr;
        int rc = factor_create(A, B, fi, const_cast<zolo_symbolic_s *>(S), &o, (cudaStream_t)stream, true, &h);
        if (rc) return rc;
        std::vector<int> neg(nb);
        rc = cuda_check(cudaMemcpy(neg.data(), h->d_negcnt, nb * sizeof(int), cudaMemcpyDeviceToHost), "inertia");
        for (int i = 0; i < nb && !rc; ++i) count[i0 + i] = neg[i];
        zolo_factor_destroy(h);
        if (rc) return rc;
    }
    return ZOLO_OK;
}

int zolo_profile_begin(int32_t gemm_events) {
    clear_error();
    prof_collect_ms();
    counters() = LaunchCounters();
    prof_set(gemm_events);
    return ZOLO_OK;
}

int zolo_profile_end(void *stream, int64_t *launches, int64_t *gemm_launches, double *gemm_ms, double *gemm_flops) {
    clear_error();
    int rc = cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "profile");
    const double ms = prof_collect_ms();
    prof_set(0);
    if (launches) *launches = counters().launches;
    if (gemm_launches) *gemm_launches = counters().gemm_launches;
    if (gemm_ms) *gemm_ms = ms;
    if (gemm_flops) *gemm_flops = counters().gemm_flops;
    return rc;
}

int zolo_profile_bytes(double *gemm_bytes, double *tc_bytes) {
    clear_error();
    if (gemm_bytes) *gemm_bytes = counters().gemm_bytes;
    if (tc_bytes) *tc_bytes = counters().tc_bytes;
    return ZOLO_OK;
}

int zolo_profile_tc(int64_t *launches, double *ms, double *flops) {
    clear_error();
    if (launches) *launches = counters().tc_launches;
    if (ms) *ms = counters().tc_ms;
    if (flops) *flops = counters().tc_flops;
    return ZOLO_OK;
}

int zolo_refactor(zolo_factor_h h, void *stream) {
    clear_error();
    if (!h) return set_error(ZOLO_EINVAL, "null handle");
    return factor_numeric(h, (cudaStream_t)stream);
}

void zolo_factor_destroy(zolo_factor_h h) {
    if (!h) return;
    krylov_free(h->kw);
    h->kw = nullptr;
    for (auto &b : h->owned) cudaFree(b.p);
    h->owned.clear();
    delete h;
}

int zolo_factor_get_stats(zolo_factor_h h, zolo_stats *out) {
    clear_error();
    if (!h || !out) return set_error(ZOLO_EINVAL, "null argument");
    *out = h->stats;
    return ZOLO_OK;
}

int zolo_solve(zolo_factor_h h, int32_t pole, int32_t herm, int64_t k, const void *Bk, int64_t ldb, void *X,
               int64_t ldx, void *stream) {
    clear_error();
    if (!h || !Bk || !X || k <= 0 || ldb < k || ldx < k || pole < 0 || pole >= h->r1 || (herm != 0 && herm != 1))
        return set_error(ZOLO_EINVAL, "bad argument");
    const int p = pole, hh = herm;
    const c128 *in[1] = {(const c128 *)Bk};
    c128 *outp[1] = {(c128 *)X};
    int nref = 0;
    int rc = solve_refined(h, 1, &p, &hh, k, in, ldb, outp, ldx, (cudaStream_t)stream, &nref);
    if (rc) return rc;
    h->stats.n_refine_max = std::max(h->stats.n_refine_max, nref);
    return cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "solve");
}

int zolo_matmul(zolo_factor_h h, int32_t which, int64_t k, const void *X, int64_t ldx, void *Y, int64_t ldy,
                void *stream) {
    clear_error();
    if (!h || !X || !Y || k <= 0 || ldx < k || ldy < k || (which != 0 && which != 1))
        return set_error(ZOLO_EINVAL, "bad argument");
    launch_spmm(which ? h->B : h->A, k, (const c128 *)X, ldx, (c128 *)Y, ldy, c128{1.0, 0.0}, false,
                (cudaStream_t)stream);
    return cuda_check(cudaGetLastError(), "spmm");
}

int zolo_apply_inner(zolo_factor_h h, int64_t k, const void *X, int64_t ldx, void *Y, int64_t ldy, void *stream) {
    clear_error();
    if (!h || !X || !Y || k <= 0 || ldx < k || ldy < k) return set_error(ZOLO_EINVAL, "bad argument");
    bool rx = false;
    int rc = ZOLO_OK;
    if (pencil_is_real(h) && h->opts.real_block) rc = block_is_real(h, k, (const c128 *)X, ldx, (cudaStream_t)stream, &rx);
    if (rc) return rc;
    h->realx = rx;
    rc = apply_inner(h, k, (const c128 *)X, ldx, (c128 *)Y, ldy, (cudaStream_t)stream);
    h->realx = false;
    if (rc) return rc;
    return cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "apply_inner");
}

}  // extern "C"
