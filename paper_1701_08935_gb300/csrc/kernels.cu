// Kernels of the multifrontal factorisation and the block triangular solves
// (Section 2.3: K_j = A - sigma_j B factored once, then applied to blocks of vectors),
// plus the CSR SpMM.  Every kernel is batched: blockIdx.z selects an instance
// (a pole, or a (pole, K^-1 / K^-H) pair) and job lists built on the host describe
// all fronts of one tree level, so one launch covers a whole level.
#include "kernels.cuh"
#include "df64.cuh"

#include <vector>

namespace zolo {

namespace {
LaunchCounters g_counters;
int g_prof = 0;                      // bit 0: time complex64 GEMMs, bit 1: complex128
std::vector<cudaEvent_t> g_ev;       // start/stop pairs of profiled GEMM launches
struct EvInfo {
    bool tc;                         // launched on the tensor-core kernel
    double flops;                    // executed flops of the launch
    double bytes;                    // its algorithmic bytes (operands read once, C read if accumulated, written)
};
std::vector<EvInfo> g_ev_info;       // one per pair
std::vector<cudaEvent_t> g_ev_pool;
cudaEvent_t get_event() {
    if (!g_ev_pool.empty()) {
        cudaEvent_t e = g_ev_pool.back();
        g_ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

LaunchCounters &counters() { return g_counters; }
// Launch counts come from every calling thread: relaxed atomic increments (the profiling
// fields below are process-wide and documented as not thread-safe).
void count_launch(int64_t n) { __atomic_fetch_add(&g_counters.launches, n, __ATOMIC_RELAXED); }
void prof_set(int mask) { g_prof = mask; }
double prof_collect_ms() {
    double ms = 0.0;
    for (size_t i = 0; i + 1 < g_ev.size(); i += 2) {
        cudaEventSynchronize(g_ev[i + 1]);
        float t = 0.f;
        cudaEventElapsedTime(&t, g_ev[i], g_ev[i + 1]);
        ms += t;
        const EvInfo &f = g_ev_info[i / 2];
        if (f.tc) {
            g_counters.tc_launches++;
            g_counters.tc_ms += t;
            g_counters.tc_flops += f.flops;
            g_counters.tc_bytes += f.bytes;
        }
    }
    for (cudaEvent_t e : g_ev) g_ev_pool.push_back(e);
    g_ev.clear();
    g_ev_info.clear();
    return ms;
}

// ============================================================== batched GEMM
// 8-byte asynchronous global -> shared copy; src_size 0 fills zeros (no global read)
__device__ __forceinline__ void cp_async_8(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Job of a row / extend-add / identity / transpose tile: the launch's tile map when it has
// one, else a binary search of tile0.
__device__ __forceinline__ int find_rjob(const int32_t *tmap, const RJob *jobs, int njobs, int tile) {
    if (tmap) return tmap[tile];
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Job of a tile: the launch's tile map when it has one, else a binary search of tile0.
__device__ __forceinline__ int find_job(const int32_t *tmap, const GJob *jobs, int njobs, int tile) {
    if (tmap) return tmap[tile];
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// C (=|-=) op(A) op(B) for every job in the list; one CTA per BM x BN tile (64 x 64, or
// 32 x 128 for fronts with few pivot rows).
// The whole kk extent of a tile is read before its C block is written, so a job
// whose C aliases A (with n <= BN) or B (with m <= BM) is computed in place.
// complex64: three CTAs per SM (<= 85 registers): tiles of the deep tree levels are short
// in kk, so their global-memory latency is hidden by resident CTAs rather than the k-loop.
// RE: the operands hold real values (zero imaginary parts) -- one real FMA per product
// instead of four; the imaginary parts of C are left as they are.
template <class T, int BM, int BN, int BK, bool RE = false>
__global__ void __launch_bounds__(BM * BN / 16, sizeof(T) == 4 ? 3 * 4096 / (BM * BN) : 1) k_gemm(GemmArgs<T> g) {
    const int z = blockIdx.z;
    const int tile = blockIdx.x;
    if (tile >= g.ntiles[z]) return;
    const GJob *jobs = g.jobs[z];
    __shared__ int s_job;
    // complex64: two buffers filled by cp.async; complex128: one buffer filled from registers
    constexpr int NBUF = sizeof(T) == 4 ? 2 : 1;
    __shared__ __align__(16) cx<T> As2[NBUF][BK][BM];
    __shared__ __align__(16) cx<T> Bs2[NBUF][BK][BN];
    auto &As = As2[0];
    auto &Bs = Bs2[0];
    const int tid = threadIdx.x;
    if (tid == 0) s_job = find_job(g.tmap[z], jobs, g.njobs[z], tile);
    __syncthreads();
    const GJob J = jobs[s_job];
    int t = tile - J.tile0;
    const int tmn = J.tm * ((J.n + BN - 1) / BN);
    const int kslice = t / tmn;
    t -= kslice * tmn;
    const int i0 = (t % J.tm) * BM, j0 = (t / J.tm) * BN;
    const int ksp = J.ks > 1 ? J.ks : 1;
    const int kchunk = (((J.k + ksp - 1) / ksp) + BK - 1) / BK * BK;
    const int kbeg = kslice * kchunk, kend = min(J.k, kbeg + kchunk);
    const cx<T> *__restrict__ A = g.A[z] + J.a;
    const cx<T> *__restrict__ B = g.B[z] + J.b;
    const bool conjA = J.flags & GJ_CONJA, conjB = J.flags & GJ_CONJB;
    constexpr int TX = BN / 4, TY = BM / 4;             // TX * TY threads, 4 x 4 outputs each
    constexpr int NT = TX * TY;
    static_assert((BM * BK) % NT == 0 && (BN * BK) % NT == 0, "tile must split evenly over the threads");
    const int tx = tid % TX, ty = tid / TX;
    cx<T> acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = mk<T>(0, 0);

    if constexpr (sizeof(T) == 4) {
        // complex64: double-buffered cp.async staging (zero fill at the edges), so the loads of
        // k-tile s + 1 are in flight while tile s is consumed; conjugation is applied on read
        const int nst = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
        auto issue = [&](int l0, int buf) {
#pragma unroll
            for (int q = 0; q < (BM * BK) / NT; ++q) {
                const int e = tid + NT * q;
                int i, l;
                if (J.ars == 1) { i = e % BM; l = e / BM; } else { l = e % BK; i = e / BK; }
                const bool v = (i0 + i < J.m) && (l0 + l < kend);
                const cx<T> *src = v ? A + (int64_t)(i0 + i) * J.ars + (int64_t)(l0 + l) * J.acs : A;
                cp_async_8((uint32_t)__cvta_generic_to_shared(&As2[buf][l][i]), src, v);
            }
#pragma unroll
            for (int q = 0; q < (BN * BK) / NT; ++q) {
                const int e = tid + NT * q;
                int j, l;
                if (J.brs == 1) { l = e % BK; j = e / BK; } else { j = e % BN; l = e / BN; }
                const bool v = (j0 + j < J.n) && (l0 + l < kend);
                const cx<T> *src = v ? B + (int64_t)(l0 + l) * J.brs + (int64_t)(j0 + j) * J.bcs : B;
                cp_async_8((uint32_t)__cvta_generic_to_shared(&Bs2[buf][l][j]), src, v);
            }
        };
        if (nst > 0) issue(kbeg, 0);
        cp_async_commit_group();
        for (int s = 0; s < nst; ++s) {
            if (s + 1 < nst) issue(kbeg + (s + 1) * BK, (s + 1) & 1);
            cp_async_commit_group();
            cp_async_wait_group<1>();
            __syncthreads();
            const int b = s & 1;
#pragma unroll 4
            for (int l = 0; l < BK; ++l) {
                cx<T> a[4], bv[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    a[r] = As2[b][l][ty + TY * r];
                    if (conjA) a[r].im = -a[r].im;
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    bv[c] = Bs2[b][l][tx + TX * c];
                    if (conjB) bv[c].im = -bv[c].im;
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) fma_acc(acc[r][c], a[r], bv[c]);
            }
            __syncthreads();
        }
    } else
    for (int l0 = kbeg; l0 < kend; l0 += BK) {
        // ---- stage A tile (BM x BK) and B tile (BK x BN)
#pragma unroll
        for (int q = 0; q < (BM * BK) / NT; ++q) {
            const int e = tid + NT * q;
            int i, l;
            if (J.ars == 1) { i = e % BM; l = e / BM; } else { l = e % BK; i = e / BK; }
            cx<T> v = mk<T>(0, 0);
            if (i0 + i < J.m && l0 + l < kend) v = A[(int64_t)(i0 + i) * J.ars + (int64_t)(l0 + l) * J.acs];
            As[l][i] = conjA ? conj(v) : v;
        }
#pragma unroll
        for (int q = 0; q < (BN * BK) / NT; ++q) {
            const int e = tid + NT * q;
            int j, l;
            if (J.brs == 1) { l = e % BK; j = e / BK; } else { j = e % BN; l = e / BN; }
            cx<T> v = mk<T>(0, 0);
            if (j0 + j < J.n && l0 + l < kend) v = B[(int64_t)(l0 + l) * J.brs + (int64_t)(j0 + j) * J.bcs];
            Bs[l][j] = conjB ? conj(v) : v;
        }
        __syncthreads();
#pragma unroll 4
        for (int l = 0; l < BK; ++l) {
            cx<T> a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[l][ty + TY * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[l][tx + TX * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if constexpr (RE)
                        acc[r][c].re = fma(a[r].re, b[c].re, acc[r][c].re);
                    else
                        fma_acc(acc[r][c], a[r], b[c]);
                }
        }
        __syncthreads();
    }
    cx<T> *__restrict__ C = g.C[z] + J.c;
    const bool sub = J.flags & GJ_SUB, add = J.flags & GJ_ACC, atom = J.ks > 1;
    // Accumulating products read every C element of the thread first (16 independent loads in
    // flight) and only then write: interleaved read-modify-writes would make each load wait for
    // the previous store, one global round trip per element.
    if ((sub || add) && !atom) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = i0 + ty + TY * r;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = j0 + tx + TX * c;
                if (i < J.m && j < J.n) {
                    const cx<T> o = C[(int64_t)i * J.crs + (int64_t)j * J.ccs];
                    acc[r][c] = sub ? o - acc[r][c] : o + acc[r][c];
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = i0 + ty + TY * r;
        if (i >= J.m) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = j0 + tx + TX * c;
            if (j >= J.n) continue;
            cx<T> *p = C + (int64_t)i * J.crs + (int64_t)j * J.ccs;
            if (atom) {
                const cx<T> v = sub ? mk<T>(-acc[r][c].re, -acc[r][c].im) : acc[r][c];
                atomicAdd(&p->re, v.re);
                atomicAdd(&p->im, v.im);
            } else {
                *p = acc[r][c];
            }
        }
    }
}

// Complex64 variant for the FP32 pipe: 128 x 64 C tile per CTA, each thread an 8 x 4 block of
// complex outputs (rows ty*4 + {0..3} and 64 + ty*4 + {0..3}, columns tx*2 + {0,1} and
// 32 + tx*2 + {0,1}) fed by 128-bit shared-memory reads; the next k-tile is prefetched into
// registers while the current one is consumed.  Same job semantics (and in-place rules)
// as k_gemm, with tiles of GEMM_BM_C64 rows.
constexpr int G2_BM = 128, G2_BN = 64, G2_BK = 16;
__global__ void __launch_bounds__(256) k_gemm_c64(GemmArgs<float> g) {
    const int z = blockIdx.z;
    const int tile = blockIdx.x;
    if (tile >= g.ntiles[z]) return;
    const GJob *jobs = g.jobs[z];
    __shared__ int s_job;
    __shared__ __align__(16) c64 As[G2_BK][G2_BM];
    __shared__ __align__(16) c64 Bs[G2_BK][G2_BN];
    const int tid = threadIdx.x;
    if (tid == 0) s_job = find_job(g.tmap[z], jobs, g.njobs[z], tile);
    __syncthreads();
    const GJob J = jobs[s_job];
    int t = tile - J.tile0;
    const int tmn = J.tm * ((J.n + G2_BN - 1) / G2_BN);
    const int kslice = t / tmn;
    t -= kslice * tmn;
    const int i0 = (t % J.tm) * G2_BM, j0 = (t / J.tm) * G2_BN;
    const int ksp = J.ks > 1 ? J.ks : 1;
    const int kchunk = (((J.k + ksp - 1) / ksp) + G2_BK - 1) / G2_BK * G2_BK;
    const int kbeg = kslice * kchunk, kend = min(J.k, kbeg + kchunk);
    const c64 *__restrict__ A = g.A[z] + J.a;
    const c64 *__restrict__ B = g.B[z] + J.b;
    const bool conjA = J.flags & GJ_CONJA, conjB = J.flags & GJ_CONJB;
    const bool a_rowfast = (J.ars == 1), b_rowfast = (J.brs == 1);
    const int tx = tid & 15, ty = tid >> 4;
    float acc[8][4][2];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c][0] = acc[r][c][1] = 0.f;
    c64 ra[8], rb[4];
    auto load = [&](int l0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = tid + 256 * q;
            int i, l;
            if (a_rowfast) { i = e % G2_BM; l = e / G2_BM; } else { l = e % G2_BK; i = e / G2_BK; }
            c64 v = mk<float>(0, 0);
            if (i0 + i < J.m && l0 + l < kend) v = A[(int64_t)(i0 + i) * J.ars + (int64_t)(l0 + l) * J.acs];
            ra[q] = conjA ? conj(v) : v;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            int j, l;
            if (b_rowfast) { l = e % G2_BK; j = e / G2_BK; } else { j = e % G2_BN; l = e / G2_BN; }
            c64 v = mk<float>(0, 0);
            if (j0 + j < J.n && l0 + l < kend) v = B[(int64_t)(l0 + l) * J.brs + (int64_t)(j0 + j) * J.bcs];
            rb[q] = conjB ? conj(v) : v;
        }
    };
    auto store = [&]() {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = tid + 256 * q;
            int i, l;
            if (a_rowfast) { i = e % G2_BM; l = e / G2_BM; } else { l = e % G2_BK; i = e / G2_BK; }
            As[l][i] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            int j, l;
            if (b_rowfast) { l = e % G2_BK; j = e / G2_BK; } else { j = e % G2_BN; l = e / G2_BN; }
            Bs[l][j] = rb[q];
        }
    };
    load(kbeg);
    for (int l0 = kbeg; l0 < kend; l0 += G2_BK) {
        __syncthreads();
        store();
        __syncthreads();
        if (l0 + G2_BK < kend) load(l0 + G2_BK);
#pragma unroll 4
        for (int l = 0; l < G2_BK; ++l) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[l][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[l][ty * 4 + 2]);
            const float4 a2 = *reinterpret_cast<const float4 *>(&As[l][64 + ty * 4]);
            const float4 a3 = *reinterpret_cast<const float4 *>(&As[l][64 + ty * 4 + 2]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[l][tx * 2]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[l][32 + tx * 2]);
            const float ar[8] = {a0.x, a0.z, a1.x, a1.z, a2.x, a2.z, a3.x, a3.z};
            const float ai[8] = {a0.y, a0.w, a1.y, a1.w, a2.y, a2.w, a3.y, a3.w};
            const float br[4] = {b0.x, b0.z, b1.x, b1.z};
            const float bi[4] = {b0.y, b0.w, b1.y, b1.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    acc[r][c][0] = fmaf(ar[r], br[c], acc[r][c][0]);
                    acc[r][c][0] = fmaf(-ai[r], bi[c], acc[r][c][0]);
                    acc[r][c][1] = fmaf(ar[r], bi[c], acc[r][c][1]);
                    acc[r][c][1] = fmaf(ai[r], br[c], acc[r][c][1]);
                }
        }
    }
    c64 *__restrict__ C = g.C[z] + J.c;
    const bool sub = J.flags & GJ_SUB, add = J.flags & GJ_ACC, atom = J.ks > 1;
    // read all C elements of the thread before any write (see k_gemm)
    if ((sub || add) && !atom) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int i = i0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = j0 + (c < 2 ? tx * 2 + c : 32 + tx * 2 + (c - 2));
                if (i < J.m && j < J.n) {
                    const c64 o = C[(int64_t)i * J.crs + (int64_t)j * J.ccs];
                    acc[r][c][0] = sub ? o.re - acc[r][c][0] : o.re + acc[r][c][0];
                    acc[r][c][1] = sub ? o.im - acc[r][c][1] : o.im + acc[r][c][1];
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int i = i0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
        if (i >= J.m) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = j0 + (c < 2 ? tx * 2 + c : 32 + tx * 2 + (c - 2));
            if (j >= J.n) continue;
            c64 *p = C + (int64_t)i * J.crs + (int64_t)j * J.ccs;
            if (atom) {
                const float vr = sub ? -acc[r][c][0] : acc[r][c][0], vi = sub ? -acc[r][c][1] : acc[r][c][1];
                atomicAdd(reinterpret_cast<float2 *>(p), make_float2(vr, vi));
            } else {
                *p = mk<float>(acc[r][c][0], acc[r][c][1]);
            }
        }
    }
}

template <class T>
void launch_gemm(const GemmArgs<T> &g, int ninst, cudaStream_t st, double flops, double bytes) {
    int mx = 0;
    for (int z = 0; z < ninst; ++z) mx = g.ntiles[z] > mx ? g.ntiles[z] : mx;
    if (mx == 0) return;
    dim3 grid(mx, 1, ninst);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool timed = (g_prof & (sizeof(T) == 4 ? 1 : 2)) != 0;
    if (timed) {
        e0 = get_event();
        e1 = get_event();
        cudaEventRecord(e0, st);
    }
    bool tc = false;
    if constexpr (sizeof(T) == 4) {
        tc = (g.bm == 128 && g.bn == 128);
        if (tc)
            launch_gemm_tc(g, grid, st);
        else if (g.bn == 32 && g.bm == 32)               // narrow blocks (n <= 32): no padded columns
            k_gemm<T, 32, 32, 8><<<grid, 64, 0, st>>>(g);
        else if (g.bn == 32 && g.bm == 64)
            k_gemm<T, 64, 32, 8><<<grid, 128, 0, st>>>(g);
        else if (g.bn == 32)
            k_gemm<T, 128, 32, 16><<<grid, 256, 0, st>>>(g);
        else if (g.bm == G2_BM)
            k_gemm_c64<<<grid, 256, 0, st>>>(g);
        else if (g.bm == 32)
            k_gemm<T, 32, 128, 16><<<grid, 256, 0, st>>>(g);
        else
            k_gemm<T, 64, 64, 16><<<grid, 256, 0, st>>>(g);
    } else if (g.real) {
        k_gemm<T, 64, 64, 16, true><<<grid, 256, 0, st>>>(g);
    } else {
        k_gemm<T, 64, 64, 16><<<grid, 256, 0, st>>>(g);
    }
    if (timed) {
        cudaEventRecord(e1, st);
        g_ev.push_back(e0);
        g_ev.push_back(e1);
        g_ev_info.push_back({tc, flops, bytes});
    }
    count_launch();
    if (timed) {
        g_counters.gemm_launches++;
        g_counters.gemm_flops += flops;
        g_counters.gemm_bytes += bytes;
    }
}

// ============================================================== diagonal blocks
// No-pivot LU of an nb x nb diagonal block in FP64 shared memory, then the explicit
// inverses of its unit-lower L and upper U (one thread per column, substitution).
// A zero or non-finite pivot sets bit 1 of *err; the block is still written.
template <class T>
__global__ void __launch_bounds__(256) k_diag_lu(DiagArgs<T> g) {
    const int z = blockIdx.z;
    if ((int)blockIdx.x >= g.njobs) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c128 *blk = reinterpret_cast<c128 *>(smem_raw);          // NB x NB, ld NB
    c128 *X = blk + NB * NB;                                  // inverse column buffer
    const DJob J = g.jobs[blockIdx.x];
    cx<T> *F = g.pool[z] + J.off;
    const int nb = J.nb, tid = threadIdx.x;
    for (int e = tid; e < nb * nb; e += 256) {
        const int i = e % nb, j = e / nb;
        blk[i + j * NB] = cvt<double>(F[i + (int64_t)j * J.ld]);
    }
    __syncthreads();
    double minpiv = 1e300;
    int neg = 0;
    for (int p = 0; p < nb; ++p) {
        const c128 piv = blk[p + p * NB];
        const double a2 = abs2(piv);
        if (tid == 0) {
            minpiv = fmin(minpiv, sqrt(a2));
            neg += piv.re < 0.0 ? 1 : 0;
            if (!(a2 > 0.0) || !isfinite(a2)) atomicOr(g.err, 1);
        }
        const c128 ip = (a2 > 0.0 && isfinite(a2)) ? cdiv(mk<double>(1, 0), piv) : mk<double>(0, 0);
        for (int i = p + 1 + tid; i < nb; i += 256) blk[i + p * NB] = blk[i + p * NB] * ip;
        __syncthreads();
        const int r = nb - p - 1;
        for (int e = tid; e < r * r; e += 256) {
            const int i = p + 1 + e % r, j = p + 1 + e / r;
            blk[i + j * NB] = blk[i + j * NB] - blk[i + p * NB] * blk[p + j * NB];
        }
        __syncthreads();
    }
    if (tid == 0) {
        g.minpiv[(int64_t)z * g.njobs + blockIdx.x] = minpiv;
        if (g.negcnt) atomicAdd(g.negcnt + z, neg);
    }
    cx<T> *Li = g.inv[z] + J.inv;
    cx<T> *Ui = Li + NB * NB;
    // Linv: column j solves L x = e_j (unit lower)
    if (tid < nb) {
        const int j = tid;
        X[j + j * NB] = mk<double>(1, 0);
        for (int i = j + 1; i < nb; ++i) {
            c128 s = mk<double>(0, 0);
            for (int t = j; t < i; ++t) fma_acc(s, blk[i + t * NB], X[t + j * NB]);
            X[i + j * NB] = mk<double>(-s.re, -s.im);
        }
    }
    __syncthreads();
    for (int e = tid; e < nb * nb; e += 256) {
        const int i = e % nb, j = e / nb;
        Li[i + j * NB] = (i >= j) ? cvt<T>(X[i + j * NB]) : mk<T>(0, 0);
    }
    __syncthreads();
    // Uinv: column j solves U x = e_j (upper)
    if (tid < nb) {
        const int j = tid;
        X[j + j * NB] = cdiv(mk<double>(1, 0), blk[j + j * NB]);
        for (int i = j - 1; i >= 0; --i) {
            c128 s = mk<double>(0, 0);
            for (int t = i + 1; t <= j; ++t) fma_acc(s, blk[i + t * NB], X[t + j * NB]);
            X[i + j * NB] = cdiv(mk<double>(-s.re, -s.im), blk[i + i * NB]);
        }
    }
    __syncthreads();
    for (int e = tid; e < nb * nb; e += 256) {
        const int i = e % nb, j = e / nb;
        Ui[i + j * NB] = (i <= j) ? cvt<T>(X[i + j * NB]) : mk<T>(0, 0);
        F[i + (int64_t)j * J.ld] = cvt<T>(blk[i + j * NB]);
    }
}

template <class T>
void launch_diag_lu(const DiagArgs<T> &g, int ninst, cudaStream_t st) {
    if (g.njobs == 0) return;
    const size_t smem = 2 * NB * NB * sizeof(c128);
    static bool attr_set[64] = {};                  // per device: the kernel's shared-memory opt-in
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        cudaFuncSetAttribute(k_diag_lu<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set[dev] = true;
    }
    dim3 grid(g.njobs, 1, ninst);
    k_diag_lu<T><<<grid, 256, smem, st>>>(g);
    count_launch();
}

// ============================================================== assembly
// F[dst[e]] += scale_z * val[src[e]]  (entries of A, then of B with scale -sigma_z)
template <class T>
__global__ void k_assemble(AsmArgs<T> g) {
    const int z = blockIdx.z;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= g.count) return;
    const c128 v = g.val[g.src[e]];
    const c128 s = g.scale[z];
    cx<T> *p = g.pool[z] + g.dst[e];
    *p = *p + cvt<T>(s * v);
}

template <class T>
void launch_assemble(const AsmArgs<T> &g, int ninst, cudaStream_t st) {
    if (g.count == 0) return;
    dim3 grid((unsigned)((g.count + 255) / 256), 1, ninst);
    k_assemble<T><<<grid, 256, 0, st>>>(g);
    count_launch();
}

// ============================================================== matrix extend-add
// Parent front += child's Schur block, scattered through the child's relative map:
// F_p[rel[i] + rel[j] ld_p] += F_c[i + j ld_c]  over a 32 x 32 tile per CTA.
template <class T>
__global__ void __launch_bounds__(256) k_extend_add(EaddArgs<T> g) {
    const int z = blockIdx.z;
    const int tile = blockIdx.x;
    if (tile >= g.ntiles) return;
    __shared__ int s_job;
    if (threadIdx.x == 0) s_job = find_rjob(g.tmap, g.jobs, g.njobs, tile);
    __syncthreads();
    const RJob J = g.jobs[s_job];
    const int t = tile - J.tile0;
    const int bi = (t % J.tr) * 32, bj = (t / J.tr) * 32;
    const int32_t *rel = g.rel + J.map;
    const cx<T> *S = g.pool[z] + J.src;
    cx<T> *P = g.pool[z] + J.dst;
    const int i = bi + (threadIdx.x & 31);
    if (i >= J.rows) return;
    const int ri = rel[i];
    cx<T> v[4];
    cx<T> *p[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {                    // loads first, then the stores
        const int j = bj + (threadIdx.x >> 5) + 8 * q;
        p[q] = nullptr;
        if (j < J.rows) {
            p[q] = P + ri + (int64_t)rel[j] * J.ld_dst;
            v[q] = *p[q] + S[i + (int64_t)j * J.ld_src];
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (p[q]) *p[q] = v[q];
}

template <class T>
void launch_extend_add(const EaddArgs<T> &g, int ninst, cudaStream_t st) {
    if (g.ntiles == 0) return;
    dim3 grid(g.ntiles, 1, ninst);
    k_extend_add<T><<<grid, 256, 0, st>>>(g);
    count_launch();
}

// ============================================================== row moves
// mode ROW_GATHER : W[dst + r ldw + c]            = X[map[r] ldx + c]     (X c128 -> W T)
// mode ROW_SCATTER: X[map[r] ldx + c]             = W[src + r ldw + c]    (W T -> X c128)
// mode ROW_EADD   : W[dst + map[r] ldw + c]      += W[src + r ldw + c]    (child -> parent)
template <class T>
__global__ void __launch_bounds__(256) k_rows(RowArgs<T> g) {
    const int z = blockIdx.z;
    const int tile = blockIdx.x;
    if (tile >= g.ntiles) return;
    __shared__ int s_job;
    if (threadIdx.x == 0) s_job = find_rjob(g.tmap, g.jobs, g.njobs, tile);
    __syncthreads();
    const RJob J = g.jobs[s_job];
    const int r0 = (tile - J.tile0) * g.rpt;
    const int32_t *map = g.map + J.map;
    const int k = g.k;
    cx<T> *W = g.W[z];
    c128 *X = g.X[z];
    if (g.mode == ROW_EADD) {
        // batches of 8 elements per thread: all loads, then the stores (an interleaved
        // read-modify-write would wait one global round trip per element)
        for (int e0 = 0; e0 < g.rpt * k; e0 += 8 * 256) {
            cx<T> v[8];
            cx<T> *p[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = e0 + threadIdx.x + 256 * q;
                const int rr = e / k, c = e - rr * k, r = r0 + rr;
                p[q] = nullptr;
                if (e < g.rpt * k && r < J.rows) {
                    p[q] = W + J.dst + (int64_t)map[r] * g.ldw + c;
                    v[q] = *p[q] + W[J.src + (int64_t)r * g.ldw + c];
                }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (p[q]) *p[q] = v[q];
        }
        return;
    }
    for (int e = threadIdx.x; e < g.rpt * k; e += 256) {
        const int rr = e / k, c = e - rr * k;
        const int r = r0 + rr;
        if (r >= J.rows) break;
        if (g.mode == ROW_GATHER) {
            W[J.dst + (int64_t)r * g.ldw + c] = cvt<T>(X[(int64_t)map[r] * g.ldx + c]);
        } else if (g.mode == ROW_SCATTER) {
            X[(int64_t)map[r] * g.ldx + c] = cvt<double>(W[J.src + (int64_t)r * g.ldw + c]);
        } else {
            W[J.dst + (int64_t)r * g.ldw + c] = mk<T>(0, 0);
        }
    }
}

template <class T>
void launch_rows(const RowArgs<T> &g, int ninst, cudaStream_t st) {
    if (g.ntiles == 0) return;
    dim3 grid(g.ntiles, 1, ninst);
    k_rows<T><<<grid, 256, 0, st>>>(g);
    count_launch();
}

// ============================================================== identity starts
template <class T>
__global__ void __launch_bounds__(256) k_eye_blocks(EyeArgs<T> g) {
    const int z = blockIdx.z;
    const int tile = blockIdx.x;
    if (tile >= g.ntiles) return;
    __shared__ int s_job;
    if (threadIdx.x == 0) s_job = find_rjob(g.tmap, g.jobs, g.njobs, tile);
    __syncthreads();
    const RJob J = g.jobs[s_job];
    const int i = (tile - J.tile0) * 256 + threadIdx.x;
    if (i >= J.rows) return;
    const int64_t r = J.rows;
    g.P[z][J.dst + i * (r + 1)] = mk<T>(1, 0);
    g.P[z][J.dst + r * r + i * (r + 1)] = mk<T>(1, 0);
}

template <class T>
void launch_eye(const EyeArgs<T> &g, int ninst, cudaStream_t st) {
    if (g.ntiles == 0) return;
    dim3 grid(g.ntiles, 1, ninst);
    k_eye_blocks<T><<<grid, 256, 0, st>>>(g);
    count_launch();
}

// ============================================================== SpMM
// Y[i, c] = s * sum_e M[i, col_e] X[col_e, c] (+ Y[i, c] if acc), complex128, row-major
// blocks.  One warp per row, lanes across the k columns (each nonzero reads a
// contiguous row of X).
__global__ void __launch_bounds__(256) k_spmm(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                              const c128 *__restrict__ v, int64_t n, int k,
                                              const c128 *__restrict__ X, int64_t ldx, c128 *__restrict__ Y,
                                              int64_t ldy, c128 s, int acc) {
    const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= n) return;
    const int lane = threadIdx.x & 31;
    const int64_t b = rp[row], e = rp[row + 1];
    for (int c = lane; c < k; c += 32) {
        c128 sum = mk<double>(0, 0);
        for (int64_t p = b; p < e; ++p) fma_acc(sum, v[p], X[(int64_t)ci[p] * ldx + c]);
        c128 *y = Y + row * ldy + c;
        *y = acc ? (*y + s * sum) : (s * sum);
    }
}

// real-valued matrix (e.g. a mass matrix): 2 real FMAs per entry instead of 4
__global__ void __launch_bounds__(256) k_spmm_real(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                   const double *__restrict__ v, int64_t n, int k,
                                                   const c128 *__restrict__ X, int64_t ldx, c128 *__restrict__ Y,
                                                   int64_t ldy, c128 s, int acc) {
    const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= n) return;
    const int lane = threadIdx.x & 31;
    const int64_t b = rp[row], e = rp[row + 1];
    for (int c = lane; c < k; c += 32) {
        double sr = 0.0, si = 0.0;
        for (int64_t p = b; p < e; ++p) {
            const double a = v[p];
            const c128 x = X[(int64_t)ci[p] * ldx + c];
            sr = fma(a, x.re, sr);
            si = fma(a, x.im, si);
        }
        c128 *y = Y + row * ldy + c;
        const c128 t = s * mk<double>(sr, si);
        *y = acc ? (*y + t) : t;
    }
}

void launch_spmm(const DevCSR &M, int64_t k, const c128 *X, int64_t ldx, c128 *Y, int64_t ldy, c128 s,
                 bool acc, cudaStream_t st) {
    if (M.n == 0 || k == 0) return;
    dim3 grid((unsigned)((M.n + 7) / 8));
    if (M.vr)
        k_spmm_real<<<grid, 256, 0, st>>>(M.rp, M.ci, M.vr, M.n, (int)k, X, ldx, Y, ldy, s, acc ? 1 : 0);
    else
        k_spmm<<<grid, 256, 0, st>>>(M.rp, M.ci, M.v, M.n, (int)k, X, ldx, Y, ldy, s, acc ? 1 : 0);
    count_launch();
}

// Refinement residuals of all instances in one pass over the rows of A and M
__global__ void __launch_bounds__(256) k_refine_resid(DevCSR A, DevCSR M, ResidArgs r) {
    const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= A.n) return;
    const int lane = threadIdx.x & 31;
    const int64_t ab = A.rp[row], ae = A.rp[row + 1], mb = M.rp[row], me = M.rp[row + 1];
    for (int z = 0; z < r.ninst; ++z) {
        const c128 *X = r.Xz[z];
        for (int c = lane; c < r.k; c += 32) {
            c128 ax = mk<double>(0, 0);
            if (A.vr) {                                  // real matrix: 2 FMAs per entry instead of 4
                for (int64_t p = ab; p < ae; ++p) {
                    const c128 x = X[(int64_t)A.ci[p] * r.ldx + c];
                    ax.re = fma(A.vr[p], x.re, ax.re);
                    ax.im = fma(A.vr[p], x.im, ax.im);
                }
            } else {
                for (int64_t p = ab; p < ae; ++p) fma_acc(ax, A.v[p], X[(int64_t)A.ci[p] * r.ldx + c]);
            }
            double mr = 0.0, mi = 0.0;
            c128 mx = mk<double>(0, 0);
            if (M.vr) {
                for (int64_t p = mb; p < me; ++p) {
                    const c128 x = X[(int64_t)M.ci[p] * r.ldx + c];
                    mr = fma(M.vr[p], x.re, mr);
                    mi = fma(M.vr[p], x.im, mi);
                }
                mx = mk<double>(mr, mi);
            } else {
                for (int64_t p = mb; p < me; ++p) fma_acc(mx, M.v[p], X[(int64_t)M.ci[p] * r.ldx + c]);
            }
            const c128 b = r.Bz[z][row * r.ldb + c];
            r.Rz[z][row * r.ldr + c] = b - ax + r.s[z] * mx;
        }
    }
}

void launch_refine_resid(const DevCSR &A, const DevCSR &M, const ResidArgs &r, cudaStream_t st) {
    if (A.n == 0 || r.k == 0 || r.ninst == 0) return;
    k_refine_resid<<<(unsigned)((A.n + 7) / 8), 256, 0, st>>>(A, M, r);
    count_launch();
}

// Double-float variant: the sums over the rows of A and M, sigma M x and b - A x + sigma M x
// all in df64 on the FP32 pipe (no FP64 instruction per non-zero).
__global__ void __launch_bounds__(256) k_refine_resid_df(DevCSR A, DevCSR M, ResidDfArgs r) {
    const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= A.n) return;
    const int lane = threadIdx.x & 31;
    const int64_t ab = A.rp[row], ae = A.rp[row + 1], mb = M.rp[row], me = M.rp[row + 1];
    for (int z = 0; z < r.ninst; ++z) {
        const float4 *__restrict__ X = r.Xs[z];
        const float4 sg = r.s[z];
        for (int c = lane; c < r.k; c += 32) {
            float arh = 0.f, arl = 0.f, aih = 0.f, ail = 0.f;     // A x
            if (A.vrdf) {
                for (int64_t p = ab; p < ae; ++p) {
                    const float2 a = A.vrdf[p];
                    const float4 x = X[(int64_t)A.ci[p] * r.k + c];
                    df_fma(arh, arl, a.x, a.y, x.x, x.y);
                    df_fma(aih, ail, a.x, a.y, x.z, x.w);
                }
            } else {
                for (int64_t p = ab; p < ae; ++p) {
                    const float4 a = A.vdf[p];
                    const float4 x = X[(int64_t)A.ci[p] * r.k + c];
                    df_fma(arh, arl, a.x, a.y, x.x, x.y);             // ar xr
                    df_fma(arh, arl, -a.z, -a.w, x.z, x.w);           // - ai xi
                    df_fma(aih, ail, a.x, a.y, x.z, x.w);             // ar xi
                    df_fma(aih, ail, a.z, a.w, x.x, x.y);             // ai xr
                }
            }
            float mrh = 0.f, mrl = 0.f, mih = 0.f, mil = 0.f;     // M x
            if (M.vrdf) {
                for (int64_t p = mb; p < me; ++p) {
                    const float2 a = M.vrdf[p];
                    const float4 x = X[(int64_t)M.ci[p] * r.k + c];
                    df_fma(mrh, mrl, a.x, a.y, x.x, x.y);
                    df_fma(mih, mil, a.x, a.y, x.z, x.w);
                }
            } else {
                for (int64_t p = mb; p < me; ++p) {
                    const float4 a = M.vdf[p];
                    const float4 x = X[(int64_t)M.ci[p] * r.k + c];
                    df_fma(mrh, mrl, a.x, a.y, x.x, x.y);
                    df_fma(mrh, mrl, -a.z, -a.w, x.z, x.w);
                    df_fma(mih, mil, a.x, a.y, x.z, x.w);
                    df_fma(mih, mil, a.z, a.w, x.x, x.y);
                }
            }
            df_norm(mrh, mrl);
            df_norm(mih, mil);
            // t = b - A x + s (M x)
            const c128 b = r.Bz[z][row * r.ldb + c];
            float trh, trl, tih, til;
            df_split(b.re, trh, trl);
            df_split(b.im, tih, til);
            df_add(trh, trl, -arh, -arl);
            df_add(tih, til, -aih, -ail);
            df_fma(trh, trl, sg.x, sg.y, mrh, mrl);                 // sr (Mx)r
            df_fma(trh, trl, -sg.z, -sg.w, mih, mil);               // - si (Mx)i
            df_fma(tih, til, sg.x, sg.y, mih, mil);                 // sr (Mx)i
            df_fma(tih, til, sg.z, sg.w, mrh, mrl);                 // si (Mx)r
            r.Rz[z][row * r.ldr + c] = mk<double>(df_widen(__fadd_rn(trh, trl)), df_widen(__fadd_rn(tih, til)));
        }
    }
}

void launch_refine_resid_df(const DevCSR &A, const DevCSR &M, const ResidDfArgs &r, cudaStream_t st) {
    if (A.n == 0 || r.k == 0 || r.ninst == 0) return;
    k_refine_resid_df<<<(unsigned)((A.n + 7) / 8), 256, 0, st>>>(A, M, r);
    count_launch();
}

__global__ void __launch_bounds__(256) k_spmm_df(DevCSR M, int k, const float2 *__restrict__ Xs,
                                                 c128 *__restrict__ Y) {
    const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= M.n) return;
    const int lane = threadIdx.x & 31;
    const int64_t b = M.rp[row], e = M.rp[row + 1], nk = M.n * k;
    for (int c = lane; c < k; c += 32) {
        float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
        if (M.vrdf) {
            for (int64_t p = b; p < e; ++p) {
                const float2 a = M.vrdf[p];
                const int64_t x = (int64_t)M.ci[p] * k + c;
                const float2 xh = Xs[x], xl = Xs[nk + x];
                df_fma(rh, rl, a.x, a.y, xh.x, xl.x);
                df_fma(ih, il, a.x, a.y, xh.y, xl.y);
            }
        } else {
            for (int64_t p = b; p < e; ++p) {
                const float4 a = M.vdf[p];
                const int64_t x = (int64_t)M.ci[p] * k + c;
                const float2 xh = Xs[x], xl = Xs[nk + x];
                df_fma(rh, rl, a.x, a.y, xh.x, xl.x);             // ar xr
                df_fma(rh, rl, -a.z, -a.w, xh.y, xl.y);           // - ai xi
                df_fma(ih, il, a.x, a.y, xh.y, xl.y);             // ar xi
                df_fma(ih, il, a.z, a.w, xh.x, xl.x);             // ai xr
            }
        }
        Y[row * k + c] = mk<double>(df_widen(rh) + df_widen(rl), df_widen(ih) + df_widen(il));
    }
}

void launch_spmm_df(const DevCSR &M, int64_t k, const float2 *Xs, c128 *Y, cudaStream_t st) {
    if (M.n == 0 || k == 0) return;
    k_spmm_df<<<(unsigned)((M.n + 7) / 8), 256, 0, st>>>(M, (int)k, Xs, Y);
    count_launch();
}

__global__ void k_split_df(int64_t n, int k, const c128 *__restrict__ X, int64_t ldx, float4 *__restrict__ Xs) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * k) return;
    const int64_t i = idx / k, c = idx - i * k;
    const c128 x = X[i * ldx + c];
    float4 o;
    df_split(x.re, o.x, o.y);
    df_split(x.im, o.z, o.w);
    Xs[idx] = o;
}

void launch_split_df(int64_t n, int64_t k, const c128 *X, int64_t ldx, float4 *Xs, cudaStream_t st) {
    const int64_t tot = n * k;
    if (tot == 0) return;
    k_split_df<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, (int)k, X, ldx, Xs);
    count_launch();
}

// ============================================================== elementwise
// Y = sum_t coef[t] * X_t   (t < nterm, every operand n x k with its own ld)
__global__ void k_lincomb(LinArgs a) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.n * a.k) return;
    const int64_t i = idx / a.k, c = idx - i * a.k;
    c128 s = mk<double>(0, 0);
    for (int t = 0; t < a.nterm; ++t) fma_acc(s, a.coef[t], a.X[t][i * a.ldx[t] + c]);
    if (a.real_out) s.im = 0.0;
    a.Y[i * a.ldy + c] = s;
}

void launch_lincomb(const LinArgs &a, cudaStream_t st) {
    const int64_t tot = a.n * a.k;
    if (tot == 0) return;
    k_lincomb<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(a);
    count_launch();
}

// ============================================================== column norms
// stage 1: CTA b sums a contiguous chunk of rows into part[b * k + c]: for k <= 256 the
// threads form 256 / k row groups of k consecutive columns, so a warp reads consecutive
// addresses of a row-major block; the groups' sums are added in a fixed order through shared
// memory.  stage 2: one warp per column adds the COLNORM_PARTS partial sums (fixed order:
// deterministic).
__global__ void __launch_bounds__(256) k_colnorm_part(int64_t n, int k, const c128 *__restrict__ X, int64_t ldx,
                                                      double *__restrict__ part, int imag_only) {
    __shared__ double red[256];
    const int64_t rpc = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rpc, r1 = r0 + rpc < n ? r0 + rpc : n;
    if (k <= 256) {
        const int rpp = 256 / k, c = threadIdx.x % k, rr = threadIdx.x / k;
        double s = 0.0;
        if (rr < rpp) {
            if (imag_only)
                for (int64_t i = r0 + rr; i < r1; i += rpp) s = fma(X[i * ldx + c].im, X[i * ldx + c].im, s);
            else
                for (int64_t i = r0 + rr; i < r1; i += rpp) s += abs2(X[i * ldx + c]);
        }
        red[threadIdx.x] = s;
        __syncthreads();
        if (threadIdx.x < k) {
            double t = 0.0;
            for (int q = 0; q < rpp; ++q) t += red[q * k + threadIdx.x];
            part[(int64_t)blockIdx.x * k + threadIdx.x] = t;
        }
        return;
    }
    for (int c = threadIdx.x; c < k; c += 256) {
        double s = 0.0;
        if (imag_only)
            for (int64_t i = r0; i < r1; ++i) s = fma(X[i * ldx + c].im, X[i * ldx + c].im, s);
        else
            for (int64_t i = r0; i < r1; ++i) s += abs2(X[i * ldx + c]);
        part[(int64_t)blockIdx.x * k + c] = s;
    }
}
__global__ void __launch_bounds__(256) k_colnorm_sum(int k, int parts, const double *__restrict__ part,
                                                     double *__restrict__ out) {
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (c >= k) return;
    double s = 0.0;
    for (int b = lane; b < parts; b += 32) s += part[(int64_t)b * k + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[c] = s;
}

void launch_colnorm2(int64_t n, int64_t k, const c128 *X, int64_t ldx, double *out, double *part, cudaStream_t st,
                     bool imag_only) {
    if (k <= 0) return;
    k_colnorm_part<<<COLNORM_PARTS, 256, 0, st>>>(n, (int)k, X, ldx, part, imag_only ? 1 : 0);
    k_colnorm_sum<<<(unsigned)((k + 7) / 8), 256, 0, st>>>((int)k, COLNORM_PARTS, part, out);
    count_launch(2);
}

// ============================================================== square transposes
template <class T>
__global__ void __launch_bounds__(256) k_transpose_sq(EyeArgs<T> g) {
    const int z = blockIdx.z;
    const int tile = blockIdx.x;
    if (tile >= g.ntiles) return;
    __shared__ int s_job;
    __shared__ cx<T> ta[32][33], tb[32][33];
    if (threadIdx.x == 0) s_job = find_rjob(g.tmap, g.jobs, g.njobs, tile);
    __syncthreads();
    const RJob J = g.jobs[s_job];
    int loc = tile - J.tile0, bi = 0;
    while (loc >= J.tr - bi) {            // row bi of the upper triangle holds tr - bi tile pairs
        loc -= J.tr - bi;
        ++bi;
    }
    const int bj = bi + loc;
    const int64_t n = J.rows;
    cx<T> *M = g.P[z] + J.dst;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
        const int64_t i1 = 32 * bi + r, j1 = 32 * bj + tx;      // (bi, bj) tile
        const int64_t i2 = 32 * bj + r, j2 = 32 * bi + tx;      // (bj, bi) tile
        if (i1 < n && j1 < n) ta[r][tx] = M[i1 + j1 * n];
        if (i2 < n && j2 < n) tb[r][tx] = M[i2 + j2 * n];
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t i1 = 32 * bi + r, j1 = 32 * bj + tx;
        const int64_t i2 = 32 * bj + r, j2 = 32 * bi + tx;
        if (i1 < n && j1 < n) M[i1 + j1 * n] = tb[tx][r];        // M(i1, j1) <- old M(j1, i1)
        if (i2 < n && j2 < n) M[i2 + j2 * n] = ta[tx][r];
    }
}

template <class T>
void launch_transpose_sq(const EyeArgs<T> &g, int ninst, cudaStream_t st) {
    if (g.ntiles == 0) return;
    dim3 grid(g.ntiles, 1, ninst);
    k_transpose_sq<T><<<grid, 256, 0, st>>>(g);
    count_launch();
}

// explicit instantiations
template void launch_gemm<double>(const GemmArgs<double> &, int, cudaStream_t, double, double);
template void launch_gemm<float>(const GemmArgs<float> &, int, cudaStream_t, double, double);
template void launch_diag_lu<double>(const DiagArgs<double> &, int, cudaStream_t);
template void launch_diag_lu<float>(const DiagArgs<float> &, int, cudaStream_t);
template void launch_assemble<double>(const AsmArgs<double> &, int, cudaStream_t);
template void launch_assemble<float>(const AsmArgs<float> &, int, cudaStream_t);
template void launch_extend_add<double>(const EaddArgs<double> &, int, cudaStream_t);
template void launch_extend_add<float>(const EaddArgs<float> &, int, cudaStream_t);
template void launch_rows<double>(const RowArgs<double> &, int, cudaStream_t);
template void launch_eye<double>(const EyeArgs<double> &, int, cudaStream_t);
template void launch_eye<float>(const EyeArgs<float> &, int, cudaStream_t);
template void launch_transpose_sq<double>(const EyeArgs<double> &, int, cudaStream_t);
template void launch_transpose_sq<float>(const EyeArgs<float> &, int, cudaStream_t);
template void launch_rows<float>(const RowArgs<float> &, int, cudaStream_t);

}  // namespace zolo
