// Complex64 batched GEMM on the 5th-generation tensor cores (tcgen05, kind::tf32).
//
// Same job semantics as k_gemm / k_gemm_c64 (C (=|-=|+=) op(A) op(B) per job, split-K by
// atomic adds, in-place when C aliases A with n <= the tile width or B with m <= 128), used
// for the front updates and block solves of the multifrontal factor (Section 2.3) in the
// mixed-precision mode.
//
// Arithmetic: every complex64 operand x is split into two TF32 numbers, x = hi + lo with
// hi = x rounded to 11 significant bits and lo = (x - hi) rounded the same way (3xTF32:
// the products hi*hi + hi*lo + lo*hi are accumulated in FP32 in tensor memory, the
// lo*lo term, at most 2^-24 of the product, is dropped).  The real and imaginary parts of a
// w-column C tile sit side by side in one 2w-column accumulator D = [Cr | Ci], and the B
// operand is staged as four 2w-row planes
//      B0 = [Br_hi ; Bi_hi], B1 = [Br_lo ; Bi_lo], B2 = [-Bi_hi ; Br_hi], B3 = [-Bi_lo ; Br_lo],
// so one k-step of 8 is six MMAs of 128 x 2w x 8:
//      D += Ar_hi B0 + Ar_hi B1 + Ar_lo B0 + Ai_hi B2 + Ai_hi B3 + Ai_lo B2,
// which gives Cr = Ar Br - Ai Bi and Ci = Ar Bi + Ai Br (conjugated operands are conjugated
// while they are staged).  The tensor core's FP32 accumulation truncates, so products are
// ~5-10x less accurate than with FP32 FMAs (~1e-6 relative at k = 64); the FP64 refinement of
// every mixed-precision solve absorbs this.
//
// Pre-split operands: a job flagged GJ_PRESPLIT (the block solves' column-major factor
// operands, mixed precision) has its A already stored as the four TF32 planes of every
// 128 x 8 stage (16 KB blocks, k_presplit below, built once per factorisation).  Its A stage
// is then one bulk copy straight into the MMA stage (thread 0 adds the bytes to the stage's
// "full" mbarrier), and the converters only split B: no A staging, no A conversion.
//
// Tiles: one CTA per 128 x w tile of C, w <= 128 columns chosen per job so that the
// ceil(n / 128) column tiles have equal width (a multiple of 16); 256 tensor-memory columns
// per CTA.
//
// Pipeline (warp-specialised): eight converter warps stream the operands through a ring of
// P raw stages (k = 8 complex each) filled by cp.async (8-byte copies with zero fill at the
// edges), P - 1 stages in flight; each converts the oldest raw stage (conjugation, hi/lo
// split) into one of NB MMA stages in the canonical no-swizzle K-major layout and arrives on
// that stage's "full" mbarrier.  A ninth warp issues each stage's six MMAs once it is full and
// commits them to the stage's "empty" mbarrier, which the converters wait on before they
// overwrite it, so the MMA issue never holds up the conversion.  The plan depends on the
// widest tile of the launch (WMAX = 32, 64, 128: NB = 3, 2, 2 and P = 4, 4, 3), two CTAs per
// SM; 128-wide tiles keep Cr and Ci in separate accumulators (twelve MMAs of N = w per
// k-step) to fit.  Every wait on an mbarrier is bounded in time (2 s): on expiry the thread skips
// its remaining waits, the CTA skips its epilogue, records ZOLO_ETIMEOUT in a device status
// word (read by gemm_tc_status) and releases its tensor memory.
#include "kernels.cuh"
#include "zolo.h"

#include <cstdint>

namespace zolo {

namespace {

constexpr int TC_BM = 128;                 // rows of a C tile (MMA M)
constexpr int TC_BN = 128;                 // widest C tile (MMA N)
constexpr int TC_BK = 8;                   // complex k-extent of a stage (one MMA k-step)
constexpr int TC_PLANE_A = TC_BM * TC_BK * 4;        // bytes of one A plane (4 KB)
constexpr uint32_t TC_TMEM_COLS = 256;
constexpr uint64_t TC_WAIT_NS = 2000000000ull;              // 2 s per mbarrier wait at most

// Shared-memory plan of a launch whose tiles are at most WMAX wide.
template <int WMAX> struct TcPlan {
    // FUSED: [Cr | Ci] in one 2w-column accumulator, six MMAs of N = 2w per k-step (B staged
    // as 2w-row planes); otherwise Cr and Ci in separate 128-column accumulators, twelve MMAs
    // of N = w (w-row B planes, -Ai Bi through the instruction's negate-A bit), which keeps
    // the 128-wide tiles of the factorisation at two CTAs per SM
    static constexpr bool FUSED = WMAX <= 64;
    static constexpr int PLANE_B = (FUSED ? 2 : 1) * WMAX * TC_BK * 4;
    static constexpr int MMA_STAGE = 4 * TC_PLANE_A + 4 * PLANE_B;   // A and B planes of a k-step
    static constexpr int RAW_A = TC_BM * TC_BK * 8;                   // raw complex64 A stage (8 KB)
    static constexpr int RAW_STAGE = RAW_A + WMAX * TC_BK * 8;
    static constexpr int CTAS = 2;                                    // CTAs per SM
    // MMA stages (a pre-split A stage is in flight only while its MMA stage waits: three of
    // them for the 32-wide solve tiles) and raw stages in the ring
    static constexpr int NB = WMAX <= 32 ? 3 : 2;
    static constexpr int P = WMAX <= 32 ? 4 : (WMAX <= 64 ? 4 : 3);
    static constexpr int BAR = 128;                                   // mbarriers, TMEM slot, job
    static constexpr int SMEM = NB * MMA_STAGE + P * RAW_STAGE + BAR;
    static_assert(SMEM * CTAS + 1024 * CTAS <= 233472, "shared memory plan too large");
};
constexpr int TC_THREADS = 288;              // 8 converter warps + 1 MMA warp

__device__ int g_tc_status = 0;

// Byte offset of the 4-element group q (kk = 4q .. 4q+3, q < 2) of row `row` inside a plane
// in the canonical no-swizzle K-major layout: 8-row x 16-byte core matrices stored
// contiguously (128 B each), the two core matrices of a row group adjacent along K
// (LBO = 128 B) and row groups 256 B apart (SBO).
__device__ __forceinline__ uint32_t core_off(int row, int q) {
    return (uint32_t)(((row >> 3) * 2 + q) * 128 + (row & 7) * 16);
}

// Shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), version 1,
// no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    const uint64_t lbo = 128 >> 4, sbo = 256 >> 4;
    return (uint64_t)((addr & 0x3FFFF) >> 4) | (lbo << 16) | (sbo << 32) | (1ull << 46);
}

// Instruction descriptor for kind::tf32: FP32 accumulator, TF32 A and B, both K-major,
// N = n, M = 128, optional negation of A.
__device__ __forceinline__ uint32_t instr_desc(int n, bool neg_a) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (neg_a ? (1u << 13) : 0u) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// Non-blocking test of a phase (test_wait never suspends the thread, so a completed phase is
// seen at the next poll).
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait for the given phase parity, for TC_WAIT_NS of wall time at most (the bound is on
// time, not on polls); false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    while (!mbar_try(mbar, parity))
        if (global_ns() - t0 > TC_WAIT_NS) return false;
    return true;
}

__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// x rounded to TF32 (11 significant bits), ties away from zero, with two integer
// operations (full-rate ALU; a cvt.rna.tf32 conversion per operand was measured slower).
__device__ __forceinline__ float tf32_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Four complex values (one row, four consecutive kk) split and stored into the four
// planes (re hi, re lo, im hi, im lo) at byte offset `off`.
__device__ __forceinline__ void put4(unsigned char *planes, int plane_bytes, uint32_t off, const c64 *v) {
    float rh[4], rl[4], ih[4], il[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        rh[e] = tf32_round(v[e].re);
        rl[e] = tf32_round(v[e].re - rh[e]);
        ih[e] = tf32_round(v[e].im);
        il[e] = tf32_round(v[e].im - ih[e]);
    }
    *reinterpret_cast<float4 *>(planes + off) = make_float4(rh[0], rh[1], rh[2], rh[3]);
    *reinterpret_cast<float4 *>(planes + plane_bytes + off) = make_float4(rl[0], rl[1], rl[2], rl[3]);
    *reinterpret_cast<float4 *>(planes + 2 * plane_bytes + off) = make_float4(ih[0], ih[1], ih[2], ih[3]);
    *reinterpret_cast<float4 *>(planes + 3 * plane_bytes + off) = make_float4(il[0], il[1], il[2], il[3]);
}

// Complex element (row, l) of a raw A stage, l < 8, as a complex64 index: the four k of a
// (row, q = l / 4) unit sit in two 16-byte halves h = (l / 2) % 2, and unit u is the thread
// index that converts it, so each half is read by the warp as one contiguous 512-byte run.
__device__ __forceinline__ int raw_index(int row, int l, int units) {
    const int q = l >> 2, h = (l >> 1) & 1, e = l & 1;
    const int u = (((row >> 3) << 1) + q) * 8 + (row & 7);
    return h * 2 * units + u * 2 + e;
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void converters_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Split four complex B values (row j of the w-row tile, one k-group) into the four 2w-row
// planes B0 = [Br_hi ; Bi_hi], B1 = [Br_lo ; Bi_lo], B2 = [-Bi_hi ; Br_hi], B3 = [-Bi_lo ; Br_lo].
__device__ __forceinline__ void put4_b(unsigned char *planes, int plane_bytes, uint32_t off_top, uint32_t off_bot,
                                       const c64 *v) {
    float rh[4], rl[4], ih[4], il[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        rh[e] = tf32_round(v[e].re);
        rl[e] = tf32_round(v[e].re - rh[e]);
        ih[e] = tf32_round(v[e].im);
        il[e] = tf32_round(v[e].im - ih[e]);
    }
    unsigned char *p0 = planes, *p1 = planes + plane_bytes, *p2 = planes + 2 * plane_bytes,
                  *p3 = planes + 3 * plane_bytes;
    *reinterpret_cast<float4 *>(p0 + off_top) = make_float4(rh[0], rh[1], rh[2], rh[3]);
    *reinterpret_cast<float4 *>(p0 + off_bot) = make_float4(ih[0], ih[1], ih[2], ih[3]);
    *reinterpret_cast<float4 *>(p1 + off_top) = make_float4(rl[0], rl[1], rl[2], rl[3]);
    *reinterpret_cast<float4 *>(p1 + off_bot) = make_float4(il[0], il[1], il[2], il[3]);
    *reinterpret_cast<float4 *>(p2 + off_top) = make_float4(-ih[0], -ih[1], -ih[2], -ih[3]);
    *reinterpret_cast<float4 *>(p2 + off_bot) = make_float4(rh[0], rh[1], rh[2], rh[3]);
    *reinterpret_cast<float4 *>(p3 + off_top) = make_float4(-il[0], -il[1], -il[2], -il[3]);
    *reinterpret_cast<float4 *>(p3 + off_bot) = make_float4(rl[0], rl[1], rl[2], rl[3]);
}

template <int WMAX>
__global__ void __launch_bounds__(TC_THREADS, TcPlan<WMAX>::CTAS) k_gemm_tc(GemmArgs<float> g) {
    using PL = TcPlan<WMAX>;
    constexpr int P = PL::P, NB = PL::NB;
    const int z = blockIdx.z;
    const int tile = blockIdx.x;
    if (tile >= g.ntiles[z]) return;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *raw = smem + NB * PL::MMA_STAGE;
    unsigned char *ctl = raw + P * PL::RAW_STAGE;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(ctl);                 // full[0..NB), empty[0..NB)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(ctl + 16 * NB);
    int *s_job = reinterpret_cast<int *>(ctl + 16 * NB + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const GJob *jobs = g.jobs[z];
    if (tid == 0) {
        if (g.tmap[z]) {
            *s_job = g.tmap[z][tile];
        } else {
            int lo = 0, hi = g.njobs[z] - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (jobs[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
            }
            *s_job = lo;
        }
    }
    __syncthreads();
    const GJob J = jobs[*s_job];
    int t = tile - J.tile0;
    const int ntn = (J.n + TC_BN - 1) / TC_BN;
    const int w = ((J.n + ntn - 1) / ntn + 15) / 16 * 16;     // tile width, <= WMAX (checked at planning)
    const int tmn = J.tm * ntn;
    const int kslice = t / tmn;
    t -= kslice * tmn;
    const int i0 = (t % J.tm) * TC_BM, j0 = (t / J.tm) * w;
    const int ksp = J.ks > 1 ? J.ks : 1;
    const int kchunk = (((J.k + ksp - 1) / ksp) + TC_BK - 1) / TC_BK * TC_BK;
    const int kbeg = kslice * kchunk, kend = min(J.k, kbeg + kchunk);
    const int nst = kend > kbeg ? (kend - kbeg + TC_BK - 1) / TC_BK : 0;
    c64 *__restrict__ C = g.C[z] + J.c;
    const bool sub = J.flags & GJ_SUB, add = J.flags & GJ_ACC, atom = J.ks > 1;
    if (nst == 0) {                       // empty k-slice: only a plain product writes (zeros)
        if (!(sub || add || atom))
            for (int e = tid; e < TC_BM * w; e += TC_THREADS) {
                const int i = i0 + e / w, j = j0 + e % w;
                if (i < J.m && j < J.n) C[(int64_t)i * J.crs + (int64_t)j * J.ccs] = mk<float>(0, 0);
            }
        return;
    }

    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t rbase = (uint32_t)__cvta_generic_to_shared(raw);
    const uint32_t mfull = (uint32_t)__cvta_generic_to_shared(mbar), mempty = mfull + 8 * NB;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < NB; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 256;" ::"r"(mfull + 8 * b) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mempty + 8 * b) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 8) {
        // ---- MMA warp: one thread issues every stage's six MMAs once the stage is full
        if (lane == 0) {
            const uint32_t idesc = instr_desc(PL::FUSED ? 2 * w : w, false), idneg = instr_desc(w, true);
            const uint32_t t_re = tmem, t_im = tmem + 128;
            for (int s = 0; s < nst && ok; ++s) {
                const int buf = s % NB;
                if (!mbar_wait(mfull + 8 * buf, (s / NB) & 1)) {
                    ok = false;
                    break;
                }
                fence_after_sync();
                const uint32_t sa = sbase + buf * PL::MMA_STAGE, sb = sa + 4 * TC_PLANE_A;
                const uint64_t a0 = smem_desc(sa), a1 = smem_desc(sa + TC_PLANE_A),
                               a2 = smem_desc(sa + 2 * TC_PLANE_A), a3 = smem_desc(sa + 3 * TC_PLANE_A);
                const uint64_t b0 = smem_desc(sb), b1 = smem_desc(sb + PL::PLANE_B),
                               b2 = smem_desc(sb + 2 * PL::PLANE_B), b3 = smem_desc(sb + 3 * PL::PLANE_B);
                const uint32_t first = s > 0 ? 1u : 0u;
                if constexpr (PL::FUSED) {
                    mma_tf32(tmem, a0, b0, idesc, first);          // Ar_hi [Br_hi | Bi_hi]
                    mma_tf32(tmem, a0, b1, idesc, 1u);             // Ar_hi [Br_lo | Bi_lo]
                    mma_tf32(tmem, a1, b0, idesc, 1u);             // Ar_lo [Br_hi | Bi_hi]
                    mma_tf32(tmem, a2, b2, idesc, 1u);             // Ai_hi [-Bi_hi | Br_hi]
                    mma_tf32(tmem, a2, b3, idesc, 1u);             // Ai_hi [-Bi_lo | Br_lo]
                    mma_tf32(tmem, a3, b2, idesc, 1u);             // Ai_lo [-Bi_hi | Br_hi]
                } else {                                           // b0..b3: Br_hi, Br_lo, Bi_hi, Bi_lo
                    mma_tf32(t_re, a0, b0, idesc, first);          // Ar Br
                    mma_tf32(t_re, a0, b1, idesc, 1u);
                    mma_tf32(t_re, a1, b0, idesc, 1u);
                    mma_tf32(t_re, a2, b2, idneg, 1u);             // - Ai Bi
                    mma_tf32(t_re, a2, b3, idneg, 1u);
                    mma_tf32(t_re, a3, b2, idneg, 1u);
                    mma_tf32(t_im, a0, b2, idesc, first);          // Ar Bi
                    mma_tf32(t_im, a0, b3, idesc, 1u);
                    mma_tf32(t_im, a1, b2, idesc, 1u);
                    mma_tf32(t_im, a2, b0, idesc, 1u);             // Ai Br
                    mma_tf32(t_im, a2, b1, idesc, 1u);
                    mma_tf32(t_im, a3, b0, idesc, 1u);
                }
                mma_commit(mempty + 8 * buf);
            }
        }
        __syncwarp();
    } else {
        // ---- converter warps
        const c64 *__restrict__ A = g.A[z] + J.a;
        const c64 *__restrict__ B = g.B[z] + J.b;
        const bool conjA = J.flags & GJ_CONJA, conjB = J.flags & GJ_CONJB;
        // pre-split A: the job's blocks of this tile row, from this CTA's first k-step on
        const bool pre = (J.flags & GJ_PRESPLIT) && g.ps[z] != nullptr;
        const float *psrc = pre ? g.ps[z] + J.ps +
                                      ((int64_t)(i0 / TC_BM) * ((J.k + TC_BK - 1) / TC_BK) + kbeg / TC_BK) * 4096
                                : nullptr;
        // cp.async of one raw stage (k = l0 .. l0 + 7): 1024 A elements (4 per thread) and
        // w x 8 B elements, mapped so that consecutive threads read consecutive addresses
        const bool a_rows = (J.ars == 1), b_cols = (J.bcs == 1);
        auto issue = [&](int st, int slot) {
            const int l0 = kbeg + TC_BK * st;
            const uint32_t ra = rbase + slot * PL::RAW_STAGE, rb = ra + PL::RAW_A;
#pragma unroll
            for (int q = 0; q < 4 && !pre; ++q) {
                const int e = tid + 256 * q;
                const int row = a_rows ? (e & 127) : (e >> 3), l = a_rows ? (e >> 7) : (e & 7);
                const bool v = (i0 + row < J.m) && (l0 + l < kend);
                const c64 *src = v ? A + (int64_t)(i0 + row) * J.ars + (int64_t)(l0 + l) * J.acs : A;
                cp_async8(ra + 8 * raw_index(row, l, TC_BM * 2), src, v);
            }
            for (int e = tid; e < w * TC_BK; e += 256) {
                const int j = b_cols ? (e % w) : (e >> 3), l = b_cols ? (e / w) : (e & 7);
                const bool v = (j0 + j < J.n) && (l0 + l < kend);
                const c64 *src = v ? B + (int64_t)(l0 + l) * J.brs + (int64_t)(j0 + j) * J.bcs : B;
                cp_async8(rb + 8 * raw_index(j, l, WMAX * 2), src, v);
            }
        };
        // conversion unit of a thread: row r = 8 (tid / 16) + tid % 8 and k-group q = (tid / 8) % 2
        // of A (and of B when r < w); its raw unit index is tid
        const int ur = 8 * (tid >> 4) + (tid & 7), uq = (tid >> 3) & 1;
        const uint32_t uoff = core_off(ur, uq);
        const uint32_t boff_bot = core_off(ur + w, uq);
        auto convert = [&](int slot, int buf) {
            const unsigned char *ra = raw + slot * PL::RAW_STAGE;
            unsigned char *pa = smem + buf * PL::MMA_STAGE;
            c64 v[4];
            if (!pre) {
                const float4 h0 = *reinterpret_cast<const float4 *>(ra + 16 * tid);
                const float4 h1 = *reinterpret_cast<const float4 *>(ra + 16 * (TC_BM * 2) + 16 * tid);
                v[0] = mk<float>(h0.x, h0.y); v[1] = mk<float>(h0.z, h0.w);
                v[2] = mk<float>(h1.x, h1.y); v[3] = mk<float>(h1.z, h1.w);
                if (conjA)
#pragma unroll
                    for (int e = 0; e < 4; ++e) v[e].im = -v[e].im;
                put4(pa, TC_PLANE_A, uoff, v);
            }
            if (ur < w) {
                const unsigned char *rb = ra + PL::RAW_A;
                const float4 h0 = *reinterpret_cast<const float4 *>(rb + 16 * tid);
                const float4 h1 = *reinterpret_cast<const float4 *>(rb + 16 * (WMAX * 2) + 16 * tid);
                v[0] = mk<float>(h0.x, h0.y); v[1] = mk<float>(h0.z, h0.w);
                v[2] = mk<float>(h1.x, h1.y); v[3] = mk<float>(h1.z, h1.w);
                if (conjB)
#pragma unroll
                    for (int e = 0; e < 4; ++e) v[e].im = -v[e].im;
                if constexpr (PL::FUSED)
                    put4_b(pa + 4 * TC_PLANE_A, PL::PLANE_B, uoff, boff_bot, v);
                else
                    put4(pa + 4 * TC_PLANE_A, PL::PLANE_B, uoff, v);
            }
        };
        for (int p = 0; p < P - 1; ++p) {           // prologue: P - 1 raw stages in flight
            if (p < nst) issue(p, p);
            cp_async_commit();
        }
        for (int s = 0; s < nst; ++s) {
            cp_async_wait<P - 2>();                 // raw stage s has landed (this thread's copies)
            converters_sync();                      // ... everybody's; stage s - 1 is converted
            if (s + P - 1 < nst) issue(s + P - 1, (s + P - 1) % P);
            cp_async_commit();
            const int buf = s % NB;
            if (s >= NB && ok && !mbar_wait(mempty + 8 * buf, ((s - NB) / NB) & 1)) ok = false;
            if (pre && tid == 0 && ok) {            // the stage's A planes: one 16 KB bulk copy
                asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(mfull + 8 * buf),
                             "r"(4 * TC_PLANE_A)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        sbase + (uint32_t)(buf * PL::MMA_STAGE)),
                    "l"(psrc + (int64_t)s * 4096), "r"(4 * TC_PLANE_A), "r"(mfull + 8 * buf)
                    : "memory");
            }
            convert(s % P, buf);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(mfull + 8 * buf);
        }
        cp_async_wait<0>();
        const int p = nst - 1;                      // its commit covers every earlier MMA
        if (ok && !mbar_wait(mempty + 8 * (p % NB), (p / NB) & 1)) ok = false;
        // after a timeout, the last stages' bulk copies may still be in flight: wait for their
        // stages to fill (bounded) before the CTA's shared memory is released
        if (pre && tid == 0 && !ok)
            for (int q = nst > NB ? nst - NB : 0; q < nst; ++q) mbar_wait(mfull + 8 * (q % NB), (q / NB) & 1);
        fence_after_sync();
    }
    ok = __syncthreads_and(ok);

    if (ok && warp < 8) {
        // epilogue: warp v reads TMEM lanes 32 (v % 4) .. + 31 (C rows); column chunks of 16
        // alternate between warps v and v + 4; Cr sits in columns [0, w), Ci in [w, 2w) (FUSED) or
        // [128, 128 + w)
        const int qd = warp & 3, hf = warp >> 2;
        const int i = i0 + 32 * qd + lane;
        const int nch = w / 16;
        for (int c = hf; c < nch; c += 2) {
            float re[16], im[16];
            const uint32_t ta = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(16 * c);
            tmem_ld16(ta, re);
            tmem_ld16(ta + (uint32_t)(PL::FUSED ? w : 128), im);
            if (i < J.m) {
                // accumulating products: all 16 loads first, then the stores (an interleaved
                // read-modify-write would wait one global round trip per element)
                if ((sub || add) && !atom) {
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        const int j = j0 + 16 * c + jj;
                        if (j < J.n) {
                            const c64 o = C[(int64_t)i * J.crs + (int64_t)j * J.ccs];
                            re[jj] = sub ? o.re - re[jj] : o.re + re[jj];
                            im[jj] = sub ? o.im - im[jj] : o.im + im[jj];
                        }
                    }
                }
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const int j = j0 + 16 * c + jj;
                    if (j >= J.n) continue;
                    c64 *q = C + (int64_t)i * J.crs + (int64_t)j * J.ccs;
                    if (atom) {
                        const float vr = sub ? -re[jj] : re[jj], vi = sub ? -im[jj] : im[jj];
                        atomicAdd(reinterpret_cast<float2 *>(q), make_float2(vr, vi));
                    } else {
                        *q = mk<float>(re[jj], im[jj]);
                    }
                }
            }
        }
    } else if (!ok && tid == 0) {
        atomicExch(&g_tc_status, ZOLO_ETIMEOUT);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
}

}  // namespace

// One 16 KB pre-split block per CTA: the 128 x 8 tile (rt, ks) of a PJob's operand, read
// column by column (rows contiguous) into shared memory, then written as the four TF32 planes
// in the canonical layout (each thread four consecutive floats: one row, four k), zero outside
// the operand.  The split is the converters' (tf32_round), so both paths give the same planes.
__global__ void __launch_bounds__(256) k_presplit(PresplitArgs g) {
    const int z = blockIdx.z;
    const int64_t blk = blockIdx.x;
    const int tid = threadIdx.x;
    __shared__ c64 tile[TC_BK][TC_BM];
    __shared__ int s_job;
    if (tid == 0) {
        int lo = 0, hi = g.njobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (g.jobs[mid].blk0 <= blk) lo = mid; else hi = mid - 1;
        }
        s_job = lo;
    }
    __syncthreads();
    const PJob J = g.jobs[s_job];
    const int nks = (J.k + TC_BK - 1) / TC_BK;
    const int64_t rel = blk - J.blk0;
    const int rt = (int)(rel / nks), ks = (int)(rel % nks);
    const c64 *__restrict__ A = (J.base ? g.finv[z] : g.pool[z]) + J.a;
    for (int e = tid; e < TC_BM * TC_BK; e += 256) {
        const int r = e & (TC_BM - 1), kk = e / TC_BM;
        const int i = rt * TC_BM + r, l = ks * TC_BK + kk;
        tile[kk][r] = (i < J.m && l < J.k) ? A[i + (int64_t)l * J.acs] : mk<float>(0.f, 0.f);
    }
    __syncthreads();
    float *out = g.out[z] + J.ps + rel * 4096;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int f = 4 * (tid + 256 * q);        // four consecutive floats of the block
        const int pl = f >> 10, w = f & 1023;     // plane, offset in the plane
        const int cm = w >> 5;                    // core matrix: row group * 2 + k-group
        const int row = (cm >> 1) * 8 + ((w & 31) >> 2), kk0 = (cm & 1) * 4;
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const c64 x = tile[kk0 + e][row];
            const float c = (pl < 2) ? x.re : x.im;
            const float hi = tf32_round(c);
            v[e] = (pl & 1) ? tf32_round(c - hi) : hi;
        }
        *reinterpret_cast<float4 *>(out + f) = make_float4(v[0], v[1], v[2], v[3]);
    }
}

template <int WMAX> void launch_tc_w(const GemmArgs<float> &g, dim3 grid, cudaStream_t st) {
    static bool attr_set[64] = {};                  // per device: the kernel's shared-memory opt-in
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        cudaFuncSetAttribute(k_gemm_tc<WMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcPlan<WMAX>::SMEM);
        attr_set[dev] = true;
    }
    k_gemm_tc<WMAX><<<grid, TC_THREADS, TcPlan<WMAX>::SMEM, st>>>(g);
}

void launch_presplit(const PresplitArgs &g, int64_t nblocks, int ninst, cudaStream_t st) {
    if (nblocks <= 0 || g.njobs <= 0) return;
    k_presplit<<<dim3((unsigned)nblocks, 1, ninst), 256, 0, st>>>(g);
    count_launch();
}

void launch_gemm_tc(const GemmArgs<float> &g, dim3 grid, cudaStream_t st) {
    const int wm = g.wmax > 0 ? g.wmax : 128;      // unplanned launches take the widest plan
    if (wm <= 32)
        launch_tc_w<32>(g, grid, st);
    else if (wm <= 64)
        launch_tc_w<64>(g, grid, st);
    else
        launch_tc_w<128>(g, grid, st);
}

int gemm_tc_status(bool reset) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(int)) != cudaSuccess) return ZOLO_ECUDA;
    if (v && reset) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(int));
    }
    return v;
}

}  // namespace zolo
