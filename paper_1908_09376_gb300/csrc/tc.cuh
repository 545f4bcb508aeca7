// Tensor-core (tcgen05) apply for many right-hand sides, sm_103a.
//
// Both kernels compute, for one block of a stage and a tile of 128 output
// rows, the complex product Z (128 x R) = A (128 x K) Y (K x R) on the
// 5th-generation tensor cores with FP32 accumulation in tensor memory (TMEM):
//   * k_s_tc:   A is a middle-factor block S (Sec. 3.5) made on the fly from
//               the split phase of its rows and columns;
//   * k_blk_tc: A is a V or U block of interpolative decompositions
//               (Sec. 3.2), read from dense BF16 tile images.
// The complex product runs through a real embedding of A: with
//   A_top = (Re A, -Im A) and A_bot = (Im A, Re A) interleaved along K, and
//   B     = (Re Y, Im Y)  interleaved along K (row n of B = RHS n),
// D_top = A_top B^T = Re(A Y) and D_bot = A_bot B^T = Im(A Y).  D_top sits in
// TMEM columns [0, 256), D_bot in [256, 512), so one pass covers 256 RHS.
// With refinement every operand is split into BF16 hi + lo (lo = bf16(v -
// hi)) and D accumulates hi*hi + hi*lo + lo*hi (the lo*lo product is of the
// order of the FP32 accumulation's rounding).
//
// Operands live in shared memory in the no-swizzle K-major core-matrix
// layout (8 rows x 16 bytes per core matrix; byte offset 128 between core
// matrices along K, (K/8)*128 between 8-row groups).  A CTA is 8 producer
// warps and one MMA warp around a ring of S stages of 16 complex columns:
// producers fill stage s and arrive on full[s]; the MMA warp's first lane
// issues the MMAs of the stage and commits them to empty[s].  Producers
// gather the right-hand sides of the next stage while they fill this one.  In k_blk_tc
// the MMA warp also issues the bulk copies of the A tiles, S - 1 chunks
// ahead.  Every wait is bounded: a wait that gives up sets the plan's status
// word to MIDBF_ETIMEOUT and the CTA winds down without writing outputs.
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "kernels.cuh"

namespace midbf_dev {

constexpr int kTcM = 128;                      // rows per item (TMEM lanes)
constexpr int kTcKc = 16;                      // complex columns per ring stage
constexpr int kTcK = 2 * kTcKc;                // K of a stage: (re, im) interleaved
constexpr int kTcR = 256;                      // RHS per pass
constexpr int kTcProducers = 512;              // producer threads (16 warps)
constexpr int kTcThreads = kTcProducers + 32;  // + the MMA warp
constexpr int kTcColStride = 12;               // reals per column of phase-split data (1 + P + Q <= 12)
constexpr int kTcAElems = kTcM * kTcK;         // BF16 elements of one A part (8 KB)
constexpr int kTcBElems = kTcR * kTcK;         // BF16 elements of one B part (16 KB)
constexpr int kTcTileElems = kTcAElems;        // one image tile part: 128 rows x 16 complex columns

template <bool REFINE>
struct TcCfg {
    static constexpr int NP = REFINE ? 2 : 1;  // BF16 parts per operand (hi, lo)
    static constexpr int S = REFINE ? 3 : 4;   // ring stages
    // one stage: A_top[NP], A_bot[NP], B[NP]
    static constexpr size_t stage_elems = (size_t)NP * (2 * kTcAElems + kTcBElems);
    static constexpr size_t bar_bytes = 256;   // mbarriers, TMEM address
    static constexpr size_t smem = (size_t)S * stage_elems * 2 + bar_bytes;
};

template <bool REFINE>
__host__ __device__ constexpr size_t tc_smem_bytes() {
    return TcCfg<REFINE>::smem;
}

// Small-RHS ring of k_blk_tc (Rpad <= kTcRSmall): a stage holds A_top, B and
// B2 = (Im Y, -Re Y) instead of A_top and A_bot, since D_bot = A_top B2^T as
// well; with small B parts that is half the bytes, so twice the stages (and
// twice the A-tile bytes in flight).
constexpr int kTcRSmall = 64;

template <bool REFINE>
struct TcCfgSmall {
    static constexpr int NP = REFINE ? 2 : 1;
    static constexpr int S = REFINE ? 6 : 8;
    static constexpr size_t b_elems = (size_t)kTcRSmall * kTcK;   // one B part
    // one stage: A_top[NP], B[NP], B2[NP]
    static constexpr size_t stage_elems = (size_t)NP * (kTcAElems + 2 * b_elems);
    static constexpr size_t bar_bytes = 256;
    static constexpr size_t smem = (size_t)S * stage_elems * 2 + bar_bytes;
};

// Offset (elements) of (row r, k) in the K-major core-matrix layout with K columns.
__host__ __device__ __forceinline__ int core_off(int r, int k, int K) {
    return ((r >> 3) * (K >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of tcgen05; no swizzle, base offset 0
    return d;
}

// kind::f16 instruction descriptor: BF16 A and B (K-major), FP32 D, M x N.
__device__ __forceinline__ uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr uint64_t kTcWaitNs = 2000000000ull;  // 2 s: far above any wait of a working pipeline

// Bounded wait for the completion of the mbarrier phase with the given
// parity.  Gives up after kTcWaitNs, or at once when the status word shows
// that some CTA has already given up (so one failure does not make every
// later CTA wait out its own limit).  status = nullptr: the time limit only
// (the drain waits before TMEM is released and the CTA exits).
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, const int* status) {
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63) == 63) {
            if (status && *reinterpret_cast<const volatile int*>(status) != 0) return false;
            if (global_ns() - t0 > kTcWaitNs) return false;
        }
    }
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(mbar))
        : "memory");
}

// Producer-only named barrier (barrier 1, the 8 producer warps) that returns
// the AND of a predicate over them, so that the outcome of a bounded wait is
// uniform before any producer acts on it.
__device__ __forceinline__ bool producers_and(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.b32 q, %1, 0;\n\t"
        "bar.red.and.pred p, 1, %2, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kTcProducers)
        : "memory");
    return r != 0;
}

// (re, im) -> packed BF16 pair (re in the low half), and the pair of the
// remainders v - bf16(v) rounded to BF16.
__device__ __forceinline__ void split_pair(float re, float im, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    const float rh = __uint_as_float(hi << 16), ih = __uint_as_float(hi & 0xffff0000u);
    const __nv_bfloat162 l = __floats2bfloat162_rn(re - rh, im - ih);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Packed BF16 pairs: (a, b) -> (a, -b); (a, b) -> (b, a); (a, -b) -> (b, a).
__device__ __forceinline__ uint32_t neg_high(uint32_t w) { return w ^ 0x80000000u; }
__device__ __forceinline__ uint32_t swap_halves(uint32_t w) { return __byte_perm(w, 0, 0x1032); }
__device__ __forceinline__ uint32_t top_to_bot(uint32_t w) { return swap_halves(w) ^ 0x00008000u; }

// Shared-memory control block after the ring.
template <int S>
struct TcBars {
    uint64_t full[S];    // producers -> MMA warp (count kTcProducers)
    uint64_t empty[S];   // MMAs of the stage complete (tcgen05.commit)
    uint64_t load[S];    // bulk copies into the stage landed (B image; A tile in k_blk_tc)
    uint64_t done;       // all MMAs complete
    uint64_t fin;        // teardown: every MMA issued has completed
    uint32_t taddr;
};

// B image of one chunk: NP parts (hi, lo) of Rpad rows (RHS) x 32 (16 complex
// columns, re/im interleaved) in the core-matrix layout.
__host__ __device__ inline size_t tc_bimg_elems(int Rpad, bool refine) {
    return (size_t)(refine ? 2 : 1) * (size_t)Rpad * kTcK;
}

// MMAs of one ring stage: D_top += A_top B^T and D_bot += A_bot B^T over the
// stage's K = 32, plus the hi/lo refinement products.  The B lo part sits
// b_lo bytes after the B hi part.
template <bool REFINE>
__device__ __forceinline__ void tc_issue_stage(uint32_t tmem, const __nv_bfloat16* stage, uint32_t idesc,
                                               uint32_t b_lo, bool first) {
    constexpr int NP = REFINE ? 2 : 1;
    constexpr uint32_t sbo = (kTcK / 8) * 128;
    const uint32_t aT = smem_u32(stage);
    const uint32_t aB = aT + NP * kTcAElems * 2;
    const uint32_t bB = aT + 2 * NP * kTcAElems * 2;
#pragma unroll
    for (int kk = 0; kk < kTcK; kk += 16) {
        const uint32_t ko = (uint32_t)(kk / 8) * 128;
        const uint32_t acc = (first && kk == 0) ? 0u : 1u;
        const uint64_t bh = umma_desc(bB + ko, 128, sbo);
        const uint64_t th = umma_desc(aT + ko, 128, sbo);
        const uint64_t uh = umma_desc(aB + ko, 128, sbo);
        umma_bf16(tmem, th, bh, idesc, acc);
        umma_bf16(tmem + kTcR, uh, bh, idesc, acc);
        if (REFINE) {
            const uint64_t bl = umma_desc(bB + b_lo + ko, 128, sbo);
            const uint64_t tl = umma_desc(aT + kTcAElems * 2 + ko, 128, sbo);
            const uint64_t ul = umma_desc(aB + kTcAElems * 2 + ko, 128, sbo);
            umma_bf16(tmem, th, bl, idesc, 1u);
            umma_bf16(tmem, tl, bh, idesc, 1u);
            umma_bf16(tmem + kTcR, uh, bl, idesc, 1u);
            umma_bf16(tmem + kTcR, ul, bh, idesc, 1u);
        }
    }
}

// MMAs of one small-RHS stage: D_top += A_top B^T, D_bot += A_top B2^T.
template <bool REFINE>
__device__ __forceinline__ void tc_issue_stage_b2(uint32_t tmem, const __nv_bfloat16* stage, uint32_t idesc,
                                                  uint32_t b_lo, bool first) {
    using Cfg = TcCfgSmall<REFINE>;
    constexpr int NP = Cfg::NP;
    constexpr uint32_t sbo = (kTcK / 8) * 128;
    const uint32_t aT = smem_u32(stage);
    const uint32_t bB = aT + NP * kTcAElems * 2;
    const uint32_t b2B = bB + (uint32_t)(NP * Cfg::b_elems * 2);
#pragma unroll
    for (int kk = 0; kk < kTcK; kk += 16) {
        const uint32_t ko = (uint32_t)(kk / 8) * 128;
        const uint32_t acc = (first && kk == 0) ? 0u : 1u;
        const uint64_t th = umma_desc(aT + ko, 128, sbo);
        const uint64_t bh = umma_desc(bB + ko, 128, sbo);
        const uint64_t ch = umma_desc(b2B + ko, 128, sbo);
        umma_bf16(tmem, th, bh, idesc, acc);
        umma_bf16(tmem + kTcR, th, ch, idesc, acc);
        if (REFINE) {
            const uint64_t tl = umma_desc(aT + kTcAElems * 2 + ko, 128, sbo);
            const uint64_t bl = umma_desc(bB + b_lo + ko, 128, sbo);
            const uint64_t cl = umma_desc(b2B + b_lo + ko, 128, sbo);
            umma_bf16(tmem, th, bl, idesc, 1u);
            umma_bf16(tmem, tl, bh, idesc, 1u);
            umma_bf16(tmem + kTcR, th, cl, idesc, 1u);
            umma_bf16(tmem + kTcR, tl, ch, idesc, 1u);
        }
    }
}

// ---------------------------------------------------------------------------
// Right-hand sides.  Before a tensor-core stage runs, k_pack_b gathers its
// input once per (block, 16-column chunk) and writes the chunk's B image:
// row n = RHS n, (Re y, Im y) of the 16 columns interleaved along K, BF16 hi
// (and lo) in the core-matrix layout, so that the MMA warp moves it with one
// bulk copy.  Chunk q holds the columns at positions pos[chunks[q].x + j],
// j < chunks[q].y (<= 16); the rest of the chunk is zero.
struct TcPack {
    const int2* chunks;
    const int* pos;
    int nchunks;
};

template <bool REFINE>
__global__ void __launch_bounds__(256) k_pack_b(TcPack pk, VecRef<float> src, int R, int Rpad, __nv_bfloat16* img) {
    const size_t ce = tc_bimg_elems(Rpad, REFINE);
    for (int q = blockIdx.x; q < pk.nchunks; q += gridDim.x) {
        const int2 ch = pk.chunks[q];
        __nv_bfloat16* out = img + (size_t)q * ce;
        for (int e = threadIdx.x; e < Rpad * 4; e += blockDim.x) {
            const int n = e % Rpad, jq = e / Rpad;   // consecutive threads: consecutive RHS
            uint32_t h[4], l[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int jj = jq * 4 + u;
                float re = 0.f, im = 0.f;
                if (n < R && jj < ch.y) {
                    const cx<float> y = src.ptr[(long long)__ldg(pk.pos + ch.x + jj) * src.ps + (long long)n * src.rs];
                    re = y.x;
                    im = y.y;
                }
                split_pair(re, im, h[u], l[u]);
            }
            const int o = core_off(n, 8 * jq, kTcK);
            *reinterpret_cast<uint4*>(out + o) = make_uint4(h[0], h[1], h[2], h[3]);
            if (REFINE) *reinterpret_cast<uint4*>(out + (size_t)Rpad * kTcK + o) = make_uint4(l[0], l[1], l[2], l[3]);
        }
    }
}

// Epilogue: producer warp w reads TMEM lanes 32 (w & 3) + lane (its row),
// column groups of 8 RHS round robin over the four warps of a lane quarter;
// Re from D_top, Im from D_bot.
__device__ __forceinline__ void tc_epilogue(uint32_t tmem, int warp, int lane, int Rpad, int R, bool rowok, int op,
                                            VecRef<float> dst, bool zero) {
    constexpr int kQuarterWarps = kTcProducers / 32 / 4;
    const int q = warp & 3;
    for (int c0 = 8 * (warp >> 2); c0 < Rpad; c0 += 8 * kQuarterWarps) {
        uint32_t v[8], w[8];
        const uint32_t a = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                     : "r"(a));
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
                     : "r"(a + kTcR));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (rowok) {
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int n = c0 + t;
                if (n < R) {
                    const float re = zero ? 0.f : __uint_as_float(v[t]);
                    const float im = zero ? 0.f : __uint_as_float(w[t]);
                    dst.ptr[(long long)op * dst.ps + (long long)n * dst.rs] = cx<float>{re, im};
                }
            }
        }
    }
}

template <int S>
__device__ __forceinline__ void tc_setup(TcBars<S>* bars, int tid, int warp) {
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&bars->full[s], kTcProducers);
            mbar_init(&bars->empty[s], 1);
            mbar_init(&bars->load[s], 1);
        }
        mbar_init(&bars->done, 1);
        mbar_init(&bars->fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&bars->taddr)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
}

__device__ __forceinline__ void tc_teardown(uint32_t tmem, int warp) {
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// The MMA warp's side of the ring, shared by both kernels.  Chunk g's bulk
// copies go out S - 1 chunks ahead: into the stage of chunk g - 1 once that
// chunk's MMAs are done (the MMAs of chunk g are queued behind them, so the
// tensor pipe stays fed).  Before the MMAs of chunk g it waits for the
// producers (full) and the copies (load).  Last, a commit that arrives once
// every MMA has completed is awaited (time-bounded only) before TMEM is
// released, and so are copies issued but never awaited.
template <int S, bool REFINE, bool B2, class Copy>
__device__ __forceinline__ void tc_mma_loop(TcBars<S>* bars, __nv_bfloat16* ring, size_t stage_elems, uint32_t tmem,
                                            int nchunk, int Rpad, int lane, int* status, Copy copy) {
    bool ok = true;
    int issued = 0;
    for (; issued < nchunk && issued < S; ++issued) copy(issued);
    const uint32_t idesc = umma_idesc_bf16(kTcM, Rpad);
    const uint32_t b_lo = (uint32_t)Rpad * kTcK * 2;
    for (int c = 0; c < nchunk; ++c) {
        const int s = c % S;
        const uint32_t ph = (uint32_t)(c / S) & 1;
        if (!mbar_wait(&bars->full[s], ph, status) || !mbar_wait(&bars->load[s], ph, status)) {
            ok = false;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (lane == 0) {
            if (B2) tc_issue_stage_b2<REFINE>(tmem, ring + (size_t)s * stage_elems, idesc, b_lo, c == 0);
            else tc_issue_stage<REFINE>(tmem, ring + (size_t)s * stage_elems, idesc, b_lo, c == 0);
            umma_commit(&bars->empty[s]);
        }
        __syncwarp();
        if (c >= 1 && issued < nchunk && issued == c + S - 1) {
            if (!mbar_wait(&bars->empty[(c - 1) % S], (uint32_t)((c - 1) / S) & 1, status)) {
                ok = false;
                break;
            }
            copy(issued);
            ++issued;
        }
    }
    if (lane == 0) umma_commit(&bars->done);   // arrives at once when no MMA was issued
    __syncwarp();
    if (!ok && lane == 0) atomicExch(status, MIDBF_ETIMEOUT);
    if (lane == 0) {
        umma_commit(&bars->fin);
        if (!mbar_wait(&bars->fin, 0, nullptr)) atomicExch(status, MIDBF_ETIMEOUT);
        for (int gg = issued - 1; gg >= 0 && gg >= issued - S; --gg)
            mbar_wait(&bars->load[gg % S], (uint32_t)(gg / S) & 1, nullptr);
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Middle factor.  One CTA per item (block, 128 role-rows) and at most kTcR
// RHS; role rows/cols as in k_s_fly (row_is_row = 1 forward, 0 adjoint with
// CONJ).  bimg + chunk0[b] * (chunk size) is the block's first B image.
//
// Producer iteration for chunk c (ring slot s = c mod S): wait until the
// stage's MMAs of chunk c - S are done; threads < 16 put the phase data of
// chunk c + 1 (loaded one iteration earlier) into slot (c + 1) mod S and
// load that of chunk c + 2; a producer barrier; generate A_top / A_bot of
// chunk c; arrive on full[s].  A slot is rewritten S - 1 iterations after it
// was last read; S >= 3 and the barrier of every iteration keep that ordered.
template <int PQ, bool REFINE, bool CONJ>
__global__ void __launch_bounds__(kTcThreads, 1) k_s_tc(SStage<float> st, SSide<float> rs, SSide<float> cs,
                                                        const int* chunk0, const __nv_bfloat16* bimg,
                                                        VecRef<float> dst, int R, int row_is_row, int* status) {
    using Cfg = TcCfg<REFINE>;
    constexpr int S = Cfg::S, NP = Cfg::NP;
    static_assert(S >= 3, "slot reuse needs three ring stages");
    using Sh = PhaseShape<PQ>;
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __nv_bfloat16* ring = reinterpret_cast<__nv_bfloat16*>(tc_smem_raw);
    TcBars<S>* bars = reinterpret_cast<TcBars<S>*>(tc_smem_raw + S * Cfg::stage_elems * 2);
    __shared__ float scol[S][kTcKc * kTcColStride];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int2 it = st.items[blockIdx.x];
    const int b = it.x;
    const int ro = row_is_row ? st.blk_rows[b] : st.blk_cols[b];
    const int co = row_is_row ? st.blk_cols[b] : st.blk_rows[b];
    const int nrow = row_is_row ? st.blk_nrow[b] : st.blk_ncol[b];
    const int ncol = row_is_row ? st.blk_ncol[b] : st.blk_nrow[b];
    const int P = Sh::fixed ? Sh::P : st.P;
    const int Q = Sh::fixed ? Sh::Q : st.Q;
    const int nchunk = (ncol + kTcKc - 1) / kTcKc;
    const int Rpad = (R + 15) & ~15;
    const size_t bce = tc_bimg_elems(Rpad, REFINE);
    const __nv_bfloat16* b0 = bimg + (size_t)chunk0[b] * bce;

    tc_setup<S>(bars, tid, warp);
    const uint32_t tmem = bars->taddr;

    if (warp == kTcProducers / 32) {
        // ---- MMA warp: B images by bulk copy, MMAs
        auto copy = [&](int g) {
            const int s = g % S;
            if (lane == 0) {
                mbar_expect_tx(&bars->load[s], (uint32_t)(bce * 2));
                bulk_g2s(ring + (size_t)s * Cfg::stage_elems + 2 * NP * kTcAElems, b0 + (size_t)g * bce,
                         (uint32_t)(bce * 2), &bars->load[s]);
            }
        };
        tc_mma_loop<S, REFINE, false>(bars, ring, Cfg::stage_elems, tmem, nchunk, Rpad, lane, status, copy);
    } else {
        // ---- producers: thread = (row, quarter of the stage's 16 columns)
        const int ptid = tid;
        const int row = ptid & (kTcM - 1), cq = ptid >> 7;
        const int i = it.y + row;
        const bool rok = i < nrow;
        float ra = 0.f, ru[Sh::PA], rc[Sh::QA];
        {
            const int ii = rok ? i : 0;
            ra = rs.a[ro + ii];
#pragma unroll
            for (int p = 0; p < Sh::P; ++p) ru[p] = p < P ? rs.u[(size_t)(ro + ii) * P + p] : 0.f;
#pragma unroll
            for (int q = 0; q < Sh::Q; ++q) rc[q] = q < Q ? rs.c[(size_t)(ro + ii) * Q + q] : 0.f;
        }
        const int op = rok ? rs.pos[ro + i] : 0;
        // phase data of one column, prefetched into registers by threads < 16
        float cpre[kTcColStride];
        auto fetch = [&](int c) {
            const int j = c * kTcKc + ptid;
            if (ptid < kTcKc && c < nchunk) {
#pragma unroll
                for (int q = 0; q < kTcColStride; ++q) cpre[q] = 0.f;
                if (j < ncol) {
                    const int e = co + j;
                    cpre[0] = cs.a[e];
#pragma unroll
                    for (int q = 0; q < Sh::P; ++q)
                        if (Sh::fixed || q < P) cpre[1 + q] = cs.u[(size_t)e * P + q];
#pragma unroll
                    for (int q = 0; q < Sh::Q; ++q)
                        if (Sh::fixed || q < Q) cpre[1 + P + q] = cs.c[(size_t)e * Q + q];
                }
            }
        };
        auto put = [&](int c) {
            if (ptid < kTcKc && c < nchunk) {
                float* cj = scol[c % S] + ptid * kTcColStride;
#pragma unroll
                for (int q = 0; q < kTcColStride; ++q) cj[q] = cpre[q];
            }
        };
        bool ok = true;
        fetch(0);
        put(0);
        fetch(1);
        producers_and(true);
        for (int c = 0; c < nchunk; ++c) {
            const int s = c % S;
            const uint32_t u = (uint32_t)(c / S);
            // the stage's previous MMAs (chunk c - S) must be done before it is overwritten
            bool w = true;
            if (u > 0) w = mbar_wait(&bars->empty[s], (u - 1) & 1, status);
            put(c + 1);
            fetch(c + 2);
            ok = producers_and(w);
            if (!ok) break;
            __nv_bfloat16* stg = ring + (size_t)s * Cfg::stage_elems;
            const int j0 = c * kTcKc;
            // this thread's row, columns 4 cq .. 4 cq + 3 = one core row of A_top and of A_bot
            uint32_t th[4], tl[4], bh[4], bl[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int jj = cq * 4 + v;
                float er = 0.f, ei = 0.f;
                if (rok && j0 + jj < ncol) {
                    const float* cj = scol[s] + jj * kTcColStride;
                    float thp = ra + cj[0];
#pragma unroll
                    for (int q = 0; q < Sh::P; ++q)
                        if (Sh::fixed || q < P) thp = fmaf(ru[q], cj[1 + q], thp);
                    if (Sh::Q > 0 && (Sh::fixed || Q > 0)) {
                        float sq = 0.f;
#pragma unroll
                        for (int q = 0; q < Sh::Q; ++q) {
                            if (!(Sh::fixed || q < Q)) continue;
                            if constexpr (Sh::dist) {
                                const float dq = rc[q] - cj[1 + P + q];
                                sq = fmaf(dq, dq, sq);
                            } else {
                                sq = fmaf(rc[q], cj[1 + P + q], sq);
                            }
                        }
                        thp += sqrt_nr(sq);
                    }
                    thp = frac_rn(thp);
                    sincos2pi(thp, &ei, &er);
                    if (CONJ) ei = -ei;
                }
                uint32_t h, l;
                split_pair(er, ei, h, l);
                th[v] = neg_high(h);
                tl[v] = neg_high(l);
                bh[v] = swap_halves(h);
                bl[v] = swap_halves(l);
            }
            const int o = core_off(row, 8 * cq, kTcK);
            *reinterpret_cast<uint4*>(stg + o) = make_uint4(th[0], th[1], th[2], th[3]);
            *reinterpret_cast<uint4*>(stg + NP * kTcAElems + o) = make_uint4(bh[0], bh[1], bh[2], bh[3]);
            if (REFINE) {
                *reinterpret_cast<uint4*>(stg + kTcAElems + o) = make_uint4(tl[0], tl[1], tl[2], tl[3]);
                *reinterpret_cast<uint4*>(stg + (NP + 1) * kTcAElems + o) = make_uint4(bl[0], bl[1], bl[2], bl[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;");
            mbar_arrive(&bars->full[s]);
        }
        if (ok) ok = producers_and(mbar_wait(&bars->done, 0, status));
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            tc_epilogue(tmem, warp, lane, Rpad, R, rok, op, dst, nchunk == 0);
        }
        if (!ok && ptid == 0) atomicExch(status, MIDBF_ETIMEOUT);
    }
    tc_teardown(tmem, warp);
}

// ---------------------------------------------------------------------------
// Interpolation / transfer stages (V, U) on the tensor cores.
//
// In the tensor-core modes every V or U block is also stored densely (its
// identity entries included) as BF16 tile images: tile (row tile rt, column
// chunk c) holds A_top = (Re, -Im) of rows [128 rt, 128 rt + 128) x complex
// columns [16 c, 16 c + 16) in exactly the core-matrix layout of a ring stage
// (hi part, then lo part), so one cp.async.bulk moves it; A_bot is derived
// from it in shared memory.  Two orientations are stored: the block itself
// (forward) and its conjugate transpose (adjoint).  The item is (block, row
// tile); the block's B images start at chunk0.
struct TcBlock {
    long long img_off;   // element offset (BF16) of the block's first tile image
    int rows, cols;      // complex rows (outputs) and columns (inputs)
    int out_off;         // offset into the output positions
    int chunk0;          // index of the block's first B image
};

struct TcStage {
    const TcBlock* blocks;
    const int* out_pos;     // positions of block outputs in the destination space
    const __nv_bfloat16* img;
    const int2* items;      // (block, row tile)
};

// SMALL (Rpad <= kTcRSmall): the TcCfgSmall ring; producers derive B2 from B.
// Otherwise the TcCfg ring; producers derive A_bot from A_top.
template <bool REFINE, bool SMALL>
__global__ void __launch_bounds__(kTcThreads, 1) k_blk_tc(TcStage st, const __nv_bfloat16* bimg, VecRef<float> dst,
                                                          int R, int* status) {
    using Cfg = typename std::conditional<SMALL, TcCfgSmall<REFINE>, TcCfg<REFINE>>::type;
    constexpr int S = Cfg::S, NP = Cfg::NP;
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __nv_bfloat16* ring = reinterpret_cast<__nv_bfloat16*>(tc_smem_raw);
    TcBars<S>* bars = reinterpret_cast<TcBars<S>*>(tc_smem_raw + S * Cfg::stage_elems * 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int2 it = st.items[blockIdx.x];
    const TcBlock bk = st.blocks[it.x];
    const int rt = it.y;
    const int nchunk = (bk.cols + kTcKc - 1) / kTcKc;
    const int Rpad = (R + 15) & ~15;
    const size_t bce = tc_bimg_elems(Rpad, REFINE);
    const __nv_bfloat16* tile0 = st.img + bk.img_off + (size_t)rt * nchunk * NP * kTcTileElems;
    const __nv_bfloat16* b0 = bimg + (size_t)bk.chunk0 * bce;
    constexpr uint32_t kABytes = NP * kTcTileElems * 2;

    tc_setup<S>(bars, tid, warp);
    const uint32_t tmem = bars->taddr;

    if (warp == kTcProducers / 32) {
        // ---- MMA warp: A tile and B image of each chunk by bulk copy, MMAs
        // offset of the B region in a stage: after A_top and A_bot, or (SMALL) after A_top
        constexpr size_t b_at = (SMALL ? 1 : 2) * (size_t)NP * kTcAElems;
        auto copy = [&](int g) {
            const int s = g % S;
            if (lane == 0) {
                __nv_bfloat16* stg = ring + (size_t)s * Cfg::stage_elems;
                mbar_expect_tx(&bars->load[s], kABytes + (uint32_t)(bce * 2));
                bulk_g2s(stg, tile0 + (size_t)g * NP * kTcTileElems, kABytes, &bars->load[s]);
                bulk_g2s(stg + b_at, b0 + (size_t)g * bce, (uint32_t)(bce * 2), &bars->load[s]);
            }
        };
        tc_mma_loop<S, REFINE, SMALL>(bars, ring, Cfg::stage_elems, tmem, nchunk, Rpad, lane, status, copy);
    } else {
        // ---- producers: A_bot = (Im, Re) from A_top = (Re, -Im), 512 16-byte vectors per part
        const int ptid = tid;
        const int row = ptid & (kTcM - 1);
        const int i = rt * kTcM + row;
        const bool rok = i < bk.rows;
        const int op = rok ? st.out_pos[bk.out_off + i] : 0;
        bool ok = true;
        for (int c = 0; c < nchunk; ++c) {
            const int s = c % S;
            ok = producers_and(mbar_wait(&bars->load[s], (uint32_t)(c / S) & 1, status));
            if (!ok) break;
            __nv_bfloat16* stg = ring + (size_t)s * Cfg::stage_elems;
            if constexpr (SMALL) {
                // B2 = (Im Y, -Re Y) word by word from B = (Re Y, Im Y), hi and lo parts
                const uint4* b = reinterpret_cast<const uint4*>(stg + NP * kTcAElems);
                uint4* b2 = reinterpret_cast<uint4*>(stg + NP * kTcAElems + NP * Cfg::b_elems);
                const int nv = (int)(bce / 8);   // 16-byte vectors of the B image
                for (int v = ptid; v < nv; v += kTcProducers) {
                    const uint4 w = b[v];
                    b2[v] = make_uint4(neg_high(swap_halves(w.x)), neg_high(swap_halves(w.y)),
                                       neg_high(swap_halves(w.z)), neg_high(swap_halves(w.w)));
                }
            } else {
#pragma unroll
                for (int part = 0; part < NP; ++part) {
                    const uint4 a = reinterpret_cast<const uint4*>(stg + part * kTcAElems)[ptid];
                    reinterpret_cast<uint4*>(stg + (NP + part) * kTcAElems)[ptid] =
                        make_uint4(top_to_bot(a.x), top_to_bot(a.y), top_to_bot(a.z), top_to_bot(a.w));
                }
            }
            asm volatile("fence.proxy.async.shared::cta;");
            mbar_arrive(&bars->full[s]);
        }
        if (ok) ok = producers_and(mbar_wait(&bars->done, 0, status));
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            tc_epilogue(tmem, warp, lane, Rpad, R, rok, op, dst, nchunk == 0);
        }
        if (!ok && ptid == 0) atomicExch(status, MIDBF_ETIMEOUT);
    }
    tc_teardown(tmem, warp);
}

}  // namespace midbf_dev

