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
    uint64_t aload[S];   // bulk copy of the stage's A tiles landed (k_blk_tc)
    uint64_t done;       // all MMAs of a pass complete
    uint64_t tfree;      // the epilogue of a pass has read TMEM (count kTcProducers)
    uint64_t fin;        // teardown: every MMA issued has completed
    uint32_t taddr;
};

// MMAs of one ring stage: D_top += A_top B^T and D_bot += A_bot B^T over the
// stage's K = 32, plus the hi/lo refinement products.
template <bool REFINE>
__device__ __forceinline__ void tc_issue_stage(uint32_t tmem, const __nv_bfloat16* stage, uint32_t idesc,
                                               bool first) {
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
            const uint64_t bl = umma_desc(bB + kTcBElems * 2 + ko, 128, sbo);
            const uint64_t tl = umma_desc(aT + kTcAElems * 2 + ko, 128, sbo);
            const uint64_t ul = umma_desc(aB + kTcAElems * 2 + ko, 128, sbo);
            umma_bf16(tmem, th, bl, idesc, 1u);
            umma_bf16(tmem, tl, bh, idesc, 1u);
            umma_bf16(tmem + kTcR, uh, bl, idesc, 1u);
            umma_bf16(tmem + kTcR, ul, bh, idesc, 1u);
        }
    }
}

// Right-hand sides of one ring stage: rows n < Rpad of B from the stage's 16
// columns at positions pos[0..16) of src (zero past ncol_left or R).  Item e
// = (n, quad jq): 4 consecutive columns of RHS n = one 16-byte core row;
// consecutive threads take consecutive RHS.  The item coordinates depend on
// the pass only, so they are set once per pass (TcBItems).
constexpr int kTcBItems = (kTcR * kTcKc / 4 + kTcProducers - 1) / kTcProducers;  // items per thread

struct TcBItems {
    int n[kTcBItems], jq[kTcBItems];
    long long roff[kTcBItems];   // (r0 + n) * rs
    bool on[kTcBItems];          // item exists (e < Rpad * 4)
    bool live[kTcBItems];        // RHS exists (n < R)
};

__device__ __forceinline__ void tc_b_items(TcBItems& I, VecRef<float> src, int r0, int R, int Rpad, int ptid) {
#pragma unroll
    for (int it = 0; it < kTcBItems; ++it) {
        const int e = ptid + it * kTcProducers;
        I.on[it] = e < Rpad * 4;
        I.n[it] = e % Rpad;
        I.jq[it] = e / Rpad;
        I.live[it] = I.on[it] && I.n[it] < R;
        I.roff[it] = (long long)(r0 + I.n[it]) * src.rs;
    }
}

struct TcBLoad {
    float2 y[kTcBItems][4];
};

__device__ __forceinline__ void tc_load_b(TcBLoad& L, const TcBItems& I, const int* pos, int ncol_left,
                                          VecRef<float> src) {
#pragma unroll
    for (int it = 0; it < kTcBItems; ++it) {
        const int4 p4 = *reinterpret_cast<const int4*>(pos + 4 * (I.jq[it] & 3));
        const int pp[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float2 v = make_float2(0.f, 0.f);
            if (I.live[it] && I.jq[it] * 4 + u < ncol_left) {
                const cx<float> y = src.ptr[(long long)pp[u] * src.ps + I.roff[it]];
                v = make_float2(y.x, y.y);
            }
            L.y[it][u] = v;
        }
    }
}

template <bool REFINE>
__device__ __forceinline__ void tc_store_b(const TcBLoad& L, const TcBItems& I, __nv_bfloat16* B) {
#pragma unroll
    for (int it = 0; it < kTcBItems; ++it) {
        if (I.on[it]) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) split_pair(L.y[it][u].x, L.y[it][u].y, h[u], l[u]);
            const int o = core_off(I.n[it], 8 * I.jq[it], kTcK);
            *reinterpret_cast<uint4*>(B + o) = make_uint4(h[0], h[1], h[2], h[3]);
            if (REFINE) *reinterpret_cast<uint4*>(B + kTcBElems + o) = make_uint4(l[0], l[1], l[2], l[3]);
        }
    }
}

// Epilogue of a pass: producer warp w reads TMEM lanes 32 (w & 3) + lane
// (its row), column groups of 8 RHS round robin over the four warps of a lane
// quarter; Re from D_top, Im from D_bot.
__device__ __forceinline__ void tc_epilogue(uint32_t tmem, int warp, int lane, int Rpad, int R, int r0, bool rowok,
                                            int op, VecRef<float> dst, bool zero) {
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
                    dst.ptr[(long long)op * dst.ps + (long long)(r0 + n) * dst.rs] = cx<float>{re, im};
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
            mbar_init(&bars->aload[s], 1);
        }
        mbar_init(&bars->done, 1);
        mbar_init(&bars->tfree, kTcProducers);
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

template <int S>
__device__ __forceinline__ void tc_teardown(uint32_t tmem, int warp) {
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// The MMA warp's last step: a commit that arrives once every MMA it issued
// has completed, awaited (bounded) before the tensor memory is released.
__device__ __forceinline__ void tc_mma_drain(uint64_t* fin, int lane, int* status) {
    if (lane == 0) {
        umma_commit(fin);
        if (!mbar_wait(fin, 0, nullptr)) atomicExch(status, MIDBF_ETIMEOUT);
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Middle factor.  One CTA per item (block, 128 role-rows); role rows/cols as
// in k_s_fly (row_is_row = 1 forward, 0 adjoint with CONJ).
//
// Producer iteration for chunk c (ring slot s = g mod S):
//   wait until the stage's MMAs of chunk g - S are done; threads < 16 stage
//   the phase data and positions of chunk c + 1 in slot (g + 1) mod S; a
//   producer barrier; gather the RHS of chunk c + 1 into registers; generate
//   A_top / A_bot of chunk c; store the RHS of chunk c (gathered one
//   iteration earlier) as B; arrive on full[s].
// A slot is rewritten S - 1 iterations after it was last read; S >= 3 and the
// barrier of every iteration keep that ordered.
template <int PQ, bool REFINE, bool CONJ>
__global__ void __launch_bounds__(kTcThreads, 1) k_s_tc(SStage<float> st, SSide<float> rs, SSide<float> cs,
                                                        VecRef<float> src, VecRef<float> dst, int nrhs,
                                                        int row_is_row, int* status) {
    using Cfg = TcCfg<REFINE>;
    constexpr int S = Cfg::S, NP = Cfg::NP;
    static_assert(S >= 3, "slot reuse needs three ring stages");
    using Sh = PhaseShape<PQ>;
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __nv_bfloat16* ring = reinterpret_cast<__nv_bfloat16*>(tc_smem_raw);
    TcBars<S>* bars = reinterpret_cast<TcBars<S>*>(tc_smem_raw + S * Cfg::stage_elems * 2);
    __shared__ float scol[S][kTcKc * kTcColStride];
    __shared__ __align__(16) int spos[S][kTcKc];
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
    const int npass = (nrhs + kTcR - 1) / kTcR;

    tc_setup<S>(bars, tid, warp);
    const uint32_t tmem = bars->taddr;

    if (warp == kTcProducers / 32) {
        // ---- MMA warp
        bool ok = true;
        int g = 0;
        for (int p = 0; p < npass && ok; ++p) {
            const int R = min(kTcR, nrhs - p * kTcR), Rpad = (R + 15) & ~15;
            const uint32_t idesc = umma_idesc_bf16(kTcM, Rpad);
            if (p > 0 && !mbar_wait(&bars->tfree, (uint32_t)(p - 1) & 1, status)) {
                ok = false;
                break;
            }
            for (int c = 0; c < nchunk; ++c, ++g) {
                const int s = g % S;
                if (!mbar_wait(&bars->full[s], (uint32_t)(g / S) & 1, status)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                if (lane == 0) {
                    tc_issue_stage<REFINE>(tmem, ring + (size_t)s * Cfg::stage_elems, idesc, c == 0);
                    umma_commit(&bars->empty[s]);
                }
                __syncwarp();
            }
            if (!ok) break;
            if (lane == 0) umma_commit(&bars->done);
            __syncwarp();
        }
        if (!ok && lane == 0) atomicExch(status, MIDBF_ETIMEOUT);
        tc_mma_drain(&bars->fin, lane, status);
    } else {
        // ---- producers: thread = (row, quarter of the stage's 16 columns)
        const int ptid = tid;
        const int row = ptid & (kTcM - 1), cq = ptid >> 7;
        const int i = it.y + row;
        const bool rok = i < nrow;
        float ra = 0.f, ru[Sh::P], rc[Sh::Q > 0 ? Sh::Q : 1];
        {
            const int ii = rok ? i : 0;
            ra = rs.a[ro + ii];
#pragma unroll
            for (int p = 0; p < Sh::P; ++p) ru[p] = p < P ? rs.u[(size_t)(ro + ii) * P + p] : 0.f;
#pragma unroll
            for (int q = 0; q < Sh::Q; ++q) rc[q] = q < Q ? rs.c[(size_t)(ro + ii) * Q + q] : 0.f;
        }
        const int op = rok ? rs.pos[ro + i] : 0;
        // phase data and positions of chunk c into ring slot `slot` (threads < 16)
        auto stage_cols = [&](int c, int slot) {
            if (ptid < kTcKc) {
                const int j = c * kTcKc + ptid;
                float* cj = scol[slot] + ptid * kTcColStride;
                if (j < ncol) {
                    const int e = co + j;
                    cj[0] = cs.a[e];
                    for (int q = 0; q < P; ++q) cj[1 + q] = cs.u[(size_t)e * P + q];
                    for (int q = 0; q < Q; ++q) cj[1 + P + q] = cs.c[(size_t)e * Q + q];
                    spos[slot][ptid] = cs.pos[e];
                } else {
                    spos[slot][ptid] = 0;
                }
            }
        };
        bool ok = true;
        int g = 0;
        for (int p = 0; p < npass && ok; ++p) {
            const int r0 = p * kTcR;
            const int R = min(kTcR, nrhs - r0), Rpad = (R + 15) & ~15;
            TcBItems I;
            tc_b_items(I, src, r0, R, Rpad, ptid);
            TcBLoad Lcur, Lnext;
            if (nchunk > 0) {
                stage_cols(0, g % S);
                producers_and(true);
                tc_load_b(Lcur, I, spos[g % S], ncol, src);
            }
            for (int c = 0; c < nchunk; ++c, ++g) {
                const int s = g % S, s1 = (g + 1) % S;
                const uint32_t u = (uint32_t)(g / S);
                // the stage's previous MMAs (chunk g - S) must be done before it is overwritten
                bool w = true;
                if (u > 0) w = mbar_wait(&bars->empty[s], (u - 1) & 1, status);
                const bool more = c + 1 < nchunk;
                if (more) stage_cols(c + 1, s1);
                ok = producers_and(w);
                if (!ok) break;
                if (more) tc_load_b(Lnext, I, spos[s1], ncol - (c + 1) * kTcKc, src);
                __nv_bfloat16* stg = ring + (size_t)s * Cfg::stage_elems;
                const int j0 = c * kTcKc;
                // A: this thread's row, columns 4 cq .. 4 cq + 3 = one core row of A_top and of A_bot
                {
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
                                for (int q = 0; q < Sh::Q; ++q)
                                    if (Sh::fixed || q < Q) sq = fmaf(rc[q], cj[1 + P + q], sq);
                                thp += sqrtf(sq);
                            }
                            thp -= rintf(thp);
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
                        *reinterpret_cast<uint4*>(stg + (NP + 1) * kTcAElems + o) =
                            make_uint4(bl[0], bl[1], bl[2], bl[3]);
                    }
                }
                tc_store_b<REFINE>(Lcur, I, stg + 2 * NP * kTcAElems);
                asm volatile("fence.proxy.async.shared::cta;");
                mbar_arrive(&bars->full[s]);
                if (more) Lcur = Lnext;
            }
            if (!ok) break;
            ok = producers_and(mbar_wait(&bars->done, (uint32_t)p & 1, status));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            tc_epilogue(tmem, warp, lane, Rpad, R, r0, rok, op, dst, nchunk == 0);
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(&bars->tfree);
        }
        if (!ok && ptid == 0) atomicExch(status, MIDBF_ETIMEOUT);
    }
    tc_teardown<S>(tmem, warp);
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
// tile); the right-hand sides come from the block's input positions.
struct TcBlock {
    long long img_off;   // element offset (BF16) of the block's first tile image
    int rows, cols;      // complex rows (outputs) and columns (inputs)
    int in_off, out_off; // offsets into the position arrays
};

struct TcStage {
    const TcBlock* blocks;
    const int* in_pos;      // positions of block inputs in the source space
    const int* out_pos;     // positions of block outputs in the destination space
    const __nv_bfloat16* img;
    const int2* items;      // (block, row tile)
};

template <bool REFINE>
__global__ void __launch_bounds__(kTcThreads, 1) k_blk_tc(TcStage st, VecRef<float> src, VecRef<float> dst, int nrhs,
                                                          int* status) {
    using Cfg = TcCfg<REFINE>;
    constexpr int S = Cfg::S, NP = Cfg::NP;
    static_assert(S >= 3, "slot reuse needs three ring stages");
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __nv_bfloat16* ring = reinterpret_cast<__nv_bfloat16*>(tc_smem_raw);
    TcBars<S>* bars = reinterpret_cast<TcBars<S>*>(tc_smem_raw + S * Cfg::stage_elems * 2);
    __shared__ __align__(16) int spos[S][kTcKc];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int2 it = st.items[blockIdx.x];
    const TcBlock bk = st.blocks[it.x];
    const int rt = it.y;
    const int nchunk = (bk.cols + kTcKc - 1) / kTcKc;
    const int npass = (nrhs + kTcR - 1) / kTcR;
    const int total = npass * nchunk;
    const __nv_bfloat16* tile0 = st.img + bk.img_off + (size_t)rt * nchunk * NP * kTcTileElems;
    constexpr uint32_t kCopyBytes = NP * kTcTileElems * 2;

    tc_setup<S>(bars, tid, warp);
    const uint32_t tmem = bars->taddr;

    if (warp == kTcProducers / 32) {
        // ---- MMA warp: bulk copies of the A tiles S - 1 chunks ahead, then the MMAs
        bool ok = true;
        int issued = 0;
        auto copy = [&](int gg) {
            const int s = gg % S;
            if (lane == 0) {
                mbar_expect_tx(&bars->aload[s], kCopyBytes);
                bulk_g2s(ring + (size_t)s * Cfg::stage_elems, tile0 + (size_t)(gg % nchunk) * NP * kTcTileElems,
                         kCopyBytes, &bars->aload[s]);
            }
        };
        for (; issued < total && issued < S; ++issued) copy(issued);
        int g = 0;
        for (int p = 0; p < npass && ok; ++p) {
            const int R = min(kTcR, nrhs - p * kTcR), Rpad = (R + 15) & ~15;
            const uint32_t idesc = umma_idesc_bf16(kTcM, Rpad);
            if (p > 0 && !mbar_wait(&bars->tfree, (uint32_t)(p - 1) & 1, status)) {
                ok = false;
                break;
            }
            for (int c = 0; c < nchunk; ++c, ++g) {
                const int s = g % S;
                if (!mbar_wait(&bars->full[s], (uint32_t)(g / S) & 1, status)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                if (lane == 0) {
                    tc_issue_stage<REFINE>(tmem, ring + (size_t)s * Cfg::stage_elems, idesc, c == 0);
                    umma_commit(&bars->empty[s]);
                }
                __syncwarp();
                // chunk g + S - 1 takes the stage of chunk g - 1 once its MMAs are done
                // (the MMAs of chunk g are queued behind them, so the tensor pipe stays fed)
                if (g >= 1 && issued < total && issued == g + S - 1) {
                    if (!mbar_wait(&bars->empty[(g - 1) % S], (uint32_t)((g - 1) / S) & 1, status)) {
                        ok = false;
                        break;
                    }
                    copy(issued);
                    ++issued;
                }
            }
            if (!ok) break;
            if (lane == 0) umma_commit(&bars->done);
            __syncwarp();
        }
        if (!ok && lane == 0) atomicExch(status, MIDBF_ETIMEOUT);
        tc_mma_drain(&bars->fin, lane, status);
        // copies that no producer waited for (after a timeout) land before the CTA exits
        if (lane == 0) {
            for (int gg = issued - 1; gg >= 0 && gg >= issued - S; --gg)
                mbar_wait(&bars->aload[gg % S], (uint32_t)(gg / S) & 1, nullptr);
        }
        __syncwarp();
    } else {
        // ---- producers
        const int ptid = tid;
        const int row = ptid & (kTcM - 1);
        const int i = rt * kTcM + row;
        const bool rok = i < bk.rows;
        const int op = rok ? st.out_pos[bk.out_off + i] : 0;
        auto stage_pos = [&](int c, int slot) {
            if (ptid < kTcKc) {
                const int j = c * kTcKc + ptid;
                spos[slot][ptid] = j < bk.cols ? st.in_pos[bk.in_off + j] : 0;
            }
        };
        bool ok = true;
        int g = 0;
        for (int p = 0; p < npass && ok; ++p) {
            const int r0 = p * kTcR;
            const int R = min(kTcR, nrhs - r0), Rpad = (R + 15) & ~15;
            TcBItems I;
            tc_b_items(I, src, r0, R, Rpad, ptid);
            TcBLoad Lcur, Lnext;
            if (nchunk > 0) {
                stage_pos(0, g % S);
                producers_and(true);
                tc_load_b(Lcur, I, spos[g % S], bk.cols, src);
            }
            for (int c = 0; c < nchunk; ++c, ++g) {
                const int s = g % S, s1 = (g + 1) % S;
                const bool more = c + 1 < nchunk;
                if (more) stage_pos(c + 1, s1);
                // the stage's A tiles have landed (and its previous MMAs are done: the
                // copy was issued after them)
                ok = producers_and(mbar_wait(&bars->aload[s], (uint32_t)(g / S) & 1, status));
                if (!ok) break;
                if (more) tc_load_b(Lnext, I, spos[s1], bk.cols - (c + 1) * kTcKc, src);
                __nv_bfloat16* stg = ring + (size_t)s * Cfg::stage_elems;
                // A_bot = (Im, Re) from A_top = (Re, -Im): 512 16-byte vectors per part
#pragma unroll
                for (int part = 0; part < NP; ++part) {
                    const uint4 a = reinterpret_cast<const uint4*>(stg + part * kTcAElems)[ptid];
                    reinterpret_cast<uint4*>(stg + (NP + part) * kTcAElems)[ptid] =
                        make_uint4(top_to_bot(a.x), top_to_bot(a.y), top_to_bot(a.z), top_to_bot(a.w));
                }
                tc_store_b<REFINE>(Lcur, I, stg + 2 * NP * kTcAElems);
                asm volatile("fence.proxy.async.shared::cta;");
                mbar_arrive(&bars->full[s]);
                if (more) Lcur = Lnext;
            }
            if (!ok) break;
            ok = producers_and(mbar_wait(&bars->done, (uint32_t)p & 1, status));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            tc_epilogue(tmem, warp, lane, Rpad, R, r0, rok, op, dst, nchunk == 0);
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(&bars->tfree);
        }
        if (!ok && ptid == 0) atomicExch(status, MIDBF_ETIMEOUT);
    }
    tc_teardown<S>(tmem, warp);
}

}  // namespace midbf_dev
