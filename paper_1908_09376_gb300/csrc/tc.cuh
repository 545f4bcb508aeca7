// Tensor-core (tcgen05) middle factor for many right-hand sides, sm_103a.
//
// For one S block (Sec. 3.5) and a tile of 128 rows, D (128 x 2R') =
// A (128 x 2K) * B' (2K x 2R') on the 5th-generation tensor cores, where
//   A  = the block's kernel entries exp(2 pi i Phi) generated on the fly in
//        BF16, complex entries interleaved (re, im) along K;
//   B' = the real embedding of the RHS block Y (K x R'):
//        B'[2k][2n] = Re Y, B'[2k][2n+1] = Im Y, B'[2k+1][2n] = -Im Y,
//        B'[2k+1][2n+1] = Re Y,
// so that D[:, 2n] + i D[:, 2n+1] = (S Y)[:, n] with FP32 accumulation in
// tensor memory.  With refinement each operand is split into BF16 hi + lo
// (lo = bf16(v - hi)) and D accumulates A_hi B_hi + A_hi B_lo + A_lo B_hi.
//
// Operands live in shared memory in the no-swizzle K-major core-matrix layout
// (8 rows x 16 bytes per core matrix; leading byte offset 128 between core
// matrices along K, stride byte offset (K/8)*128 between 8-row groups).  One
// thread issues the MMAs; tcgen05.commit arrives on an mbarrier per pipeline
// stage, so generating column chunk c+1 overlaps the MMAs of chunk c.  Every
// wait is bounded; a wait that gives up sets the plan's status word.
#pragma once

#include <cuda_bf16.h>

#include "kernels.cuh"

namespace midbf_dev {

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

// Bounded wait for the completion of the mbarrier phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
    uint32_t done = 0;
    for (int it = 0; it < (1 << 24) && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity));
    }
    return done != 0;
}

// Offset (elements) of (row r, k) in the K-major core-matrix layout with K columns.
__device__ __forceinline__ int core_off(int r, int k, int K) {
    return ((r >> 3) * (K >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo_half, __nv_bfloat16 hi_half) {
    return (uint32_t)__bfloat16_as_ushort(lo_half) | ((uint32_t)__bfloat16_as_ushort(hi_half) << 16);
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

constexpr int kTcM = 128;         // rows per item
constexpr int kTcCols = 32;       // complex columns per pipeline chunk (K' = 64)
constexpr int kTcK = 2 * kTcCols;
constexpr int kTcThreads = 256;
constexpr int kTcMaxR = 128;      // RHS per accumulator (N = 2 R' <= 256)
constexpr int kTcColStride = 12;  // reals per column of phase-split data (1 + P + Q <= 12)

template <bool REFINE>
__host__ __device__ constexpr size_t tc_smem_bytes() {
    // per stage: A (128 x 64) and B' (256 x 64) BF16, doubled for hi/lo
    return (size_t)2 * (REFINE ? 2 : 1) * ((size_t)kTcM * kTcK + (size_t)2 * kTcMaxR * kTcK) * 2 + 256;
}

// One CTA per item (block, 128 role-rows).  role rows/cols as in k_s_fly.
template <int PQ, bool REFINE, bool CONJ>
__global__ void __launch_bounds__(kTcThreads, 1) k_s_tc(SStage<float> st, SSide<float> rs, SSide<float> cs,
                                                        VecRef<float> src, VecRef<float> dst, int nrhs,
                                                        int row_is_row, int* status) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    using Sh = PhaseShape<PQ>;
    constexpr int NP = REFINE ? 2 : 1;
    __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(tc_smem_raw);                 // [stage][part][128*64]
    __nv_bfloat16* sB = sA + 2 * NP * kTcM * kTcK;                                    // [stage][part][256*64]
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sB + 2 * NP * 2 * kTcMaxR * kTcK);  // [2]
    uint32_t* taddr = reinterpret_cast<uint32_t*>(mbar + 2);
    __shared__ float scol[kTcCols * kTcColStride];
    __shared__ int spos[kTcCols];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int2 it = st.items[blockIdx.x];
    const int b = it.x;
    const int ro = row_is_row ? st.blk_rows[b] : st.blk_cols[b];
    const int co = row_is_row ? st.blk_cols[b] : st.blk_rows[b];
    const int nrow = row_is_row ? st.blk_nrow[b] : st.blk_ncol[b];
    const int ncol = row_is_row ? st.blk_ncol[b] : st.blk_nrow[b];
    const int P = Sh::fixed ? Sh::P : st.P;
    const int Q = Sh::fixed ? Sh::Q : st.Q;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(taddr)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *taddr;

    // this thread's row of the item (two threads per row, 16 columns each)
    const int row = tid & (kTcM - 1), half = tid >> 7;
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
    uint32_t commits[2] = {0, 0};   // commits issued per stage
    bool pending[2] = {false, false};  // latest commit of the stage not yet waited for
    bool ok = true;
    const int nchunk = (ncol + kTcCols - 1) / kTcCols;
    for (int r0 = 0; r0 < nrhs && ok; r0 += kTcMaxR) {
        const int nr = min(kTcMaxR, nrhs - r0);
        const int N = ((2 * nr + 15) / 16) * 16;
        const uint32_t idesc = umma_idesc_bf16(kTcM, N);
        for (int c = 0; c < nchunk && ok; ++c) {
            const int s = c & 1;
            // the stage's previous MMAs (chunk c-2) must be done before overwriting it;
            // the outcome of the bounded wait is made block-uniform before acting on it
            if (pending[s]) {
                const bool w = mbar_wait(&mbar[s], (commits[s] - 1) & 1);
                ok = __syncthreads_and(w) != 0;
                if (!ok) break;
                pending[s] = false;
            }
            // this chunk's column data (phase split, positions) into shared memory
            {
                const int jb = c * kTcCols;
                if (tid < kTcCols) {
                    const int j = jb + tid;
                    float* cj = scol + tid * kTcColStride;
                    if (j < ncol) {
                        const int e = co + j;
                        cj[0] = cs.a[e];
                        for (int p = 0; p < P; ++p) cj[1 + p] = cs.u[(size_t)e * P + p];
                        for (int q = 0; q < Q; ++q) cj[1 + P + q] = cs.c[(size_t)e * Q + q];
                        spos[tid] = cs.pos[e];
                    } else {
                        spos[tid] = 0;
                    }
                }
                __syncthreads();
            }
            __nv_bfloat16* A0 = sA + (size_t)(s * NP) * kTcM * kTcK;
            __nv_bfloat16* B0 = sB + (size_t)(s * NP) * 2 * kTcMaxR * kTcK;
            const int j0 = c * kTcCols;
            // A: this thread's row, 16 complex columns = 4 core-matrix rows of
            // 8 BF16 (4 complex entries) each, stored as 16-byte vectors
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
                uint32_t hv[4], lv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int jj = half * 16 + q4 * 4 + u;
                    const int j = j0 + jj;
                    float er = 0.f, ei = 0.f;
                    if (rok && j < ncol) {
                        const float* cj = scol + jj * kTcColStride;
                        float th = ra + cj[0];
#pragma unroll
                        for (int p = 0; p < Sh::P; ++p)
                            if (Sh::fixed || p < P) th = fmaf(ru[p], cj[1 + p], th);
                        if (Sh::Q > 0 && (Sh::fixed || Q > 0)) {
                            float sq = 0.f;
#pragma unroll
                            for (int q = 0; q < Sh::Q; ++q)
                                if (Sh::fixed || q < Q) sq = fmaf(rc[q], cj[1 + P + q], sq);
                            th += sqrtf(sq);
                        }
                        th -= rintf(th);
                        sincos2pi(th, &ei, &er);
                        if (CONJ) ei = -ei;
                    }
                    __nv_bfloat16 h0, l0, h1, l1;
                    split_bf16(er, h0, l0);
                    split_bf16(ei, h1, l1);
                    hv[u] = pack_bf16(h0, h1);
                    lv[u] = pack_bf16(l0, l1);
                }
                const int off = core_off(row, 2 * (half * 16 + q4 * 4), kTcK);
                *reinterpret_cast<uint4*>(A0 + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                if (REFINE) *reinterpret_cast<uint4*>(A0 + kTcM * kTcK + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
            }
            // B': for RHS n and 4 consecutive columns, rows 2n and 2n+1 of the
            // embedding are each one 16-byte core-matrix row
            for (int e = tid; e < (N / 2) * (kTcCols / 4); e += kTcThreads) {
                const int jq = e / (N / 2), n = e % (N / 2);   // consecutive threads: consecutive RHS
                uint32_t h0[4], h1[4], l0[4], l1[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int jj = jq * 4 + u;
                    const int j = j0 + jj;
                    float yr = 0.f, yi = 0.f;
                    if (n < nr && j < ncol) {
                        const cx<float> y = src.ptr[spos[jj] * src.ps + (r0 + n) * src.rs];
                        yr = y.x;
                        yi = y.y;
                    }
                    __nv_bfloat16 rh, rl, ih, il;
                    split_bf16(yr, rh, rl);
                    split_bf16(yi, ih, il);
                    h0[u] = pack_bf16(rh, __hneg(ih));   // row 2n:   ( Re, -Im )
                    h1[u] = pack_bf16(ih, rh);           // row 2n+1: ( Im,  Re )
                    l0[u] = pack_bf16(rl, __hneg(il));
                    l1[u] = pack_bf16(il, rl);
                }
                const int o0 = core_off(2 * n, 8 * jq, kTcK), o1 = core_off(2 * n + 1, 8 * jq, kTcK);
                *reinterpret_cast<uint4*>(B0 + o0) = make_uint4(h0[0], h0[1], h0[2], h0[3]);
                *reinterpret_cast<uint4*>(B0 + o1) = make_uint4(h1[0], h1[1], h1[2], h1[3]);
                if (REFINE) {
                    *reinterpret_cast<uint4*>(B0 + 2 * kTcMaxR * kTcK + o0) = make_uint4(l0[0], l0[1], l0[2], l0[3]);
                    *reinterpret_cast<uint4*>(B0 + 2 * kTcMaxR * kTcK + o1) = make_uint4(l1[0], l1[1], l1[2], l1[3]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t sbo_a = (kTcK / 8) * 128, sbo_b = (kTcK / 8) * 128;
                for (int kk = 0; kk < kTcK; kk += 16) {
                    const uint32_t koff = (uint32_t)(kk / 8) * 128;
                    const uint64_t ah = umma_desc(smem_u32(A0) + koff, 128, sbo_a);
                    const uint64_t bh = umma_desc(smem_u32(B0) + koff, 128, sbo_b);
                    const uint32_t acc0 = (c > 0 || kk > 0) ? 1u : 0u;
                    umma_bf16(tmem, ah, bh, idesc, acc0);
                    if (REFINE) {
                        const uint64_t al = umma_desc(smem_u32(A0 + kTcM * kTcK) + koff, 128, sbo_a);
                        const uint64_t bl = umma_desc(smem_u32(B0 + 2 * kTcMaxR * kTcK) + koff, 128, sbo_b);
                        umma_bf16(tmem, ah, bl, idesc, 1u);
                        umma_bf16(tmem, al, bh, idesc, 1u);
                    }
                }
                umma_commit(&mbar[s]);
            }
            commits[s]++;
            pending[s] = true;
        }
        if (!ok) break;
        // wait for the outstanding commits, the older stage first
        {
            const int last = (nchunk - 1) & 1;
            const int order[2] = {last ^ 1, last};
            for (int q = 0; q < 2 && ok; ++q) {
                const int sw = order[q];
                if (pending[sw]) {
                    const bool w = mbar_wait(&mbar[sw], (commits[sw] - 1) & 1);
                    ok = __syncthreads_and(w) != 0;
                    if (ok) pending[sw] = false;
                }
            }
        }
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        // epilogue: warps 0-3 columns [0, N/2), warps 4-7 columns [N/2, N), lanes = rows
        {
            const int wq = warp & 3;
            const int rr = wq * 32 + lane;
            const int ii = it.y + rr;
            const int cbeg = (warp >> 2) * (N / 2), cend = cbeg + N / 2;
            for (int c0 = cbeg; c0 < cend; c0 += 8) {
                uint32_t v[8];
                const uint32_t addr = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)c0;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                               "=r"(v[7])
                             : "r"(addr));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (ii < nrow) {
                    const int op = rs.pos[ro + ii];
#pragma unroll
                    for (int q = 0; q < 8; q += 2) {
                        const int n = (c0 + q) >> 1;
                        if (n < nr) dst.ptr[op * dst.ps + (r0 + n) * dst.rs] = cx<float>{__uint_as_float(v[q]), __uint_as_float(v[q + 1])};
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    if (!ok) {
        // report, then give the MMAs still in flight one more bounded wait
        // before the tensor memory is released
        if (tid == 0) atomicExch(status, MIDBF_ETIMEOUT);
        for (int sw = 0; sw < 2; ++sw)
            if (pending[sw]) mbar_wait(&mbar[sw], (commits[sw] - 1) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

}  // namespace midbf_dev

namespace midbf_dev {

// ---------------------------------------------------------------------------
// Tensor-core block GEMM for the interpolation/transfer stages (many RHS).
//
// In the tensor-core modes every V or U block is also stored densely (its
// identity entries included) as pre-tiled BF16 images: tile (row tile rt,
// column chunk c) holds rows [128 rt, 128 rt + 128) x complex columns
// [32 c, 32 c + 32) in exactly the shared-memory core-matrix layout used by
// the MMA (hi part, then lo part), so one cp.async.bulk moves a tile.  Two
// orientations are stored: the block itself (forward) and its conjugate
// transpose (adjoint).  The item is (block, row tile); the right-hand sides
// come from the block's input positions and are embedded into B' as in k_s_tc.
struct TcBlock {
    long long img_off;   // element offset (bf16) of the first tile image
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

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(mbar))
        : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}

constexpr int kTcTileElems = kTcM * kTcK;   // bf16 elements per tile part (16 KB)

template <bool REFINE>
__host__ __device__ constexpr size_t tcb_smem_bytes() {
    return (size_t)2 * (REFINE ? 2 : 1) * ((size_t)kTcM * kTcK + (size_t)2 * kTcMaxR * kTcK) * 2 + 256;
}

template <bool REFINE>
__global__ void __launch_bounds__(kTcThreads, 1) k_blk_tc(TcStage st, VecRef<float> src, VecRef<float> dst, int nrhs,
                                                          int* status) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    constexpr int NP = REFINE ? 2 : 1;
    __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(tc_smem_raw);                 // [stage][part][128*64]
    __nv_bfloat16* sB = sA + 2 * NP * kTcM * kTcK;                                    // [stage][part][256*64]
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sB + 2 * NP * 2 * kTcMaxR * kTcK);  // [2] MMA done
    uint64_t* fbar = mbar + 2;                                                        // [2] A tile landed
    uint32_t* taddr = reinterpret_cast<uint32_t*>(fbar + 2);
    __shared__ int spos[kTcCols];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int2 it = st.items[blockIdx.x];
    const TcBlock bk = st.blocks[it.x];
    const int rt = it.y;
    const int nchunk = (bk.cols + kTcCols - 1) / kTcCols;
    if (tid == 0) {
        for (int q = 0; q < 4; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[q])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(taddr)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *taddr;
    uint32_t commits[2] = {0, 0}, loads[2] = {0, 0}, issued[2] = {0, 0};
    bool pending[2] = {false, false};
    bool ok = true;
    const __nv_bfloat16* tile0 = st.img + bk.img_off + (size_t)rt * nchunk * NP * kTcTileElems;
    for (int r0 = 0; r0 < nrhs && ok; r0 += kTcMaxR) {
        const int nr = min(kTcMaxR, nrhs - r0);
        const int N = ((2 * nr + 15) / 16) * 16;
        const uint32_t idesc = umma_idesc_bf16(kTcM, N);
        for (int c = 0; c < nchunk && ok; ++c) {
            const int s = c & 1;
            if (pending[s]) {
                const bool w = mbar_wait(&mbar[s], (commits[s] - 1) & 1);
                ok = __syncthreads_and(w) != 0;
                if (!ok) break;
                pending[s] = false;
            }
            __nv_bfloat16* A0 = sA + (size_t)(s * NP) * kTcM * kTcK;
            __nv_bfloat16* B0 = sB + (size_t)(s * NP) * 2 * kTcMaxR * kTcK;
            // A tile(s) by one bulk copy
            if (tid == 0) {
                const uint32_t bytes = (uint32_t)(NP * kTcTileElems * 2);
                mbar_expect_tx(&fbar[s], bytes);
                bulk_g2s(A0, tile0 + (size_t)c * NP * kTcTileElems, bytes, &fbar[s]);
            }
            issued[s]++;
            if (tid < kTcCols) {
                const int j = c * kTcCols + tid;
                spos[tid] = j < bk.cols ? st.in_pos[bk.in_off + j] : 0;
            }
            __syncthreads();
            for (int e = tid; e < (N / 2) * (kTcCols / 4); e += kTcThreads) {
                const int jq = e / (N / 2), n = e % (N / 2);
                uint32_t h0[4], h1[4], l0[4], l1[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int jj = jq * 4 + u;
                    const int j = c * kTcCols + jj;
                    float yr = 0.f, yi = 0.f;
                    if (n < nr && j < bk.cols) {
                        const cx<float> y = src.ptr[spos[jj] * src.ps + (r0 + n) * src.rs];
                        yr = y.x;
                        yi = y.y;
                    }
                    __nv_bfloat16 rh, rl, ih, il;
                    split_bf16(yr, rh, rl);
                    split_bf16(yi, ih, il);
                    h0[u] = pack_bf16(rh, __hneg(ih));
                    h1[u] = pack_bf16(ih, rh);
                    l0[u] = pack_bf16(rl, __hneg(il));
                    l1[u] = pack_bf16(il, rl);
                }
                const int o0 = core_off(2 * n, 8 * jq, kTcK), o1 = core_off(2 * n + 1, 8 * jq, kTcK);
                *reinterpret_cast<uint4*>(B0 + o0) = make_uint4(h0[0], h0[1], h0[2], h0[3]);
                *reinterpret_cast<uint4*>(B0 + o1) = make_uint4(h1[0], h1[1], h1[2], h1[3]);
                if (REFINE) {
                    *reinterpret_cast<uint4*>(B0 + 2 * kTcMaxR * kTcK + o0) = make_uint4(l0[0], l0[1], l0[2], l0[3]);
                    *reinterpret_cast<uint4*>(B0 + 2 * kTcMaxR * kTcK + o1) = make_uint4(l1[0], l1[1], l1[2], l1[3]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;");
            {
                const bool w = mbar_wait(&fbar[s], loads[s] & 1);
                ok = __syncthreads_and(w) != 0;
                if (!ok) break;
                loads[s]++;
            }
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t sbo = (kTcK / 8) * 128;
                for (int kk = 0; kk < kTcK; kk += 16) {
                    const uint32_t koff = (uint32_t)(kk / 8) * 128;
                    const uint64_t ah = umma_desc(smem_u32(A0) + koff, 128, sbo);
                    const uint64_t bh = umma_desc(smem_u32(B0) + koff, 128, sbo);
                    umma_bf16(tmem, ah, bh, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                    if (REFINE) {
                        const uint64_t al = umma_desc(smem_u32(A0 + kTcM * kTcK) + koff, 128, sbo);
                        const uint64_t bl = umma_desc(smem_u32(B0 + 2 * kTcMaxR * kTcK) + koff, 128, sbo);
                        umma_bf16(tmem, ah, bl, idesc, 1u);
                        umma_bf16(tmem, al, bh, idesc, 1u);
                    }
                }
                umma_commit(&mbar[s]);
            }
            commits[s]++;
            pending[s] = true;
        }
        if (!ok) break;
        {
            const int last = (nchunk - 1) & 1;
            const int order[2] = {last ^ 1, last};
            for (int q = 0; q < 2 && ok; ++q) {
                const int sw = order[q];
                if (pending[sw]) {
                    const bool w = mbar_wait(&mbar[sw], (commits[sw] - 1) & 1);
                    ok = __syncthreads_and(w) != 0;
                    if (ok) pending[sw] = false;
                }
            }
        }
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        {
            const int wq = warp & 3;
            const int rr = wq * 32 + lane;
            const int ii = rt * kTcM + rr;
            const int cbeg = (warp >> 2) * (N / 2), cend = cbeg + N / 2;
            for (int c0 = cbeg; c0 < cend; c0 += 8) {
                uint32_t v[8];
                const uint32_t addr = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)c0;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                               "=r"(v[7])
                             : "r"(addr));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (nchunk == 0) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[q] = 0u;   // empty input side: the product is zero
                }
                if (ii < bk.rows) {
                    const int op = st.out_pos[bk.out_off + ii];
#pragma unroll
                    for (int q = 0; q < 8; q += 2) {
                        const int n = (c0 + q) >> 1;
                        if (n < nr)
                            dst.ptr[op * dst.ps + (r0 + n) * dst.rs] =
                                cx<float>{__uint_as_float(v[q]), __uint_as_float(v[q + 1])};
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    if (!ok) {
        if (tid == 0) atomicExch(status, MIDBF_ETIMEOUT);
        for (int sw = 0; sw < 2; ++sw) {
            if (pending[sw]) mbar_wait(&mbar[sw], (commits[sw] - 1) & 1);
            if (issued[sw] > loads[sw]) mbar_wait(&fbar[sw], loads[sw] & 1);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

}  // namespace midbf_dev
