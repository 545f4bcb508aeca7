// Launchers of the tensor-core stages: RHS packing, middle factor, V / U blocks.
#include "dev_plan.cuh"

namespace midbf_gpu {

// Tensor-core stages run in groups of at most kTcR RHS.  Each group first
// packs the stage input into per-chunk B images (k_pack_b, in the workspace
// area tc_bimg) and then multiplies.
inline VecRef<float> rhs_shift(VecRef<float> v, int r0) {
    v.ptr += (long long)r0 * v.rs;
    return v;
}

void launch_pack(const TcPack& pk, VecRef<float> src, int R, bool refine, __nv_bfloat16* bimg, cudaStream_t s) {
    if (pk.nchunks == 0) return;
    const int Rpad = (R + 15) & ~15;
    const int grid = std::min(pk.nchunks, 152 * 8);
    if (refine) k_pack_b<true><<<grid, 256, 0, s>>>(pk, src, R, Rpad, bimg);
    else k_pack_b<false><<<grid, 256, 0, s>>>(pk, src, R, Rpad, bimg);
}

template <int PQ, bool RF, bool CJ>
void launch_tc_t(const DevStage<float>& ds, VecRef<float> dst, int R, const __nv_bfloat16* bimg, int* status,
                 cudaStream_t s) {
    SStage<float> st = ds.ss;
    const size_t sm = tc_smem_bytes<RF>();
    auto kf = k_s_tc<PQ, RF, CJ>;
    set_smem(kf, sm);
    if (!CJ) {
        st.items = ds.items_rows4;
        kf<<<ds.n_items_rows4, kTcThreads, sm, s>>>(st, ds.srows, ds.scols, ds.chunk0_s[0], bimg, dst, R, 1, status);
    } else {
        st.items = ds.items_cols4;
        kf<<<ds.n_items_cols4, kTcThreads, sm, s>>>(st, ds.scols, ds.srows, ds.chunk0_s[1], bimg, dst, R, 0, status);
    }
}

template <bool RF, bool CJ>
void launch_tc_rc(const DevStage<float>& ds, VecRef<float> dst, int R, const __nv_bfloat16* bimg, int* status,
                  cudaStream_t s) {
    switch (s_shape(ds)) {
        case 1: launch_tc_t<1, RF, CJ>(ds, dst, R, bimg, status, s); break;
        case 2: launch_tc_t<2, RF, CJ>(ds, dst, R, bimg, status, s); break;
        case 3: launch_tc_t<3, RF, CJ>(ds, dst, R, bimg, status, s); break;
        case 4: launch_tc_t<4, RF, CJ>(ds, dst, R, bimg, status, s); break;
        case 5: launch_tc_t<5, RF, CJ>(ds, dst, R, bimg, status, s); break;
        case kShapeDistance: launch_tc_t<kShapeDistance, RF, CJ>(ds, dst, R, bimg, status, s); break;
        default: launch_tc_t<0, RF, CJ>(ds, dst, R, bimg, status, s);
    }
}

// Middle factor on the tensor cores.
void launch_tc(const DevStage<float>& ds, VecRef<float> src, VecRef<float> dst, int nrhs, bool adjoint, bool refine,
               __nv_bfloat16* bimg, int* status, cudaStream_t s) {
    const int o = adjoint ? 1 : 0;
    for (int r0 = 0; r0 < nrhs; r0 += kTcR) {
        const int R = std::min(kTcR, nrhs - r0);
        launch_pack(ds.pk[o], rhs_shift(src, r0), R, refine, bimg, s);
        const VecRef<float> d = rhs_shift(dst, r0);
        if (refine) {
            if (adjoint) launch_tc_rc<true, true>(ds, d, R, bimg, status, s);
            else launch_tc_rc<true, false>(ds, d, R, bimg, status, s);
        } else {
            if (adjoint) launch_tc_rc<false, true>(ds, d, R, bimg, status, s);
            else launch_tc_rc<false, false>(ds, d, R, bimg, status, s);
        }
    }
    CK(cudaGetLastError());
}

// V / U stage on the tensor cores: o = 0 forward, 1 adjoint orientation.
void launch_blk_tc(const DevStage<float>& ds, int o, VecRef<float> src, VecRef<float> dst, int nrhs, bool refine,
                   __nv_bfloat16* bimg, int* status, cudaStream_t s) {
    if (ds.n_tc_items[o] == 0) return;
    for (int r0 = 0; r0 < nrhs; r0 += kTcR) {
        const int R = std::min(kTcR, nrhs - r0);
        launch_pack(ds.pk[o], rhs_shift(src, r0), R, refine, bimg, s);
        const VecRef<float> d = rhs_shift(dst, r0);
        const bool small = ((R + 15) & ~15) <= kTcRSmall;
        auto go = [&](auto kf, size_t sm) {
            set_smem(kf, sm);
            kf<<<ds.n_tc_items[o], kTcThreads, sm, s>>>(ds.tcs[o], bimg, d, R, status);
        };
        if (refine) {
            if (small) go(k_blk_tc<true, true>, TcCfgSmall<true>::smem);
            else go(k_blk_tc<true, false>, TcCfg<true>::smem);
        } else {
            if (small) go(k_blk_tc<false, true>, TcCfgSmall<false>::smem);
            else go(k_blk_tc<false, false>, TcCfg<false>::smem);
        }
    }
    CK(cudaGetLastError());
}

// Bytes of the B-image area of the workspace for nrhs RHS (0 outside the
// tensor-core modes): the largest stage's chunks at one group of <= kTcR RHS.

// Self-test of the failure detection: one thread per CTA waits, with the
// bounded wait of the tensor-core pipelines, on an mbarrier that nothing
// arrives on.  The wait gives up after its time limit (or at once when
// another CTA has already set the status word), the thread sets
// MIDBF_ETIMEOUT and the CTA exits; no TMEM, no bulk copy is involved.
__global__ void k_wait_selftest(int* status) {
    __shared__ __align__(8) uint64_t bar;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    if (!mbar_wait(&bar, 0, status)) atomicExch(status, MIDBF_ETIMEOUT);
}

void launch_wait_selftest(int* status, int ctas, cudaStream_t s) {
    k_wait_selftest<<<ctas, 1, 0, s>>>(status);
    CK(cudaGetLastError());
}
}  // namespace midbf_gpu
