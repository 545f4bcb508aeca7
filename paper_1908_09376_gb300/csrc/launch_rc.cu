// Launchers of the interpolation / transfer stages on the SIMT kernels
// (pattern R: narrow from wide; pattern C: wide from narrow; Sec. 3.2 IDs).
#include "dev_plan.cuh"

namespace midbf_gpu {

template <class R, int RT, int NR, bool CJ>
void launch_r_t(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, cudaStream_t s, bool persist) {
    const size_t sm = pattern_r_smem<R>(ds.max_nred, RT, NR);
    const int n = ds.n_items_r;
    if (persist) {
        auto kf = k_pattern_r_p<R, RT, NR, CJ>;
        set_smem(kf, sm);
        kf<<<grid_for(reinterpret_cast<const void*>(kf), sm, n, true), kThreads, sm, s>>>(ds.ids, src, dst, nrhs, n);
    } else {
        auto kf = NR >= 16 ? k_pattern_r16<R, RT, NR, CJ> : k_pattern_r<R, RT, NR, CJ>;
        set_smem(kf, sm);
        kf<<<n, kThreads, sm, s>>>(ds.ids, src, dst, nrhs);
    }
}

template <class R, int RT, bool CJ>
void launch_r_nr(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, int nr, cudaStream_t s, bool persist) {
    switch (nr) {
        case 1: launch_r_t<R, RT, 1, CJ>(ds, src, dst, nrhs, s, persist); break;
        case 2: launch_r_t<R, RT, 2, CJ>(ds, src, dst, nrhs, s, persist); break;
        case 4: launch_r_t<R, RT, 4, CJ>(ds, src, dst, nrhs, s, persist); break;
        case 8: launch_r_t<R, RT, 8, CJ>(ds, src, dst, nrhs, s, persist); break;
        default:
            if constexpr (sizeof(R) == 4) launch_r_t<R, RT, 16, CJ>(ds, src, dst, nrhs, s, persist);
            else launch_r_t<R, RT, 8, CJ>(ds, src, dst, nrhs, s, persist);
    }
}

// The one-RHS cluster form (k_pattern_r_cl): a cluster of cl CTAs per item.
template <class R, int RT, bool CJ>
void launch_r_cl_t(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int cl, cudaStream_t s) {
    const size_t sm = pattern_r_cl_smem<R>(ds.max_nred, RT);
    auto kf = k_pattern_r_cl<R, RT, CJ>;
    set_smem(kf, sm);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ds.n_items_r * (unsigned)cl, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, kf, ds.ids, src, dst));
}

template <class R>
void launch_r_cluster(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, bool conj, int cl, cudaStream_t s) {
    if (ds.n_items_r == 0) return;
    if (cl < 2 || cl > kMaxRowCluster) fail(MIDBF_EINTERNAL, "row cluster size out of range");
    if (ds.rt == 1) {
        if (conj) launch_r_cl_t<R, 1, true>(ds, src, dst, cl, s);
        else launch_r_cl_t<R, 1, false>(ds, src, dst, cl, s);
    } else {
        if (conj) launch_r_cl_t<R, 2, true>(ds, src, dst, cl, s);
        else launch_r_cl_t<R, 2, false>(ds, src, dst, cl, s);
    }
}

template <class R>
void launch_r(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, bool conj, cudaStream_t s, int force,
              bool persist) {
    if (ds.n_items_r == 0) return;
    const int nr = forced_or_pick<R>(force, nrhs, [&](int q) { return pattern_r_smem<R>(ds.max_nred, ds.rt, q); });
    if (ds.rt == 1) {
        if (conj) launch_r_nr<R, 1, true>(ds, src, dst, nrhs, nr, s, persist);
        else launch_r_nr<R, 1, false>(ds, src, dst, nrhs, nr, s, persist);
    } else {
        if (conj) launch_r_nr<R, 2, true>(ds, src, dst, nrhs, nr, s, persist);
        else launch_r_nr<R, 2, false>(ds, src, dst, nrhs, nr, s, persist);
    }
    CK(cudaGetLastError());
}

template <class R, int NR, bool CJ>
void launch_c_t(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, cudaStream_t s, bool persist) {
    const size_t sm = pattern_c_smem<R>(ds.max_narrow, ds.max_nsub, kRangeC, NR);
    const int n = ds.n_items_c;
    if (persist) {
        auto kf = k_pattern_c_p<R, NR, CJ>;
        set_smem(kf, sm);
        kf<<<grid_for(reinterpret_cast<const void*>(kf), sm, n, true), kThreads, sm, s>>>(ds.ids, src, dst, nrhs, n);
    } else {
        auto kf = k_pattern_c<R, NR, CJ>;
        set_smem(kf, sm);
        kf<<<n, kThreads, sm, s>>>(ds.ids, src, dst, nrhs);
    }
}

template <class R, bool CJ>
void launch_c_nr(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, int nr, cudaStream_t s, bool persist) {
    switch (nr) {
        case 1: launch_c_t<R, 1, CJ>(ds, src, dst, nrhs, s, persist); break;
        case 2: launch_c_t<R, 2, CJ>(ds, src, dst, nrhs, s, persist); break;
        case 4: launch_c_t<R, 4, CJ>(ds, src, dst, nrhs, s, persist); break;
        case 8: launch_c_t<R, 8, CJ>(ds, src, dst, nrhs, s, persist); break;
        default:
            if constexpr (sizeof(R) == 4) launch_c_t<R, 16, CJ>(ds, src, dst, nrhs, s, persist);
            else launch_c_t<R, 8, CJ>(ds, src, dst, nrhs, s, persist);
    }
}

template <class R>
void launch_c(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, bool conj, cudaStream_t s, int force,
              bool persist) {
    if (ds.n_items_c == 0) return;
    if (nrhs == 1 && (force == 0 || force == MIDBF_CHOICE_COLUMN1)) {
        const size_t sm = pattern_c1_smem<R>(ds.max_narrow, ds.max_nsub);
        if (sm <= kSmemCap) {
            const int n = ds.n_items_c1;
            if (persist) {
                auto kf = conj ? k_pattern_c1_p<R, true> : k_pattern_c1_p<R, false>;
                set_smem(kf, sm);
                kf<<<grid_for(reinterpret_cast<const void*>(kf), sm, n, true), kThreads, sm, s>>>(ds.ids1, src, dst, n);
            } else {
                auto kf = conj ? k_pattern_c1<R, true> : k_pattern_c1<R, false>;
                set_smem(kf, sm);
                kf<<<n, kThreads, sm, s>>>(ds.ids1, src, dst);
            }
            CK(cudaGetLastError());
            return;
        }
    }
    const int nr = forced_or_pick<R>(force, nrhs, [&](int q) { return pattern_c_smem<R>(ds.max_narrow, ds.max_nsub, kRangeC, q); });
    if (conj) launch_c_nr<R, true>(ds, src, dst, nrhs, nr, s, persist);
    else launch_c_nr<R, false>(ds, src, dst, nrhs, nr, s, persist);
    CK(cudaGetLastError());
}

// One RHS, narrow IDs (every rank <= 64): a warp per sub-block for pattern R,
// a lane per column for pattern C.
template <class R>
void launch_r_narrow(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, bool conj, cudaStream_t s) {
    if (ds.n_subs == 0) return;
    const int grid = (ds.n_subs + kWarps - 1) / kWarps;
    if (ds.max_k <= 32) {
        if (conj) k_pattern_r1n<R, 1, true><<<grid, kThreads, 0, s>>>(ds.ids, src, dst, ds.n_subs);
        else k_pattern_r1n<R, 1, false><<<grid, kThreads, 0, s>>>(ds.ids, src, dst, ds.n_subs);
    } else {
        if (conj) k_pattern_r1n<R, 2, true><<<grid, kThreads, 0, s>>>(ds.ids, src, dst, ds.n_subs);
        else k_pattern_r1n<R, 2, false><<<grid, kThreads, 0, s>>>(ds.ids, src, dst, ds.n_subs);
    }
    CK(cudaGetLastError());
}

template <class R>
void launch_c_narrow(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, bool conj, cudaStream_t s) {
    if (ds.n_items_c1 == 0) return;
    // many small blocks: a warp per block (the same results bit for bit)
    const int per_warp = ds.max_narrow + ds.max_m;
    const size_t smw = (size_t)kWarps * per_warp * sizeof(cx<R>);
    if (ds.n_blocks >= kWarpBlocksPerSm * sm_count() && smw <= kWarpBlockSmem) {
        auto kw = conj ? k_pattern_c1w<R, true> : k_pattern_c1w<R, false>;
        set_smem(kw, smw);
        kw<<<(ds.n_blocks + kWarps - 1) / kWarps, kThreads, smw, s>>>(ds.ids1, src, dst, ds.n_blocks, per_warp);
        CK(cudaGetLastError());
        return;
    }
    const size_t sm = pattern_c_smem<R>(ds.max_narrow, ds.max_nsub, kRangeC1, 1);
    auto kf = conj ? k_pattern_c1n<R, true> : k_pattern_c1n<R, false>;
    set_smem(kf, sm);
    kf<<<ds.n_items_c1, kThreads, sm, s>>>(ds.ids1, src, dst);
    CK(cudaGetLastError());
}

// Many RHS in FP32: the column pattern as a register-tiled GEMM (k_c_gemm)
// over the pattern-C items.
void launch_c_gemm(const DevStage<float>& ds, VecRef<float> src, VecRef<float> dst, int nrhs, bool conj,
                   cudaStream_t s) {
    if (ds.n_items_c == 0) return;
    const size_t sm = c_gemm_smem();
    auto kf = conj ? k_c_gemm<true> : k_c_gemm<false>;
    set_smem(kf, sm);
    kf<<<ds.n_items_c, kThreads, sm, s>>>(ds.ids, src, dst, nrhs);
    CK(cudaGetLastError());
}

// Many RHS in FP32: the row pattern as a register-tiled GEMM (k_r_gemm) over
// the row items (32 or 64 rows each).
void launch_r_gemm(const DevStage<float>& ds, VecRef<float> src, VecRef<float> dst, int nrhs, bool conj,
                   cudaStream_t s) {
    if (ds.n_items_r == 0) return;
    const int rows = 32 * ds.rt;
    if (rows > kRgRows) fail(MIDBF_EINTERNAL, "row items larger than the row GEMM tile");
    const size_t sm = r_gemm_smem();
    auto kf = conj ? k_r_gemm<true> : k_r_gemm<false>;
    set_smem(kf, sm);
    kf<<<ds.n_items_r, kThreads, sm, s>>>(ds.ids, src, dst, nrhs, rows);
    CK(cudaGetLastError());
}

template void launch_r_narrow<float>(const DevStage<float>&, VecRef<float>, VecRef<float>, bool, cudaStream_t);
template void launch_r_narrow<double>(const DevStage<double>&, VecRef<double>, VecRef<double>, bool, cudaStream_t);
template void launch_c_narrow<float>(const DevStage<float>&, VecRef<float>, VecRef<float>, bool, cudaStream_t);
template void launch_c_narrow<double>(const DevStage<double>&, VecRef<double>, VecRef<double>, bool, cudaStream_t);

template void launch_r_cluster<float>(const DevStage<float>&, VecRef<float>, VecRef<float>, bool, int, cudaStream_t);
template void launch_r_cluster<double>(const DevStage<double>&, VecRef<double>, VecRef<double>, bool, int, cudaStream_t);
template void launch_r<float>(const DevStage<float>&, VecRef<float>, VecRef<float>, int, bool, cudaStream_t, int, bool);
template void launch_r<double>(const DevStage<double>&, VecRef<double>, VecRef<double>, int, bool, cudaStream_t, int, bool);
template void launch_c<float>(const DevStage<float>&, VecRef<float>, VecRef<float>, int, bool, cudaStream_t, int, bool);
template void launch_c<double>(const DevStage<double>&, VecRef<double>, VecRef<double>, int, bool, cudaStream_t, int, bool);

}  // namespace midbf_gpu
