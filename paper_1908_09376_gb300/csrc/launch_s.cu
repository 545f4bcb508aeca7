// Launchers of the middle factor made on the fly on the SIMT kernels (Sec. 3.5).
#include "dev_plan.cuh"

namespace midbf_gpu {

template <class R, int RT, int NR, bool CJ, int PQ>
void launch_s_t(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, cudaStream_t s, bool persist) {
    SStage<R> st = ds.ss;
    const size_t sm = s_fly_smem<R>(st.P, st.Q, RT, NR);
    const bool four = RT == 4;
    st.items = !CJ ? (four ? ds.items_rows4 : ds.items_rows) : (four ? ds.items_cols4 : ds.items_cols);
    const int n = !CJ ? (four ? ds.n_items_rows4 : ds.n_items_rows) : (four ? ds.n_items_cols4 : ds.n_items_cols);
    if (n == 0) return;
    const SSide<R>& rside = !CJ ? ds.srows : ds.scols;
    const SSide<R>& cside = !CJ ? ds.scols : ds.srows;
    if (persist) {
        auto kf = k_s_fly_p<R, RT, NR, CJ, PQ>;
        set_smem(kf, sm);
        kf<<<grid_for(reinterpret_cast<const void*>(kf), sm, n, true), kThreads, sm, s>>>(st, rside, cside, !CJ ? 1 : 0,
                                                                                       src, dst, nrhs, n);
    } else {
        auto kf = k_s_fly<R, RT, NR, CJ, PQ>;
        set_smem(kf, sm);
        kf<<<n, kThreads, sm, s>>>(st, rside, cside, !CJ ? 1 : 0, src, dst, nrhs);
    }
}

// FP32: 128-row items for up to 4 RHS per pass, phase shape fixed at compile
// time for the workload families; one RHS on a middle factor of few large
// blocks (fewer 128-row items than two per SM) runs as 64-row items, which
// doubles the CTAs.  FP64: the general shape or the distance form (the plain
// form stores the middle factor by default).
template <class R, bool CJ, int PQ>
void launch_s_pq(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, int nr, cudaStream_t s, bool persist) {
    if constexpr (sizeof(R) == 4) {
        const bool few = (CJ ? ds.n4_cols_stage : ds.n4_rows_stage) < 2 * sm_count();
        switch (nr) {
            case 1:
                if (few) launch_s_t<R, 2, 1, CJ, PQ>(ds, src, dst, nrhs, s, persist);
                else launch_s_t<R, 4, 1, CJ, PQ>(ds, src, dst, nrhs, s, persist);
                break;
            case 2: launch_s_t<R, 4, 2, CJ, PQ>(ds, src, dst, nrhs, s, persist); break;
            case 4: launch_s_t<R, 4, 4, CJ, PQ>(ds, src, dst, nrhs, s, persist); break;
            case 8: launch_s_t<R, 2, 8, CJ, PQ>(ds, src, dst, nrhs, s, persist); break;
            default: launch_s_t<R, 2, 16, CJ, PQ>(ds, src, dst, nrhs, s, persist);
        }
    } else {
        constexpr int PQ64 = PQ == kShapeDistance ? kShapeDistance : 0;
        switch (nr) {
            case 1: launch_s_t<R, 2, 1, CJ, PQ64>(ds, src, dst, nrhs, s, persist); break;
            case 2: launch_s_t<R, 2, 2, CJ, PQ64>(ds, src, dst, nrhs, s, persist); break;
            case 4: launch_s_t<R, 2, 4, CJ, PQ64>(ds, src, dst, nrhs, s, persist); break;
            default: launch_s_t<R, 2, 8, CJ, PQ64>(ds, src, dst, nrhs, s, persist);
        }
    }
}

template <class R, bool CJ>
void launch_s_nr(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, int nr, cudaStream_t s, bool persist) {
    switch (s_shape(ds)) {
        case 1: launch_s_pq<R, CJ, 1>(ds, src, dst, nrhs, nr, s, persist); break;
        case 2: launch_s_pq<R, CJ, 2>(ds, src, dst, nrhs, nr, s, persist); break;
        case 3: launch_s_pq<R, CJ, 3>(ds, src, dst, nrhs, nr, s, persist); break;
        case 4: launch_s_pq<R, CJ, 4>(ds, src, dst, nrhs, nr, s, persist); break;
        case 5: launch_s_pq<R, CJ, 5>(ds, src, dst, nrhs, nr, s, persist); break;
        case kShapeDistance: launch_s_pq<R, CJ, kShapeDistance>(ds, src, dst, nrhs, nr, s, persist); break;
        default: launch_s_pq<R, CJ, 0>(ds, src, dst, nrhs, nr, s, persist);
    }
}

// The accurate phase (FP32, one RHS per pass, 64-row items).
template <bool CJ, int PQ>
void launch_s_df_t(const DevStage<float>& ds, VecRef<float> src, VecRef<float> dst, int nrhs, cudaStream_t s,
                   bool persist) {
    SStage<float> st = ds.ss;
    const size_t sm = s_fly_df_smem(st.P, st.Q, 2);
    st.items = !CJ ? ds.items_rows : ds.items_cols;
    const int n = !CJ ? ds.n_items_rows : ds.n_items_cols;
    if (n == 0) return;
    const SSide<float>& rside = !CJ ? ds.srows : ds.scols;
    const SSide<float>& cside = !CJ ? ds.scols : ds.srows;
    if (persist) {
        auto kf = k_s_fly_df_p<2, CJ, PQ>;
        set_smem(kf, sm);
        kf<<<grid_for(reinterpret_cast<const void*>(kf), sm, n, true), kThreads, sm, s>>>(st, rside, cside, !CJ ? 1 : 0,
                                                                                       src, dst, nrhs, n);
    } else {
        auto kf = k_s_fly_df<2, CJ, PQ>;
        set_smem(kf, sm);
        kf<<<n, kThreads, sm, s>>>(st, rside, cside, !CJ ? 1 : 0, src, dst, nrhs);
    }
}

template <bool CJ>
void launch_s_df(const DevStage<float>& ds, VecRef<float> src, VecRef<float> dst, int nrhs, cudaStream_t s,
                 bool persist) {
    switch (phase_shape_code(ds.ss.P, ds.ss.Q)) {
        case 1: launch_s_df_t<CJ, 1>(ds, src, dst, nrhs, s, persist); break;
        case 2: launch_s_df_t<CJ, 2>(ds, src, dst, nrhs, s, persist); break;
        case 3: launch_s_df_t<CJ, 3>(ds, src, dst, nrhs, s, persist); break;
        case 4: launch_s_df_t<CJ, 4>(ds, src, dst, nrhs, s, persist); break;
        case 5: launch_s_df_t<CJ, 5>(ds, src, dst, nrhs, s, persist); break;
        default: launch_s_df_t<CJ, 0>(ds, src, dst, nrhs, s, persist);
    }
}

template <class R>
void launch_s(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, bool adjoint, cudaStream_t s, int force,
              bool persist) {
    if constexpr (sizeof(R) == 4) {
        if (ds.s_df) {
            if (adjoint) launch_s_df<true>(ds, src, dst, nrhs, s, persist);
            else launch_s_df<false>(ds, src, dst, nrhs, s, persist);
            CK(cudaGetLastError());
            return;
        }
    }
    const int nr = forced_or_pick<R>(force, nrhs, [&](int q) { return s_fly_smem<R>(ds.ss.P, ds.ss.Q, q <= 4 && sizeof(R) == 4 ? 4 : 2, q); });
    if (adjoint) launch_s_nr<R, true>(ds, src, dst, nrhs, nr, s, persist);
    else launch_s_nr<R, false>(ds, src, dst, nrhs, nr, s, persist);
    CK(cudaGetLastError());
}

// Many RHS in FP32: the register-tiled GEMM form of the middle factor
// (k_s_gemm), 64-row items.
template <bool CJ, int PQ>
void launch_s_gemm_t(const DevStage<float>& ds, VecRef<float> src, VecRef<float> dst, int nrhs, cudaStream_t s) {
    SStage<float> st = ds.ss;
    st.items = !CJ ? ds.items_rows : ds.items_cols;
    const int n = !CJ ? ds.n_items_rows : ds.n_items_cols;
    if (n == 0) return;
    const size_t sm = s_gemm_smem(st.P, st.Q);
    auto kf = k_s_gemm<CJ, PQ>;
    set_smem(kf, sm);
    kf<<<n, kThreads, sm, s>>>(st, !CJ ? ds.srows : ds.scols, !CJ ? ds.scols : ds.srows, !CJ ? 1 : 0, src, dst, nrhs);
}

template <bool CJ>
void launch_s_gemm_cj(const DevStage<float>& ds, VecRef<float> src, VecRef<float> dst, int nrhs, cudaStream_t s) {
    switch (s_shape(ds)) {
        case 1: launch_s_gemm_t<CJ, 1>(ds, src, dst, nrhs, s); break;
        case 2: launch_s_gemm_t<CJ, 2>(ds, src, dst, nrhs, s); break;
        case 3: launch_s_gemm_t<CJ, 3>(ds, src, dst, nrhs, s); break;
        case 4: launch_s_gemm_t<CJ, 4>(ds, src, dst, nrhs, s); break;
        case 5: launch_s_gemm_t<CJ, 5>(ds, src, dst, nrhs, s); break;
        case kShapeDistance: launch_s_gemm_t<CJ, kShapeDistance>(ds, src, dst, nrhs, s); break;
        default: launch_s_gemm_t<CJ, 0>(ds, src, dst, nrhs, s);
    }
}

void launch_s_gemm(const DevStage<float>& ds, VecRef<float> src, VecRef<float> dst, int nrhs, bool adjoint,
                   cudaStream_t s) {
    if (ds.s_df) fail(MIDBF_EINTERNAL, "the GEMM form of the middle factor takes the FP32 phase");
    if (adjoint) launch_s_gemm_cj<true>(ds, src, dst, nrhs, s);
    else launch_s_gemm_cj<false>(ds, src, dst, nrhs, s);
    CK(cudaGetLastError());
}

template void launch_s<float>(const DevStage<float>&, VecRef<float>, VecRef<float>, int, bool, cudaStream_t, int, bool);
template void launch_s<double>(const DevStage<double>&, VecRef<double>, VecRef<double>, int, bool, cudaStream_t, int, bool);

}  // namespace midbf_gpu
