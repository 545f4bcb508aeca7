// Batched apply over many instances (midbf_apply_batched).
#include "dev_plan.cuh"

namespace midbf_gpu {

// ---------------------------------------------------------------------------
// Batched apply: level index q of every instance in one group of launches.
// Forward instances run their stage q, adjoint instances their stage ns-1-q;
// instances are grouped by kernel variant (pattern, rows per lane, RHS tile,
// phase shape) and up to kBatch instances share a launch.
template <class R>
const std::vector<DevStage<R>>& stages_of(const midbf_dplan* dp);
template <>
const std::vector<DevStage<float>>& stages_of<float>(const midbf_dplan* dp) { return dp->st32; }
template <>
const std::vector<DevStage<double>>& stages_of<double>(const midbf_dplan* dp) { return dp->st64; }

size_t instance_workspace(const midbf_dplan* dp, int nrhs) {
    const size_t ce = dp->precision == MIDBF_FP32 ? 8 : 16;
    const size_t b = 2 * (size_t)std::max<int64_t>(dp->max_space, 1) * (size_t)nrhs * ce;
    return (b + 255) / 256 * 256;
}

enum { BT_R = 0, BT_C = 1, BT_C1 = 2, BT_S = 3 };

template <class R, class E>
void launch_batch_group(const midbf_dplan* const* dps, const std::array<int, 4>& key, const E* ents, int n,
                        const int* nrhs, const int* adjoint, cudaStream_t s) {
    const int type = key[0], rt = key[1], nr = key[2], pq = key[3];
    if (type == BT_S) {
        BatchS<R> a{};
        a.ninst = n;
        size_t sm = 0;
        int items = 0;
        for (int k = 0; k < n; ++k) {
            const E& e = ents[k];
            const DevStage<R>& ds = stages_of<R>(dps[e.i])[e.sidx];
            const bool adj = adjoint[e.i] != 0;
            a.st[k] = ds.ss;
            const bool four = rt == 4;
            a.st[k].items = adj ? (four ? ds.items_cols4 : ds.items_cols) : (four ? ds.items_rows4 : ds.items_rows);
            a.rs[k] = adj ? ds.scols : ds.srows;
            a.cs[k] = adj ? ds.srows : ds.scols;
            a.src[k] = e.src;
            a.dst[k] = e.dst;
            a.nrhs[k] = nrhs[e.i];
            a.conj[k] = adj;
            a.item0[k] = items;
            items += adj ? (four ? ds.n_items_cols4 : ds.n_items_cols) : (four ? ds.n_items_rows4 : ds.n_items_rows);
            sm = std::max(sm, s_fly_smem<R>(ds.ss.P, ds.ss.Q, rt, nr));
        }
        a.item0[n] = items;
        if (items == 0) return;
#define LB(RT_, NR_, PQ_)                                        \
    {                                                            \
        auto kf = k_batch_s<R, RT_, NR_, PQ_>;                   \
        set_smem(kf, sm);                                        \
        kf<<<items, kThreads, sm, s>>>(a);                       \
    }
        if constexpr (sizeof(R) == 4) {
            auto go = [&](auto pqc) {
                constexpr int P_ = decltype(pqc)::value;
                switch (nr) {
                    case 1: LB(4, 1, P_) break;
                    case 2: LB(4, 2, P_) break;
                    case 4: LB(4, 4, P_) break;
                    case 8: LB(2, 8, P_) break;
                    default: LB(2, 16, P_)
                }
            };
            switch (pq) {
                case 1: go(std::integral_constant<int, 1>{}); break;
                case 2: go(std::integral_constant<int, 2>{}); break;
                case 3: go(std::integral_constant<int, 3>{}); break;
                case 4: go(std::integral_constant<int, 4>{}); break;
                case 5: go(std::integral_constant<int, 5>{}); break;
                case kShapeDistance: go(std::integral_constant<int, kShapeDistance>{}); break;
                default: go(std::integral_constant<int, 0>{});
            }
        } else if (pq == kShapeDistance) {
            switch (nr) {
                case 1: LB(2, 1, kShapeDistance) break;
                case 2: LB(2, 2, kShapeDistance) break;
                case 4: LB(2, 4, kShapeDistance) break;
                default: LB(2, 8, kShapeDistance)
            }
        } else {
            switch (nr) {
                case 1: LB(2, 1, 0) break;
                case 2: LB(2, 2, 0) break;
                case 4: LB(2, 4, 0) break;
                default: LB(2, 8, 0)
            }
        }
#undef LB
        CK(cudaGetLastError());
        return;
    }
    BatchId<R> a{};
    a.ninst = n;
    size_t sm = 0;
    int items = 0;
    for (int k = 0; k < n; ++k) {
        const E& e = ents[k];
        const DevStage<R>& ds = stages_of<R>(dps[e.i])[e.sidx];
        a.st[k] = type == BT_C1 ? ds.ids1 : ds.ids;
        a.src[k] = e.src;
        a.dst[k] = e.dst;
        a.nrhs[k] = nrhs[e.i];
        a.conj[k] = adjoint[e.i] != 0;
        a.item0[k] = items;
        if (type == BT_R) {
            items += ds.n_items_r;
            sm = std::max(sm, pattern_r_smem<R>(ds.max_nred, rt, nr));
        } else if (type == BT_C1) {
            items += ds.n_items_c1;
            sm = std::max(sm, pattern_c1_smem<R>(ds.max_narrow, ds.max_nsub));
        } else {
            items += ds.n_items_c;
            sm = std::max(sm, pattern_c_smem<R>(ds.max_narrow, ds.max_nsub, kRangeC, nr));
        }
    }
    a.item0[n] = items;
    if (items == 0) return;
#define LK(KF)                                \
    {                                         \
        auto kf = KF;                         \
        set_smem(kf, sm);                     \
        kf<<<items, kThreads, sm, s>>>(a);    \
    }
    if (type == BT_C1) {
        LK(k_batch_c1<R>)
    } else if (type == BT_R) {
        auto go = [&](auto rtc) {
            constexpr int RT_ = decltype(rtc)::value;
            switch (nr) {
                case 1: LK((k_batch_r<R, RT_, 1>)) break;
                case 2: LK((k_batch_r<R, RT_, 2>)) break;
                case 4: LK((k_batch_r<R, RT_, 4>)) break;
                case 8: LK((k_batch_r<R, RT_, 8>)) break;
                default:
                    if constexpr (sizeof(R) == 4) LK((k_batch_r<R, RT_, 16>))
                    else LK((k_batch_r<R, RT_, 8>))
            }
        };
        if (rt == 1) go(std::integral_constant<int, 1>{});
        else go(std::integral_constant<int, 2>{});
    } else {
        switch (nr) {
            case 1: LK((k_batch_c<R, 1>)) break;
            case 2: LK((k_batch_c<R, 2>)) break;
            case 4: LK((k_batch_c<R, 4>)) break;
            case 8: LK((k_batch_c<R, 8>)) break;
            default:
                if constexpr (sizeof(R) == 4) LK((k_batch_c<R, 16>))
                else LK((k_batch_c<R, 8>))
        }
    }
#undef LK
    CK(cudaGetLastError());
}

template <class R>
// Returns the number of launches; dry = true only counts them.
int run_batched(int count, const midbf_dplan* const* dps, const int* adjoint, const void* const* in,
                const int64_t* ldin, void* const* out, const int64_t* ldout, const int* nrhs, cudaStream_t s,
                char* ws, bool dry) {
    int launches = 0;
    std::vector<cx<R>*> b0(count), b1(count);
    size_t off = 0;
    int maxst = 0;
    for (int i = 0; i < count; ++i) {
        if (!dry) {
            b0[i] = reinterpret_cast<cx<R>*>(ws + off);
            b1[i] = b0[i] + dps[i]->max_space * nrhs[i];
        }
        off += instance_workspace(dps[i], nrhs[i]);
        maxst = std::max(maxst, (int)stages_of<R>(dps[i]).size());
    }
    for (int q = 0; q < maxst; ++q) {
        struct Entry { int i, sidx; VecRef<R> src, dst; };
        std::map<std::array<int, 4>, std::vector<Entry>> groups;
        // one-RHS ID stages that the single-instance apply runs on the narrow-ID
        // or cluster kernels run the same launch here (one per instance), so
        // every output equals the single-instance apply's bit for bit
        struct Solo { Entry e; const DevStage<R>* ds; bool use_r, narrow; int cl; bool gemm; };
        std::vector<Solo> solo;
        for (int i = 0; i < count; ++i) {
            const auto& sts = stages_of<R>(dps[i]);
            const int ns = (int)sts.size();
            if (q >= ns) continue;
            const bool adj = adjoint[i] != 0;
            const int sidx = adj ? ns - 1 - q : q;
            const DevStage<R>& ds = sts[sidx];
            const int nr = nrhs[i];
            VecRef<R> uin{(cx<R>*)in[i], 1, ldin[i]}, uout{(cx<R>*)out[i], 1, ldout[i]};
            auto internal = [&](int space) { return VecRef<R>{(space & 1) ? b1[i] : b0[i], nr, 1}; };
            VecRef<R> fin = sidx == 0 ? (adj ? uout : uin) : internal(sidx - 1);
            VecRef<R> fout = ds.out_user ? (adj ? uin : uout) : internal(sidx);
            Entry e{i, sidx, adj ? fout : fin, adj ? fin : fout};
            std::array<int, 4> key{};
            // a tuned SIMT tile for this instance's RHS count, if any
            const int force = choice_tile(tuned_choice(dps[i], nr, sidx, adj));
            if (ds.id) {
                const bool wide_is_fwd_input = ds.kind != KIND_U;
                const bool use_r = adj ? !wide_is_fwd_input : wide_is_fwd_input;
                if (use_gemm(ds, nr, tuned_choice(dps[i], nr, sidx, adj), use_r)) {
                    solo.push_back({e, &ds, use_r, false, 1, true});
                    continue;
                }
                if (nr == 1) {
                    const int ch = tuned_choice(dps[i], nr, sidx, adj);
                    const bool narrow = use_narrow(ds, 1, ch, use_r);
                    const int cl = (use_r && !narrow) ? row_cluster_for(ds, ch) : 1;
                    if (narrow || cl > 1) {
                        solo.push_back({e, &ds, use_r, narrow, cl, false});
                        continue;
                    }
                }
                if (use_r) {
                    const int t = forced_or_pick<R>(force, nr, [&](int qq) { return pattern_r_smem<R>(ds.max_nred, ds.rt, qq); });
                    key = {BT_R, ds.rt, t, 0};
                } else if (nr == 1 && force == 0 && pattern_c1_smem<R>(ds.max_narrow, ds.max_nsub) <= kSmemCap) {
                    key = {BT_C1, 0, 1, 0};
                } else {
                    const int t = forced_or_pick<R>(force, nr, [&](int qq) { return pattern_c_smem<R>(ds.max_narrow, ds.max_nsub, kRangeC, qq); });
                    key = {BT_C, 0, t, 0};
                }
            } else {
                if (use_gemm(ds, nr, tuned_choice(dps[i], nr, sidx, adj), false)) {
                    solo.push_back({e, &ds, false, false, 1, true});
                    continue;
                }
                const int t = forced_or_pick<R>(force, nr, [&](int qq) {
                    return s_fly_smem<R>(ds.ss.P, ds.ss.Q, qq <= 4 && sizeof(R) == 4 ? 4 : 2, qq);
                });
                const int rt = (t <= 4 && sizeof(R) == 4) ? 4 : 2;
                const int pq = s_shape(ds);
                key = {BT_S, rt, t, pq};
            }
            groups[key].push_back(e);
        }
        for (auto& kv : groups) {
            const auto& key = kv.first;
            const auto& ents = kv.second;
            for (size_t g0 = 0; g0 < ents.size(); g0 += kBatch) {
                const int n = (int)std::min<size_t>(kBatch, ents.size() - g0);
                if (!dry) launch_batch_group<R>(dps, key, &ents[g0], n, nrhs, adjoint, s);
                ++launches;
            }
        }
        for (const Solo& o : solo) {
            if (!dry) {
                const bool conj = adjoint[o.e.i] != 0;
                if (o.gemm) {
                    if constexpr (sizeof(R) == 4) {
                        if (o.ds->id && o.use_r) launch_r_gemm(*o.ds, o.e.src, o.e.dst, nrhs[o.e.i], conj, s);
                        else if (o.ds->id) launch_c_gemm(*o.ds, o.e.src, o.e.dst, nrhs[o.e.i], conj, s);
                        else launch_s_gemm(*o.ds, o.e.src, o.e.dst, nrhs[o.e.i], conj, s);
                    }
                } else if (o.cl > 1) launch_r_cluster<R>(*o.ds, o.e.src, o.e.dst, conj, o.cl, s);
                else if (o.use_r) launch_r_narrow<R>(*o.ds, o.e.src, o.e.dst, conj, s);
                else launch_c_narrow<R>(*o.ds, o.e.src, o.e.dst, conj, s);
            }
            ++launches;
        }
    }
    return launches;
}

template int run_batched<float>(int, const midbf_dplan* const*, const int*, const void* const*, const int64_t*, void* const*, const int64_t*, const int*, cudaStream_t, char*, bool);
template int run_batched<double>(int, const midbf_dplan* const*, const int*, const void* const*, const int64_t*, void* const*, const int64_t*, const int*, cudaStream_t, char*, bool);

}  // namespace midbf_gpu
