// Device-resident plans and the apply launcher (host code + kernel launches).
//
// midbf_dplan_create turns a host plan (factor stages of eq. (finishIDBF),
// Sec. 3.5) into device arrays in one precision:
//   * ID blocks: T of every interpolative decomposition (Sec. 3.2) column-major
//     with its redundant indices sorted ascending, block/sub descriptors, the
//     wide/narrow position maps and the work-item lists of both patterns;
//   * the middle factor: per-entry phase-split data for on-the-fly generation
//     (or the dense entries, MIDBF_S_STORED).
// midbf_apply runs the stages in order (forward) or reverse order with
// conjugated factors (adjoint), ping-ponging between two workspace vectors.
#include <algorithm>
#include <cstdio>
#include <functional>
#include <mutex>
#include <array>
#include <map>
#include <set>
#include <type_traits>
#include <numeric>
#include <thread>
#include <tuple>

#include "internal.hpp"
#include "kernels.cuh"
#include "tc.cuh"

using namespace midbf;
using namespace midbf_dev;

namespace {

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) fail(MIDBF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

constexpr int kRangeC = 64;   // output entries per pattern-C item
constexpr size_t kSmemCap = 200 * 1024;  // dynamic shared memory budget per CTA

struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
};

struct DevStageBase {
    int kind = KIND_V;
    int64_t in_len = 0, out_len = 0;
    bool out_user = false, in_user = false;
};

template <class R>
struct DevStage : DevStageBase {
    // ID stages (and stored S)
    bool id = false;
    IdStage<R> ids{};
    IdStage<R> ids1{};   // same data, items for the one-RHS pattern-C kernel
    int n_items_r = 0, n_items_c = 0, n_items_c1 = 0, rt = 1;
    int max_nred = 0, max_narrow = 0, max_nsub = 1;
    // on-the-fly S
    SStage<R> ss{};
    SSide<R> srows{}, scols{};
    const int2* items_rows = nullptr;   // 64-row items (RT = 2)
    const int2* items_cols = nullptr;
    const int2* items_rows4 = nullptr;  // 128-row items (RT = 4)
    const int2* items_cols4 = nullptr;
    int n_items_rows = 0, n_items_cols = 0, n_items_rows4 = 0, n_items_cols4 = 0, rt_rows = 1, rt_cols = 1;
    // tensor-core modes: dense BF16 tile images of the V/U blocks,
    // [0] forward orientation (stage input -> output), [1] adjoint
    bool tc = false;
    TcStage tcs[2]{};
    int n_tc_items[2] = {0, 0};
    double tc_bytes[2] = {0, 0};
    // B-image chunks of the stage input, per orientation (V/U and middle factor)
    TcPack pk[2]{};
    const int* chunk0_s[2] = {nullptr, nullptr};   // middle factor: first chunk of each block
};

}  // namespace

struct midbf_dplan {
    int precision = MIDBF_FP32;   // storage: MIDBF_FP32 (also for the BF16 modes) or MIDBF_FP64
    int tc_mode = 0;              // 0: SIMT only; 1: BF16 tensor cores; 2: BF16 + refinement
    int* d_status = nullptr;      // device status word written by bounded waits
    int s_mode = MIDBF_S_ONTHEFLY;
    int device = 0;
    int64_t nx = 0, nw = 0;
    int64_t max_space = 0;        // longest internal vector space
    size_t factor_bytes = 0, index_bytes = 0;
    size_t tc_image_bytes = 0;    // dense BF16 tile images (tensor-core modes)
    int max_tc_chunks = 0;        // most B-image chunks of one tensor-core stage launch
    std::vector<void*> allocs;
    std::vector<DevStage<float>> st32;
    std::vector<DevStage<double>> st64;
    int launches = 0;
    // per stage, in forward order: stored bytes streamed once per apply, and
    // the input + output vector lengths (entries per right-hand side)
    std::vector<double> stage_fixed_bytes;
    std::vector<int64_t> stage_vec_entries;
    std::vector<int> stage_kind;
    // per stage: complex entries of the method's factor (T entries of the IDs,
    // or rows x cols of the middle-factor blocks) and of the dense blocks
    // (identity parts of the IDs included)
    std::vector<int64_t> stage_entries, stage_dense;
    // kernel choices per RHS count: [stage][0 forward, 1 adjoint] (midbf_autotune)
    std::map<int, std::vector<std::array<int, 2>>> tuned;
    // measurement hooks (midbf_dplan_profile / midbf_stage_times)
    bool profile = false;
    mutable std::vector<cudaEvent_t> ev;
    mutable std::vector<int> ev_stage;   // stage index of each event pair of the last apply
    mutable int last_nrhs = 1;
    ~midbf_dplan() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (d_status) cudaFree(d_status);
        for (void* p : allocs) cudaFree(p);
    }
};

namespace {

template <class T>
T* upload(midbf_dplan* dp, const std::vector<T>& v, size_t* counter) {
    if (v.empty()) return nullptr;
    void* p = nullptr;
    size_t bytes = v.size() * sizeof(T);
    if (cudaMalloc(&p, bytes) != cudaSuccess) fail(MIDBF_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    dp->allocs.push_back(p);
    CK(cudaMemcpy(p, v.data(), bytes, cudaMemcpyHostToDevice));
    if (counter) *counter += bytes;
    return static_cast<T*>(p);
}

inline double frac(double v) { return v - std::nearbyint(v); }

int rows_per_lane(int maxk) { return maxk <= 32 ? 1 : 2; }

// IEEE binary32 -> bfloat16 with round-to-nearest-even on the 16 dropped
// bits (NaN stays a quiet NaN).
uint16_t bf16_bits(float v) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

float bf16_value(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Dense tile images of the blocks of a V or U stage for k_blk_tc.
//
// Per block, G is the narrow x wide matrix of its interpolative
// decompositions (Sec. 3.2): row c of sub-block s has a one in the column of
// its skeleton skel_c and T_s(c, r) in the column of redundant index red_r.
// The oriented matrices are
//   V stage: forward G,   adjoint G^H;
//   U stage: forward G^T, adjoint conj(G),
// each cut into 128-row x 16-column tiles.  A tile image holds the real
// embedding row (Re a, -Im a) of every entry a, interleaved along K, as BF16
// (hi, then lo in the refined mode) in the core-matrix layout of the MMA.
template <class R>
void make_tc_images(midbf_dplan* dp, const Stage& st, DevStage<R>& ds) {
    const bool is_v = st.kind == KIND_V;
    const int NP = dp->tc_mode == 2 ? 2 : 1;
    const int nb = (int)st.blocks.size();
    for (int o = 0; o < 2; ++o) {
        std::vector<TcBlock> tb(nb);
        std::vector<int> ipos, opos;
        std::vector<int2> items, chunks;
        long long off = 0;
        for (int b = 0; b < nb; ++b) {
            const Block& bk = st.blocks[b];
            const std::vector<int64_t>& src = o == 0 ? bk.in_idx : bk.out_idx;
            const std::vector<int64_t>& dst = o == 0 ? bk.out_idx : bk.in_idx;
            TcBlock& t = tb[b];
            t.rows = (int)dst.size();
            t.cols = (int)src.size();
            t.out_off = (int)opos.size();
            t.chunk0 = (int)chunks.size();
            t.img_off = off;
            const int in_off = (int)ipos.size();
            for (int64_t v : src) ipos.push_back((int)v);
            for (int64_t v : dst) opos.push_back((int)v);
            const int nrt = (t.rows + kTcM - 1) / kTcM, nch = (t.cols + kTcKc - 1) / kTcKc;
            for (int c = 0; c < nch; ++c) chunks.push_back(make_int2(in_off + c * kTcKc, std::min(kTcKc, t.cols - c * kTcKc)));
            for (int r = 0; r < nrt; ++r) items.push_back(make_int2(b, r));
            off += (long long)nrt * nch * NP * kTcTileElems;
        }
        std::vector<uint16_t> img((size_t)off, 0);
        auto fill = [&](int b) {
            const Block& bk = st.blocks[b];
            const TcBlock& t = tb[b];
            const int nch = (t.cols + kTcKc - 1) / kTcKc;
            auto put = [&](int i, int j, float re, float im) {
                const int rt = i / kTcM, r = i % kTcM, c = j / kTcKc, jj = j % kTcKc;
                uint16_t* tile = &img[(size_t)t.img_off + ((size_t)rt * nch + c) * NP * kTcTileElems];
                const float v[2] = {re, -im};
                for (int q = 0; q < 2; ++q) {
                    const size_t e = (size_t)core_off(r, 2 * jj + q, kTcK);
                    const uint16_t hi = bf16_bits(v[q]);
                    tile[e] = hi;
                    if (NP == 2) tile[kTcTileElems + e] = bf16_bits(v[q] - bf16_value(hi));
                }
            };
            // (narrow row, wide column, value of G) -> entry of the oriented matrix
            auto emit = [&](int nrow, int wcol, cplx g) {
                const float re = (float)g.real(), im = (float)g.imag();
                if (is_v) {
                    if (o == 0) put(nrow, wcol, re, im);
                    else put(wcol, nrow, re, -im);
                } else {
                    if (o == 0) put(wcol, nrow, re, im);
                    else put(nrow, wcol, re, -im);
                }
            };
            int noff = 0;
            for (const Sub& sb : bk.subs) {
                const int nred = sb.m - sb.k;
                for (int c = 0; c < sb.k; ++c) {
                    emit(noff + c, sb.skel[c], cplx(1.0, 0.0));
                    for (int r = 0; r < nred; ++r) emit(noff + c, sb.red[r], sb.t((size_t)c * nred + r));
                }
                noff += sb.k;
            }
        };
        const int nthreads = std::max(1u, std::thread::hardware_concurrency());
        std::vector<std::thread> th;
        for (int w = 0; w < nthreads; ++w)
            th.emplace_back([&, w]() {
                for (int b = w; b < nb; b += nthreads) fill(b);
            });
        for (auto& t : th) t.join();
        ds.tcs[o].blocks = upload(dp, tb, &dp->index_bytes);
        ds.tcs[o].out_pos = upload(dp, opos, &dp->index_bytes);
        ds.pk[o].pos = upload(dp, ipos, &dp->index_bytes);
        ds.pk[o].chunks = upload(dp, chunks, &dp->index_bytes);
        ds.pk[o].nchunks = (int)chunks.size();
        dp->max_tc_chunks = std::max(dp->max_tc_chunks, (int)chunks.size());
        ds.tcs[o].items = upload(dp, items, &dp->index_bytes);
        ds.tcs[o].img = reinterpret_cast<const __nv_bfloat16*>(upload(dp, img, &dp->tc_image_bytes));
        ds.n_tc_items[o] = (int)items.size();
        ds.tc_bytes[o] = (double)img.size() * 2.0;
    }
    ds.tc = true;
}

// Build the device arrays of an ID stage (V or U), or of a stored S stage
// seen as dense blocks with no skeleton.
template <class R>
void make_id_stage(midbf_dplan* dp, const Plan& pl, const Stage& st, DevStage<R>& ds, bool stored_s) {
    std::vector<SubDesc> subs;
    std::vector<BlockDesc> blocks;
    std::vector<int> skel, red, wide_pos, narrow_pos;
    std::vector<ItemR> items_r;
    std::vector<ItemC> items_c, items_c1;
    std::vector<cx<R>> T;
    int maxk = 1;
    size_t max_nred = 0, max_narrow = 0, max_nsub = 1;
    const bool is_v = st.kind == KIND_V || st.kind == KIND_S;  // S stored: wide = input like V
    for (size_t b = 0; b < st.blocks.size(); ++b) {
        const Block& bk = st.blocks[b];
        BlockDesc bd{};
        const std::vector<int64_t>& wide = is_v ? bk.in_idx : bk.out_idx;
        const std::vector<int64_t>& narrow = is_v ? bk.out_idx : bk.in_idx;
        bd.m = (int)wide.size();
        bd.wide_off = (int)wide_pos.size();
        bd.narrow_off = (int)narrow_pos.size();
        bd.nnarrow = (int)narrow.size();
        bd.sub0 = (int)subs.size();
        for (int64_t v : wide) wide_pos.push_back((int)v);
        for (int64_t v : narrow) narrow_pos.push_back((int)v);
        int noff = bd.narrow_off;
        if (stored_s) {
            // dense block: one "sub" with k = nrow rows, all columns redundant
            SubDesc sd{};
            sd.k = (int)bk.out_idx.size();
            sd.nskel = 0;
            sd.skel_off = (int)skel.size();
            sd.red_off = (int)red.size();
            sd.narrow_off = noff;
            sd.block = (int)b;
            sd.t_off = (long long)T.size();
            for (int j = 0; j < bd.m; ++j) red.push_back(j);
            const size_t base = T.size();
            T.resize(base + (size_t)sd.k * bd.m);
            const int nthreads = std::max(1u, std::thread::hardware_concurrency());
            std::vector<std::thread> th;
            for (int w = 0; w < nthreads; ++w)
                th.emplace_back([&, w]() {
                    for (int j = w; j < bd.m; j += nthreads)
                        for (int i = 0; i < sd.k; ++i) {
                            cplx kv = pl.phase.kernel(bk.xidx[i], bk.widx[j]);
                            T[base + (size_t)j * sd.k + i] = {(R)kv.real(), (R)kv.imag()};
                        }
                });
            for (auto& t : th) t.join();
            subs.push_back(sd);
            maxk = std::max(maxk, sd.k);
            max_nred = std::max(max_nred, (size_t)bd.m);
        } else {
            for (const Sub& sb : bk.subs) {
                SubDesc sd{};
                sd.k = sb.k;
                sd.nskel = sb.k;
                sd.skel_off = (int)skel.size();
                sd.red_off = (int)red.size();
                sd.narrow_off = noff;
                sd.block = (int)b;
                sd.t_off = (long long)T.size();
                noff += sb.k;
                for (int v : sb.skel) skel.push_back(v);
                const int nred = sb.m - sb.k;
                std::vector<int> perm(nred);
                std::iota(perm.begin(), perm.end(), 0);
                std::sort(perm.begin(), perm.end(), [&](int a, int c) { return sb.red[a] < sb.red[c]; });
                for (int jj = 0; jj < nred; ++jj) red.push_back(sb.red[perm[jj]]);
                for (int jj = 0; jj < nred; ++jj)
                    for (int i = 0; i < sb.k; ++i) {
                        const cplx v = sb.t((size_t)i * nred + perm[jj]);
                        T.push_back({(R)v.real(), (R)v.imag()});
                    }
                subs.push_back(sd);
                maxk = std::max(maxk, sb.k);
                max_nred = std::max(max_nred, (size_t)nred);
            }
        }
        bd.nsub = (int)subs.size() - bd.sub0;
        max_nsub = std::max(max_nsub, (size_t)bd.nsub);
        max_narrow = std::max(max_narrow, (size_t)bd.nnarrow);
        blocks.push_back(bd);
        for (int o0 = 0; o0 < bd.m; o0 += kRangeC) items_c.push_back({(int)b, o0, std::min(bd.m, o0 + kRangeC), 0});
        for (int o0 = 0; o0 < bd.m; o0 += kRangeC1) items_c1.push_back({(int)b, o0, std::min(bd.m, o0 + kRangeC1), 0});
    }
    if (max_nsub > 16) fail(MIDBF_EINTERNAL, "more than 16 sub-blocks in a block");
    const int rt = rows_per_lane(maxk);
    for (size_t s = 0; s < subs.size(); ++s)
        for (int r0 = 0; r0 < subs[s].k; r0 += 32 * rt) items_r.push_back({(int)s, r0});
    ds.id = true;
    ds.rt = rt;
    ds.n_items_r = (int)items_r.size();
    ds.n_items_c = (int)items_c.size();
    ds.max_nred = (int)max_nred;
    ds.max_narrow = (int)max_narrow;
    ds.max_nsub = (int)max_nsub;
    if (pattern_r_smem<R>((int)max_nred, rt, 1) > kSmemCap || pattern_c_smem<R>((int)max_narrow, (int)max_nsub, kRangeC, 1) > kSmemCap)
        fail(MIDBF_EINTERNAL, "block too wide for shared memory");
    ds.ids.subs = upload(dp, subs, &dp->index_bytes);
    ds.ids.blocks = upload(dp, blocks, &dp->index_bytes);
    ds.ids.skel = upload(dp, skel, &dp->index_bytes);
    ds.ids.red = upload(dp, red, &dp->index_bytes);
    ds.ids.wide_pos = upload(dp, wide_pos, &dp->index_bytes);
    ds.ids.narrow_pos = upload(dp, narrow_pos, &dp->index_bytes);
    ds.ids.T = upload(dp, T, &dp->factor_bytes);
    ds.ids.items_r = upload(dp, items_r, &dp->index_bytes);
    ds.ids.items_c = upload(dp, items_c, &dp->index_bytes);
    ds.ids1 = ds.ids;
    ds.ids1.items_c = upload(dp, items_c1, &dp->index_bytes);
    ds.n_items_c1 = (int)items_c1.size();
    if constexpr (sizeof(R) == 4) {
        if (dp->tc_mode && !stored_s) make_tc_images<R>(dp, st, ds);
    }
}

// Split of the phase for one S block (see kernels.cuh): rows get (a, u, C),
// columns (b, v, W), all computed in FP64 and rounded to R at the end.
struct SplitOut {
    std::vector<double> a, u, c;
};

void phase_split(const Phase& ph, const Block& bk, int P, int Q, SplitOut& rows, SplitOut& cols) {
    const int d = ph.d;
    const int64_t i0 = bk.xidx[0], j0 = bk.widx[0];
    const size_t nr = bk.xidx.size(), nc = bk.widx.size();
    rows.a.resize(nr);
    rows.u.resize(nr * P);
    rows.c.resize(nr * Q);
    cols.a.resize(nc);
    cols.u.resize(nc * P);
    cols.c.resize(nc * Q);
    const int fam = ph.family;
    if (fam == MIDBF_PHASE_LOWRANK) {
        const double* U0 = &ph.U[(size_t)i0 * ph.r];
        const double* V0 = &ph.V[(size_t)j0 * ph.r];
        for (size_t i = 0; i < nr; ++i) {
            const double* Ui = &ph.U[(size_t)bk.xidx[i] * ph.r];
            double s = 0.0;
            for (int t = 0; t < ph.r; ++t) {
                s += (Ui[t] - U0[t]) * V0[t];
                rows.u[i * P + t] = Ui[t] - U0[t];
            }
            rows.a[i] = frac(s);
        }
        for (size_t j = 0; j < nc; ++j) {
            const double* Vj = &ph.V[(size_t)bk.widx[j] * ph.r];
            double s = 0.0;
            for (int t = 0; t < ph.r; ++t) {
                s += U0[t] * Vj[t];
                cols.u[j * P + t] = Vj[t] - V0[t];
            }
            cols.a[j] = frac(s);
        }
        return;
    }
    if (fam == MIDBF_PHASE_ZERO || fam == MIDBF_PHASE_SEPARABLE) {
        // Phi = a(x) + b(xi): a split with no mixed term
        const double z[3] = {0, 0, 0};
        for (size_t i = 0; i < nr; ++i) {
            double v = ph.eval_xy(&ph.X[(size_t)bk.xidx[i] * d], z);
            rows.a[i] = frac(v);
        }
        for (size_t j = 0; j < nc; ++j) {
            double v = ph.eval_xy(z, &ph.W[(size_t)bk.widx[j] * d]) - ph.eval_xy(z, z);
            cols.a[j] = frac(v);
        }
        return;
    }
    // DOT and FIO families: x.xi = x0.xi + (x - x0).xi0 + (x - x0).(xi - xi0)
    const double* x0 = &ph.X[(size_t)i0 * d];
    const double* w0 = &ph.W[(size_t)j0 * d];
    const bool jump = fam == MIDBF_PHASE_FIO2D_JUMP;
    const double sg0 = (x0[0] - 0.5 >= 0.0) ? 1.0 : -1.0;
    const double twopi = 2.0 * M_PI;
    for (size_t i = 0; i < nr; ++i) {
        const double* x = &ph.X[(size_t)bk.xidx[i] * d];
        double s = 0.0;
        for (int k = 0; k < d; ++k) {
            s += (x[k] - x0[k]) * w0[k];
            rows.u[i * P + k] = x[k] - x0[k];
        }
        rows.a[i] = frac(s);
        if (jump) rows.u[i * P + d] = 0.5 * (((x[0] - 0.5 >= 0.0) ? 1.0 : -1.0) - sg0);
        if (Q) {
            if (d == 2) {
                const double c1 = (2.0 + std::sin(twopi * x[0]) * std::sin(twopi * x[1])) / 16.0;
                const double c2 = (2.0 + std::cos(twopi * x[0]) * std::cos(twopi * x[1])) / 16.0;
                rows.c[i * Q + 0] = c1 * c1;
                rows.c[i * Q + 1] = c2 * c2;
            } else {
                for (int k = 0; k < 3; ++k) {
                    const double ck = (2.0 + std::sin(twopi * x[k]) * std::cos(twopi * x[(k + 1) % 3])) / 16.0;
                    rows.c[i * Q + k] = ck * ck;
                }
            }
        }
    }
    for (size_t j = 0; j < nc; ++j) {
        const double* w = &ph.W[(size_t)bk.widx[j] * d];
        double s = 0.0, nrm = 0.0;
        for (int k = 0; k < d; ++k) {
            s += x0[k] * w[k];
            cols.u[j * P + k] = w[k] - w0[k];
            nrm += w[k] * w[k];
            if (Q) cols.c[j * Q + k] = w[k] * w[k];
        }
        if (jump) {
            nrm = std::sqrt(nrm);
            s += 0.5 * nrm * sg0;
            cols.u[j * P + d] = frac(nrm) < 0 ? frac(nrm) + 1.0 : frac(nrm);
        }
        cols.a[j] = frac(s);
    }
}

template <class R>
void make_s_stage(midbf_dplan* dp, const Plan& pl, const Stage& st, DevStage<R>& ds) {
    const Phase& ph = pl.phase;
    int P = 0, Q = 0;
    switch (ph.family) {
        case MIDBF_PHASE_LOWRANK: P = ph.r; break;
        case MIDBF_PHASE_DOT: P = ph.d; break;
        case MIDBF_PHASE_FIO2D: case MIDBF_PHASE_FIO3D: P = ph.d; Q = ph.d; break;
        case MIDBF_PHASE_FIO2D_JUMP: P = ph.d + 1; Q = ph.d; break;
        default: break;
    }
    if (P > 8 || Q > 3) fail(MIDBF_EINVAL, "on-the-fly middle factor supports at most 8 low-rank terms");
    std::vector<int> blk_rows, blk_cols, blk_nrow, blk_ncol, rpos, cpos;
    std::vector<R> ra, ru, rc, ca, cu, cc;
    std::vector<int2> it_rows, it_cols, it_rows4, it_cols4;
    int maxr = 1, maxc = 1;
    for (size_t b = 0; b < st.blocks.size(); ++b) {
        const Block& bk = st.blocks[b];
        SplitOut r, c;
        phase_split(ph, bk, P, Q, r, c);
        blk_rows.push_back((int)ra.size());
        blk_cols.push_back((int)ca.size());
        blk_nrow.push_back((int)bk.xidx.size());
        blk_ncol.push_back((int)bk.widx.size());
        maxr = std::max(maxr, (int)bk.xidx.size());
        maxc = std::max(maxc, (int)bk.widx.size());
        for (double v : r.a) ra.push_back((R)v);
        for (double v : r.u) ru.push_back((R)v);
        for (double v : r.c) rc.push_back((R)v);
        for (double v : c.a) ca.push_back((R)v);
        for (double v : c.u) cu.push_back((R)v);
        for (double v : c.c) cc.push_back((R)v);
        for (int64_t v : bk.out_idx) rpos.push_back((int)v);
        for (int64_t v : bk.in_idx) cpos.push_back((int)v);
    }
    ds.rt_rows = 2;  // k_s_fly launches use 64 rows per item
    ds.rt_cols = 2;
    for (size_t b = 0; b < st.blocks.size(); ++b) {
        for (int r0 = 0; r0 < blk_nrow[b]; r0 += 32 * ds.rt_rows) it_rows.push_back(make_int2((int)b, r0));
        for (int c0 = 0; c0 < blk_ncol[b]; c0 += 32 * ds.rt_cols) it_cols.push_back(make_int2((int)b, c0));
        for (int r0 = 0; r0 < blk_nrow[b]; r0 += 128) it_rows4.push_back(make_int2((int)b, r0));
        for (int c0 = 0; c0 < blk_ncol[b]; c0 += 128) it_cols4.push_back(make_int2((int)b, c0));
    }
    ds.ss.P = P;
    ds.ss.Q = Q;
    ds.ss.blk_rows = upload(dp, blk_rows, &dp->index_bytes);
    ds.ss.blk_cols = upload(dp, blk_cols, &dp->index_bytes);
    ds.ss.blk_nrow = upload(dp, blk_nrow, &dp->index_bytes);
    ds.ss.blk_ncol = upload(dp, blk_ncol, &dp->index_bytes);
    ds.srows.a = upload(dp, ra, &dp->factor_bytes);
    ds.srows.u = upload(dp, ru, &dp->factor_bytes);
    ds.srows.c = upload(dp, rc, &dp->factor_bytes);
    ds.srows.pos = upload(dp, rpos, &dp->index_bytes);
    ds.scols.a = upload(dp, ca, &dp->factor_bytes);
    ds.scols.u = upload(dp, cu, &dp->factor_bytes);
    ds.scols.c = upload(dp, cc, &dp->factor_bytes);
    ds.scols.pos = upload(dp, cpos, &dp->index_bytes);
    ds.items_rows = upload(dp, it_rows, &dp->index_bytes);
    ds.items_cols = upload(dp, it_cols, &dp->index_bytes);
    ds.items_rows4 = upload(dp, it_rows4, &dp->index_bytes);
    ds.items_cols4 = upload(dp, it_cols4, &dp->index_bytes);
    ds.n_items_rows = (int)it_rows.size();
    ds.n_items_cols = (int)it_cols.size();
    ds.n_items_rows4 = (int)it_rows4.size();
    ds.n_items_cols4 = (int)it_cols4.size();
    if constexpr (sizeof(R) == 4) {
        if (dp->tc_mode) {
            // B-image chunks of the middle factor's input: forward the columns
            // (Omega side) of each block, adjoint its rows (X side)
            for (int o = 0; o < 2; ++o) {
                const std::vector<int>& off = o == 0 ? blk_cols : blk_rows;
                const std::vector<int>& cnt = o == 0 ? blk_ncol : blk_nrow;
                std::vector<int2> chunks;
                std::vector<int> c0(st.blocks.size());
                for (size_t b = 0; b < st.blocks.size(); ++b) {
                    c0[b] = (int)chunks.size();
                    for (int c = 0; c * kTcKc < cnt[b]; ++c)
                        chunks.push_back(make_int2(off[b] + c * kTcKc, std::min(kTcKc, cnt[b] - c * kTcKc)));
                }
                ds.pk[o].pos = o == 0 ? ds.scols.pos : ds.srows.pos;
                ds.pk[o].chunks = upload(dp, chunks, &dp->index_bytes);
                ds.pk[o].nchunks = (int)chunks.size();
                ds.chunk0_s[o] = upload(dp, c0, &dp->index_bytes);
                dp->max_tc_chunks = std::max(dp->max_tc_chunks, (int)chunks.size());
            }
        }
    }
}

template <class R>
void make_stages(midbf_dplan* dp, const Plan& pl, std::vector<DevStage<R>>& out) {
    int64_t in_len = pl.phase.nw;
    for (size_t s = 0; s < pl.stages.size(); ++s) {
        const Stage& st = pl.stages[s];
        DevStage<R> ds;
        ds.kind = st.kind;
        ds.in_len = in_len;
        ds.out_len = st.out_len;
        ds.in_user = s == 0;
        ds.out_user = st.out_user != 0;
        const size_t f0 = dp->factor_bytes, i0 = dp->index_bytes;
        if (st.kind == KIND_S) {
            if (dp->s_mode == MIDBF_S_STORED) make_id_stage<R>(dp, pl, st, ds, true);
            else make_s_stage<R>(dp, pl, st, ds);
        } else {
            make_id_stage<R>(dp, pl, st, ds, false);
        }
        // algorithmic bytes: factor data and position maps once, vectors per RHS
        // (work-item lists and descriptors are bookkeeping, counted too)
        dp->stage_fixed_bytes.push_back((double)(dp->factor_bytes - f0) + (double)(dp->index_bytes - i0));
        dp->stage_vec_entries.push_back(in_len + st.out_len);
        dp->stage_kind.push_back(st.kind);
        int64_t ent = 0, dense = 0;
        for (const Block& bk : st.blocks) {
            if (st.kind == KIND_S) {
                ent += (int64_t)bk.xidx.size() * (int64_t)bk.widx.size();
                dense += (int64_t)bk.xidx.size() * (int64_t)bk.widx.size();
            } else {
                for (const Sub& sb : bk.subs) {
                    ent += (int64_t)sb.k * (sb.m - sb.k);
                    dense += (int64_t)sb.k * sb.m;
                }
            }
        }
        dp->stage_entries.push_back(ent);
        dp->stage_dense.push_back(dense);
        if (!ds.in_user) dp->max_space = std::max(dp->max_space, in_len);
        if (!ds.out_user) dp->max_space = std::max(dp->max_space, st.out_len);
        in_len = st.out_len;
        out.push_back(std::move(ds));
    }
}

// Raise a kernel's dynamic shared-memory limit to the library's cap, once per
// kernel and device, so apply calls issue no attribute calls afterwards.
void set_smem_ptr(const void* kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return;
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(mu);
    if (done.count({kernel, dev})) return;
    CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap));
    done.insert({kernel, dev});
}

template <class K>
void set_smem(K kernel, size_t bytes) {
    set_smem_ptr(reinterpret_cast<const void*>(kernel), bytes);
}

// Right-hand sides per kernel pass: the smallest tile that covers nrhs (at
// most 16 for FP32, 8 for FP64), halved while the shared-memory need is
// above the budget.
template <class R>
int pick_nr(int nrhs, const std::function<size_t(int)>& smem) {
    const int cap = sizeof(R) == 4 ? 16 : 8;
    int nr = 1;
    while (nr < nrhs && nr < cap) nr *= 2;
    while (nr > 1 && smem(nr) > kSmemCap) nr /= 2;
    return nr;
}

// Grid of a SIMT launch: one CTA per work item, or (persistent) as many CTAs
// as are resident on the GPU at once, each looping over the items with the
// grid size as stride (the kernels' item loops).
int grid_for(const void* kernel, size_t smem, int nitems, bool persist) {
    if (!persist || nitems <= 0) return nitems;
    static std::mutex mu;
    static std::map<std::tuple<const void*, size_t, int>, int> cache;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    const auto key = std::make_tuple(kernel, smem, dev);
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return std::min(nitems, it->second);
    }
    int per_sm = 0, nsm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void*>(kernel), kThreads, smem));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int cap = std::max(1, per_sm) * std::max(1, nsm);
    std::lock_guard<std::mutex> g(mu);
    cache[key] = cap;
    return std::min(nitems, cap);
}

template <class R, int RT, int NR, bool CJ>
void launch_r_t(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, cudaStream_t s, bool persist) {
    const size_t sm = pattern_r_smem<R>(ds.max_nred, RT, NR);
    auto kf = k_pattern_r<R, RT, NR, CJ>;
    set_smem(kf, sm);
    const int n = ds.n_items_r;
    kf<<<grid_for(reinterpret_cast<const void*>(kf), sm, n, persist), kThreads, sm, s>>>(ds.ids, src, dst, nrhs, n);
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

// A forced RHS tile (from the autotuner) is taken when it is one of the
// compiled tiles and fits the shared-memory budget; otherwise pick_nr decides.
template <class R>
int forced_or_pick(int force, int nrhs, const std::function<size_t(int)>& smem) {
    const int cap = sizeof(R) == 4 ? 16 : 8;
    if (force > 0 && force <= cap && (force & (force - 1)) == 0 && smem(force) <= kSmemCap) return force;
    return pick_nr<R>(nrhs, smem);
}

template <class R>
void launch_r(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, bool conj, cudaStream_t s, int force = 0,
              bool persist = false) {
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
    auto kf = k_pattern_c<R, NR, CJ>;
    set_smem(kf, sm);
    const int n = ds.n_items_c;
    kf<<<grid_for(reinterpret_cast<const void*>(kf), sm, n, persist), kThreads, sm, s>>>(ds.ids, src, dst, nrhs, n);
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
void launch_c(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, bool conj, cudaStream_t s, int force = 0,
              bool persist = false) {
    if (ds.n_items_c == 0) return;
    if (nrhs == 1 && (force == 0 || force == MIDBF_CHOICE_COLUMN1)) {
        const size_t sm = pattern_c_smem<R>(ds.max_narrow, ds.max_nsub, kRangeC1, 1);
        if (sm <= kSmemCap) {
            if (conj) {
                auto kf = k_pattern_c1<R, true>;
                set_smem(kf, sm);
                kf<<<grid_for(reinterpret_cast<const void*>(kf), sm, ds.n_items_c1, persist), kThreads, sm, s>>>(ds.ids1, src, dst, ds.n_items_c1);
            } else {
                auto kf = k_pattern_c1<R, false>;
                set_smem(kf, sm);
                kf<<<grid_for(reinterpret_cast<const void*>(kf), sm, ds.n_items_c1, persist), kThreads, sm, s>>>(ds.ids1, src, dst, ds.n_items_c1);
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

template <class R, int RT, int NR, bool CJ, int PQ>
void launch_s_t(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, cudaStream_t s, bool persist) {
    SStage<R> st = ds.ss;
    const size_t sm = s_fly_smem<R>(st.P, st.Q, RT, NR);
    auto kf = k_s_fly<R, RT, NR, CJ, PQ>;
    set_smem(kf, sm);
    const bool four = RT == 4;
    if (!CJ) {
        st.items = four ? ds.items_rows4 : ds.items_rows;
        const int n = four ? ds.n_items_rows4 : ds.n_items_rows;
        kf<<<grid_for(reinterpret_cast<const void*>(kf), sm, n, persist), kThreads, sm, s>>>(st, ds.srows, ds.scols, 1, src,
                                                                                          dst, nrhs, n);
    } else {
        st.items = four ? ds.items_cols4 : ds.items_cols;
        const int n = four ? ds.n_items_cols4 : ds.n_items_cols;
        kf<<<grid_for(reinterpret_cast<const void*>(kf), sm, n, persist), kThreads, sm, s>>>(st, ds.scols, ds.srows, 0, src,
                                                                                          dst, nrhs, n);
    }
}

// FP32: 128-row items for up to 4 RHS per pass, phase shape fixed at compile
// time for the workload families.  FP64: the general shape (the plain form
// stores the middle factor by default).
template <class R, bool CJ, int PQ>
void launch_s_pq(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, int nr, cudaStream_t s, bool persist) {
    if constexpr (sizeof(R) == 4) {
        switch (nr) {
            case 1: launch_s_t<R, 4, 1, CJ, PQ>(ds, src, dst, nrhs, s, persist); break;
            case 2: launch_s_t<R, 4, 2, CJ, PQ>(ds, src, dst, nrhs, s, persist); break;
            case 4: launch_s_t<R, 4, 4, CJ, PQ>(ds, src, dst, nrhs, s, persist); break;
            case 8: launch_s_t<R, 2, 8, CJ, PQ>(ds, src, dst, nrhs, s, persist); break;
            default: launch_s_t<R, 2, 16, CJ, PQ>(ds, src, dst, nrhs, s, persist);
        }
    } else {
        switch (nr) {
            case 1: launch_s_t<R, 2, 1, CJ, 0>(ds, src, dst, nrhs, s, persist); break;
            case 2: launch_s_t<R, 2, 2, CJ, 0>(ds, src, dst, nrhs, s, persist); break;
            case 4: launch_s_t<R, 2, 4, CJ, 0>(ds, src, dst, nrhs, s, persist); break;
            default: launch_s_t<R, 2, 8, CJ, 0>(ds, src, dst, nrhs, s, persist);
        }
    }
}

template <class R, bool CJ>
void launch_s_nr(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, int nr, cudaStream_t s, bool persist) {
    switch (sizeof(R) == 4 ? phase_shape_code(ds.ss.P, ds.ss.Q) : 0) {
        case 1: launch_s_pq<R, CJ, 1>(ds, src, dst, nrhs, nr, s, persist); break;
        case 2: launch_s_pq<R, CJ, 2>(ds, src, dst, nrhs, nr, s, persist); break;
        case 3: launch_s_pq<R, CJ, 3>(ds, src, dst, nrhs, nr, s, persist); break;
        case 4: launch_s_pq<R, CJ, 4>(ds, src, dst, nrhs, nr, s, persist); break;
        case 5: launch_s_pq<R, CJ, 5>(ds, src, dst, nrhs, nr, s, persist); break;
        default: launch_s_pq<R, CJ, 0>(ds, src, dst, nrhs, nr, s, persist);
    }
}

template <class R>
void launch_s(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, bool adjoint, cudaStream_t s, int force = 0,
              bool persist = false) {
    const int nr = forced_or_pick<R>(force, nrhs, [&](int q) { return s_fly_smem<R>(ds.ss.P, ds.ss.Q, q <= 4 && sizeof(R) == 4 ? 4 : 2, q); });
    if (adjoint) launch_s_nr<R, true>(ds, src, dst, nrhs, nr, s, persist);
    else launch_s_nr<R, false>(ds, src, dst, nrhs, nr, s, persist);
    CK(cudaGetLastError());
}

constexpr int kTcMinRhs = 16;     // tensor cores for the middle factor from this many RHS on
constexpr int kTcBlkMinRhs = 16;  // and for the V / U stages

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
    switch (phase_shape_code(ds.ss.P, ds.ss.Q)) {
        case 1: launch_tc_t<1, RF, CJ>(ds, dst, R, bimg, status, s); break;
        case 2: launch_tc_t<2, RF, CJ>(ds, dst, R, bimg, status, s); break;
        case 3: launch_tc_t<3, RF, CJ>(ds, dst, R, bimg, status, s); break;
        case 4: launch_tc_t<4, RF, CJ>(ds, dst, R, bimg, status, s); break;
        case 5: launch_tc_t<5, RF, CJ>(ds, dst, R, bimg, status, s); break;
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
    const size_t sm = refine ? tc_smem_bytes<true>() : tc_smem_bytes<false>();
    for (int r0 = 0; r0 < nrhs; r0 += kTcR) {
        const int R = std::min(kTcR, nrhs - r0);
        launch_pack(ds.pk[o], rhs_shift(src, r0), R, refine, bimg, s);
        const VecRef<float> d = rhs_shift(dst, r0);
        if (refine) {
            auto kf = k_blk_tc<true>;
            set_smem(kf, sm);
            kf<<<ds.n_tc_items[o], kTcThreads, sm, s>>>(ds.tcs[o], bimg, d, R, status);
        } else {
            auto kf = k_blk_tc<false>;
            set_smem(kf, sm);
            kf<<<ds.n_tc_items[o], kTcThreads, sm, s>>>(ds.tcs[o], bimg, d, R, status);
        }
    }
    CK(cudaGetLastError());
}

// Bytes of the B-image area of the workspace for nrhs RHS (0 outside the
// tensor-core modes): the largest stage's chunks at one group of <= kTcR RHS.
// Bytes of the two ping-pong vectors of the workspace, rounded up to 256.
size_t vec_workspace_bytes(const midbf_dplan* dp, int nrhs) {
    const size_t ce = dp->precision == MIDBF_FP32 ? 8 : 16;
    const size_t b = 2 * (size_t)std::max<int64_t>(dp->max_space, 1) * (size_t)nrhs * ce;
    return (b + 255) / 256 * 256;
}

size_t tc_bimg_bytes(const midbf_dplan* dp, int nrhs) {
    if (!dp->tc_mode || dp->max_tc_chunks == 0) return 0;
    const int Rpad = (std::min(nrhs, kTcR) + 15) & ~15;
    const size_t b = (size_t)dp->max_tc_chunks * tc_bimg_elems(Rpad, dp->tc_mode == 2) * 2;
    return (b + 255) / 256 * 256;
}

template <class R>
int count_launches(const std::vector<DevStage<R>>& st) {
    int n = 0;
    for (auto& s : st) n += 1;
    return n;
}

// SIMT RHS tile named by a choice (0: none).
inline int choice_tile(int choice) {
    const int base = choice == MIDBF_CHOICE_TENSOR ? 0 : (choice & ~MIDBF_CHOICE_PERSIST);
    return base >= 1 && base <= 16 ? base : 0;
}

inline bool valid_choice(int choice) {
    if (choice == MIDBF_CHOICE_TENSOR) return true;
    const int base = choice & ~MIDBF_CHOICE_PERSIST;
    return base == MIDBF_CHOICE_DEFAULT || base == MIDBF_CHOICE_COLUMN1 || base == 1 || base == 2 || base == 4 ||
           base == 8 || base == 16;
}

// One stage launch.  choice: MIDBF_CHOICE_DEFAULT (the built-in rules: tensor
// cores in the BF16 modes from kTcMinRhs / kTcBlkMinRhs RHS on, else the SIMT
// kernel with the RHS tile of pick_nr), a SIMT RHS tile (1, 2, 4, 8, 16) or
// MIDBF_CHOICE_COLUMN1 (the one-RHS pattern-C kernel), optionally with
// MIDBF_CHOICE_PERSIST, or MIDBF_CHOICE_TENSOR.
template <class R>
void launch_stage(const midbf_dplan* dp, const DevStage<R>& ds, bool adjoint, VecRef<R> src, VecRef<R> dst, int nrhs,
                  int choice, __nv_bfloat16* bimg, cudaStream_t s) {
    if constexpr (sizeof(R) == 4) {
        const bool tc_ok = ds.id ? ds.tc : dp->tc_mode != 0;
        const bool use_tc = tc_ok && (choice == MIDBF_CHOICE_TENSOR ||
                                      (choice == MIDBF_CHOICE_DEFAULT && nrhs >= (ds.id ? kTcBlkMinRhs : kTcMinRhs)));
        if (use_tc) {
            if (ds.id) launch_blk_tc(ds, adjoint ? 1 : 0, src, dst, nrhs, dp->tc_mode == 2, bimg, dp->d_status, s);
            else launch_tc(ds, src, dst, nrhs, adjoint, dp->tc_mode == 2, bimg, dp->d_status, s);
            return;
        }
    }
    const bool persist = choice != MIDBF_CHOICE_TENSOR && (choice & MIDBF_CHOICE_PERSIST) != 0;
    const int tile = choice_tile(choice);
    const bool col1 = choice != MIDBF_CHOICE_TENSOR && (choice & ~MIDBF_CHOICE_PERSIST) == MIDBF_CHOICE_COLUMN1;
    if (ds.id) {
        const bool wide_is_fwd_input = ds.kind != KIND_U;  // V and stored S
        // pattern R computes narrow from wide; pattern C wide from narrow.
        const bool use_r = adjoint ? !wide_is_fwd_input : wide_is_fwd_input;
        if (use_r) launch_r<R>(ds, src, dst, nrhs, adjoint, s, tile, persist);
        else launch_c<R>(ds, src, dst, nrhs, adjoint, s, col1 ? MIDBF_CHOICE_COLUMN1 : tile, persist);
    } else {
        launch_s<R>(ds, src, dst, nrhs, adjoint, s, tile, persist);
    }
}

// Choice recorded by the autotuner (or midbf_set_choice) for this RHS count,
// stage and direction; MIDBF_CHOICE_DEFAULT when there is none.
int tuned_choice(const midbf_dplan* dp, int nrhs, int sidx, bool adjoint);

// Run all stages.  user_in/user_out: caller vectors (column-major with ld).
template <class R>
void run(const midbf_dplan* dp, const std::vector<DevStage<R>>& stages, bool adjoint, const void* in, int64_t ldin,
         void* out, int64_t ldout, int nrhs, cudaStream_t s, void* ws) {
    const int ns = (int)stages.size();
    cx<R>* buf[2] = {static_cast<cx<R>*>(ws), static_cast<cx<R>*>(ws) + dp->max_space * nrhs};
    __nv_bfloat16* bimg = reinterpret_cast<__nv_bfloat16*>(static_cast<char*>(ws) + vec_workspace_bytes(dp, nrhs));
    VecRef<R> uin{(cx<R>*)in, 1, ldin};
    VecRef<R> uout{(cx<R>*)out, 1, ldout};
    auto internal = [&](int space) { return VecRef<R>{buf[space & 1], nrhs, 1}; };
    if (dp->profile) {
        while ((int)dp->ev.size() < 2 * ns) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            dp->ev.push_back(e);
        }
        dp->ev_stage.assign(ns, 0);
        dp->last_nrhs = nrhs;
    }
    for (int q = 0; q < ns; ++q) {
        const int sidx = adjoint ? ns - 1 - q : q;
        const DevStage<R>& ds = stages[sidx];
        if (dp->profile) {
            dp->ev_stage[q] = sidx;
            CK(cudaEventRecord(dp->ev[2 * q], s));
        }
        // forward: stage sidx reads space sidx-1 (user in for 0) and writes space sidx.
        VecRef<R> fin = sidx == 0 ? (adjoint ? uout : uin) : internal(sidx - 1);
        VecRef<R> fout = ds.out_user ? (adjoint ? uin : uout) : internal(sidx);
        VecRef<R> src = adjoint ? fout : fin;
        VecRef<R> dst = adjoint ? fin : fout;
        launch_stage<R>(dp, ds, adjoint, src, dst, nrhs, tuned_choice(dp, nrhs, sidx, adjoint), bimg, s);
        if (dp->profile) CK(cudaEventRecord(dp->ev[2 * q + 1], s));
    }
}


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
                default: go(std::integral_constant<int, 0>{});
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
            sm = std::max(sm, pattern_c_smem<R>(ds.max_narrow, ds.max_nsub, kRangeC1, 1));
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
                char* ws, bool dry = false) {
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
                if (use_r) {
                    const int t = forced_or_pick<R>(force, nr, [&](int qq) { return pattern_r_smem<R>(ds.max_nred, ds.rt, qq); });
                    key = {BT_R, ds.rt, t, 0};
                } else if (nr == 1 && force == 0 && pattern_c_smem<R>(ds.max_narrow, ds.max_nsub, kRangeC1, 1) <= kSmemCap) {
                    key = {BT_C1, 0, 1, 0};
                } else {
                    const int t = forced_or_pick<R>(force, nr, [&](int qq) { return pattern_c_smem<R>(ds.max_narrow, ds.max_nsub, kRangeC, qq); });
                    key = {BT_C, 0, t, 0};
                }
            } else {
                const int t = forced_or_pick<R>(force, nr, [&](int qq) {
                    return s_fly_smem<R>(ds.ss.P, ds.ss.Q, qq <= 4 && sizeof(R) == 4 ? 4 : 2, qq);
                });
                const int rt = (t <= 4 && sizeof(R) == 4) ? 4 : 2;
                const int pq = sizeof(R) == 4 ? phase_shape_code(ds.ss.P, ds.ss.Q) : 0;
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
    }
    return launches;
}

int tuned_choice(const midbf_dplan* dp, int nrhs, int sidx, bool adjoint) {
    if (dp->tuned.empty()) return MIDBF_CHOICE_DEFAULT;
    auto it = dp->tuned.find(nrhs);
    if (it == dp->tuned.end() || sidx >= (int)it->second.size()) return MIDBF_CHOICE_DEFAULT;
    return it->second[sidx][adjoint ? 1 : 0];
}

// Kernel variants worth timing for a stage and direction.
template <class R>
std::vector<int> stage_candidates(const midbf_dplan* dp, const DevStage<R>& ds, bool adjoint, int nrhs) {
    std::vector<int> c;
    const int cap = sizeof(R) == 4 ? 16 : 8;
    int top = 1;
    while (top < nrhs && top < cap) top *= 2;
    bool use_r = false;
    if (ds.id) {
        const bool wide_is_fwd_input = ds.kind != KIND_U;
        use_r = adjoint ? !wide_is_fwd_input : wide_is_fwd_input;
    }
    for (int nr = 1; nr <= top; nr *= 2) {
        size_t sm = 0;
        if (ds.id) sm = use_r ? pattern_r_smem<R>(ds.max_nred, ds.rt, nr) : pattern_c_smem<R>(ds.max_narrow, ds.max_nsub, kRangeC, nr);
        else sm = s_fly_smem<R>(ds.ss.P, ds.ss.Q, nr <= 4 && sizeof(R) == 4 ? 4 : 2, nr);
        if (sm <= kSmemCap) {
            c.push_back(nr);
            c.push_back(nr | MIDBF_CHOICE_PERSIST);
        }
    }
    if (ds.id && !use_r && nrhs == 1 && pattern_c_smem<R>(ds.max_narrow, ds.max_nsub, kRangeC1, 1) <= kSmemCap) {
        c.push_back(MIDBF_CHOICE_COLUMN1);
        c.push_back(MIDBF_CHOICE_COLUMN1 | MIDBF_CHOICE_PERSIST);
    }
    if (sizeof(R) == 4 && (ds.id ? ds.tc : dp->tc_mode != 0)) c.push_back(MIDBF_CHOICE_TENSOR);
    return c;
}

// Time every candidate of every stage in both directions on zero vectors of
// the plan's sizes (the kernels' cost does not depend on the values) and keep
// the fastest: one untimed launch, then the minimum of three timed ones.
template <class R>
void autotune(midbf_dplan* dp, const std::vector<DevStage<R>>& stages, int nrhs, cudaStream_t s) {
    const size_t ce = sizeof(cx<R>);
    const int64_t nuser = std::max(dp->nx, dp->nw);
    const size_t ub = (size_t)nuser * nrhs * ce, ib = (size_t)std::max<int64_t>(dp->max_space, 1) * nrhs * ce;
    const size_t bb = tc_bimg_bytes(dp, nrhs);
    void* mem = nullptr;
    if (cudaMalloc(&mem, 2 * ub + 2 * ib + bb) != cudaSuccess)
        fail(MIDBF_ENOMEM, "autotune: cudaMalloc of the trial vectors failed");
    struct Free {
        void* p;
        ~Free() { cudaFree(p); }
    } guard{mem};
    CK(cudaMemsetAsync(mem, 0, 2 * ub + 2 * ib + bb, s));
    cx<R>* ubuf[2] = {static_cast<cx<R>*>(mem), reinterpret_cast<cx<R>*>(static_cast<char*>(mem) + ub)};
    cx<R>* ibuf[2] = {reinterpret_cast<cx<R>*>(static_cast<char*>(mem) + 2 * ub),
                      reinterpret_cast<cx<R>*>(static_cast<char*>(mem) + 2 * ub + ib)};
    __nv_bfloat16* bimg = reinterpret_cast<__nv_bfloat16*>(static_cast<char*>(mem) + 2 * ub + 2 * ib);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int ns = (int)stages.size();
    std::vector<std::array<int, 2>> best(ns, {MIDBF_CHOICE_DEFAULT, MIDBF_CHOICE_DEFAULT});
    try {
        for (int sidx = 0; sidx < ns; ++sidx) {
            const DevStage<R>& ds = stages[sidx];
            for (int a = 0; a < 2; ++a) {
                const bool adjoint = a == 1;
                // the same vector roles as run(): user vectors at the ends, internal spaces between
                VecRef<R> fin = sidx == 0 ? VecRef<R>{ubuf[0], 1, nuser} : VecRef<R>{ibuf[(sidx - 1) & 1], nrhs, 1};
                VecRef<R> fout = ds.out_user ? VecRef<R>{ubuf[1], 1, nuser} : VecRef<R>{ibuf[sidx & 1], nrhs, 1};
                VecRef<R> src = adjoint ? fout : fin, dst = adjoint ? fin : fout;
                float best_ms = 1e30f;
                for (int cand : stage_candidates<R>(dp, ds, adjoint, nrhs)) {
                    launch_stage<R>(dp, ds, adjoint, src, dst, nrhs, cand, bimg, s);
                    float t = 1e30f;
                    for (int rep = 0; rep < 3; ++rep) {
                        CK(cudaEventRecord(e0, s));
                        launch_stage<R>(dp, ds, adjoint, src, dst, nrhs, cand, bimg, s);
                        CK(cudaEventRecord(e1, s));
                        CK(cudaEventSynchronize(e1));
                        float ms = 0.f;
                        CK(cudaEventElapsedTime(&ms, e0, e1));
                        t = std::min(t, ms);
                    }
                    if (t < best_ms) {
                        best_ms = t;
                        best[sidx][a] = cand;
                    }
                }
            }
        }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dp->tuned[nrhs] = best;
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &st));
    return st != cudaStreamCaptureStatusNone;
}

}  // namespace

// A recorded sequence of apply calls (midbf_capture_begin / _end).
struct midbf_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~midbf_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

// ---------------------------------------------------------------------------
// C ABI
extern "C" {

int midbf_autotune(midbf_dplan* dp, int nrhs, void* stream) {
    try {
        if (!dp || nrhs <= 0) fail(MIDBF_EINVAL, "bad argument");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (capturing(s)) fail(MIDBF_EINVAL, "midbf_autotune cannot run while the stream records a graph");
        if (dp->precision == MIDBF_FP32) autotune<float>(dp, dp->st32, nrhs, s);
        else autotune<double>(dp, dp->st64, nrhs, s);
        int st = 0;
        CK(cudaMemcpy(&st, dp->d_status, sizeof(int), cudaMemcpyDeviceToHost));
        if (st != 0) fail(MIDBF_ETIMEOUT, "a tensor-core wait gave up during tuning");
        return MIDBF_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::bad_alloc&) {
        set_last_error("host allocation failed");
        return MIDBF_ENOMEM;
    }
}

int midbf_set_choice(midbf_dplan* dp, int nrhs, int stage, int adjoint, int choice) {
    if (!dp || nrhs <= 0 || stage < 0 || stage >= (int)dp->stage_kind.size()) {
        set_last_error("midbf_set_choice: bad argument");
        return MIDBF_EINVAL;
    }
    if (!valid_choice(choice)) {
        set_last_error("midbf_set_choice: unknown choice");
        return MIDBF_EINVAL;
    }
    auto& v = dp->tuned[nrhs];
    if (v.empty()) v.assign(dp->stage_kind.size(), {MIDBF_CHOICE_DEFAULT, MIDBF_CHOICE_DEFAULT});
    v[stage][adjoint ? 1 : 0] = choice;
    return MIDBF_OK;
}

int midbf_get_choice(const midbf_dplan* dp, int nrhs, int stage, int adjoint, int* choice) {
    if (!dp || !choice || nrhs <= 0 || stage < 0 || stage >= (int)dp->stage_kind.size()) {
        set_last_error("midbf_get_choice: bad argument");
        return MIDBF_EINVAL;
    }
    *choice = tuned_choice(dp, nrhs, stage, adjoint != 0);
    return MIDBF_OK;
}

int midbf_capture_begin(void* stream) {
    try {
        if (!stream) fail(MIDBF_EINVAL, "the legacy default stream cannot record a graph");
        CK(cudaStreamBeginCapture(static_cast<cudaStream_t>(stream), cudaStreamCaptureModeThreadLocal));
        return MIDBF_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    }
}

int midbf_capture_end(void* stream, midbf_graph** graph) {
    try {
        if (!stream || !graph) fail(MIDBF_EINVAL, "null argument");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (!capturing(s)) fail(MIDBF_EINVAL, "no recording in progress on this stream");
        auto g = std::make_unique<midbf_graph>();
        cudaError_t e = cudaStreamEndCapture(s, &g->graph);
        if (e != cudaSuccess) fail(MIDBF_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&g->exec, g->graph, 0);
        if (e != cudaSuccess) fail(MIDBF_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        *graph = g.release();
        return MIDBF_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    }
}

int midbf_graph_launch(const midbf_graph* graph, void* stream) {
    try {
        if (!graph) fail(MIDBF_EINVAL, "null graph");
        CK(cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream)));
        return MIDBF_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    }
}

void midbf_graph_destroy(midbf_graph* graph) { delete graph; }


int midbf_dplan_create(const midbf_plan* plan, int precision, int s_mode, midbf_dplan** out) {
    try {
        if (!plan || !out) fail(MIDBF_EINVAL, "null argument");
        const int base = precision & ~MIDBF_REFINE;
        if (base != MIDBF_FP64 && base != MIDBF_FP32 && base != MIDBF_BF16) fail(MIDBF_EINVAL, "unknown precision");
        if ((precision & MIDBF_REFINE) && base != MIDBF_BF16) fail(MIDBF_EINVAL, "MIDBF_REFINE applies to MIDBF_BF16");
        if (s_mode != MIDBF_S_ONTHEFLY && s_mode != MIDBF_S_STORED) fail(MIDBF_EINVAL, "unknown middle-factor mode");
        const Plan& pl = *reinterpret_cast<const Plan*>(plan);
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) fail(MIDBF_ECUDA, "no CUDA device");
        auto dp = std::make_unique<midbf_dplan>();
        dp->precision = base == MIDBF_FP64 ? MIDBF_FP64 : MIDBF_FP32;
        dp->tc_mode = base == MIDBF_BF16 ? ((precision & MIDBF_REFINE) ? 2 : 1) : 0;
        if (dp->tc_mode && s_mode != MIDBF_S_ONTHEFLY) fail(MIDBF_EINVAL, "the tensor-core modes generate the middle factor on the fly");
        dp->s_mode = s_mode;
        CK(cudaGetDevice(&dp->device));
        dp->nx = pl.nx();
        dp->nw = pl.nw();
        if (cudaMalloc(&dp->d_status, sizeof(int)) != cudaSuccess) fail(MIDBF_ENOMEM, "cudaMalloc of the status word failed");
        CK(cudaMemset(dp->d_status, 0, sizeof(int)));
        if (dp->precision == MIDBF_FP32) make_stages<float>(dp.get(), pl, dp->st32);
        else make_stages<double>(dp.get(), pl, dp->st64);
        dp->launches = dp->precision == MIDBF_FP32 ? count_launches(dp->st32) : count_launches(dp->st64);
        CK(cudaDeviceSynchronize());
        *out = dp.release();
        return MIDBF_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::bad_alloc&) {
        set_last_error("host allocation failed");
        return MIDBF_ENOMEM;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return MIDBF_EINTERNAL;
    }
}

void midbf_dplan_destroy(midbf_dplan* dp) { delete dp; }

int midbf_dplan_status(const midbf_dplan* dp, int reset, int* status) {
    try {
        if (!dp || !status) fail(MIDBF_EINVAL, "null argument");
        int v = 0;
        CK(cudaMemcpy(&v, dp->d_status, sizeof(int), cudaMemcpyDeviceToHost));
        if (reset) CK(cudaMemset(dp->d_status, 0, sizeof(int)));
        *status = v;
        return MIDBF_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    }
}

int midbf_workspace_size(const midbf_dplan* dp, int nrhs, size_t* bytes) {
    if (!dp || !bytes || nrhs <= 0) {
        set_last_error("midbf_workspace_size: bad argument");
        return MIDBF_EINVAL;
    }
    *bytes = vec_workspace_bytes(dp, nrhs) + tc_bimg_bytes(dp, nrhs);
    return MIDBF_OK;
}

int midbf_dplan_bytes(const midbf_dplan* dp, size_t* factor_bytes, size_t* index_bytes) {
    if (!dp) {
        set_last_error("midbf_dplan_bytes: null plan");
        return MIDBF_EINVAL;
    }
    if (factor_bytes) *factor_bytes = dp->factor_bytes;
    if (index_bytes) *index_bytes = dp->index_bytes;
    return MIDBF_OK;
}

int midbf_apply_launches(const midbf_dplan* dp, int nrhs, int* launches) {
    if (!dp || !launches || nrhs <= 0) {
        set_last_error("midbf_apply_launches: bad argument");
        return MIDBF_EINVAL;
    }
    // mirrors launch_stage: a tensor-core stage runs a pack and a multiply per
    // group of kTcR RHS, a SIMT stage one launch
    int n = 0;
    const int groups = (nrhs + kTcR - 1) / kTcR;
    auto count = [&](const auto& stages) {
        for (size_t q = 0; q < stages.size(); ++q) {
            const auto& ds = stages[q];
            const int ch = tuned_choice(dp, nrhs, (int)q, false);
            bool tc = false;
            if (dp->precision == MIDBF_FP32) {
                const bool tc_ok = ds.id ? ds.tc : dp->tc_mode != 0;
                tc = tc_ok && (ch == MIDBF_CHOICE_TENSOR ||
                               (ch == MIDBF_CHOICE_DEFAULT && nrhs >= (ds.id ? kTcBlkMinRhs : kTcMinRhs)));
            }
            n += tc ? 2 * groups : 1;
        }
    };
    if (dp->precision == MIDBF_FP32) count(dp->st32);
    else count(dp->st64);
    *launches = n;
    return MIDBF_OK;
}

int midbf_dplan_profile(midbf_dplan* dp, int enable) {
    if (!dp) {
        set_last_error("midbf_dplan_profile: null plan");
        return MIDBF_EINVAL;
    }
    dp->profile = enable != 0;
    return MIDBF_OK;
}

int midbf_stage_times(const midbf_dplan* dp, int max_stages, float* ms, int* kinds, double* bytes, int* n_stages) {
    try {
        if (!dp || !n_stages || max_stages < 0) fail(MIDBF_EINVAL, "bad argument");
        if (!dp->profile || dp->ev_stage.empty()) fail(MIDBF_EINVAL, "no profiled apply recorded");
        const int ns = (int)dp->ev_stage.size();
        const size_t ce = dp->precision == MIDBF_FP32 ? 8 : 16;
        CK(cudaEventSynchronize(dp->ev[2 * ns - 1]));
        for (int q = 0; q < ns && q < max_stages; ++q) {
            const int sidx = dp->ev_stage[q];
            if (ms) CK(cudaEventElapsedTime(&ms[q], dp->ev[2 * q], dp->ev[2 * q + 1]));
            if (kinds) kinds[q] = dp->stage_kind[sidx];
            if (bytes)
                bytes[q] = dp->stage_fixed_bytes[sidx] + (double)dp->stage_vec_entries[sidx] * dp->last_nrhs * (double)ce;
        }
        *n_stages = ns;
        return MIDBF_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    }
}

int midbf_stage_info(const midbf_dplan* dp, int max_stages, int* kinds, int64_t* entries, int64_t* dense,
                     int* n_stages) {
    if (!dp || !n_stages || max_stages < 0) {
        set_last_error("midbf_stage_info: bad argument");
        return MIDBF_EINVAL;
    }
    const int ns = (int)dp->stage_kind.size();
    for (int q = 0; q < ns && q < max_stages; ++q) {
        if (kinds) kinds[q] = dp->stage_kind[q];
        if (entries) entries[q] = dp->stage_entries[q];
        if (dense) dense[q] = dp->stage_dense[q];
    }
    *n_stages = ns;
    return MIDBF_OK;
}

int midbf_apply(const midbf_dplan* dp, int adjoint, const void* in, int64_t ldin, void* out, int64_t ldout,
                int nrhs, void* stream, void* workspace, size_t workspace_bytes) {
    try {
        if (!dp || !in || !out) fail(MIDBF_EINVAL, "null argument");
        if (nrhs <= 0) fail(MIDBF_EINVAL, "nrhs must be positive");
        const int64_t nin = adjoint ? dp->nx : dp->nw;
        const int64_t nout = adjoint ? dp->nw : dp->nx;
        if (ldin < nin || ldout < nout) fail(MIDBF_EINVAL, "leading dimension smaller than the vector length");
        size_t need = 0;
        midbf_workspace_size(dp, nrhs, &need);
        if (!workspace || workspace_bytes < need) fail(MIDBF_EINVAL, "workspace too small: need " + std::to_string(need) + " bytes");
        const size_t ce = dp->precision == MIDBF_FP32 ? 8 : 16;
        const char* ib = static_cast<const char*>(in);
        const char* ob = static_cast<const char*>(out);
        const size_t inb = ((size_t)(nrhs - 1) * ldin + nin) * ce, outb = ((size_t)(nrhs - 1) * ldout + nout) * ce;
        if (ib < ob + outb && ob < ib + inb) fail(MIDBF_EINVAL, "input and output overlap");
        if (dp->nw >= (1LL << 31) || dp->nx >= (1LL << 31)) fail(MIDBF_EINVAL, "vectors longer than 2^31");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (dp->profile && capturing(s)) fail(MIDBF_EINVAL, "profiling is on: the apply cannot be recorded into a graph");
        if (dp->precision == MIDBF_FP32) run<float>(dp, dp->st32, adjoint != 0, in, ldin, out, ldout, nrhs, s, workspace);
        else run<double>(dp, dp->st64, adjoint != 0, in, ldin, out, ldout, nrhs, s, workspace);
        return MIDBF_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return MIDBF_EINTERNAL;
    }
}


int midbf_batched_workspace_size(int count, const midbf_dplan* const* dps, const int* nrhs, size_t* bytes) {
    if (count <= 0 || !dps || !nrhs || !bytes) {
        set_last_error("midbf_batched_workspace_size: bad argument");
        return MIDBF_EINVAL;
    }
    size_t b = 0;
    for (int i = 0; i < count; ++i) {
        if (!dps[i] || nrhs[i] <= 0) {
            set_last_error("midbf_batched_workspace_size: bad instance");
            return MIDBF_EINVAL;
        }
        b += instance_workspace(dps[i], nrhs[i]);
    }
    *bytes = b;
    return MIDBF_OK;
}

int midbf_batched_launches(int count, const midbf_dplan* const* dps, const int* adjoint, const int* nrhs,
                           int* launches) {
    try {
        if (count <= 0 || !dps || !adjoint || !nrhs || !launches) fail(MIDBF_EINVAL, "null argument");
        const int prec = dps[0] ? dps[0]->precision : -1;
        for (int i = 0; i < count; ++i)
            if (!dps[i] || nrhs[i] <= 0 || dps[i]->precision != prec) fail(MIDBF_EINVAL, "bad instance " + std::to_string(i));
        std::vector<const void*> in(count, nullptr);
        std::vector<void*> out(count, nullptr);
        std::vector<int64_t> ld(count, 0);
        *launches = prec == MIDBF_FP32
                        ? run_batched<float>(count, dps, adjoint, in.data(), ld.data(), out.data(), ld.data(), nrhs,
                                             nullptr, nullptr, true)
                        : run_batched<double>(count, dps, adjoint, in.data(), ld.data(), out.data(), ld.data(), nrhs,
                                              nullptr, nullptr, true);
        return MIDBF_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    }
}

int midbf_apply_batched(int count, const midbf_dplan* const* dps, const int* adjoint, const void* const* in,
                        const int64_t* ldin, void* const* out, const int64_t* ldout, const int* nrhs, void* stream,
                        void* workspace, size_t workspace_bytes) {
    try {
        if (count <= 0 || !dps || !adjoint || !in || !ldin || !out || !ldout || !nrhs) fail(MIDBF_EINVAL, "null argument");
        const int prec = dps[0] ? dps[0]->precision : -1;
        for (int i = 0; i < count; ++i) {
            const midbf_dplan* dp = dps[i];
            if (!dp || !in[i] || !out[i] || nrhs[i] <= 0) fail(MIDBF_EINVAL, "bad instance " + std::to_string(i));
            if (dp->precision != prec) fail(MIDBF_EINVAL, "all instances must share one precision");
            if (dp->device != dps[0]->device) fail(MIDBF_EINVAL, "all instances must live on one device");
            const int64_t nin = adjoint[i] ? dp->nx : dp->nw, nout = adjoint[i] ? dp->nw : dp->nx;
            if (ldin[i] < nin || ldout[i] < nout) fail(MIDBF_EINVAL, "leading dimension too small for instance " + std::to_string(i));
        }
        size_t need = 0;
        midbf_batched_workspace_size(count, dps, nrhs, &need);
        if (!workspace || workspace_bytes < need) fail(MIDBF_EINVAL, "workspace too small: need " + std::to_string(need) + " bytes");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (prec == MIDBF_FP32) run_batched<float>(count, dps, adjoint, in, ldin, out, ldout, nrhs, s, static_cast<char*>(workspace));
        else run_batched<double>(count, dps, adjoint, in, ldin, out, ldout, nrhs, s, static_cast<char*>(workspace));
        return MIDBF_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return MIDBF_EINTERNAL;
    }
}

int midbf_apply_host(const midbf_dplan* dp, int adjoint, const void* in_host, void* out_host, int nrhs, void* stream,
                     void* workspace, size_t workspace_bytes) {
    try {
        if (!dp || !in_host || !out_host || nrhs <= 0) fail(MIDBF_EINVAL, "bad argument");
        size_t need = 0;
        midbf_workspace_size(dp, nrhs, &need);
        const size_t ce = dp->precision == MIDBF_FP32 ? 8 : 16;
        const int64_t nin = adjoint ? dp->nx : dp->nw;
        const int64_t nout = adjoint ? dp->nw : dp->nx;
        const size_t io = (size_t)(nin + nout) * nrhs * ce;
        if (!workspace || workspace_bytes < need + io) fail(MIDBF_EINVAL, "workspace too small for host I/O");
        char* base = static_cast<char*>(workspace);
        char* din = base + need;
        char* dout = din + (size_t)nin * nrhs * ce;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (capturing(s)) fail(MIDBF_EINVAL, "midbf_apply_host cannot be recorded into a graph");
        CK(cudaMemcpyAsync(din, in_host, (size_t)nin * nrhs * ce, cudaMemcpyHostToDevice, s));
        int rc = midbf_apply(dp, adjoint, din, nin, dout, nout, nrhs, stream, workspace, need);
        if (rc != MIDBF_OK) return rc;
        CK(cudaMemcpyAsync(out_host, dout, (size_t)nout * nrhs * ce, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return MIDBF_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return MIDBF_EINTERNAL;
    }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Apply without any allocation.
//
// Some callers cannot allocate device memory at the time they apply the
// operator: a service whose GPU memory is entirely owned by another allocator
// (a framework's caching allocator, a fixed memory pool), or a latency-bound
// loop where cudaMalloc would synchronize the device and stall other work.
// midbf_apply_noalloc serves them: instead of a caller workspace it uses one
// statically sized scratch array in device memory that every GPU loading this
// library holds until the process exits.  It calls no cudaMalloc, cudaFree or
// allocating library routine.
//
// The array is shared by all calls: a call overwrites what the previous call
// left there (the kernels write every scratch entry they read, so nothing has
// to start at zero), and calls that overlap on the GPU - on different streams,
// or from different host threads without ordering - race on it.
namespace {
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB
}
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256] = {};  // device address of the scratch array, per device

// Device address of the scratch array on the current device.  The host-side
// name g_noalloc_scratch is only a stand-in, never a device address, so the
// address is looked up once per device with that device current.
void* noalloc_scratch(int dev) {
    if (dev < 0 || dev >= 256) fail(MIDBF_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            fail(MIDBF_ECUDA, std::string("cudaGetSymbolAddress of the scratch array failed: ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = ptr;
    }
    return g_noalloc_ptr[dev];
}
}  // namespace

extern "C" {

size_t midbf_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }

int midbf_apply_noalloc(const midbf_dplan* dp, int adjoint, const void* in, int64_t ldin, void* out, int64_t ldout,
                        int nrhs, void* stream) {
    try {
        if (!dp || !in || !out) fail(MIDBF_EINVAL, "null argument");
        if (nrhs <= 0) fail(MIDBF_EINVAL, "nrhs must be positive");
        const int64_t nin = adjoint ? dp->nx : dp->nw;
        const int64_t nout = adjoint ? dp->nw : dp->nx;
        if (ldin < nin || ldout < nout) fail(MIDBF_EINVAL, "leading dimension smaller than the vector length");
        size_t need = 0;
        midbf_workspace_size(dp, nrhs, &need);
        if (need > kNoAllocScratchBytes)
            fail(MIDBF_EINVAL, "midbf_apply_noalloc: this plan needs " + std::to_string(need) +
                                   " bytes of scratch for " + std::to_string(nrhs) +
                                   " right-hand sides, more than the built-in " +
                                   std::to_string(kNoAllocScratchBytes) +
                                   " bytes; use midbf_apply with a caller workspace or fewer right-hand sides");
        const size_t ce = dp->precision == MIDBF_FP32 ? 8 : 16;
        const char* ib = static_cast<const char*>(in);
        const char* ob = static_cast<const char*>(out);
        const size_t inb = ((size_t)(nrhs - 1) * ldin + nin) * ce, outb = ((size_t)(nrhs - 1) * ldout + nout) * ce;
        if (ib < ob + outb && ob < ib + inb) fail(MIDBF_EINVAL, "input and output overlap");
        int dev = 0;
        CK(cudaGetDevice(&dev));
        if (dev != dp->device) fail(MIDBF_EINVAL, "the current device is not the device of this plan");
        void* scratch = noalloc_scratch(dev);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (dp->precision == MIDBF_FP32) run<float>(dp, dp->st32, adjoint != 0, in, ldin, out, ldout, nrhs, s, scratch);
        else run<double>(dp, dp->st64, adjoint != 0, in, ldin, out, ldout, nrhs, s, scratch);
        return MIDBF_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return MIDBF_EINTERNAL;
    }
}

}  // extern "C"
