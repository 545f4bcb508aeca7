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
#include "dev_plan.cuh"

#ifdef __GLIBC__
#include <malloc.h>
#endif

using namespace midbf;
using namespace midbf_dev;
using namespace midbf_gpu;

namespace midbf_gpu {

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

// Chunks for the overlap of the middle factor (stage si) with the first U
// stage (si + 1): the blocks of S that a U block reads are joined into one
// group (union-find over the U blocks' inputs, found through the positions S
// writes), then whole groups are dealt to at most nch chunks of about equal
// work (entries of S and of the U stage's T), in block order.  Every U block
// reads only S blocks of its own chunk.  Returns false when there are fewer
// than two groups.
bool overlap_chunks(const Plan& pl, int si, int nch, std::vector<int>& ck_s, std::vector<int>& ck_u) {
    if (si < 0 || si + 1 >= (int)pl.stages.size() || pl.stages[si + 1].kind != KIND_U || nch < 2) return false;
    const Stage& S = pl.stages[si];
    const Stage& U = pl.stages[si + 1];
    const int ns = (int)S.blocks.size(), nu = (int)U.blocks.size();
    std::vector<int> owner((size_t)S.out_len, -1), parent(ns);
    std::iota(parent.begin(), parent.end(), 0);
    std::function<int(int)> find = [&](int a) {
        while (parent[a] != a) a = parent[a] = parent[parent[a]];
        return a;
    };
    for (int b = 0; b < ns; ++b)
        for (int64_t p : S.blocks[b].out_idx) owner[p] = b;
    std::vector<int> first(nu, -1);
    for (int b = 0; b < nu; ++b)
        for (int64_t p : U.blocks[b].in_idx) {
            const int o = owner[p];
            if (o < 0) fail(MIDBF_EINTERNAL, "U stage reads a position the middle factor does not write");
            if (first[b] < 0) first[b] = o;
            else parent[find(o)] = find(first[b]);
        }
    // group weights and group order (by smallest S block)
    std::vector<int> gid(ns, -1);
    std::vector<double> gw;
    for (int b = 0; b < ns; ++b) {
        const int r = find(b);
        if (gid[r] < 0) {
            gid[r] = (int)gw.size();
            gw.push_back(0.0);
        }
        gid[b] = gid[r];
        gw[gid[b]] += (double)S.blocks[b].out_idx.size() * (double)S.blocks[b].in_idx.size();
    }
    for (int b = 0; b < nu; ++b) {
        if (first[b] < 0) continue;
        for (const Sub& sb : U.blocks[b].subs) gw[gid[first[b]]] += (double)sb.k * (double)(sb.m - sb.k);
    }
    const int ng = (int)gw.size();
    if (ng < 2) return false;
    nch = std::min(nch, ng);
    const double total = std::accumulate(gw.begin(), gw.end(), 0.0);
    std::vector<int> gchunk(ng);
    double acc = 0.0;
    for (int g = 0; g < ng; ++g) {
        gchunk[g] = std::min(nch - 1, (int)(acc / total * nch));
        acc += gw[g];
    }
    ck_s.assign(ns, 0);
    ck_u.assign(nu, 0);
    for (int b = 0; b < ns; ++b) ck_s[b] = gchunk[gid[b]];
    for (int b = 0; b < nu; ++b) ck_u[b] = first[b] < 0 ? 0 : gchunk[gid[first[b]]];
    return true;
}

// Stable reorder of a work-item list by the chunk of each item's block, and
// the item offset of every chunk (off has nch + 1 entries).
template <class It, class BlockOf>
void group_items(std::vector<It>& items, const std::vector<int>& chunk_of_block, int nch, BlockOf block_of, int* off) {
    std::stable_sort(items.begin(), items.end(), [&](const It& a, const It& b) {
        return chunk_of_block[block_of(a)] < chunk_of_block[block_of(b)];
    });
    for (int k = 0; k <= nch; ++k) off[k] = 0;
    for (const It& it : items) off[chunk_of_block[block_of(it)] + 1]++;
    for (int k = 0; k < nch; ++k) off[k + 1] += off[k];
}

// Column stride of T on the device: k rounded up to even, so that every
// column starts on a 16-byte boundary (the one-RHS column kernel copies 16
// bytes at a time); the padding entries are zero.
inline int even_up(int k) { return k + (k & 1); }

// Build the device arrays of an ID stage (V or U), or of a stored S stage
// seen as dense blocks with no skeleton.
template <class R>
void make_id_stage(midbf_dplan* dp, const Plan& pl, const Stage& st, DevStage<R>& ds, bool stored_s,
                   const std::vector<int>* chunk_of_block = nullptr, int nch = 0) {
    std::vector<SubDesc> subs;
    std::vector<BlockDesc> blocks;
    std::vector<int> skel, red, wide_pos, narrow_pos;
    std::vector<ItemR> items_r;
    std::vector<ItemC> items_c, items_c1;
    // T goes to the device in chunks through a bounded host buffer: the
    // largest stages hold billions of entries
    size_t nt = 0, nt_pad = 0;   // entries of T with its column padding; the padding alone
    {
        size_t ns = 0, nk = 0;
        for (const Block& bk : st.blocks) {
            if (stored_s) {
                const int k = (int)bk.out_idx.size();
                nt += (size_t)even_up(k) * bk.in_idx.size();
                nt_pad += (size_t)(even_up(k) - k) * bk.in_idx.size();
            } else {
                for (const Sub& sb : bk.subs) {
                    nt += (size_t)even_up(sb.k) * (size_t)(sb.m - sb.k);
                    nt_pad += (size_t)(even_up(sb.k) - sb.k) * (size_t)(sb.m - sb.k);
                    nk += (size_t)sb.k;
                    ns += (size_t)(sb.m - sb.k);
                }
            }
        }
        skel.reserve(nk);
        red.reserve(ns);
    }
    constexpr size_t kChunk = (size_t)64 << 20;   // entries per host-to-device copy
    cx<R>* dT = nullptr;
    if (nt) {
        const size_t bytes = nt * sizeof(cx<R>);
        if (cudaMalloc(reinterpret_cast<void**>(&dT), bytes) != cudaSuccess)
            fail(MIDBF_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
        dp->allocs.push_back(dT);
        dp->factor_bytes += bytes;
        dp->pad_bytes += nt_pad * sizeof(cx<R>);
    }
    std::vector<cx<R>> T;
    T.reserve(std::min(nt, kChunk + 4096));
    size_t t_done = 0;   // entries already copied to the device
    auto flush = [&]() {
        if (T.empty()) return;
        CK(cudaMemcpy(dT + t_done, T.data(), T.size() * sizeof(cx<R>), cudaMemcpyHostToDevice));
        t_done += T.size();
        T.clear();
    };
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
            sd.ld = even_up(sd.k);
            sd.nskel = 0;
            sd.skel_off = (int)skel.size();
            sd.red_off = (int)red.size();
            sd.narrow_off = noff;
            sd.block = (int)b;
            if (T.size() + (size_t)sd.ld * bd.m > kChunk) flush();
            sd.t_off = (long long)(t_done + T.size());
            for (int j = 0; j < bd.m; ++j) red.push_back(j);
            const size_t base = T.size();
            T.resize(base + (size_t)sd.ld * bd.m);   // the padding rows stay zero
            const int nthreads = std::max(1u, std::thread::hardware_concurrency());
            std::vector<std::thread> th;
            for (int w = 0; w < nthreads; ++w)
                th.emplace_back([&, w]() {
                    for (int j = w; j < bd.m; j += nthreads)
                        for (int i = 0; i < sd.k; ++i) {
                            cplx kv = pl.phase.kernel(bk.xidx[i], bk.widx[j]);
                            T[base + (size_t)j * sd.ld + i] = {(R)kv.real(), (R)kv.imag()};
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
                sd.ld = even_up(sb.k);
                sd.nskel = sb.k;
                sd.skel_off = (int)skel.size();
                sd.red_off = (int)red.size();
                sd.narrow_off = noff;
                sd.block = (int)b;
                if (T.size() + (size_t)sd.ld * (sb.m - sb.k) > kChunk) flush();
                sd.t_off = (long long)(t_done + T.size());
                noff += sb.k;
                for (int v : sb.skel) skel.push_back(v);
                const int nred = sb.m - sb.k;
                std::vector<int> perm(nred);
                std::iota(perm.begin(), perm.end(), 0);
                std::sort(perm.begin(), perm.end(), [&](int a, int c) { return sb.red[a] < sb.red[c]; });
                for (int jj = 0; jj < nred; ++jj) red.push_back(sb.red[perm[jj]]);
                for (int jj = 0; jj < nred; ++jj) {
                    for (int i = 0; i < sb.k; ++i) {
                        const cplx v = sb.t((size_t)i * nred + perm[jj]);
                        T.push_back({(R)v.real(), (R)v.imag()});
                    }
                    if (sd.ld > sb.k) T.push_back({R(0), R(0)});   // pad the column to ld entries
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
    }
    if (max_nsub > 16) fail(MIDBF_EINTERNAL, "more than 16 sub-blocks in a block");
    // One-RHS column items: kRangeC1 outputs each, or fewer when a stage has
    // too few wide blocks to give every SM several items (a CTA streams one
    // item's columns at a latency-bound rate, so a short grid leaves the HBM
    // idle); ranges of 64 or 32 outputs split the same columns over more CTAs.
    // Every item gathers all of its block's narrow inputs, so a range is
    // halved only while those gathers stay within 1/8 of the stage's T
    // entries (a block with little T, mostly skeleton, keeps its range).
    {
        const int target = 4 * sm_count();
        int range = kRangeC1;
        auto count = [&](int rg) {
            size_t c = 0;
            for (const BlockDesc& bd : blocks) c += (size_t)((bd.m + rg - 1) / rg);
            return c;
        };
        auto gathers = [&](int rg) {
            size_t g = 0;
            for (const BlockDesc& bd : blocks) g += (size_t)bd.nnarrow * (size_t)((bd.m + rg - 1) / rg);
            return g;
        };
        const size_t t_stage = nt - nt_pad;
        while (range > 32 && count(range) < (size_t)target && 8 * gathers(range / 2) <= t_stage) range /= 2;
        for (size_t b = 0; b < blocks.size(); ++b)
            for (int o0 = 0; o0 < blocks[b].m; o0 += range)
                items_c1.push_back({(int)b, o0, std::min(blocks[b].m, o0 + range), 0});
        ds.range_c1 = range;
    }
    const int rt = rows_per_lane(maxk);
    for (size_t s = 0; s < subs.size(); ++s)
        for (int r0 = 0; r0 < subs[s].k; r0 += 32 * rt) items_r.push_back({(int)s, r0});
    if (chunk_of_block && nch > 1) {
        group_items(items_r, *chunk_of_block, nch, [&](const ItemR& it) { return subs[it.sub].block; }, ds.ck_r);
        group_items(items_c, *chunk_of_block, nch, [](const ItemC& it) { return it.block; }, ds.ck_c);
        group_items(items_c1, *chunk_of_block, nch, [](const ItemC& it) { return it.block; }, ds.ck_c1);
        ds.nchunks = nch;
    }
    // the column range of every (column item, sub-block): one host-side binary
    // search over the sorted redundant indices, instead of one per CTA
    auto make_jr = [&](std::vector<ItemC>& items) {
        std::vector<int2> jr;
        for (ItemC& it : items) {
            const BlockDesc& bd = blocks[it.block];
            it.jr_off = (int)jr.size();
            for (int c = 0; c < bd.nsub; ++c) {
                const SubDesc& sd = subs[bd.sub0 + c];
                const int* r = red.data() + sd.red_off;
                const int* e = r + (bd.m - sd.nskel);
                jr.push_back(make_int2((int)(std::lower_bound(r, e, it.o0) - r), (int)(std::lower_bound(r, e, it.o1) - r)));
            }
        }
        return jr;
    };
    const std::vector<int2> jr_c = make_jr(items_c), jr_c1 = make_jr(items_c1);
    ds.id = true;
    ds.rt = rt;
    ds.n_subs = (int)subs.size();
    ds.max_k = maxk;
    ds.n_items_r = (int)items_r.size();
    ds.row_cl = row_cluster_size(ds.n_items_r, (int)max_nred);
    ds.n_items_c = (int)items_c.size();
    ds.max_nred = (int)max_nred;
    ds.max_narrow = (int)max_narrow;
    ds.n_blocks = (int)blocks.size();
    for (const BlockDesc& bd : blocks) ds.max_m = std::max(ds.max_m, bd.m);
    ds.max_nsub = (int)max_nsub;
    if (pattern_r_smem<R>((int)max_nred, rt, 1) > kSmemCap || pattern_c_smem<R>((int)max_narrow, (int)max_nsub, kRangeC, 1) > kSmemCap)
        fail(MIDBF_EINTERNAL, "block too wide for shared memory");
    ds.ids.subs = upload(dp, subs, &dp->index_bytes);
    ds.ids.blocks = upload(dp, blocks, &dp->index_bytes);
    ds.ids.skel = upload(dp, skel, &dp->index_bytes);
    ds.ids.red = upload(dp, red, &dp->index_bytes);
    ds.ids.wide_pos = upload(dp, wide_pos, &dp->index_bytes);
    ds.ids.narrow_pos = upload(dp, narrow_pos, &dp->index_bytes);
    flush();
    if (t_done != nt) fail(MIDBF_EINTERNAL, "coefficient count mismatch");
    ds.ids.T = dT;
    ds.ids.items_r = upload(dp, items_r, &dp->index_bytes);
    ds.ids.items_c = upload(dp, items_c, &dp->index_bytes);
    ds.ids.jr = upload(dp, jr_c, &dp->index_bytes);
    ds.ids1 = ds.ids;
    ds.ids1.items_c = upload(dp, items_c1, &dp->index_bytes);
    ds.ids1.jr = upload(dp, jr_c1, &dp->index_bytes);
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
    if (fam == MIDBF_PHASE_DISTANCE) {
        // |x - xi| in the distance form: coordinates relative to the block's
        // first column point xi0 (formed in FP64), missing axes zero
        const double* w0 = &ph.W[(size_t)j0 * d];
        for (size_t i = 0; i < nr; ++i) {
            const double* x = &ph.X[(size_t)bk.xidx[i] * d];
            rows.a[i] = 0.0;
            for (int k = 0; k < Q; ++k) rows.c[i * Q + k] = k < d ? x[k] - w0[k] : 0.0;
        }
        for (size_t j = 0; j < nc; ++j) {
            const double* w = &ph.W[(size_t)bk.widx[j] * d];
            cols.a[j] = 0.0;
            for (int k = 0; k < Q; ++k) cols.c[j * Q + k] = k < d ? w[k] - w0[k] : 0.0;
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
void make_s_stage(midbf_dplan* dp, const Plan& pl, const Stage& st, DevStage<R>& ds,
                  const std::vector<int>* chunk_of_block = nullptr, int nch = 0) {
    const Phase& ph = pl.phase;
    int P = 0, Q = 0;
    switch (ph.family) {
        case MIDBF_PHASE_LOWRANK: P = ph.r; break;
        case MIDBF_PHASE_DOT: P = ph.d; break;
        case MIDBF_PHASE_FIO2D: case MIDBF_PHASE_FIO3D: P = ph.d; Q = ph.d; break;
        case MIDBF_PHASE_FIO2D_JUMP: P = ph.d + 1; Q = ph.d; break;
        case MIDBF_PHASE_DISTANCE: P = 0; Q = 3; ds.s_dist = true; break;
        default: break;
    }
    if (P > 8 || Q > 3) fail(MIDBF_EINVAL, "on-the-fly middle factor supports at most 8 low-rank terms");
    std::vector<int> blk_rows, blk_cols, blk_nrow, blk_ncol, rpos, cpos;
    std::vector<R> ra, ru, rc, ca, cu, cc;
    std::vector<double> da_r, du_r, dc_r, da_c, du_c, dc_c;   // the FP64 values (accurate phase only)
    const bool keep64 = dp->s_mode == MIDBF_S_ONTHEFLY_DF;
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
        if (keep64) {
            da_r.insert(da_r.end(), r.a.begin(), r.a.end());
            du_r.insert(du_r.end(), r.u.begin(), r.u.end());
            dc_r.insert(dc_r.end(), r.c.begin(), r.c.end());
            da_c.insert(da_c.end(), c.a.begin(), c.a.end());
            du_c.insert(du_c.end(), c.u.begin(), c.u.end());
            dc_c.insert(dc_c.end(), c.c.begin(), c.c.end());
        }
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
    if (chunk_of_block && nch > 1) {
        auto blk = [](const int2& it) { return it.x; };
        group_items(it_rows, *chunk_of_block, nch, blk, ds.ck_rows);
        group_items(it_cols, *chunk_of_block, nch, blk, ds.ck_cols);
        group_items(it_rows4, *chunk_of_block, nch, blk, ds.ck_rows4);
        group_items(it_cols4, *chunk_of_block, nch, blk, ds.ck_cols4);
        ds.nchunks = nch;
    }
    ds.ss.P = P;
    ds.ss.Q = Q;
    ds.ss.blk_rows = upload(dp, blk_rows, &dp->index_bytes);
    ds.ss.blk_cols = upload(dp, blk_cols, &dp->index_bytes);
    ds.ss.blk_nrow = upload(dp, blk_nrow, &dp->index_bytes);
    ds.ss.blk_ncol = upload(dp, blk_ncol, &dp->index_bytes);
    if (dp->s_mode == MIDBF_S_ONTHEFLY_DF) {
        if constexpr (sizeof(R) != 4) fail(MIDBF_EINVAL, "the accurate phase applies to MIDBF_FP32 plans");
        if (ds.s_dist) fail(MIDBF_EINVAL, "the accurate phase takes the inner-product phases, not the distance form");
        // hi + lo of every FP64 value: hi = float(v), lo = float(v - hi)
        auto lo_of = [](const std::vector<double>& v, std::vector<R>& hi) {
            std::vector<R> lo(v.size());
            for (size_t i = 0; i < v.size(); ++i) lo[i] = (R)(v[i] - (double)hi[i]);
            return lo;
        };
        ds.srows.a_lo = upload(dp, lo_of(da_r, ra), &dp->factor_bytes);
        ds.srows.u_lo = upload(dp, lo_of(du_r, ru), &dp->factor_bytes);
        ds.srows.c_lo = upload(dp, lo_of(dc_r, rc), &dp->factor_bytes);
        ds.scols.a_lo = upload(dp, lo_of(da_c, ca), &dp->factor_bytes);
        ds.scols.u_lo = upload(dp, lo_of(du_c, cu), &dp->factor_bytes);
        ds.scols.c_lo = upload(dp, lo_of(dc_c, cc), &dp->factor_bytes);
        ds.s_df = true;
    }
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
    ds.n4_rows_stage = ds.n_items_rows4;
    ds.n4_cols_stage = ds.n_items_cols4;
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

// consume: the same plan, writable; each stage's ID coefficients are released
// from it once they are on the device.
template <class R>
void make_stages(midbf_dplan* dp, const Plan& pl, std::vector<DevStage<R>>& out, Plan* consume, bool overlap) {
    int64_t in_len = pl.phase.nw;
    // overlap groups of the middle factor and the U stage after it
    std::vector<int> ck_s, ck_u;
    int si = -1;
    for (size_t s = 0; s < pl.stages.size(); ++s)
        if (pl.stages[s].kind == KIND_S) si = (int)s;
    dp->s_stage = si;
    const bool grouped = overlap && overlap_chunks(pl, si, kDefaultChunks, ck_s, ck_u);
    int nch = 0;
    if (grouped) nch = 1 + std::max(*std::max_element(ck_s.begin(), ck_s.end()), *std::max_element(ck_u.begin(), ck_u.end()));
    dp->chunks_built = grouped ? nch : 0;
    dp->chunks = dp->chunks_built;
    for (size_t s = 0; s < pl.stages.size(); ++s) {
        const Stage& st = pl.stages[s];
        const std::vector<int>* ck = !grouped ? nullptr : (int)s == si ? &ck_s : (int)s == si + 1 ? &ck_u : nullptr;
        DevStage<R> ds;
        ds.kind = st.kind;
        ds.in_len = in_len;
        ds.out_len = st.out_len;
        ds.in_user = s == 0;
        ds.out_user = st.out_user != 0;
        const size_t f0 = dp->factor_bytes, i0 = dp->index_bytes, p0 = dp->pad_bytes;
        if (st.kind == KIND_S) {
            if (dp->s_mode == MIDBF_S_STORED) make_id_stage<R>(dp, pl, st, ds, true, ck, nch);
            else make_s_stage<R>(dp, pl, st, ds, ck, nch);
        } else {
            make_id_stage<R>(dp, pl, st, ds, false, ck, nch);
            if (consume) {
                for (Block& bk : consume->stages[s].blocks)
                    for (Sub& sb : bk.subs) {
                        std::vector<cplx>().swap(sb.T);
                        std::vector<std::complex<float>>().swap(sb.Tf);
                    }
#ifdef __GLIBC__
                malloc_trim(0);   // hand the freed pages back to the system now
#endif
            }
        }
        // algorithmic bytes: factor data and position maps once, vectors per RHS
        // (work-item lists and descriptors are bookkeeping, counted too; the zero
        // padding of the T columns is not)
        dp->stage_fixed_bytes.push_back((double)(dp->factor_bytes - f0) - (double)(dp->pad_bytes - p0) +
                                        (double)(dp->index_bytes - i0));
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

// Streaming multiprocessors of the current device (cached per device).
int sm_count() {
    static std::mutex mu;
    static std::map<int, int> cache;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    cache[dev] = std::max(1, nsm);
    return cache[dev];
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


// One stage launch.  choice: MIDBF_CHOICE_DEFAULT (the built-in rules: tensor
// cores in the BF16 modes from kTcMinRhs / kTcBlkMinRhs RHS on, else the SIMT
// kernel with the RHS tile of pick_nr), a SIMT RHS tile (1, 2, 4, 8, 16) or
// MIDBF_CHOICE_COLUMN1 (the one-RHS pattern-C kernel), each optionally with
// MIDBF_CHOICE_PERSIST; or one of MIDBF_CHOICE_NARROW (the narrow-ID
// kernels), MIDBF_CHOICE_CLUSTER (the one-RHS row pattern on clusters of
// CTAs), MIDBF_CHOICE_GEMM (the FP32 middle factor as a register-tiled GEMM)
// and MIDBF_CHOICE_TENSOR.
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
    const bool wide_is_fwd_input = ds.kind != KIND_U;  // V and stored S
    // pattern R computes narrow from wide; pattern C wide from narrow.
    const bool use_r = adjoint ? !wide_is_fwd_input : wide_is_fwd_input;
    const bool narrow = use_narrow(ds, nrhs, choice, use_r);
    const bool persist = !whole_choice(choice) && (choice & MIDBF_CHOICE_PERSIST) != 0;
    const int tile = choice_tile(choice);
    const bool col1 = !whole_choice(choice) && (choice & ~MIDBF_CHOICE_PERSIST) == MIDBF_CHOICE_COLUMN1;
    // one RHS, row pattern: a cluster of CTAs per item when asked for, or by
    // default when the stage has few items
    const int cl = (ds.id && use_r && !narrow && nrhs == 1) ? row_cluster_for(ds, choice) : 1;
    if (ds.id) {
        if (cl > 1) {
            launch_r_cluster<R>(ds, src, dst, adjoint, cl, s);
        } else if (narrow) {
            if (use_r) launch_r_narrow<R>(ds, src, dst, adjoint, s);
            else launch_c_narrow<R>(ds, src, dst, adjoint, s);
        } else if (use_gemm(ds, nrhs, choice, use_r)) {
            if constexpr (sizeof(R) == 4) {
                if (use_r) launch_r_gemm(ds, src, dst, nrhs, adjoint, s);
                else launch_c_gemm(ds, src, dst, nrhs, adjoint, s);
            }
        } else if (use_r) {
            launch_r<R>(ds, src, dst, nrhs, adjoint, s, tile, persist);
        } else {
            launch_c<R>(ds, src, dst, nrhs, adjoint, s, col1 ? MIDBF_CHOICE_COLUMN1 : tile, persist);
        }
    } else if constexpr (sizeof(R) == 4) {
        if (use_gemm(ds, nrhs, choice, false)) launch_s_gemm(ds, src, dst, nrhs, adjoint, s);
        else launch_s<R>(ds, src, dst, nrhs, adjoint, s, tile, persist);
    } else {
        launch_s<R>(ds, src, dst, nrhs, adjoint, s, tile, persist);
    }
}

// The work items of chunk k of a split stage: a shallow copy whose item lists
// and counts cover that chunk only.
template <class R>
DevStage<R> chunk_view(const DevStage<R>& ds, int k) {
    DevStage<R> v = ds;
    auto cut = [k](auto& ptr, int& n, const int* off) {
        if (ptr) ptr += off[k];
        n = off[k + 1] - off[k];
    };
    if (ds.id) {
        cut(v.ids.items_r, v.n_items_r, ds.ck_r);
        cut(v.ids.items_c, v.n_items_c, ds.ck_c);
        cut(v.ids1.items_c, v.n_items_c1, ds.ck_c1);
    } else {
        cut(v.items_rows, v.n_items_rows, ds.ck_rows);
        cut(v.items_rows4, v.n_items_rows4, ds.ck_rows4);
        cut(v.items_cols, v.n_items_cols, ds.ck_cols);
        cut(v.items_cols4, v.n_items_cols4, ds.ck_cols4);
    }
    return v;
}

// Whether a stage launch runs on the tensor cores (mirrors launch_stage).
template <class R>
bool stage_uses_tc(const midbf_dplan* dp, const DevStage<R>& ds, int nrhs, int choice) {
    if (sizeof(R) != 4) return false;
    const bool tc_ok = ds.id ? ds.tc : dp->tc_mode != 0;
    return tc_ok && (choice == MIDBF_CHOICE_TENSOR ||
                     (choice == MIDBF_CHOICE_DEFAULT && nrhs >= (ds.id ? kTcBlkMinRhs : kTcMinRhs)));
}

// Whether an apply overlaps the middle factor with its U stage: chunks on,
// profiling off (per-stage events need the stages one after the other), and
// both stages on the SIMT kernels.
template <class R>
bool overlapped(const midbf_dplan* dp, const std::vector<DevStage<R>>& stages, int nrhs, bool adjoint) {
    const int si = dp->s_stage;
    if (dp->chunks < 2 || dp->profile || si < 0 || si + 1 >= (int)stages.size()) return false;
    if (stages[si].nchunks != dp->chunks_built || stages[si + 1].nchunks != dp->chunks_built) return false;
    return !stage_uses_tc(dp, stages[si], nrhs, tuned_choice(dp, nrhs, si, adjoint)) &&
           !stage_uses_tc(dp, stages[si + 1], nrhs, tuned_choice(dp, nrhs, si + 1, adjoint));
}

// Run all stages.  user_in/user_out: caller vectors (column-major with ld).
//
// With the overlap on, the middle factor S (stage si) and the U stage after
// it run as chunks: forward, chunk k of S on the caller's stream, then chunk
// k of U on the plan's side stream after an event; adjoint, chunk k of U's
// adjoint first, then chunk k of S's adjoint on the side stream.  The side
// stream forks from the caller's stream before the pair and joins it after,
// so the apply stays ordered on the caller's stream (and records into a
// graph as one fork and join).  U's internal output space lives in the third
// workspace vector: with two, it would share a buffer with the input of S,
// which later chunks of S still read.
template <class R>
void run(const midbf_dplan* dp, const std::vector<DevStage<R>>& stages, bool adjoint, const void* in, int64_t ldin,
         void* out, int64_t ldout, int nrhs, cudaStream_t s, void* ws) {
    const int ns = (int)stages.size();
    cx<R>* buf[3] = {static_cast<cx<R>*>(ws), static_cast<cx<R>*>(ws) + dp->max_space * nrhs,
                     static_cast<cx<R>*>(ws) + 2 * dp->max_space * nrhs};
    __nv_bfloat16* bimg = reinterpret_cast<__nv_bfloat16*>(static_cast<char*>(ws) + vec_workspace_bytes(dp, nrhs));
    VecRef<R> uin{(cx<R>*)in, 1, ldin};
    VecRef<R> uout{(cx<R>*)out, 1, ldout};
    const bool third = vec_buffers(dp) == 3;
    auto internal = [&](int space) {
        return VecRef<R>{third && space == dp->s_stage + 1 ? buf[2] : buf[space & 1], nrhs, 1};
    };
    const bool pipe = overlapped(dp, stages, nrhs, adjoint);
    std::unique_lock<std::mutex> lk(dp->pipe_mu, std::defer_lock);
    if (pipe) lk.lock();
    if (dp->profile) {
        while ((int)dp->ev.size() < 2 * ns) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            dp->ev.push_back(e);
        }
        dp->ev_stage.assign(ns, 0);
        dp->last_nrhs = nrhs;
    }
    // forward: stage sidx reads space sidx-1 (user in for 0) and writes space sidx.
    auto io = [&](int sidx, VecRef<R>& src, VecRef<R>& dst) {
        VecRef<R> fin = sidx == 0 ? (adjoint ? uout : uin) : internal(sidx - 1);
        VecRef<R> fout = stages[sidx].out_user ? (adjoint ? uin : uout) : internal(sidx);
        src = adjoint ? fout : fin;
        dst = adjoint ? fin : fout;
    };
    for (int q = 0; q < ns; ++q) {
        const int sidx = adjoint ? ns - 1 - q : q;
        const DevStage<R>& ds = stages[sidx];
        VecRef<R> src, dst;
        io(sidx, src, dst);
        if (pipe && sidx == (adjoint ? dp->s_stage + 1 : dp->s_stage)) {
            // the overlapped pair: this stage (first) and the next one in launch order (second)
            const int sidx2 = adjoint ? dp->s_stage : dp->s_stage + 1;
            VecRef<R> src2, dst2;
            io(sidx2, src2, dst2);
            const int c1 = tuned_choice(dp, nrhs, sidx, adjoint), c2 = tuned_choice(dp, nrhs, sidx2, adjoint);
            CK(cudaEventRecord(dp->ev_fork, s));
            CK(cudaStreamWaitEvent(dp->side, dp->ev_fork, 0));
            for (int k = 0; k < dp->chunks; ++k) {
                launch_stage<R>(dp, chunk_view(ds, k), adjoint, src, dst, nrhs, c1, bimg, s);
                CK(cudaEventRecord(dp->ev_ck[k], s));
                CK(cudaStreamWaitEvent(dp->side, dp->ev_ck[k], 0));
                launch_stage<R>(dp, chunk_view(stages[sidx2], k), adjoint, src2, dst2, nrhs, c2, bimg, dp->side);
            }
            CK(cudaEventRecord(dp->ev_join, dp->side));
            CK(cudaStreamWaitEvent(s, dp->ev_join, 0));
            ++q;
            continue;
        }
        if (dp->profile) {
            dp->ev_stage[q] = sidx;
            CK(cudaEventRecord(dp->ev[2 * q], s));
        }
        launch_stage<R>(dp, ds, adjoint, src, dst, nrhs, tuned_choice(dp, nrhs, sidx, adjoint), bimg, s);
        if (dp->profile) CK(cudaEventRecord(dp->ev[2 * q + 1], s));
    }
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
    if (ds.id && !use_r && nrhs == 1 && pattern_c1_smem<R>(ds.max_narrow, ds.max_nsub) <= kSmemCap) {
        c.push_back(MIDBF_CHOICE_COLUMN1);
        c.push_back(MIDBF_CHOICE_COLUMN1 | MIDBF_CHOICE_PERSIST);
    }
    if (ds.id && nrhs == 1 && ds.nchunks == 0 && ds.max_k <= 64 &&
        (use_r || pattern_c_smem<R>(ds.max_narrow, ds.max_nsub, kRangeC1, 1) <= kSmemCap))
        c.push_back(MIDBF_CHOICE_NARROW);
    if (ds.id && use_r && nrhs == 1) c.push_back(MIDBF_CHOICE_CLUSTER);
    if (sizeof(R) == 4 && (ds.id || !ds.s_df) && nrhs >= 8) c.push_back(MIDBF_CHOICE_GEMM);
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

// Checks shared by the apply entry points (midbf_apply, midbf_apply_noalloc):
// handles and pointers, RHS count, leading dimensions, disjoint in/out, the
// 32-bit position maps, and no profiling events inside a graph recording.
void check_apply_args(const midbf_dplan* dp, int adjoint, const void* in, int64_t ldin, const void* out,
                      int64_t ldout, int nrhs, cudaStream_t s) {
    if (!dp || !in || !out) fail(MIDBF_EINVAL, "null argument");
    if (nrhs <= 0) fail(MIDBF_EINVAL, "nrhs must be positive");
    const int64_t nin = adjoint ? dp->nx : dp->nw;
    const int64_t nout = adjoint ? dp->nw : dp->nx;
    if (ldin < nin || ldout < nout) fail(MIDBF_EINVAL, "leading dimension smaller than the vector length");
    const size_t ce = dp->precision == MIDBF_FP32 ? 8 : 16;
    const char* ib = static_cast<const char*>(in);
    const char* ob = static_cast<const char*>(out);
    const size_t inb = ((size_t)(nrhs - 1) * ldin + nin) * ce, outb = ((size_t)(nrhs - 1) * ldout + nout) * ce;
    if (ib < ob + outb && ob < ib + inb) fail(MIDBF_EINVAL, "input and output overlap");
    if (dp->nw >= (1LL << 31) || dp->nx >= (1LL << 31)) fail(MIDBF_EINVAL, "vectors longer than 2^31");
    if (dp->profile && capturing(s)) fail(MIDBF_EINVAL, "profiling is on: the apply cannot be recorded into a graph");
}

// Scratch array of midbf_apply_noalloc (defined at the end of this file).
void* noalloc_lookup(std::string& err);

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
    return midbf_dplan_create_ex(const_cast<midbf_plan*>(plan), precision, s_mode, 0, out);
}

int midbf_dplan_create_ex(midbf_plan* plan, int precision, int s_mode, int flags, midbf_dplan** out) {
    try {
        if (!plan || !out) fail(MIDBF_EINVAL, "null argument");
        if (flags & ~(MIDBF_DPLAN_CONSUME | MIDBF_DPLAN_OVERLAP)) fail(MIDBF_EINVAL, "unknown flags");
        const int base = precision & ~MIDBF_REFINE;
        if (base != MIDBF_FP64 && base != MIDBF_FP32 && base != MIDBF_BF16) fail(MIDBF_EINVAL, "unknown precision");
        if ((precision & MIDBF_REFINE) && base != MIDBF_BF16) fail(MIDBF_EINVAL, "MIDBF_REFINE applies to MIDBF_BF16");
        if (s_mode != MIDBF_S_ONTHEFLY && s_mode != MIDBF_S_STORED && s_mode != MIDBF_S_ONTHEFLY_DF)
            fail(MIDBF_EINVAL, "unknown middle-factor mode");
        if (s_mode == MIDBF_S_ONTHEFLY_DF && base != MIDBF_FP32)
            fail(MIDBF_EINVAL, "the accurate phase (MIDBF_S_ONTHEFLY_DF) applies to MIDBF_FP32 plans");
        Plan& plw = *reinterpret_cast<Plan*>(plan);
        const Plan& pl = plw;
        if (pl.released) fail(MIDBF_EINVAL, "the plan's coefficients were released by an earlier consuming upload");
        Plan* consume = (flags & MIDBF_DPLAN_CONSUME) ? &plw : nullptr;
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) fail(MIDBF_ECUDA, "no CUDA device");
        auto dp = std::make_unique<midbf_dplan>();
        dp->precision = base == MIDBF_FP64 ? MIDBF_FP64 : MIDBF_FP32;
        dp->tc_mode = base == MIDBF_BF16 ? ((precision & MIDBF_REFINE) ? 2 : 1) : 0;
        if (dp->tc_mode && s_mode != MIDBF_S_ONTHEFLY) fail(MIDBF_EINVAL, "the tensor-core modes generate the middle factor on the fly");
        dp->s_mode = s_mode;
        CK(cudaGetDevice(&dp->device));
        dp->noalloc_scratch = noalloc_lookup(dp->noalloc_err);   // for midbf_apply_noalloc
        dp->nx = pl.nx();
        dp->nw = pl.nw();
        if (cudaMalloc(&dp->d_status, sizeof(int)) != cudaSuccess) fail(MIDBF_ENOMEM, "cudaMalloc of the status word failed");
        CK(cudaMemset(dp->d_status, 0, sizeof(int)));
        if (consume) plw.released = true;   // from here on, whatever happens below
        const bool overlap = (flags & MIDBF_DPLAN_OVERLAP) != 0;
        if (dp->precision == MIDBF_FP32) make_stages<float>(dp.get(), pl, dp->st32, consume, overlap);
        else make_stages<double>(dp.get(), pl, dp->st64, consume, overlap);
        if (dp->chunks_built > 1) {
            // the side stream and events of the overlap (no device memory).  The side
            // stream gets the highest priority: its chunk k becomes ready while chunk
            // k + 1 of the first stage is queued, and its CTAs must then take the SM slots
            // that free up instead of waiting behind the whole next chunk.
            int prio_lo = 0, prio_hi = 0;
            CK(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
            CK(cudaStreamCreateWithPriority(&dp->side, cudaStreamNonBlocking, prio_hi));
            CK(cudaEventCreateWithFlags(&dp->ev_fork, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&dp->ev_join, cudaEventDisableTiming));
            for (int k = 0; k < dp->chunks_built; ++k) CK(cudaEventCreateWithFlags(&dp->ev_ck[k], cudaEventDisableTiming));
        }
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

int midbf_wait_selftest(midbf_dplan* dp, int ctas, void* stream) {
    try {
        if (!dp || ctas <= 0 || ctas > 1024) fail(MIDBF_EINVAL, "bad argument");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (capturing(s)) fail(MIDBF_EINVAL, "the self-test cannot be recorded into a graph");
        midbf_gpu::launch_wait_selftest(dp->d_status, ctas, s);
        return MIDBF_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    }
}

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
    // the overlapped pair runs each of its two stages as one launch per chunk
    const bool pipe = dp->precision == MIDBF_FP32 ? overlapped(dp, dp->st32, nrhs, false)
                                                  : overlapped(dp, dp->st64, nrhs, false);
    if (pipe) n += 2 * (dp->chunks - 1);
    *launches = n;
    return MIDBF_OK;
}

int midbf_dplan_set_overlap(midbf_dplan* dp, int enable) {
    if (!dp) {
        set_last_error("midbf_dplan_set_overlap: null plan");
        return MIDBF_EINVAL;
    }
    dp->chunks = enable ? dp->chunks_built : 0;
    return MIDBF_OK;
}

int midbf_dplan_overlap(const midbf_dplan* dp, int* chunks) {
    if (!dp || !chunks) {
        set_last_error("midbf_dplan_overlap: null argument");
        return MIDBF_EINVAL;
    }
    *chunks = dp->chunks;
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
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        check_apply_args(dp, adjoint, in, ldin, out, ldout, nrhs, s);
        size_t need = 0;
        midbf_workspace_size(dp, nrhs, &need);
        if (!workspace || workspace_bytes < need) fail(MIDBF_EINVAL, "workspace too small: need " + std::to_string(need) + " bytes");
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
            if (dp->s_mode == MIDBF_S_ONTHEFLY_DF) fail(MIDBF_EINVAL, "the batched apply does not take accurate-phase plans");
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

namespace midbf_gpu {
// Device address of the scratch array in the current device's context.  The
// host-side name g_noalloc_scratch is only a stand-in, never a device address,
// so midbf_dplan_create_ex looks the address up with the plan's device
// current and keeps it in the plan: a plan, like its device memory, lives in
// one context, and the lookup (which may load the module) happens at set-up,
// before any stream capture.
void* noalloc_lookup(std::string& err) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
        err = std::string("cudaGetSymbolAddress of the scratch array failed: ") + cudaGetErrorString(e);
        return nullptr;
    }
    return ptr;
}
}  // namespace midbf_gpu

extern "C" {

size_t midbf_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }

int midbf_apply_noalloc(const midbf_dplan* dp, int adjoint, const void* in, int64_t ldin, void* out, int64_t ldout,
                        int nrhs, void* stream) {
    try {
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        check_apply_args(dp, adjoint, in, ldin, out, ldout, nrhs, s);
        size_t need = 0;
        midbf_workspace_size(dp, nrhs, &need);
        if (need > kNoAllocScratchBytes)
            fail(MIDBF_EINVAL, "midbf_apply_noalloc: this plan needs " + std::to_string(need) +
                                   " bytes of scratch for " + std::to_string(nrhs) +
                                   " right-hand sides, more than the built-in " +
                                   std::to_string(kNoAllocScratchBytes) +
                                   " bytes; use midbf_apply with a caller workspace or fewer right-hand sides");
        int dev = 0;
        CK(cudaGetDevice(&dev));
        if (dev != dp->device) fail(MIDBF_EINVAL, "the current device is not the device of this plan");
        if (!dp->noalloc_scratch) fail(MIDBF_ECUDA, dp->noalloc_err);
        if (dp->precision == MIDBF_FP32)
            run<float>(dp, dp->st32, adjoint != 0, in, ldin, out, ldout, nrhs, s, dp->noalloc_scratch);
        else run<double>(dp, dp->st64, adjoint != 0, in, ldin, out, ldout, nrhs, s, dp->noalloc_scratch);
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
