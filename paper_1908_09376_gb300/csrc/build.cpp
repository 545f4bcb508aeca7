// MIDBF construction on the host in FP64 (Sec. 3.1-3.6).
//
// Trees T_X, T_Omega of equal depth L = round(log_b(N/n0)) over the domain
// cubes (Sec. 3.1; empty nodes discarded, Sec. 3.6), Z-order child digit
// t = 2 bit(x1) + bit(x2) (3D: 4 bit(x1) + 2 bit(x2) + bit(x3)) as in Fig. 6.
//
// The recursion is the paper's recursive MSCS (Sec. 3.5) preceded, when L is
// odd, by one LRCS (Sec. 3.3) - the paper assumes even L.  Both are steps
// s = 1..ceil(L/2) with a shift delta (1 for even L, 0 for odd L): step s
// pairs X nodes a at level L-s+1 with Omega nodes Q at level s-1+delta for
// the row IDs, then Omega nodes beta at level L-s+1 with X nodes P at level
// s-1+delta for the column IDs against the new row skeletons (the order of
// the LRCS: rID of K(r_i,:), then cID of K(r_hat, c_j)).  Rows of the row ID
// of (a, Q) are the children's skeletons w.r.t. the parent of Q (the points of
// a at step 1); its columns are sampled from the column skeletons of the
// Omega nodes below Q found at the previous step (the points of Q at step 1).
//
// Every ID is a linear-scaling ID (Sec. 3.2) of a Mock-Chebyshev sample of
// the opposite side: a tensor Chebyshev grid over the candidates' bounding
// box snapped to the nearest candidate, topped up with seeded random
// candidates; the sample is regrown until it holds t * k_eps rows ("gradually
// increased if not large enough").  The first ID of each kind in a step runs
// alone and sets the starting sample size of the others, so the result does
// not depend on the thread schedule.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <atomic>
#include <functional>
#include <map>
#include <mutex>
#include <random>
#include <thread>
#include <unordered_map>

#include "internal.hpp"

namespace midbf {

namespace {

struct Node {
    int64_t z;
    int64_t begin, end;  // range in the tree's sorted point order
};

struct Tree {
    int d = 2, b = 4, L = 0;
    std::vector<int64_t> order;                 // points sorted by Morton code, then index
    std::vector<std::vector<Node>> levels;      // nodes per level, ascending z
    std::vector<std::unordered_map<int64_t, int>> index;  // z -> node position per level

    void build(const std::vector<double>& P, int64_t n, int d_, int L_, const double* box) {
        d = d_;
        b = 1 << d;
        L = L_;
        std::vector<double> lo(d);
        double side;
        if (box) {
            for (int k = 0; k < d; ++k) lo[k] = box[k];
            side = box[d];
        } else {
            std::vector<double> hi(d);
            for (int k = 0; k < d; ++k) lo[k] = hi[k] = P[k];
            for (int64_t i = 0; i < n; ++i)
                for (int k = 0; k < d; ++k) {
                    lo[k] = std::min(lo[k], P[i * d + k]);
                    hi[k] = std::max(hi[k], P[i * d + k]);
                }
            side = 0.0;
            for (int k = 0; k < d; ++k) side = std::max(side, hi[k] - lo[k]);
            if (side <= 0.0) side = 1.0;
        }
        std::vector<int64_t> code(n);
        const int64_t cells = (int64_t)1 << L;
        for (int64_t i = 0; i < n; ++i) {
            int64_t c[3];
            for (int k = 0; k < d; ++k) {
                double v = std::floor((P[i * d + k] - lo[k]) / side * (double)cells);
                int64_t cv = (int64_t)v;
                c[k] = std::min<int64_t>(std::max<int64_t>(cv, 0), cells - 1);
            }
            int64_t z = 0;
            for (int bit = L - 1; bit >= 0; --bit)
                for (int k = 0; k < d; ++k) z = (z << 1) | ((c[k] >> bit) & 1);
            code[i] = z;
        }
        order.resize(n);
        for (int64_t i = 0; i < n; ++i) order[i] = i;
        std::sort(order.begin(), order.end(), [&](int64_t a, int64_t c) {
            return code[a] != code[c] ? code[a] < code[c] : a < c;
        });
        levels.assign(L + 1, {});
        index.assign(L + 1, {});
        for (int lev = 0; lev <= L; ++lev) {
            const int sh = d * (L - lev);
            std::vector<Node>& nodes = levels[lev];
            for (int64_t p = 0; p < n; ++p) {
                int64_t z = code[order[p]] >> sh;
                if (nodes.empty() || nodes.back().z != z) nodes.push_back({z, p, p + 1});
                else nodes.back().end = p + 1;
            }
            for (size_t q = 0; q < nodes.size(); ++q) index[lev][nodes[q].z] = (int)q;
        }
    }
    int find(int lev, int64_t z) const {
        auto it = index[lev].find(z);
        return it == index[lev].end() ? -1 : it->second;
    }
    // positions (into levels[lev+1]) of the children of node q at level lev
    std::vector<int> children(int lev, int q) const {
        std::vector<int> out;
        const int64_t z = levels[lev][q].z;
        for (int t = 0; t < b; ++t) {
            int c = find(lev + 1, z * b + t);
            if (c >= 0) out.push_back(c);
        }
        return out;
    }
    // positions (into levels[down]) of the descendants of node q at level lev
    std::vector<int> descendants(int lev, int q, int down) const {
        std::vector<int> out;
        const int sh = d * (down - lev);
        const int64_t lo = levels[lev][q].z << sh, hi = (levels[lev][q].z + 1) << sh;
        const std::vector<Node>& nd = levels[down];
        auto it = std::lower_bound(nd.begin(), nd.end(), lo, [](const Node& a, int64_t v) { return a.z < v; });
        for (; it != nd.end() && it->z < hi; ++it) out.push_back((int)(it - nd.begin()));
        return out;
    }
    int ancestor(int lev, int q, int up) const { return find(up, levels[lev][q].z >> (d * (lev - up))); }
    std::vector<int64_t> points(int lev, int q) const {
        const Node& nd = levels[lev][q];
        return std::vector<int64_t>(order.begin() + nd.begin, order.begin() + nd.end);
    }
};

// Nearest-candidate queries on a uniform grid hash (Mock-Chebyshev snapping).
struct GridNN {
    int d = 2;
    std::vector<double> lo, inv;
    std::vector<int> dims;
    std::vector<int> cell_start, items;
    const std::vector<double>* coords = nullptr;  // candidate coordinates (ncand x d)
    int64_t ncand = 0;

    void build(const std::vector<double>& c, int d_) {
        d = d_;
        coords = &c;
        ncand = (int64_t)c.size() / d;
        lo.assign(d, 0.0);
        std::vector<double> hi(d);
        for (int k = 0; k < d; ++k) lo[k] = hi[k] = c[k];
        for (int64_t i = 0; i < ncand; ++i)
            for (int k = 0; k < d; ++k) {
                lo[k] = std::min(lo[k], c[i * d + k]);
                hi[k] = std::max(hi[k], c[i * d + k]);
            }
        const double per = std::pow((double)std::max<int64_t>(ncand, 1) / 2.0, 1.0 / d);
        const int g = std::max(1, std::min(1024, (int)std::ceil(per)));
        dims.assign(d, g);
        inv.assign(d, 0.0);
        for (int k = 0; k < d; ++k) inv[k] = hi[k] > lo[k] ? g / (hi[k] - lo[k]) : 0.0;
        size_t ncell = 1;
        for (int k = 0; k < d; ++k) ncell *= (size_t)g;
        std::vector<int> cnt(ncell + 1, 0);
        std::vector<int> cid(ncand);
        for (int64_t i = 0; i < ncand; ++i) {
            cid[i] = cell_of(&c[i * d]);
            cnt[cid[i] + 1]++;
        }
        for (size_t q = 0; q < ncell; ++q) cnt[q + 1] += cnt[q];
        cell_start = cnt;
        items.assign(ncand, 0);
        std::vector<int> fill(cnt.begin(), cnt.end() - 1);
        for (int64_t i = 0; i < ncand; ++i) items[fill[cid[i]]++] = (int)i;
    }
    int coord_cell(double v, int k) const {
        int c = (int)std::floor((v - lo[k]) * inv[k]);
        return std::min(std::max(c, 0), dims[k] - 1);
    }
    int cell_of(const double* x) const {
        int id = 0;
        for (int k = 0; k < d; ++k) id = id * dims[k] + coord_cell(x[k], k);
        return id;
    }
    int64_t nearest(const double* x) const {
        int c[3];
        for (int k = 0; k < d; ++k) c[k] = coord_cell(x[k], k);
        double best = 1e300;
        int64_t bi = -1;
        const int g = dims[0];
        for (int rad = 0; rad <= g; ++rad) {
            // visit the shell of cells at Chebyshev distance rad
            int lo3[3], hi3[3];
            for (int k = 0; k < 3; ++k) {
                lo3[k] = k < d ? std::max(0, c[k] - rad) : 0;
                hi3[k] = k < d ? std::min(dims[k] - 1, c[k] + rad) : 0;
            }
            for (int i0 = lo3[0]; i0 <= hi3[0]; ++i0)
                for (int i1 = lo3[1]; i1 <= hi3[1]; ++i1)
                    for (int i2 = lo3[2]; i2 <= hi3[2]; ++i2) {
                        int ii[3] = {i0, i1, i2};
                        int cheb = 0;
                        for (int k = 0; k < d; ++k) cheb = std::max(cheb, std::abs(ii[k] - c[k]));
                        if (cheb != rad) continue;
                        int id = 0;
                        for (int k = 0; k < d; ++k) id = id * dims[k] + ii[k];
                        for (int q = cell_start[id]; q < cell_start[id + 1]; ++q) {
                            const int64_t p = items[q];
                            double dd = 0.0;
                            for (int k = 0; k < d; ++k) {
                                double t = (*coords)[p * d + k] - x[k];
                                dd += t * t;
                            }
                            if (dd < best || (dd == best && p < bi)) {
                                best = dd;
                                bi = p;
                            }
                        }
                    }
            if (bi >= 0) {
                // a point in a farther shell can still be closer than this one
                double cellw = 1e300;
                for (int k = 0; k < d; ++k)
                    if (inv[k] > 0) cellw = std::min(cellw, 1.0 / inv[k]);
                if (cellw >= 1e299 || best <= (rad * cellw) * (rad * cellw)) return bi;
            }
        }
        return bi;
    }
};

uint64_t mix(uint64_t a, uint64_t b) {
    uint64_t z = a + 0x9e3779b97f4a7c15ULL * (b + 1);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// Mock-Chebyshev sample of `count` candidates (positions into the candidate list).
std::vector<int64_t> mock_chebyshev(const std::vector<double>& cc, const GridNN& nn, int d, int64_t count,
                                    uint64_t seed) {
    const int64_t ncand = (int64_t)cc.size() / d;
    std::vector<int64_t> out;
    if (ncand <= count) {
        out.resize(ncand);
        for (int64_t i = 0; i < ncand; ++i) out[i] = i;
        return out;
    }
    int p = (int)std::ceil(std::pow((double)count, 1.0 / d) - 1e-12);
    std::vector<double> lo(d), hi(d);
    for (int k = 0; k < d; ++k) lo[k] = hi[k] = cc[k];
    for (int64_t i = 0; i < ncand; ++i)
        for (int k = 0; k < d; ++k) {
            lo[k] = std::min(lo[k], cc[i * d + k]);
            hi[k] = std::max(hi[k], cc[i * d + k]);
        }
    std::vector<double> t(p);
    for (int i = 0; i < p; ++i) t[i] = (1.0 - std::cos((2.0 * i + 1.0) * M_PI / (2.0 * p))) / 2.0;
    std::vector<uint8_t> taken(ncand, 0);
    int64_t total = 1;
    for (int k = 0; k < d; ++k) total *= p;
    double x[3];
    for (int64_t q = 0; q < total; ++q) {
        int64_t r = q;
        for (int k = d - 1; k >= 0; --k) {
            x[k] = lo[k] + (hi[k] - lo[k]) * t[r % p];
            r /= p;
        }
        int64_t c = nn.nearest(x);
        if (c >= 0 && !taken[c]) {
            taken[c] = 1;
            out.push_back(c);
        }
    }
    if ((int64_t)out.size() < count) {
        std::mt19937_64 rng(seed);
        std::vector<int64_t> rest;
        rest.reserve(ncand - out.size());
        for (int64_t i = 0; i < ncand; ++i)
            if (!taken[i]) rest.push_back(i);
        const int64_t need = count - (int64_t)out.size();
        for (int64_t i = 0; i < need; ++i) {  // partial Fisher-Yates
            std::uniform_int_distribution<int64_t> U(i, (int64_t)rest.size() - 1);
            std::swap(rest[i], rest[U(rng)]);
            out.push_back(rest[i]);
        }
    }
    std::sort(out.begin(), out.end());
    return out;
}

// Candidate set shared by all IDs of one key: point indices, coordinates, NN index.
struct Cand {
    std::vector<int64_t> pts;
    std::vector<double> xy;
    GridNN nn;
};

void parallel_for(int64_t n, int nthreads, const std::function<void(int64_t)>& f) {
    if (n <= 0) return;
    if (nthreads <= 1 || n == 1) {
        for (int64_t i = 0; i < n; ++i) f(i);
        return;
    }
    std::atomic<int64_t> next(0);
    std::mutex em;
    std::string err;
    int ecode = 0;
    std::vector<std::thread> th;
    for (int w = 0; w < std::min<int64_t>(nthreads, n); ++w)
        th.emplace_back([&]() {
            for (;;) {
                int64_t i = next.fetch_add(1);
                if (i >= n) break;
                try {
                    f(i);
                } catch (const Error& e) {
                    std::lock_guard<std::mutex> g(em);
                    if (!ecode) { ecode = e.code; err = e.what(); }
                    next = n;
                } catch (const std::exception& e) {
                    std::lock_guard<std::mutex> g(em);
                    if (!ecode) { ecode = MIDBF_EINTERNAL; err = e.what(); }
                    next = n;
                }
            }
        });
    for (auto& t : th) t.join();
    if (ecode) fail(ecode, err);
}

struct IdOut {
    Sub sub;
    std::vector<int64_t> skel_pts;  // point indices of the skeleton
};

}  // namespace

// Construction timings on stderr when the environment sets MIDBF_BUILD_LOG:
// wall time per phase, and the thread-seconds spent filling kernel samples
// and in the pivoted QRs of the host IDs.
struct BuildLog {
    bool on = std::getenv("MIDBF_BUILD_LOG") != nullptr;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now(), t = t0;
    std::atomic<int64_t> ns_fill{0}, ns_qr{0}, entries{0};
    template <class F>
    auto timed(std::atomic<int64_t>& acc, F&& f) {
        if (!on) return f();
        const auto a = std::chrono::steady_clock::now();
        struct Add {
            std::atomic<int64_t>& acc;
            std::chrono::steady_clock::time_point a;
            ~Add() {
                acc += std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - a).count();
            }
        } add{acc, a};
        return f();
    }
    void totals() {
        if (!on) return;
        std::fprintf(stderr, "[midbf build] host IDs: %.2f thread-s filling %.3g kernel samples, %.2f thread-s in QRs\n",
                     ns_fill.load() * 1e-9, (double)entries.load(), ns_qr.load() * 1e-9);
    }
    void mark(const std::string& what) {
        if (!on) return;
        const auto now = std::chrono::steady_clock::now();
        std::fprintf(stderr, "[midbf build %8.2fs +%7.2fs] %s\n",
                     std::chrono::duration<double>(now - t0).count(), std::chrono::duration<double>(now - t).count(),
                     what.c_str());
        t = now;
    }
};

std::unique_ptr<Plan> build_plan(const Phase& ph, const midbf_params& prm) {
    phase_check(ph);
    BuildLog blog;
    const int d = ph.d, b = 1 << d;
    const int64_t nmax = std::max(ph.nx, ph.nw);
    int L = 0;
    if (nmax > prm.n0) L = std::max(0, (int)std::lround(std::log((double)nmax / prm.n0) / std::log((double)b)));
    if (L > 20) fail(MIDBF_EINVAL, "tree too deep");
    const int nthreads = prm.nthreads > 0 ? prm.nthreads : std::max(1u, std::thread::hardware_concurrency());
    auto pl = std::make_unique<Plan>();
    pl->d = d;
    pl->L = L;
    pl->tol = prm.tol;
    pl->phase = ph;
    if (L == 0) {
        pl->delta = 1;
        pl->nsteps = 0;
        Stage st;
        st.kind = KIND_S;
        st.in_space = -1;
        st.out_user = 1;
        st.out_len = ph.nx;
        Block bk;
        for (int64_t j = 0; j < ph.nw; ++j) bk.in_idx.push_back(j), bk.widx.push_back(j);
        for (int64_t i = 0; i < ph.nx; ++i) bk.out_idx.push_back(i), bk.xidx.push_back(i);
        st.blocks.push_back(std::move(bk));
        pl->stages.push_back(std::move(st));
        return pl;
    }
    const int delta = L % 2 == 0 ? 1 : 0;
    const int nsteps = (L + 1) / 2;
    pl->delta = delta;
    pl->nsteps = nsteps;
    Tree TX, TW;
    TX.build(ph.X, ph.nx, d, L, prm.use_box ? prm.boxX : nullptr);
    TW.build(ph.W, ph.nw, d, L, prm.use_box ? prm.boxW : nullptr);

    // factors per step: index [ia * nq + iq]
    std::vector<std::vector<IdOut>> Uf(nsteps + 1), Vf(nsteps + 1);
    std::vector<int> nq_of(nsteps + 1), np_of(nsteps + 1);
    int64_t kest_r = prm.kest, kest_c = prm.kest;

    auto kernel_fill = [&](std::vector<cplx>& M, const std::vector<int64_t>& srows, bool srows_are_x,
                           const std::vector<int64_t>& cols) {
        // M (|srows| x |cols|, column-major): entry (s, c) = K(x, w) with the
        // sample on the opposite side of the decomposed index set.
        const size_t ms = srows.size();
        M.resize(ms * cols.size());
        if (srows_are_x) ph.kernel_block(srows.data(), ms, cols.data(), cols.size(), M.data(), 1, ms);
        else ph.kernel_block(cols.data(), cols.size(), srows.data(), ms, M.data(), ms, 1);
    };

    // Column ID of the index set `cols` (points on side `cols_x`) from a sample
    // of the candidate set on the other side.
    auto sampled_id = [&](const std::vector<int64_t>& cols, bool cols_x, const Cand& cand, int64_t ns0,
                          uint64_t seed) {
        const int64_t ncand = (int64_t)cand.pts.size();
        int64_t ns = std::max<int64_t>(1, ns0);
        std::vector<cplx> M;
        for (;;) {
            std::vector<int64_t> pos = mock_chebyshev(cand.xy, cand.nn, d, ns, seed);
            std::vector<int64_t> srows(pos.size());
            for (size_t i = 0; i < pos.size(); ++i) srows[i] = cand.pts[pos[i]];
            blog.timed(blog.ns_fill, [&] { kernel_fill(M, srows, !cols_x, cols); });
            blog.entries += (int64_t)(srows.size() * cols.size());
            IdResult r = blog.timed(blog.ns_qr, [&] {
                return column_id(M, (int)srows.size(), (int)cols.size(), prm.tol, prm.kmax);
            });
            const int64_t k = (int64_t)r.skel.size();
            const int64_t need = (int64_t)std::ceil(prm.t * (double)k);
            if ((int64_t)pos.size() >= ncand || (int64_t)pos.size() >= need) {
                IdOut o;
                o.sub.k = (int32_t)k;
                o.sub.m = (int32_t)cols.size();
                o.sub.skel = r.skel;
                o.sub.red = r.red;
                o.sub.T = std::move(r.T);
                if (prm.store_fp32) o.sub.to_fp32();
                o.skel_pts.resize(k);
                for (int64_t i = 0; i < k; ++i) o.skel_pts[i] = cols[r.skel[i]];
                return o;
            }
            ns = std::min(ncand, need);
        }
    };

    auto make_cand = [&](std::vector<int64_t> pts, bool on_x) {
        auto c = std::make_unique<Cand>();
        c->pts = std::move(pts);
        const std::vector<double>& P = on_x ? ph.X : ph.W;
        c->xy.resize(c->pts.size() * d);
        for (size_t i = 0; i < c->pts.size(); ++i)
            for (int k = 0; k < d; ++k) c->xy[i * d + k] = P[c->pts[i] * d + k];
        c->nn.build(c->xy, d);
        return c;
    };

    std::unique_ptr<GpuIdContext, void (*)(GpuIdContext*)> gctx(nullptr, [](GpuIdContext*) {});
    if (prm.device_ids) gctx = gpu_id_context(ph);

    // All IDs of one kind in one step.  The first runs alone and sets the
    // starting sample size of the others (t times its rank), so the result
    // does not depend on the thread schedule or on the device path.
    auto run_phase = [&](int64_t ntot, bool cols_x, uint64_t tag, int64_t& kest, std::vector<IdOut>& outv,
                         const std::function<std::vector<int64_t>(int64_t)>& cols_fn,
                         const std::function<const Cand&(int64_t)>& cand_fn) {
        auto seed_of = [&](int64_t e) { return mix(prm.seed, tag * 1000003 + (uint64_t)e); };
        if (!gctx) {
            outv[0] = sampled_id(cols_fn(0), cols_x, cand_fn(0), (int64_t)std::ceil(prm.t * kest), seed_of(0));
            kest = outv[0].sub.k;
            const int64_t ns0 = (int64_t)std::ceil(prm.t * kest);
            parallel_for(ntot - 1, nthreads, [&](int64_t e) {
                outv[e + 1] = sampled_id(cols_fn(e + 1), cols_x, cand_fn(e + 1), ns0, seed_of(e + 1));
            });
            return;
        }
        // device path: the same sampling and regrowth rule, decompositions batched on the GPU
        std::vector<std::vector<int64_t>> colsv(ntot);
        parallel_for(ntot, nthreads, [&](int64_t e) { colsv[e] = cols_fn(e); });
        std::vector<int64_t> ns(ntot, 0);
        std::vector<char> done(ntot, 0);
        auto solve = [&](const std::vector<int64_t>& which) {
            std::vector<IdRequest> req(which.size());
            parallel_for((int64_t)which.size(), nthreads, [&](int64_t q) {
                const int64_t e = which[q];
                const Cand& cand = cand_fn(e);
                std::vector<int64_t> pos = mock_chebyshev(cand.xy, cand.nn, d, ns[e], seed_of(e));
                req[q].cols = &colsv[e];
                req[q].cols_x = cols_x;
                req[q].samples.resize(pos.size());
                for (size_t i = 0; i < pos.size(); ++i) req[q].samples[i] = cand.pts[pos[i]];
            });
            std::vector<IdReply> rep;
            gpu_id_batch(*gctx, req, prm.tol, prm.kmax, rep, prm.store_fp32 != 0);
            for (size_t q = 0; q < which.size(); ++q) {
                const int64_t e = which[q];
                const int64_t ncand = (int64_t)cand_fn(e).pts.size();
                const int64_t got = (int64_t)req[q].samples.size();
                const int64_t k = rep[q].k;
                const int64_t need = (int64_t)std::ceil(prm.t * (double)k);
                if (got >= ncand || got >= need) {
                    IdOut& o = outv[e];
                    o.sub.k = (int32_t)k;
                    o.sub.m = (int32_t)colsv[e].size();
                    o.sub.skel = std::move(rep[q].skel);
                    o.sub.red = std::move(rep[q].red);
                    o.sub.T = std::move(rep[q].T);
                    o.sub.Tf = std::move(rep[q].Tf);
                    o.skel_pts.resize(k);
                    for (int64_t i = 0; i < k; ++i) o.skel_pts[i] = colsv[e][o.sub.skel[i]];
                    done[e] = 1;
                } else {
                    ns[e] = std::min(ncand, need);
                }
            }
        };
        ns[0] = std::max<int64_t>(1, (int64_t)std::ceil(prm.t * kest));
        while (!done[0]) solve({0});
        kest = outv[0].sub.k;
        for (int64_t e = 1; e < ntot; ++e) ns[e] = std::max<int64_t>(1, (int64_t)std::ceil(prm.t * kest));
        for (;;) {
            std::vector<int64_t> which;
            for (int64_t e = 1; e < ntot; ++e)
                if (!done[e]) which.push_back(e);
            if (which.empty()) break;
            solve(which);
        }
    };

    for (int s = 1; s <= nsteps; ++s) {
        const int la = L - s + 1, lq = s - 1 + delta, lp = s - 2 + delta;
        const int na_x = (int)TX.levels[la].size(), nq_w = (int)TW.levels[lq].size();
        const int nb_w = (int)TW.levels[la].size(), np_x = (int)TX.levels[lq].size();
        nq_of[s] = nq_w;
        np_of[s] = np_x;
        blog.mark("step " + std::to_string(s) + " start");
        // ---- row IDs (a, Q) ----
        // candidate column sets keyed by (Q, ancestor of a at level lp)
        std::map<std::pair<int, int>, std::unique_ptr<Cand>> ccand;
        std::vector<std::pair<int, int>> keys(na_x * (size_t)nq_w);
        for (int iq = 0; iq < nq_w; ++iq)
            for (int ia = 0; ia < na_x; ++ia) {
                const int pa = (s == 1 || lp < 0) ? -1 : TX.ancestor(la, ia, lp);
                keys[(size_t)ia * nq_w + iq] = {iq, pa};
                ccand.emplace(std::make_pair(iq, pa), nullptr);
            }
        {
            std::vector<std::pair<int, int>> klist;
            for (auto& kv : ccand) klist.push_back(kv.first);
            std::vector<std::unique_ptr<Cand>> made(klist.size());
            parallel_for((int64_t)klist.size(), nthreads, [&](int64_t q) {
                const int iq = klist[q].first, pa = klist[q].second;
                std::vector<int64_t> pts;
                if (s == 1) {
                    pts = TW.points(lq, iq);
                } else {
                    for (int bb : TW.descendants(lq, iq, la + 1)) {
                        const IdOut& o = Vf[s - 1][(size_t)bb * np_of[s - 1] + pa];
                        pts.insert(pts.end(), o.skel_pts.begin(), o.skel_pts.end());
                    }
                }
                made[q] = make_cand(std::move(pts), false);
            });
            for (size_t q = 0; q < klist.size(); ++q) ccand[klist[q]] = std::move(made[q]);
        }
        Uf[s].resize(na_x * (size_t)nq_w);
        auto rows_of = [&](int ia, int iq) {
            if (s == 1) return TX.points(la, ia);
            const int qp = TW.ancestor(lq, iq, lp);
            std::vector<int64_t> rows;
            for (int c : TX.children(la, ia)) {
                const IdOut& o = Uf[s - 1][(size_t)c * nq_of[s - 1] + qp];
                rows.insert(rows.end(), o.skel_pts.begin(), o.skel_pts.end());
            }
            return rows;
        };
        blog.mark("step " + std::to_string(s) + " row candidates");
        run_phase((int64_t)na_x * nq_w, true, (uint64_t)(s * 4 + 1), kest_r, Uf[s],
                  [&](int64_t e) { return rows_of((int)(e / nq_w), (int)(e % nq_w)); },
                  [&](int64_t e) -> const Cand& { return *ccand[keys[e]]; });
        blog.mark("step " + std::to_string(s) + " row IDs (" + std::to_string((int64_t)na_x * nq_w) + ")");
        ccand.clear();
        // ---- column IDs (beta, P) ----
        std::vector<std::unique_ptr<Cand>> rcand((size_t)np_x * nq_w);
        parallel_for((int64_t)np_x * nq_w, nthreads, [&](int64_t q) {
            const int ip = (int)(q / nq_w), iq = (int)(q % nq_w);
            std::vector<int64_t> pts;
            for (int a : TX.descendants(lq, ip, la)) {
                const IdOut& o = Uf[s][(size_t)a * nq_w + iq];
                pts.insert(pts.end(), o.skel_pts.begin(), o.skel_pts.end());
            }
            rcand[q] = make_cand(std::move(pts), true);
        });
        Vf[s].resize(nb_w * (size_t)np_x);
        auto cols_of = [&](int ib, int ip) {
            if (s == 1) return TW.points(la, ib);
            const int pp = TX.ancestor(lq, ip, lp);
            std::vector<int64_t> cols;
            for (int c : TW.children(la, ib)) {
                const IdOut& o = Vf[s - 1][(size_t)c * np_of[s - 1] + pp];
                cols.insert(cols.end(), o.skel_pts.begin(), o.skel_pts.end());
            }
            return cols;
        };
        blog.mark("step " + std::to_string(s) + " column candidates");
        run_phase((int64_t)nb_w * np_x, false, (uint64_t)(s * 4 + 2), kest_c, Vf[s],
                  [&](int64_t e) { return cols_of((int)(e / np_x), (int)(e % np_x)); },
                  [&](int64_t e) -> const Cand& {
                      const int ib = (int)(e / np_x), ip = (int)(e % np_x);
                      return *rcand[(size_t)ip * nq_w + TW.ancestor(la, ib, lq)];
                  });
    }

    blog.mark("IDs done");
    blog.totals();
    // ---- assemble the stages in forward order ----
    // ypos[(ib, ip)] = (offset, k) of y(beta, P_k) in the previous V stage output
    std::vector<std::pair<int64_t, int>> ypos, zpos;
    for (int s = 1; s <= nsteps; ++s) {
        const int la = L - s + 1, lq = s - 1 + delta, lp = s - 2 + delta;
        const int np_x = np_of[s];
        Stage st;
        st.kind = KIND_V;
        st.in_space = s == 1 ? -1 : (int)pl->stages.size() - 1;
        std::vector<std::pair<int64_t, int>> ynew((size_t)TW.levels[la].size() * np_x, {-1, 0});
        int64_t off = 0;
        const int nparents = lp >= 0 ? (int)TX.levels[lp].size() : 1;
        for (int pp = 0; pp < nparents; ++pp) {
            std::vector<int> kids = lp >= 0 ? TX.children(lp, pp) : std::vector<int>{0};
            for (int ib = 0; ib < (int)TW.levels[la].size(); ++ib) {
                Block bk;
                if (s == 1) {
                    bk.in_idx = TW.points(la, ib);
                } else {
                    for (int c : TW.children(la, ib)) {
                        auto pr = ypos[(size_t)c * np_of[s - 1] + pp];
                        for (int q = 0; q < pr.second; ++q) bk.in_idx.push_back(pr.first + q);
                    }
                }
                for (int pk : kids) {
                    IdOut& o = Vf[s][(size_t)ib * np_x + pk];
                    ynew[(size_t)ib * np_x + pk] = {off, o.sub.k};
                    for (int q = 0; q < o.sub.k; ++q) bk.out_idx.push_back(off + q);
                    off += o.sub.k;
                    bk.subs.push_back(std::move(o.sub));
                }
                st.blocks.push_back(std::move(bk));
            }
        }
        st.out_len = off;
        pl->stages.push_back(std::move(st));
        ypos.swap(ynew);
    }
    {
        const int lS = nsteps - 1 + delta;
        const int np_x = np_of[nsteps], nq_w = nq_of[nsteps];
        Stage st;
        st.kind = KIND_S;
        st.in_space = (int)pl->stages.size() - 1;
        zpos.assign((size_t)TX.levels[lS + 1].size() * nq_w, {-1, 0});
        int64_t off = 0;
        for (int P = 0; P < (int)TX.levels[lS].size(); ++P)
            for (int Q = 0; Q < (int)TW.levels[lS].size(); ++Q) {
                Block bk;
                for (int bb : TW.children(lS, Q)) {
                    auto pr = ypos[(size_t)bb * np_x + P];
                    for (int q = 0; q < pr.second; ++q) bk.in_idx.push_back(pr.first + q);
                    const IdOut& o = Vf[nsteps][(size_t)bb * np_x + P];
                    bk.widx.insert(bk.widx.end(), o.skel_pts.begin(), o.skel_pts.end());
                }
                for (int a : TX.children(lS, P)) {
                    const IdOut& o = Uf[nsteps][(size_t)a * nq_w + Q];
                    zpos[(size_t)a * nq_w + Q] = {off, (int)o.skel_pts.size()};
                    for (size_t q = 0; q < o.skel_pts.size(); ++q) bk.out_idx.push_back(off + (int64_t)q);
                    bk.xidx.insert(bk.xidx.end(), o.skel_pts.begin(), o.skel_pts.end());
                    off += (int64_t)o.skel_pts.size();
                }
                st.blocks.push_back(std::move(bk));
            }
        st.out_len = off;
        pl->stages.push_back(std::move(st));
    }
    for (int s = nsteps; s >= 1; --s) {
        const int la = L - s + 1, lp = s - 2 + delta;
        const int nq_w = nq_of[s];
        Stage st;
        st.kind = KIND_U;
        st.in_space = (int)pl->stages.size() - 1;
        const bool last = s == 1;
        st.out_user = last ? 1 : 0;
        std::vector<std::pair<int64_t, int>> znew;
        if (!last) znew.assign((size_t)TX.levels[la + 1].size() * nq_of[s - 1], {-1, 0});
        int64_t off = 0;
        const int nparents = lp >= 0 ? (int)TW.levels[lp].size() : 1;
        for (int a = 0; a < (int)TX.levels[la].size(); ++a)
            for (int qp = 0; qp < nparents; ++qp) {
                std::vector<int> kids = lp >= 0 ? TW.children(lp, qp) : std::vector<int>{0};
                Block bk;
                for (int ql : kids) {
                    auto pr = zpos[(size_t)a * nq_w + ql];
                    for (int q = 0; q < pr.second; ++q) bk.in_idx.push_back(pr.first + q);
                    bk.subs.push_back(std::move(Uf[s][(size_t)a * nq_w + ql].sub));
                }
                if (last) {
                    bk.out_idx = TX.points(la, a);
                } else {
                    for (int c : TX.children(la, a)) {
                        const IdOut& o = Uf[s - 1][(size_t)c * nq_of[s - 1] + qp];
                        znew[(size_t)c * nq_of[s - 1] + qp] = {off, (int)o.skel_pts.size()};
                        for (size_t q = 0; q < o.skel_pts.size(); ++q) bk.out_idx.push_back(off + (int64_t)q);
                        off += (int64_t)o.skel_pts.size();
                    }
                }
                st.blocks.push_back(std::move(bk));
            }
        st.out_len = last ? ph.nx : off;
        pl->stages.push_back(std::move(st));
        zpos.swap(znew);
    }
    blog.mark("stages assembled");
    plan_validate(*pl);
    blog.mark("validated");
    return pl;
}

}  // namespace midbf
