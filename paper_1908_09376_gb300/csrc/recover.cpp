// Phase recovery from indirect access (Sec. 2.3, Algorithms 1, 4, 5, 6, 7).
//
// Recovery path (Algorithm 5, Def. 3.3): a Euclidean minimum spanning tree of
// the points, then breadth-first order from point 0 with neighbours visited in
// ascending index order.  The paper reaches the MST through the Delaunay
// triangulation (the Delaunay edges contain an EMST); this library computes
// the EMST directly with Boruvka's algorithm on a k-d tree (nearest point of
// another component), which needs no geometric predicates and so stays exact
// on the degenerate (co-circular) uniform grids.  Ties are broken by the
// total order (length, smaller index, larger index), so the tree is unique.
//
// Vector recovery (Algorithm 4): v(ed) = u(ed) - round(u(ed) - v(bg)) along
// the path, |v(ed) - v(bg)| >= tau flags ed; round half away from zero.
// Matrix recovery (Algorithm 6): discontinuities of the root column / row
// split both trees (Partition2); the root row and column of each block, then
// the sampled rows and columns, are recovered along the pieces.  tau starts at
// the caller's value and grows by 1/40 while more than max_disc points are
// flagged, up to 1/2 (Sec. 2.3.4).
// Low-rank factorization (Algorithm 7 with Algorithm 1 restricted to the
// known rows R and columns C): column pivots within C and row pivots within R
// from pivoted QRs of Psi(R, C), orthonormal bases of Psi(:, Pi_col) and
// Psi(Pi_row, :)^T, the core M = Qc(I,:)^+ Psi(I, J) (Qr(J,:)^T)^+ with
// I = R, J = C, its SVD, and V <- V Sigma.
#include <algorithm>
#include <functional>
#include <numeric>
#include <random>

#include "internal.hpp"

namespace midbf {

namespace {

// ---------------------------------------------------------------- k-d tree
struct KdTree {
    int d = 2;
    const double* P = nullptr;
    std::vector<int64_t> idx;
    struct N {
        int64_t lo, hi;      // range in idx
        int left = -1, right = -1;
        double bmin[3], bmax[3];
    };
    std::vector<N> nodes;
    std::vector<int64_t> comp_of_node;  // single component of the subtree, or -1

    void build(const double* pts, int64_t n, int d_) {
        d = d_;
        P = pts;
        idx.resize(n);
        std::iota(idx.begin(), idx.end(), 0);
        nodes.reserve(2 * (n / 8 + 1));
        make(0, n);
    }
    int make(int64_t lo, int64_t hi) {
        N nd;
        nd.lo = lo;
        nd.hi = hi;
        for (int k = 0; k < d; ++k) {
            nd.bmin[k] = 1e300;
            nd.bmax[k] = -1e300;
        }
        for (int64_t q = lo; q < hi; ++q)
            for (int k = 0; k < d; ++k) {
                nd.bmin[k] = std::min(nd.bmin[k], P[idx[q] * d + k]);
                nd.bmax[k] = std::max(nd.bmax[k], P[idx[q] * d + k]);
            }
        const int me = (int)nodes.size();
        nodes.push_back(nd);
        if (hi - lo > 8) {
            int ax = 0;
            for (int k = 1; k < d; ++k)
                if (nd.bmax[k] - nd.bmin[k] > nd.bmax[ax] - nd.bmin[ax]) ax = k;
            const int64_t mid = (lo + hi) / 2;
            std::nth_element(idx.begin() + lo, idx.begin() + mid, idx.begin() + hi, [&](int64_t a, int64_t b) {
                const double va = P[a * d + ax], vb = P[b * d + ax];
                return va != vb ? va < vb : a < b;
            });
            const int l = make(lo, mid);
            const int r = make(mid, hi);
            nodes[me].left = l;
            nodes[me].right = r;
        }
        return me;
    }
    void label(const std::vector<int64_t>& comp) {
        comp_of_node.assign(nodes.size(), -1);
        std::function<int64_t(int)> go = [&](int q) -> int64_t {
            const N& nd = nodes[q];
            int64_t c;
            if (nd.left < 0) {
                c = comp[idx[nd.lo]];
                for (int64_t t = nd.lo + 1; t < nd.hi; ++t)
                    if (comp[idx[t]] != c) {
                        c = -1;
                        break;
                    }
            } else {
                const int64_t a = go(nd.left), b = go(nd.right);
                c = (a >= 0 && a == b) ? a : -1;
            }
            comp_of_node[q] = c;
            return c;
        };
        go(0);
    }
    double box_dist2(const N& nd, const double* x) const {
        double s = 0.0;
        for (int k = 0; k < d; ++k) {
            double t = 0.0;
            if (x[k] < nd.bmin[k]) t = nd.bmin[k] - x[k];
            else if (x[k] > nd.bmax[k]) t = x[k] - nd.bmax[k];
            s += t * t;
        }
        return s;
    }
    // nearest point (by (dist2, index)) whose component differs from c
    void nearest_other(int q, const double* x, int64_t c, const std::vector<int64_t>& comp, double& best,
                       int64_t& bi) const {
        const N& nd = nodes[q];
        if (comp_of_node[q] == c) return;
        if (box_dist2(nd, x) > best) return;
        if (nd.left < 0) {
            for (int64_t t = nd.lo; t < nd.hi; ++t) {
                const int64_t p = idx[t];
                if (comp[p] == c) continue;
                double s = 0.0;
                for (int k = 0; k < d; ++k) {
                    const double u = P[p * d + k] - x[k];
                    s += u * u;
                }
                if (s < best || (s == best && p < bi)) {
                    best = s;
                    bi = p;
                }
            }
            return;
        }
        const double dl = box_dist2(nodes[nd.left], x), dr = box_dist2(nodes[nd.right], x);
        if (dl <= dr) {
            nearest_other(nd.left, x, c, comp, best, bi);
            nearest_other(nd.right, x, c, comp, best, bi);
        } else {
            nearest_other(nd.right, x, c, comp, best, bi);
            nearest_other(nd.left, x, c, comp, best, bi);
        }
    }
};

int64_t uf_find(std::vector<int64_t>& p, int64_t a) {
    while (p[a] != a) {
        p[a] = p[p[a]];
        a = p[a];
    }
    return a;
}

struct Edge {
    double w;
    int64_t a, b;  // a < b
    bool operator<(const Edge& o) const {
        if (w != o.w) return w < o.w;
        if (a != o.a) return a < o.a;
        return b < o.b;
    }
};

// Euclidean MST by Boruvka rounds.
std::vector<std::pair<int64_t, int64_t>> emst(const double* pts, int64_t n, int d) {
    std::vector<std::pair<int64_t, int64_t>> out;
    if (n <= 1) return out;
    KdTree kd;
    kd.build(pts, n, d);
    std::vector<int64_t> parent(n), comp(n);
    std::iota(parent.begin(), parent.end(), 0);
    int64_t ncomp = n;
    while (ncomp > 1) {
        for (int64_t i = 0; i < n; ++i) comp[i] = uf_find(parent, i);
        kd.label(comp);
        std::vector<Edge> best(n, Edge{1e300, -1, -1});
        for (int64_t i = 0; i < n; ++i) {
            double bd = 1e300;
            int64_t bj = -1;
            kd.nearest_other(0, pts + i * d, comp[i], comp, bd, bj);
            if (bj < 0) continue;
            Edge e{bd, std::min(i, bj), std::max(i, bj)};
            Edge& cur = best[comp[i]];
            if (cur.a < 0 || e < cur) cur = e;
        }
        bool merged = false;
        for (int64_t c = 0; c < n; ++c) {
            const Edge& e = best[c];
            if (e.a < 0) continue;
            const int64_t ra = uf_find(parent, e.a), rb = uf_find(parent, e.b);
            if (ra == rb) continue;
            parent[ra] = rb;
            out.push_back({e.a, e.b});
            --ncomp;
            merged = true;
        }
        if (!merged) fail(MIDBF_EINTERNAL, "minimum spanning tree did not progress");
    }
    return out;
}

// Recovery path P ((n-1) pairs parent -> child) by BFS from root 0 (Def. 3.3).
std::vector<std::pair<int64_t, int64_t>> bfs_path(int64_t n, const std::vector<std::pair<int64_t, int64_t>>& edges) {
    std::vector<std::vector<int64_t>> adj(n);
    for (auto& e : edges) {
        adj[e.first].push_back(e.second);
        adj[e.second].push_back(e.first);
    }
    for (auto& a : adj) std::sort(a.begin(), a.end());
    std::vector<uint8_t> seen(n, 0);
    std::vector<int64_t> queue{0};
    seen[0] = 1;
    std::vector<std::pair<int64_t, int64_t>> P;
    P.reserve(n - 1);
    for (size_t h = 0; h < queue.size(); ++h) {
        const int64_t u = queue[h];
        for (int64_t v : adj[u])
            if (!seen[v]) {
                seen[v] = 1;
                P.push_back({u, v});
                queue.push_back(v);
            }
    }
    if ((int64_t)P.size() != n - 1) fail(MIDBF_ERECOVERY, "recovery path does not reach every point");
    return P;
}

double mround(double x) { return x >= 0 ? std::floor(x + 0.5) : -std::floor(-x + 0.5); }

// Algorithm 4 along the edges E; v must hold the start value at the root of E.
void recover_along(const double* u, double* v, const std::vector<std::pair<int64_t, int64_t>>& E) {
    for (auto& e : E) v[e.second] = u[e.second] - mround(u[e.second] - v[e.first]);
}

std::vector<int64_t> detect(const std::vector<double>& u, const std::vector<std::pair<int64_t, int64_t>>& P,
                            double tau) {
    std::vector<double> v = u;
    std::vector<int64_t> D{P.empty() ? 0 : P[0].first};
    for (auto& e : P) {
        v[e.second] = u[e.second] - mround(u[e.second] - v[e.first]);
        if (std::abs(v[e.second] - v[e.first]) >= tau) D.push_back(e.second);
    }
    return D;
}

// Partition2: owner piece of every node and the edges of each piece in path order.
struct Pieces {
    std::vector<int64_t> roots;
    std::vector<int64_t> owner;  // per node: index into roots
    std::vector<std::vector<std::pair<int64_t, int64_t>>> edges;
};

Pieces partition(int64_t n, const std::vector<std::pair<int64_t, int64_t>>& P, const std::vector<int64_t>& D) {
    Pieces pc;
    pc.roots = D;
    pc.owner.assign(n, -1);
    pc.edges.resize(D.size());
    std::vector<int64_t> rootpos(n, -1);
    for (size_t i = 0; i < D.size(); ++i) rootpos[D[i]] = (int64_t)i;
    pc.owner[D[0]] = 0;
    for (auto& e : P) {
        if (rootpos[e.second] >= 0) {
            pc.owner[e.second] = rootpos[e.second];
            continue;
        }
        pc.owner[e.second] = pc.owner[e.first];
        pc.edges[pc.owner[e.first]].push_back(e);
    }
    return pc;
}

// ---------------------------------------------------------------- small dense linear algebra (real)
// Householder QR with column pivoting: returns the pivot order (first r used).
std::vector<int> pivot_order(std::vector<double> A, int m, int n, int* rank) {  // A column-major m x n
    double r00 = -1.0;
    if (rank) *rank = 0;
    std::vector<int> perm(n);
    std::iota(perm.begin(), perm.end(), 0);
    std::vector<double> nrm(n);
    for (int j = 0; j < n; ++j) {
        double s = 0;
        for (int i = 0; i < m; ++i) s += A[j * m + i] * A[j * m + i];
        nrm[j] = s;
    }
    for (int p = 0; p < std::min(m, n); ++p) {
        int jm = p;
        for (int j = p + 1; j < n; ++j)
            if (nrm[j] > nrm[jm]) jm = j;
        if (jm != p) {
            for (int i = 0; i < m; ++i) std::swap(A[p * m + i], A[jm * m + i]);
            std::swap(nrm[p], nrm[jm]);
            std::swap(perm[p], perm[jm]);
        }
        double xn = 0;
        for (int i = p; i < m; ++i) xn += A[p * m + i] * A[p * m + i];
        xn = std::sqrt(xn);
        if (p == 0) r00 = xn;
        if (rank && xn > 1e-12 * r00) *rank = p + 1;
        if (xn == 0) continue;
        const double alpha = A[p * m + p];
        const double beta = alpha >= 0 ? -xn : xn;
        std::vector<double> v(m, 0.0);
        v[p] = alpha - beta;
        for (int i = p + 1; i < m; ++i) v[i] = A[p * m + i];
        double vv = 0;
        for (int i = p; i < m; ++i) vv += v[i] * v[i];
        for (int j = p; j < n; ++j) {
            double s = 0;
            for (int i = p; i < m; ++i) s += v[i] * A[j * m + i];
            s = 2 * s / vv;
            for (int i = p; i < m; ++i) A[j * m + i] -= s * v[i];
            if (j > p) nrm[j] -= A[j * m + p] * A[j * m + p];
        }
    }
    return perm;
}

// Orthonormal basis (m x r, column-major) of the columns of A by twice-iterated
// Gram-Schmidt.  A column that is (numerically) dependent on the previous ones
// is replaced by a unit vector orthogonalized against them, so the result has
// r orthonormal columns spanning at least the column space of A (the thin Q of
// a Householder QR has the same property).
std::vector<double> orth(std::vector<double> A, int64_t m, int r) {
    auto project_out = [&](double* a, int j) {
        for (int pass = 0; pass < 2; ++pass)
            for (int q = 0; q < j; ++q) {
                const double* b = &A[(size_t)q * m];
                double s = 0;
                for (int64_t i = 0; i < m; ++i) s += a[i] * b[i];
                for (int64_t i = 0; i < m; ++i) a[i] -= s * b[i];
            }
        double s = 0;
        for (int64_t i = 0; i < m; ++i) s += a[i] * a[i];
        return std::sqrt(s);
    };
    for (int j = 0; j < r; ++j) {
        double* a = &A[(size_t)j * m];
        double s0 = 0;
        for (int64_t i = 0; i < m; ++i) s0 += a[i] * a[i];
        s0 = std::sqrt(s0);
        double s = project_out(a, j);
        for (int64_t e = 0; s <= 1e-12 * s0 || s == 0.0; ++e) {
            if (e >= m) fail(MIDBF_ERECOVERY, "cannot complete an orthonormal basis");
            std::fill(a, a + m, 0.0);
            a[e] = 1.0;
            s0 = 1.0;
            s = project_out(a, j);
            if (s < 0.5) s = 0.0;
        }
        for (int64_t i = 0; i < m; ++i) a[i] /= s;
    }
    return A;
}

// One-sided Jacobi SVD of a small m x n (m >= n) row-major matrix: A = U diag(s) V^T.
void jacobi_svd(std::vector<double> A, int m, int n, std::vector<double>& U, std::vector<double>& s,
                std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double a = 0, b = 0, c = 0;
                for (int i = 0; i < m; ++i) {
                    a += A[i * n + p] * A[i * n + p];
                    b += A[i * n + q] * A[i * n + q];
                    c += A[i * n + p] * A[i * n + q];
                }
                if (std::abs(c) <= 1e-15 * std::sqrt(a * b)) continue;
                off = std::max(off, std::abs(c) / std::sqrt(a * b));
                const double zeta = (b - a) / (2 * c);
                const double t = (zeta >= 0 ? 1 : -1) / (std::abs(zeta) + std::sqrt(1 + zeta * zeta));
                const double cs = 1 / std::sqrt(1 + t * t), sn = cs * t;
                for (int i = 0; i < m; ++i) {
                    const double x = A[i * n + p], y = A[i * n + q];
                    A[i * n + p] = cs * x - sn * y;
                    A[i * n + q] = sn * x + cs * y;
                }
                for (int i = 0; i < n; ++i) {
                    const double x = V[i * n + p], y = V[i * n + q];
                    V[i * n + p] = cs * x - sn * y;
                    V[i * n + q] = sn * x + cs * y;
                }
            }
        if (off < 1e-15) break;
    }
    s.assign(n, 0.0);
    U.assign((size_t)m * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double t = 0;
        for (int i = 0; i < m; ++i) t += A[i * n + j] * A[i * n + j];
        s[j] = std::sqrt(t);
        for (int i = 0; i < m; ++i) U[i * n + j] = s[j] > 0 ? A[i * n + j] / s[j] : 0.0;
    }
    // sort descending
    std::vector<int> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return s[a] > s[b]; });
    std::vector<double> U2(U.size()), V2(V.size()), s2(n);
    for (int j = 0; j < n; ++j) {
        s2[j] = s[ord[j]];
        for (int i = 0; i < m; ++i) U2[i * n + j] = U[i * n + ord[j]];
        for (int i = 0; i < n; ++i) V2[i * n + j] = V[i * n + ord[j]];
    }
    U.swap(U2);
    V.swap(V2);
    s.swap(s2);
}

// Pseudo-inverse of a small m x n row-major matrix (m >= n), n x m row-major.
std::vector<double> pinv(const std::vector<double>& A, int m, int n) {
    std::vector<double> U, s, V;
    jacobi_svd(A, m, n, U, s, V);
    const double cut = 1e-13 * (s.empty() ? 0 : s[0]);
    std::vector<double> out((size_t)n * m, 0.0);
    for (int k = 0; k < n; ++k) {
        if (s[k] <= cut) continue;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < m; ++j) out[i * m + j] += V[i * n + k] * U[j * n + k] / s[k];
    }
    return out;
}

double wrapped(const cplx& z) { return std::atan2(z.imag(), z.real()) / (2.0 * M_PI); }

// A kernel value e^{2 pi i Phi} has modulus one; a non-finite or zero value
// from a callback has no phase to recover.
void check_values(const std::vector<cplx>& buf, const char* what) {
    for (const cplx& z : buf)
        if (!std::isfinite(z.real()) || !std::isfinite(z.imag()) || (z.real() == 0.0 && z.imag() == 0.0))
            fail(MIDBF_ECALLBACK, std::string(what) + " callback returned a non-finite or zero value");
}

}  // namespace

std::unique_ptr<Phase> recover_phase(int d, int64_t nx, const double* X, int64_t nw, const double* W,
                                     const midbf_access& acc, int r, int q, double tau, int max_disc,
                                     uint64_t seed, midbf_recover_info* info, bool device) {
    midbf_recover_info inf{};
    auto rows_of = [&](const std::vector<int64_t>& idx) {
        std::vector<cplx> buf(idx.size() * (size_t)nw);
        if (!idx.empty() && acc.rows_fn(acc.user, idx.data(), (int64_t)idx.size(), reinterpret_cast<double*>(buf.data())))
            fail(MIDBF_ECALLBACK, "rows callback failed");
        check_values(buf, "rows");
        inf.rows_requested += (int64_t)idx.size();
        std::vector<double> u(buf.size());
        for (size_t i = 0; i < buf.size(); ++i) u[i] = wrapped(buf[i]);
        return u;  // idx.size() x nw
    };
    auto cols_of = [&](const std::vector<int64_t>& idx) {
        std::vector<cplx> buf(idx.size() * (size_t)nx);
        if (!idx.empty() && acc.cols_fn(acc.user, idx.data(), (int64_t)idx.size(), reinterpret_cast<double*>(buf.data())))
            fail(MIDBF_ECALLBACK, "columns callback failed");
        check_values(buf, "columns");
        inf.cols_requested += (int64_t)idx.size();
        std::vector<double> u(buf.size());
        for (size_t i = 0; i < buf.size(); ++i) u[i] = wrapped(buf[i]);
        return u;  // idx.size() x nx
    };
    // sampled rows and columns: index 0 plus rq - 1 seeded distinct others
    const int rq = r * q;
    std::mt19937_64 rng(seed);
    auto draw = [&](int64_t n) {
        std::vector<int64_t> s{0};
        std::vector<uint8_t> used(n, 0);
        used[0] = 1;
        std::uniform_int_distribution<int64_t> U(1, n - 1);
        while ((int)s.size() < rq) {
            int64_t v = U(rng);
            if (!used[v]) {
                used[v] = 1;
                s.push_back(v);
            }
        }
        return s;
    };
    std::vector<int64_t> R = draw(nx), Cc = draw(nw);
    auto P1 = bfs_path(nx, emst(X, nx, d));
    auto P2 = bfs_path(nw, emst(W, nw, d));
    // discontinuities along the root column (X path) and root row (Omega path)
    std::vector<double> col0 = cols_of({0}), row0 = rows_of({0});
    auto detect_sched = [&](const std::vector<double>& u, const std::vector<std::pair<int64_t, int64_t>>& P,
                            double& used) {
        double t = tau;
        for (;;) {
            auto D = device ? device_detect(u, P, t) : detect(u, P, t);
            if ((int)D.size() - 1 <= max_disc || t >= 0.5) {
                used = t;
                return D;
            }
            t = std::min(0.5, t + 1.0 / 40.0);
        }
    };
    double tr = tau, tc = tau;
    std::vector<int64_t> Dr = detect_sched(col0, P1, tr), Dc = detect_sched(row0, P2, tc);
    inf.disc_rows = (int64_t)Dr.size() - 1;
    inf.disc_cols = (int64_t)Dc.size() - 1;
    inf.tau = std::max(tr, tc);
    auto add_unique = [](std::vector<int64_t>& a, const std::vector<int64_t>& b) {
        for (int64_t v : b)
            if (std::find(a.begin(), a.end(), v) == a.end()) a.push_back(v);
    };
    add_unique(R, Dr);
    add_unique(Cc, Dc);
    const int nR = (int)R.size(), nC = (int)Cc.size();
    std::vector<double> Urow = rows_of(R), Ucol = cols_of(Cc);  // observations mod 1
    std::vector<double> rows = Urow, cols = Ucol;              // recovered values
    std::vector<int64_t> rpos(nx, -1), cpos(nw, -1);
    for (int i = 0; i < nR; ++i) rpos[R[i]] = i;
    for (int j = 0; j < nC; ++j) cpos[Cc[j]] = j;
    Pieces pc1 = partition(nx, P1, Dr), pc2 = partition(nw, P2, Dc);
    // Algorithm 4 along the edges E of one piece for a batch of vectors (u, v):
    // on the host one after the other, or on the device in one launch
    auto along = [&](int64_t n, const std::vector<std::pair<int64_t, int64_t>>& E, int64_t root,
                     const std::vector<const double*>& us, const std::vector<double*>& vs) {
        if (device) {
            device_recover_along(n, E, root, us, vs);
        } else {
            for (size_t k = 0; k < us.size(); ++k) recover_along(us[k], vs[k], E);
        }
    };
    for (size_t s = 0; s < pc1.roots.size(); ++s) {
        const int64_t rs = pc1.roots[s];
        for (size_t t = 0; t < pc2.roots.size(); ++t) {
            const int64_t ct = pc2.roots[t];
            const int i0 = (int)rpos[rs], j0 = (int)cpos[ct];
            // root row along piece t of the Omega path
            along(nw, pc2.edges[t], ct, {&Urow[(size_t)i0 * nw]}, {&rows[(size_t)i0 * nw]});
            // root column along piece s of the X path, from the recovered (rs, ct)
            cols[(size_t)j0 * nx + rs] = rows[(size_t)i0 * nw + ct];
            along(nx, pc1.edges[s], rs, {&Ucol[(size_t)j0 * nx]}, {&cols[(size_t)j0 * nx]});
            // the other sampled rows of piece s, each from the recovered root column;
            // the other sampled columns of piece t, each from the recovered root row
            std::vector<const double*> us;
            std::vector<double*> vs;
            for (int i = 0; i < nR; ++i) {
                if (pc1.owner[R[i]] != (int64_t)s || R[i] == rs) continue;
                rows[(size_t)i * nw + ct] = cols[(size_t)j0 * nx + R[i]];
                us.push_back(&Urow[(size_t)i * nw]);
                vs.push_back(&rows[(size_t)i * nw]);
            }
            along(nw, pc2.edges[t], ct, us, vs);
            us.clear();
            vs.clear();
            for (int j = 0; j < nC; ++j) {
                if (pc2.owner[Cc[j]] != (int64_t)t || Cc[j] == ct) continue;
                cols[(size_t)j * nx + rs] = rows[(size_t)i0 * nw + Cc[j]];
                us.push_back(&Ucol[(size_t)j * nx]);
                vs.push_back(&cols[(size_t)j * nx]);
            }
            along(nx, pc1.edges[s], rs, us, vs);
        }
    }
    for (int i = 0; i < nR; ++i)
        for (int j = 0; j < nC; ++j)
            if (std::abs(rows[(size_t)i * nw + Cc[j]] - cols[(size_t)j * nx + R[i]]) > 1e-9) inf.mismatches++;
    // ---- Algorithm 1 restricted to rows R and columns C ----
    if (r > std::min(nR, nC)) fail(MIDBF_ERECOVERY, "rank larger than the sample");
    std::vector<double> ARC((size_t)nR * nC), ACR((size_t)nC * nR);  // column-major
    for (int j = 0; j < nC; ++j)
        for (int i = 0; i < nR; ++i) {
            ARC[(size_t)j * nR + i] = rows[(size_t)i * nw + Cc[j]];
            ACR[(size_t)i * nC + j] = rows[(size_t)i * nw + Cc[j]];
        }
    // Numerical rank of the known block: when Psi(R, C) has rank below r (an
    // exactly low-rank phase), the factorization is carried out at that rank and
    // the remaining columns of U and V are zero.
    int rank_c = 0, rank_r = 0;
    std::vector<int> pc = pivot_order(ARC, nR, nC, &rank_c), pr = pivot_order(ACR, nC, nR, &rank_r);
    const int rfull = r;
    r = std::max(1, std::min(r, std::min(rank_c, rank_r)));
    std::vector<double> Bc((size_t)nx * r), Br((size_t)nw * r);
    for (int t = 0; t < r; ++t) {
        std::copy(cols.begin() + (size_t)pc[t] * nx, cols.begin() + (size_t)(pc[t] + 1) * nx, Bc.begin() + (size_t)t * nx);
        std::copy(rows.begin() + (size_t)pr[t] * nw, rows.begin() + (size_t)(pr[t] + 1) * nw, Br.begin() + (size_t)t * nw);
    }
    std::vector<double> Qc = orth(Bc, nx, r), Qr = orth(Br, nw, r);
    // I = R (all recovered rows), J = C (all recovered columns)
    std::vector<double> QcI((size_t)nR * r), QrJ((size_t)nC * r), AIJ((size_t)nR * nC);
    for (int i = 0; i < nR; ++i)
        for (int t = 0; t < r; ++t) QcI[(size_t)i * r + t] = Qc[(size_t)t * nx + R[i]];
    for (int j = 0; j < nC; ++j)
        for (int t = 0; t < r; ++t) QrJ[(size_t)j * r + t] = Qr[(size_t)t * nw + Cc[j]];
    for (int i = 0; i < nR; ++i)
        for (int j = 0; j < nC; ++j) AIJ[(size_t)i * nC + j] = rows[(size_t)i * nw + Cc[j]];
    std::vector<double> P1i = pinv(QcI, nR, r);  // r x nR
    std::vector<double> P2i = pinv(QrJ, nC, r);  // r x nC ; (Qr(J,:)^T)^+ = (Qr(J,:)^+)^T
    std::vector<double> T1((size_t)r * nC, 0.0), M((size_t)r * r, 0.0);
    for (int a = 0; a < r; ++a)
        for (int j = 0; j < nC; ++j) {
            double s2 = 0;
            for (int i = 0; i < nR; ++i) s2 += P1i[(size_t)a * nR + i] * AIJ[(size_t)i * nC + j];
            T1[(size_t)a * nC + j] = s2;
        }
    for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) {
            double s2 = 0;
            for (int j = 0; j < nC; ++j) s2 += T1[(size_t)a * nC + j] * P2i[(size_t)b * nC + j];
            M[(size_t)a * r + b] = s2;
        }
    std::vector<double> UM, sM, VM;
    jacobi_svd(M, r, r, UM, sM, VM);
    auto ph = std::make_unique<Phase>();
    ph->family = MIDBF_PHASE_LOWRANK;
    ph->d = d;
    ph->nx = nx;
    ph->nw = nw;
    ph->X.assign(X, X + nx * d);
    ph->W.assign(W, W + nw * d);
    ph->r = rfull;
    ph->U.assign((size_t)nx * rfull, 0.0);
    ph->V.assign((size_t)nw * rfull, 0.0);
    for (int64_t i = 0; i < nx; ++i)
        for (int t = 0; t < r; ++t) {
            double s2 = 0;
            for (int a = 0; a < r; ++a) s2 += Qc[(size_t)a * nx + i] * UM[(size_t)a * r + t];
            ph->U[(size_t)i * rfull + t] = s2;
        }
    for (int64_t j = 0; j < nw; ++j)
        for (int t = 0; t < r; ++t) {
            double s2 = 0;
            for (int a = 0; a < r; ++a) s2 += Qr[(size_t)a * nw + j] * VM[(size_t)a * r + t];
            ph->V[(size_t)j * rfull + t] = s2 * sM[t];
        }
    if (info) *info = inf;
    return ph;
}

}  // namespace midbf
