// Column-pivoted Householder QR (Businger-Golub) and the interpolative
// decomposition built from it, complex FP64 (Sec. 3.2).
//
// A(s,:) Lambda = Q R; the factorization stops at the first pivot whose
// |R(p,p)| <= tol |R(1,1)| (Sec. 3.6 adaptive rank, keeping the pivots above
// the tolerance), so only k Householder steps are spent.  Then
// T = R11^{-1} R12 by back substitution and the skeleton is Lambda(1:k).
// Column norms are downdated after each step and recomputed when
// cancellation has eaten most of them (the safeguard of LAPACK's xGEQPF).
//
// The factorization works on separate real and imaginary planes of the
// matrix, so the inner loops are plain real arithmetic over contiguous
// arrays; the trailing update takes four columns per pass over the
// Householder vector, and every sum runs as two interleaved partial sums
// (even and odd rows) added at the end: a fixed order, independent of the
// compiler's vector width.
#include <algorithm>

#include "internal.hpp"

namespace midbf {

namespace {

// s = sum_i conj(v_i) c_i over i in [i0, ms) for up to four columns c.
template <int NC>
inline void dots(const double* vr, const double* vi, const double* const* cr, const double* const* ci, int i0,
                 int ms, double* sr, double* si) {
    double ar[NC][2] = {}, ai[NC][2] = {};
    int i = i0;
    for (; i + 1 < ms; i += 2) {
        const double a0 = vr[i], b0 = vi[i], a1 = vr[i + 1], b1 = vi[i + 1];
        for (int c = 0; c < NC; ++c) {
            ar[c][0] += a0 * cr[c][i] + b0 * ci[c][i];
            ai[c][0] += a0 * ci[c][i] - b0 * cr[c][i];
            ar[c][1] += a1 * cr[c][i + 1] + b1 * ci[c][i + 1];
            ai[c][1] += a1 * ci[c][i + 1] - b1 * cr[c][i + 1];
        }
    }
    for (int c = 0; c < NC; ++c) {
        double r = ar[c][0] + ar[c][1], m = ai[c][0] + ai[c][1];
        if (i < ms) {
            r += vr[i] * cr[c][i] + vi[i] * ci[c][i];
            m += vr[i] * ci[c][i] - vi[i] * cr[c][i];
        }
        sr[c] = r;
        si[c] = m;
    }
}

// c_i -= s v_i over i in [i0, ms) for up to four columns.
template <int NC>
inline void axpys(const double* vr, const double* vi, double* const* cr, double* const* ci, int i0, int ms,
                  const double* sr, const double* si) {
    for (int i = i0; i < ms; ++i) {
        const double a = vr[i], b = vi[i];
        for (int c = 0; c < NC; ++c) {
            cr[c][i] -= sr[c] * a - si[c] * b;
            ci[c][i] -= sr[c] * b + si[c] * a;
        }
    }
}

inline double sumsq(const double* r, const double* m, int i0, int ms) {
    double s0 = 0.0, s1 = 0.0;
    int i = i0;
    for (; i + 1 < ms; i += 2) {
        s0 += r[i] * r[i] + m[i] * m[i];
        s1 += r[i + 1] * r[i + 1] + m[i + 1] * m[i + 1];
    }
    if (i < ms) s0 += r[i] * r[i] + m[i] * m[i];
    return s0 + s1;
}

}  // namespace

IdResult column_id(std::vector<cplx>& A, int ms, int n, double tol, int kmax) {
    IdResult out;
    const int kk = std::min(ms, n);
    const size_t ld = (size_t)((ms + 7) & ~7);
    std::vector<double> re(ld * n), im(ld * n);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < ms; ++i) {
            re[j * ld + i] = A[(size_t)j * ms + i].real();
            im[j * ld + i] = A[(size_t)j * ms + i].imag();
        }
    std::vector<double> nrm(n), nrm0(n);
    std::vector<int> perm(n);
    for (int j = 0; j < n; ++j) {
        nrm[j] = nrm0[j] = sumsq(&re[j * ld], &im[j * ld], 0, ms);
        perm[j] = j;
    }
    const int cap = kmax > 0 ? std::min(kmax, kk) : kk;
    double r11 = -1.0;
    int k = 0;
    for (int p = 0; p < kk; ++p) {
        int jm = p;
        for (int j = p + 1; j < n; ++j)
            if (nrm[j] > nrm[jm]) jm = j;
        if (jm != p) {
            std::swap_ranges(&re[p * ld], &re[p * ld] + ms, &re[jm * ld]);
            std::swap_ranges(&im[p * ld], &im[p * ld] + ms, &im[jm * ld]);
            std::swap(nrm[p], nrm[jm]);
            std::swap(nrm0[p], nrm0[jm]);
            std::swap(perm[p], perm[jm]);
        }
        double* pr = &re[p * ld];
        double* pi = &im[p * ld];
        const double xn = sumsq(pr, pi, p + 1, ms);
        const cplx alpha(pr[p], pi[p]);
        const double an = std::sqrt(std::norm(alpha) + xn);
        out.rdiag.push_back(an);
        if (p == 0) r11 = an;
        if (r11 <= 0.0) {  // zero matrix: keep one column, T = 0
            k = 1;
            break;
        }
        if (p > 0 && an <= tol * r11) break;
        if (p >= cap) break;
        k = p + 1;
        // Householder: H = I - tau v v^H maps column p (rows p..) to beta e1, |beta| = an
        const double aa = std::abs(alpha);
        const cplx phase = aa > 0.0 ? alpha / aa : cplx(1.0, 0.0);
        const cplx beta = -phase * an;
        if (an == 0.0) continue;
        const cplx inv = 1.0 / (alpha - beta);
        const cplx tau = (beta - alpha) / beta;
        for (int i = p + 1; i < ms; ++i) {
            const double a = pr[i], b = pi[i];
            pr[i] = a * inv.real() - b * inv.imag();
            pi[i] = a * inv.imag() + b * inv.real();
        }
        pr[p] = beta.real();
        pi[p] = beta.imag();
        // apply H to the remaining columns, four per pass over v
        for (int j0 = p + 1; j0 < n; j0 += 4) {
            const int nc = std::min(4, n - j0);
            double* cr[4];
            double* ci[4];
            for (int c = 0; c < 4; ++c) {
                const int j = j0 + std::min(c, nc - 1);
                cr[c] = &re[j * ld];
                ci[c] = &im[j * ld];
            }
            double sr[4], si[4];
            if (nc == 4) dots<4>(pr, pi, cr, ci, p + 1, ms, sr, si);
            else if (nc == 3) dots<3>(pr, pi, cr, ci, p + 1, ms, sr, si);
            else if (nc == 2) dots<2>(pr, pi, cr, ci, p + 1, ms, sr, si);
            else dots<1>(pr, pi, cr, ci, p + 1, ms, sr, si);
            for (int c = 0; c < nc; ++c) {
                // s = tau (c_p + sum conj(v) c)
                const cplx s = tau * cplx(cr[c][p] + sr[c], ci[c][p] + si[c]);
                sr[c] = s.real();
                si[c] = s.imag();
                cr[c][p] -= sr[c];
                ci[c][p] -= si[c];
            }
            if (nc == 4) axpys<4>(pr, pi, cr, ci, p + 1, ms, sr, si);
            else if (nc == 3) axpys<3>(pr, pi, cr, ci, p + 1, ms, sr, si);
            else if (nc == 2) axpys<2>(pr, pi, cr, ci, p + 1, ms, sr, si);
            else axpys<1>(pr, pi, cr, ci, p + 1, ms, sr, si);
            // downdate the trailing norms
            for (int c = 0; c < nc; ++c) {
                const int j = j0 + c;
                double t = nrm[j] - (cr[c][p] * cr[c][p] + ci[c][p] * ci[c][p]);
                if (t <= 1.5e-8 * nrm0[j] || t < 0.0) {
                    t = sumsq(cr[c], ci[c], p + 1, ms);
                    nrm0[j] = t;
                }
                nrm[j] = t;
            }
        }
    }
    if (k == 0) k = 1;
    out.skel.assign(perm.begin(), perm.begin() + k);
    out.red.assign(perm.begin() + k, perm.end());
    const int nr = n - k;
    out.T.assign((size_t)k * nr, cplx(0.0, 0.0));
    if (r11 > 0.0) {
        // T = R11^{-1} R12 by column-oriented back substitution: for each
        // column of R12, x_i = b_i / R(i,i), then b(0:i) -= x_i R(0:i, i)
        // (column i of R, contiguous in the planes)
        std::vector<double> br(k), bi(k);
        for (int j = 0; j < nr; ++j) {
            const double* col_r = &re[(size_t)(k + j) * ld];
            const double* col_i = &im[(size_t)(k + j) * ld];
            std::copy(col_r, col_r + k, br.begin());
            std::copy(col_i, col_i + k, bi.begin());
            for (int i = k - 1; i >= 0; --i) {
                const cplx x = cplx(br[i], bi[i]) / cplx(re[i * ld + i], im[i * ld + i]);
                out.T[(size_t)i * nr + j] = x;
                const double xr = x.real(), xi = x.imag();
                const double* rr = &re[i * ld];
                const double* ri = &im[i * ld];
                for (int l = 0; l < i; ++l) {
                    br[l] -= xr * rr[l] - xi * ri[l];
                    bi[l] -= xr * ri[l] + xi * rr[l];
                }
            }
        }
    }
    return out;
}

}  // namespace midbf
