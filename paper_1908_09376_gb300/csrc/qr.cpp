// Column-pivoted Householder QR (Businger-Golub) and the interpolative
// decomposition built from it, complex FP64 (Sec. 3.2).
//
// A(s,:) Lambda = Q R; the factorization stops at the first pivot whose
// |R(p,p)| <= tol |R(1,1)| (Sec. 3.6 adaptive rank, keeping the pivots above
// the tolerance), so only k Householder steps are spent.  Then
// T = R11^{-1} R12 by back substitution and the skeleton is Lambda(1:k).
// Column norms are downdated after each step and recomputed when
// cancellation has eaten most of them (the safeguard of LAPACK's xGEQPF).
#include <algorithm>

#include "internal.hpp"

namespace midbf {

IdResult column_id(std::vector<cplx>& A, int ms, int n, double tol, int kmax) {
    IdResult out;
    const int kk = std::min(ms, n);
    std::vector<double> nrm(n), nrm0(n);
    std::vector<int> perm(n);
    for (int j = 0; j < n; ++j) {
        const cplx* c = &A[(size_t)j * ms];
        double s = 0.0;
        for (int i = 0; i < ms; ++i) s += std::norm(c[i]);
        nrm[j] = nrm0[j] = s;
        perm[j] = j;
    }
    const int cap = kmax > 0 ? std::min(kmax, kk) : kk;
    double r11 = -1.0;
    int k = 0;
    std::vector<cplx> w(n);
    for (int p = 0; p < kk; ++p) {
        int jm = p;
        for (int j = p + 1; j < n; ++j)
            if (nrm[j] > nrm[jm]) jm = j;
        if (jm != p) {
            std::swap_ranges(&A[(size_t)p * ms], &A[(size_t)p * ms] + ms, &A[(size_t)jm * ms]);
            std::swap(nrm[p], nrm[jm]);
            std::swap(nrm0[p], nrm0[jm]);
            std::swap(perm[p], perm[jm]);
        }
        cplx* cp = &A[(size_t)p * ms];
        double xn = 0.0;
        for (int i = p + 1; i < ms; ++i) xn += std::norm(cp[i]);
        const cplx alpha = cp[p];
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
        // Householder: H = I - tau v v^H maps cp[p:] to beta e1, |beta| = an
        const double aa = std::abs(alpha);
        const cplx phase = aa > 0.0 ? alpha / aa : cplx(1.0, 0.0);
        const cplx beta = -phase * an;
        if (an == 0.0) continue;
        const cplx denom = alpha - beta;
        const cplx tau = (beta - alpha) / beta;
        for (int i = p + 1; i < ms; ++i) cp[i] /= denom;
        cp[p] = beta;
        // apply to the remaining columns
        for (int j = p + 1; j < n; ++j) {
            cplx* cj = &A[(size_t)j * ms];
            cplx s = cj[p];
            for (int i = p + 1; i < ms; ++i) s += std::conj(cp[i]) * cj[i];
            s *= tau;
            cj[p] -= s;
            for (int i = p + 1; i < ms; ++i) cj[i] -= s * cp[i];
            // downdate the trailing norm
            double t = nrm[j] - std::norm(cj[p]);
            if (t <= 1.5e-8 * nrm0[j] || t < 0.0) {
                t = 0.0;
                for (int i = p + 1; i < ms; ++i) t += std::norm(cj[i]);
                nrm0[j] = t;
            }
            nrm[j] = t;
        }
    }
    if (k == 0) k = 1;
    out.skel.assign(perm.begin(), perm.begin() + k);
    out.red.assign(perm.begin() + k, perm.end());
    const int nr = n - k;
    out.T.assign((size_t)k * nr, cplx(0.0, 0.0));
    if (r11 > 0.0) {
        // T = R11^{-1} R12, back substitution per column of R12
        for (int j = 0; j < nr; ++j) {
            const cplx* col = &A[(size_t)(k + j) * ms];
            for (int i = k - 1; i >= 0; --i) {
                cplx s = col[i];
                for (int l = i + 1; l < k; ++l) s -= A[(size_t)l * ms + i] * out.T[(size_t)l * nr + j];
                out.T[(size_t)i * nr + j] = s / A[(size_t)i * ms + i];
            }
        }
    }
    return out;
}

}  // namespace midbf
