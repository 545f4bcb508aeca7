// Batched interpolative decompositions on the GPU, FP64 (Sec. 3.2, 3.6).
//
// The same linear-scaling column ID as the host (qr.cpp), one CTA per
// decomposition: the sample matrix M (ns x n, column-major) of kernel values
// exp(2 pi i Phi) is generated on the device from point indices, then a
// column-pivoted Householder QR (Businger-Golub, norm downdating with
// recomputation) stops at the first pivot with |R(p,p)| <= tol |R(1,1)|,
// and T = R11^{-1} R12 is formed by back substitution.  The host keeps the
// sampling (Mock-Chebyshev with nearest-candidate snapping) and the
// regrowth rule, and assembles the factors exactly as the host build does.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "internal.hpp"

namespace midbf {
namespace gpuid {

struct Job {
    long long m_off;     // offset (complex entries) of M in the matrix pool
    long long cols_off;  // offset of the n decomposed point indices
    long long rows_off;  // offset of the ns sample point indices
    long long t_off;     // offset (complex entries) of T in the output pool
    int n, ns;
    int cols_x;          // 1: decomposed points are X points (row ID), 0: Omega points
    int pad;
};

struct PhaseDev {
    int family, d, r;
    const double* X;
    const double* W;
    const double* U;
    const double* V;
};

__device__ double phase_eval(const PhaseDev& ph, long long i, long long j) {
    if (ph.family == MIDBF_PHASE_LOWRANK) {
        double s = 0.0;
        for (int t = 0; t < ph.r; ++t) s += ph.U[i * ph.r + t] * ph.V[j * ph.r + t];
        return s;
    }
    const double* x = ph.X + i * ph.d;
    const double* w = ph.W + j * ph.d;
    double dot = 0.0;
    for (int k = 0; k < ph.d; ++k) dot += x[k] * w[k];
    switch (ph.family) {
        case MIDBF_PHASE_DOT: return dot;
        case MIDBF_PHASE_ZERO: return 0.0;
        case MIDBF_PHASE_SEPARABLE: {
            double a = 0.0, b = 0.0;
            for (int k = 0; k < ph.d; ++k) {
                a += sinpi(2.0 * x[k]);
                b += w[k] * w[k];
            }
            return a + 0.05 * b;
        }
        case MIDBF_PHASE_FIO2D:
        case MIDBF_PHASE_FIO2D_JUMP: {
            const double c1 = (2.0 + sinpi(2.0 * x[0]) * sinpi(2.0 * x[1])) / 16.0;
            const double c2 = (2.0 + cospi(2.0 * x[0]) * cospi(2.0 * x[1])) / 16.0;
            double v = dot + sqrt(c1 * c1 * w[0] * w[0] + c2 * c2 * w[1] * w[1]);
            if (ph.family == MIDBF_PHASE_FIO2D_JUMP)
                v += 0.5 * sqrt(w[0] * w[0] + w[1] * w[1]) * ((x[0] - 0.5 >= 0.0) ? 1.0 : -1.0);
            return v;
        }
        case MIDBF_PHASE_FIO3D: {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double ck = (2.0 + sinpi(2.0 * x[k]) * cospi(2.0 * x[(k + 1) % 3])) / 16.0;
                acc += ck * ck * w[k] * w[k];
            }
            return dot + sqrt(acc);
        }
        case MIDBF_PHASE_DISTANCE: {
            double s = 0.0;
            for (int k = 0; k < ph.d; ++k) s += (x[k] - w[k]) * (x[k] - w[k]);
            return sqrt(s);
        }
        default: return 0.0;   // unreachable: gpu_id_context admits the families above only
    }
}

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
    return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += red[w];
    return s;
}

// One CTA per job.  nrm/nrm0/perm/kout live in global scratch (n entries per job).
__global__ void __launch_bounds__(kThreads) k_id(const Job* jobs, PhaseDev ph, const int64_t* idx, double2* Mpool,
                                                 double* nrm_pool, double* nrm0_pool, int* perm_pool, int* kout,
                                                 double2* Tpool, double tol, int kmax, long long nrm_stride) {
    __shared__ double red[kWarps];
    __shared__ double s_val;
    __shared__ int s_idx;
    __shared__ double2 s_beta, s_denom;
    __shared__ double s_tau;
    __shared__ int s_stop;
    __shared__ int s_bi[kWarps];
    const Job jb = jobs[blockIdx.x];
    const int n = jb.n, ms = jb.ns;
    double2* M = Mpool + jb.m_off;
    const int64_t* cols = idx + jb.cols_off;
    const int64_t* rows = idx + jb.rows_off;
    double* nrm = nrm_pool + (long long)blockIdx.x * nrm_stride;
    double* nrm0 = nrm0_pool + (long long)blockIdx.x * nrm_stride;
    int* perm = perm_pool + (long long)blockIdx.x * nrm_stride;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // 1. kernel samples
    for (long long e = tid; e < (long long)ms * n; e += kThreads) {
        const int c = (int)(e / ms), s = (int)(e % ms);
        const long long xi = jb.cols_x ? cols[c] : rows[s];
        const long long wi = jb.cols_x ? rows[s] : cols[c];
        double p = phase_eval(ph, xi, wi);
        p -= rint(p);
        double sn, cs;
        sincospi(2.0 * p, &sn, &cs);
        M[e] = {cs, sn};
    }
    __syncthreads();
    // 2. column norms
    for (int j = warp; j < n; j += kWarps) {
        const double2* cj = M + (long long)j * ms;
        double s = 0.0;
        for (int i = lane; i < ms; i += 32) s += cj[i].x * cj[i].x + cj[i].y * cj[i].y;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            nrm[j] = s;
            nrm0[j] = s;
            perm[j] = j;
        }
    }
    __syncthreads();
    const int kk = min(ms, n);
    const int cap = kmax > 0 ? min(kmax, kk) : kk;
    double r11 = -1.0;
    int k = 0;
    for (int p = 0; p < kk; ++p) {
        // a. pivot: largest remaining norm, lowest index on ties
        double bv = -1.0;
        int bi = p;
        for (int j = p + tid; j < n; j += kThreads)
            if (nrm[j] > bv) {
                bv = nrm[j];
                bi = j;
            }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        __syncthreads();
        if (lane == 0) {
            red[warp] = bv;
            s_bi[warp] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            double v = red[0];
            int ix = s_bi[0];
            for (int w = 1; w < kWarps; ++w)
                if (red[w] > v || (red[w] == v && s_bi[w] < ix)) {
                    v = red[w];
                    ix = s_bi[w];
                }
            s_idx = ix;
        }
        __syncthreads();
        const int jm = s_idx;
        // b. swap columns p and jm
        if (jm != p) {
            double2* a = M + (long long)p * ms;
            double2* b2 = M + (long long)jm * ms;
            for (int i = tid; i < ms; i += kThreads) {
                const double2 t = a[i];
                a[i] = b2[i];
                b2[i] = t;
            }
            if (tid == 0) {
                double t = nrm[p];
                nrm[p] = nrm[jm];
                nrm[jm] = t;
                t = nrm0[p];
                nrm0[p] = nrm0[jm];
                nrm0[jm] = t;
                const int ti = perm[p];
                perm[p] = perm[jm];
                perm[jm] = ti;
            }
            __syncthreads();
        }
        // c. Householder reflector of column p
        double2* cp = M + (long long)p * ms;
        double xn = 0.0;
        for (int i = p + 1 + tid; i < ms; i += kThreads) xn += cp[i].x * cp[i].x + cp[i].y * cp[i].y;
        xn = block_sum(xn, red);
        if (tid == 0) {
            const double2 alpha = cp[p];
            const double aa = sqrt(alpha.x * alpha.x + alpha.y * alpha.y);
            const double an = sqrt(aa * aa + xn);
            if (p == 0) r11 = an;
            int stop = 0;
            if (r11 <= 0.0) stop = 2;
            else if (p > 0 && an <= tol * r11) stop = 1;
            else if (p >= cap) stop = 1;
            s_stop = stop;
            s_val = r11;
            if (!stop && an > 0.0) {
                const double2 ph2 = aa > 0.0 ? double2{alpha.x / aa, alpha.y / aa} : double2{1.0, 0.0};
                const double2 beta = {-ph2.x * an, -ph2.y * an};
                const double2 den = {alpha.x - beta.x, alpha.y - beta.y};
                // tau = (beta - alpha) / beta is real: 1 + |alpha| / an
                s_tau = 1.0 + aa / an;
                s_beta = beta;
                s_denom = den;
            } else {
                s_tau = 0.0;
            }
        }
        __syncthreads();
        r11 = s_val;
        if (s_stop) {
            if (s_stop == 2) k = 1;
            break;
        }
        k = p + 1;
        if (s_tau == 0.0) continue;
        {
            const double2 den = s_denom;
            const double dd = den.x * den.x + den.y * den.y;
            for (int i = p + 1 + tid; i < ms; i += kThreads) {
                const double2 v = cp[i];
                cp[i] = {(v.x * den.x + v.y * den.y) / dd, (v.y * den.x - v.x * den.y) / dd};
            }
        }
        __syncthreads();
        if (tid == 0) cp[p] = s_beta;
        // d. apply to the trailing columns, one warp per column
        const double tau = s_tau;
        for (int j = p + 1 + warp; j < n; j += kWarps) {
            double2* cj = M + (long long)j * ms;
            double2 sacc = {0.0, 0.0};
            for (int i = p + 1 + lane; i < ms; i += 32) {
                const double2 t = cmulc(cp[i], cj[i]);
                sacc.x += t.x;
                sacc.y += t.y;
            }
            for (int o = 16; o > 0; o >>= 1) {
                sacc.x += __shfl_xor_sync(0xffffffffu, sacc.x, o);
                sacc.y += __shfl_xor_sync(0xffffffffu, sacc.y, o);
            }
            double2 s2 = {cj[p].x + sacc.x, cj[p].y + sacc.y};
            s2.x *= tau;
            s2.y *= tau;
            __syncwarp();
            for (int i = p + 1 + lane; i < ms; i += 32) {
                const double2 t = cmul(s2, cp[i]);
                cj[i].x -= t.x;
                cj[i].y -= t.y;
            }
            if (lane == 0) {
                cj[p].x -= s2.x;
                cj[p].y -= s2.y;
            }
            __syncwarp();
            // downdate the trailing norm, recompute after heavy cancellation
            double t = 0.0;
            if (lane == 0) t = nrm[j] - (cj[p].x * cj[p].x + cj[p].y * cj[p].y);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t <= 1.5e-8 * nrm0[j] || t < 0.0) {
                double s3 = 0.0;
                for (int i = p + 1 + lane; i < ms; i += 32) s3 += cj[i].x * cj[i].x + cj[i].y * cj[i].y;
                for (int o = 16; o > 0; o >>= 1) s3 += __shfl_xor_sync(0xffffffffu, s3, o);
                if (lane == 0) nrm0[j] = s3;
                t = s3;
            }
            if (lane == 0) nrm[j] = t;
        }
        __syncthreads();
    }
    if (k == 0) k = 1;
    if (tid == 0) kout[blockIdx.x] = k;
    // T = R11^{-1} R12, one warp per column of R12 (serial over rows)
    const int nr = n - k;
    double2* T = Tpool + jb.t_off;
    if (r11 > 0.0) {
        for (int j = warp; j < nr; j += kWarps) {
            const double2* col = M + (long long)(k + j) * ms;
            for (int i = k - 1; i >= 0; --i) {
                double2 s = {0.0, 0.0};
                for (int l = i + 1 + lane; l < k; l += 32) {
                    const double2 t = cmul(M[(long long)l * ms + i], T[(long long)l * nr + j]);
                    s.x += t.x;
                    s.y += t.y;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
                    s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
                }
                if (lane == 0) {
                    const double2 num = {col[i].x - s.x, col[i].y - s.y};
                    const double2 d = M[(long long)i * ms + i];
                    const double dd = d.x * d.x + d.y * d.y;
                    T[(long long)i * nr + j] = {(num.x * d.x + num.y * d.y) / dd, (num.y * d.x - num.x * d.y) / dd};
                }
                __syncwarp();
            }
        }
    } else {
        for (long long e = tid; e < (long long)k * nr; e += kThreads) T[e] = {0.0, 0.0};
    }
}


#define CKG(call)                                                                                      \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) fail(MIDBF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    } while (0)

struct DevMem {
    void* p = nullptr;
    size_t n = 0;
    void ensure(size_t bytes) {
        if (bytes <= n) return;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        if (cudaMalloc(&p, bytes) != cudaSuccess) fail(MIDBF_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
        n = bytes;
    }
    ~DevMem() {
        if (p) cudaFree(p);
    }
};

}  // namespace gpuid

struct GpuIdContext {
    gpuid::PhaseDev ph{};
    gpuid::DevMem X, W, U, V, jobs, idx, M, T, nrm, nrm0, perm, kout;
};

std::unique_ptr<GpuIdContext, void (*)(GpuIdContext*)> gpu_id_context(const Phase& ph) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) fail(MIDBF_ECUDA, "no CUDA device for the device build");
    switch (ph.family) {
        case MIDBF_PHASE_LOWRANK: case MIDBF_PHASE_DOT: case MIDBF_PHASE_ZERO: case MIDBF_PHASE_SEPARABLE:
        case MIDBF_PHASE_FIO2D: case MIDBF_PHASE_FIO2D_JUMP: case MIDBF_PHASE_FIO3D: case MIDBF_PHASE_DISTANCE:
            break;
        default: fail(MIDBF_EINVAL, "phase family without a device evaluation");
    }
    std::unique_ptr<GpuIdContext, void (*)(GpuIdContext*)> c(new GpuIdContext, [](GpuIdContext* p) { delete p; });
    auto up = [](gpuid::DevMem& m, const std::vector<double>& v) -> const double* {
        if (v.empty()) return nullptr;
        m.ensure(v.size() * sizeof(double));
        CKG(cudaMemcpy(m.p, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice));
        return static_cast<const double*>(m.p);
    };
    c->ph.family = ph.family;
    c->ph.d = ph.d;
    c->ph.r = ph.r;
    c->ph.X = up(c->X, ph.X);
    c->ph.W = up(c->W, ph.W);
    c->ph.U = up(c->U, ph.U);
    c->ph.V = up(c->V, ph.V);
    return c;
}

void gpu_id_batch(GpuIdContext& ctx, const std::vector<IdRequest>& reqs, double tol, int kmax,
                  std::vector<IdReply>& out, bool fp32) {
    using gpuid::Job;
    const size_t nj = reqs.size();
    out.assign(nj, IdReply{});
    if (nj == 0) return;
    std::vector<cplx> tmp;
    // process in chunks bounded by the matrix pool size (4 GiB of M, same for T)
    const size_t kPool = (size_t)4 << 30;
    size_t j0 = 0;
    while (j0 < nj) {
        std::vector<Job> jobs;
        std::vector<int64_t> idx;
        size_t mtot = 0, maxn = 1;
        size_t j1 = j0;
        while (j1 < nj) {
            const size_t n = reqs[j1].cols->size(), ns = reqs[j1].samples.size();
            const size_t me = n * ns * sizeof(double) * 2;
            if (j1 > j0 && (mtot + me) > kPool) break;
            Job jb{};
            jb.m_off = (long long)(mtot / (sizeof(double) * 2));
            jb.t_off = jb.m_off;
            jb.n = (int)n;
            jb.ns = (int)ns;
            jb.cols_x = reqs[j1].cols_x ? 1 : 0;
            jb.cols_off = (long long)idx.size();
            idx.insert(idx.end(), reqs[j1].cols->begin(), reqs[j1].cols->end());
            jb.rows_off = (long long)idx.size();
            idx.insert(idx.end(), reqs[j1].samples.begin(), reqs[j1].samples.end());
            jobs.push_back(jb);
            mtot += me;
            maxn = std::max(maxn, n);
            ++j1;
        }
        const int njob = (int)jobs.size();
        ctx.jobs.ensure(jobs.size() * sizeof(Job));
        ctx.idx.ensure(idx.size() * sizeof(int64_t));
        ctx.M.ensure(mtot);
        ctx.T.ensure(mtot);
        ctx.nrm.ensure((size_t)njob * maxn * sizeof(double));
        ctx.nrm0.ensure((size_t)njob * maxn * sizeof(double));
        ctx.perm.ensure((size_t)njob * maxn * sizeof(int));
        ctx.kout.ensure((size_t)njob * sizeof(int));
        CKG(cudaMemcpy(ctx.jobs.p, jobs.data(), jobs.size() * sizeof(Job), cudaMemcpyHostToDevice));
        CKG(cudaMemcpy(ctx.idx.p, idx.data(), idx.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
        gpuid::k_id<<<njob, gpuid::kThreads>>>(static_cast<const Job*>(ctx.jobs.p), ctx.ph,
                                               static_cast<const int64_t*>(ctx.idx.p), static_cast<double2*>(ctx.M.p),
                                               static_cast<double*>(ctx.nrm.p), static_cast<double*>(ctx.nrm0.p),
                                               static_cast<int*>(ctx.perm.p), static_cast<int*>(ctx.kout.p),
                                               static_cast<double2*>(ctx.T.p), tol, kmax, (long long)maxn);
        CKG(cudaGetLastError());
        CKG(cudaDeviceSynchronize());
        std::vector<int> ks(njob);
        std::vector<int> perm((size_t)njob * maxn);
        CKG(cudaMemcpy(ks.data(), ctx.kout.p, njob * sizeof(int), cudaMemcpyDeviceToHost));
        CKG(cudaMemcpy(perm.data(), ctx.perm.p, perm.size() * sizeof(int), cudaMemcpyDeviceToHost));
        for (int q = 0; q < njob; ++q) {
            IdReply& r = out[j0 + q];
            const int n = jobs[q].n, k = ks[q];
            r.k = k;
            r.skel.assign(perm.begin() + (size_t)q * maxn, perm.begin() + (size_t)q * maxn + k);
            r.red.assign(perm.begin() + (size_t)q * maxn + k, perm.begin() + (size_t)q * maxn + n);
            const size_t nt = (size_t)k * (n - k);
            if (fp32) {
                // FP32 storage: convert reply by reply, so no phase-wide FP64 copy sits on the host
                tmp.resize(nt);
                if (nt)
                    CKG(cudaMemcpy(tmp.data(), static_cast<double2*>(ctx.T.p) + jobs[q].t_off, nt * sizeof(cplx),
                                   cudaMemcpyDeviceToHost));
                r.Tf.resize(nt);
                for (size_t i = 0; i < nt; ++i) r.Tf[i] = std::complex<float>((float)tmp[i].real(), (float)tmp[i].imag());
            } else {
                r.T.resize(nt);
                if (nt)
                    CKG(cudaMemcpy(r.T.data(), static_cast<double2*>(ctx.T.p) + jobs[q].t_off, nt * sizeof(cplx),
                                   cudaMemcpyDeviceToHost));
            }
        }
        j0 = j1;
    }
}

}  // namespace midbf
