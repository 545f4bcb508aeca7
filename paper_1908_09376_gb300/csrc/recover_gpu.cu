// Vector recovery (Algorithm 4, Sec. 2.3) on the GPU.
//
// Along a recovery path P (Def. 3.3: edges (parent bg, child ed) in
// breadth-first order), Algorithm 4 fixes the unwrapped value of every child
// from its parent's:  v(ed) = u(ed) - round(u(ed) - v(bg)), with round half
// away from zero, and flags ed as a discontinuity when |v(ed) - v(bg)| >= tau.
// An edge reads only its parent's final value, so all edges whose parents
// were fixed by earlier edges can run at once: the path is cut into runs of
// consecutive edges none of which has its parent set inside the same run
// (for a breadth-first path, one run per depth of the tree), and the runs run
// one after the other.  Each edge performs exactly the FP64 operations of the
// sequential loop, so the result is the same bit for bit, and so are the
// flags.  D (the root, then the children of the flagged edges in path order)
// is compacted on the device with a block scan.
//
// One CTA per vector: the 8 + 8 sampled rows and columns of Algorithm 7 (and
// the ones added for discontinuities) are recovered by one launch per path.
// The path (Algorithm 5's minimum spanning tree and its breadth-first order)
// is built on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.hpp"

#define RCK(call)                                                                                    \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) midbf::fail(MIDBF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

namespace {

constexpr int kRecThreads = 512;

// MATLAB's round: half away from zero.
__device__ __forceinline__ double round_half_away(double x) { return x >= 0.0 ? floor(x + 0.5) : -floor(-x + 0.5); }

__global__ void __launch_bounds__(kRecThreads) k_recover_path(const int* __restrict__ par, const int* __restrict__ chi,
                                                             const int* __restrict__ run_off, int nruns, int nedges,
                                                             int root, const double* __restrict__ u, long long ldu,
                                                             double* v, long long ldv, double tau, unsigned char* flags,
                                                             long long ldf, long long* D, long long ldD,
                                                             long long* nD) {
    const long long vec = blockIdx.x;
    const double* uu = u + vec * ldu;
    double* vv = v + vec * ldv;
    unsigned char* ff = flags ? flags + vec * ldf : nullptr;
    for (int r = 0; r < nruns; ++r) {
        const int e1 = run_off[r + 1];
        for (int e = run_off[r] + threadIdx.x; e < e1; e += blockDim.x) {
            const int p = par[e], c = chi[e];
            const double vb = __ldcg(vv + p);   // fixed by an earlier run (or the start value)
            const double uc = uu[c];
            const double vc = uc - round_half_away(uc - vb);
            __stcg(vv + c, vc);
            if (ff) ff[e] = fabs(vc - vb) >= tau ? 1 : 0;
        }
        __syncthreads();   // the run's values are visible to the whole CTA before the next run reads them
    }
    if (!D) return;
    // D: root, then the children of flagged edges in path order (block scan of the flags)
    __shared__ int warp_cnt[kRecThreads / 32];
    __shared__ long long base;
    long long* dd = D + vec * ldD;
    if (threadIdx.x == 0) {
        dd[0] = root;
        base = 1;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e0 = 0; e0 < nedges; e0 += blockDim.x) {
        const int e = e0 + threadIdx.x;
        const bool f = e < nedges && ff[e] != 0;
        const unsigned m = __ballot_sync(0xffffffffu, f);
        if (lane == 0) warp_cnt[w] = __popc(m);
        __syncthreads();
        int off = 0, total = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            if (k < w) off += warp_cnt[k];
            total += warp_cnt[k];
        }
        if (f) dd[base + off + __popc(m & ((1u << lane) - 1u))] = chi[e];
        __syncthreads();
        if (threadIdx.x == 0) base += total;
        __syncthreads();
    }
    if (threadIdx.x == 0 && nD) nD[vec] = base;
}

}  // namespace

// A recovery path (or a piece of one) resident on one device.
struct midbf_rpath {
    int64_t n = 0, nedges = 0, root = 0;
    int nruns = 0;
    int device = 0;
    int* par = nullptr;
    int* chi = nullptr;
    int* runs = nullptr;
    ~midbf_rpath() {
        if (par) cudaFree(par);
        if (chi) cudaFree(chi);
        if (runs) cudaFree(runs);
    }
};

namespace midbf {

namespace {

// Validate the edges (every parent already reached from root, every child
// reached once) and cut them into runs; then upload to the current device.
std::unique_ptr<midbf_rpath> make_rpath(int64_t n, int64_t nedges, const int64_t* edges, int64_t root) {
    if (n <= 0 || n >= (int64_t(1) << 31)) fail(MIDBF_EINVAL, "path length must be in [1, 2^31)");
    if (nedges < 0 || nedges > n - 1 || (nedges > 0 && !edges)) fail(MIDBF_EINVAL, "bad edge count");
    if (root < 0 || root >= n) fail(MIDBF_EINVAL, "root out of range");
    std::vector<int> par(nedges), chi(nedges), runs{0};
    std::vector<int> run_of(n, -2);   // run that fixed the node; -1: the root; -2: not reached
    run_of[root] = -1;
    int cur = 0;
    for (int64_t e = 0; e < nedges; ++e) {
        const int64_t p = edges[2 * e], c = edges[2 * e + 1];
        if (p < 0 || p >= n || c < 0 || c >= n) fail(MIDBF_EINVAL, "edge index out of range");
        if (run_of[p] == -2) fail(MIDBF_EINVAL, "edge " + std::to_string(e) + ": parent not reached by earlier edges");
        if (run_of[c] != -2) fail(MIDBF_EINVAL, "edge " + std::to_string(e) + ": child reached twice");
        if (run_of[p] == cur) {   // parent fixed in the current run: the edge starts a new one
            runs.push_back((int)e);
            ++cur;
        }
        run_of[c] = cur;
        par[e] = (int)p;
        chi[e] = (int)c;
    }
    if (nedges > 0) runs.push_back((int)nedges);
    auto rp = std::make_unique<midbf_rpath>();
    rp->n = n;
    rp->nedges = nedges;
    rp->root = root;
    rp->nruns = (int)runs.size() - 1;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) fail(MIDBF_ECUDA, "no CUDA device");
    RCK(cudaGetDevice(&rp->device));
    if (nedges > 0) {
        RCK(cudaMalloc(&rp->par, nedges * sizeof(int)));
        RCK(cudaMalloc(&rp->chi, nedges * sizeof(int)));
        RCK(cudaMalloc(&rp->runs, runs.size() * sizeof(int)));
        RCK(cudaMemcpy(rp->par, par.data(), nedges * sizeof(int), cudaMemcpyHostToDevice));
        RCK(cudaMemcpy(rp->chi, chi.data(), nedges * sizeof(int), cudaMemcpyHostToDevice));
        RCK(cudaMemcpy(rp->runs, runs.data(), runs.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    return rp;
}

void launch_recover(const midbf_rpath& rp, int nvec, const double* u, int64_t ldu, double* v, int64_t ldv, double tau,
                    uint8_t* flags, int64_t ldf, int64_t* D, int64_t ldD, int64_t* nD, cudaStream_t s) {
    if (nvec <= 0) return;
    k_recover_path<<<nvec, kRecThreads, 0, s>>>(rp.par, rp.chi, rp.runs, rp.nruns, (int)rp.nedges, (int)rp.root, u,
                                                (long long)ldu, v, (long long)ldv, tau, flags, (long long)ldf,
                                                reinterpret_cast<long long*>(D), (long long)ldD,
                                                reinterpret_cast<long long*>(nD));
    RCK(cudaGetLastError());
}

// Device buffers of one host-side recovery call, freed on every exit.
struct DevScratch {
    std::vector<void*> p;
    void* get(size_t bytes) {
        void* q = nullptr;
        if (bytes && cudaMalloc(&q, bytes) != cudaSuccess) fail(MIDBF_ENOMEM, "cudaMalloc for the recovery failed");
        p.push_back(q);
        return q;
    }
    ~DevScratch() {
        for (void* q : p)
            if (q) cudaFree(q);
    }
};

std::vector<int64_t> flat(const std::vector<std::pair<int64_t, int64_t>>& E) {
    std::vector<int64_t> f(2 * E.size());
    for (size_t e = 0; e < E.size(); ++e) {
        f[2 * e] = E[e].first;
        f[2 * e + 1] = E[e].second;
    }
    return f;
}

}  // namespace

void device_recover_along(int64_t n, const std::vector<std::pair<int64_t, int64_t>>& E, int64_t root,
                          const std::vector<const double*>& us, const std::vector<double*>& vs) {
    if (E.empty() || us.empty()) return;
    const std::vector<int64_t> f = flat(E);
    auto rp = make_rpath(n, (int64_t)E.size(), f.data(), root);
    const int nvec = (int)us.size();
    DevScratch sc;
    double* du = static_cast<double*>(sc.get((size_t)nvec * n * sizeof(double)));
    double* dv = static_cast<double*>(sc.get((size_t)nvec * n * sizeof(double)));
    for (int k = 0; k < nvec; ++k) {
        RCK(cudaMemcpy(du + (size_t)k * n, us[k], n * sizeof(double), cudaMemcpyHostToDevice));
        RCK(cudaMemcpy(dv + (size_t)k * n, vs[k], n * sizeof(double), cudaMemcpyHostToDevice));
    }
    launch_recover(*rp, nvec, du, n, dv, n, 1.0, nullptr, 0, nullptr, 0, nullptr, 0);
    for (int k = 0; k < nvec; ++k)
        RCK(cudaMemcpy(vs[k], dv + (size_t)k * n, n * sizeof(double), cudaMemcpyDeviceToHost));
}

std::vector<int64_t> device_detect(const std::vector<double>& u, const std::vector<std::pair<int64_t, int64_t>>& P,
                                   double tau) {
    const int64_t n = (int64_t)u.size();
    const int64_t root = P.empty() ? 0 : P[0].first;
    if (P.empty()) return {root};
    const std::vector<int64_t> f = flat(P);
    auto rp = make_rpath(n, (int64_t)P.size(), f.data(), root);
    DevScratch sc;
    const int64_t ne = (int64_t)P.size();
    double* du = static_cast<double*>(sc.get(n * sizeof(double)));
    double* dv = static_cast<double*>(sc.get(n * sizeof(double)));
    uint8_t* df = static_cast<uint8_t*>(sc.get(ne));
    int64_t* dD = static_cast<int64_t*>(sc.get((ne + 1) * sizeof(int64_t)));
    int64_t* dn = static_cast<int64_t*>(sc.get(sizeof(int64_t)));
    RCK(cudaMemcpy(du, u.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    RCK(cudaMemcpy(dv, u.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    launch_recover(*rp, 1, du, n, dv, n, tau, df, ne, dD, ne + 1, dn, 0);
    int64_t cnt = 0;
    RCK(cudaMemcpy(&cnt, dn, sizeof(int64_t), cudaMemcpyDeviceToHost));
    if (cnt < 1 || cnt > ne + 1) fail(MIDBF_EINTERNAL, "discontinuity count out of range");
    std::vector<int64_t> D((size_t)cnt);
    RCK(cudaMemcpy(D.data(), dD, cnt * sizeof(int64_t), cudaMemcpyDeviceToHost));
    return D;
}

}  // namespace midbf

// ---------------------------------------------------------------------------
// C ABI
extern "C" {

int midbf_rpath_create(int64_t n, int64_t nedges, const int64_t* edges, int64_t root, midbf_rpath** out) {
    try {
        if (!out) midbf::fail(MIDBF_EINVAL, "null argument");
        *out = midbf::make_rpath(n, nedges, edges, root).release();
        return MIDBF_OK;
    } catch (const midbf::Error& e) {
        midbf::set_last_error(e.what());
        return e.code;
    } catch (const std::bad_alloc&) {
        midbf::set_last_error("host allocation failed");
        return MIDBF_ENOMEM;
    }
}

void midbf_rpath_destroy(midbf_rpath* p) { delete p; }

int midbf_rpath_info(const midbf_rpath* p, int64_t* n, int64_t* nedges, int* nruns) {
    if (!p) {
        midbf::set_last_error("midbf_rpath_info: null path");
        return MIDBF_EINVAL;
    }
    if (n) *n = p->n;
    if (nedges) *nedges = p->nedges;
    if (nruns) *nruns = p->nruns;
    return MIDBF_OK;
}

int midbf_recover_vectors(const midbf_rpath* p, int nvec, const double* u, int64_t ldu, double* v, int64_t ldv,
                          double tau, uint8_t* flags, int64_t ldf, int64_t* D, int64_t ldD, int64_t* nD,
                          void* stream) {
    try {
        if (!p || nvec < 0 || (nvec > 0 && (!u || !v))) midbf::fail(MIDBF_EINVAL, "bad argument");
        if (ldu < p->n || ldv < p->n) midbf::fail(MIDBF_EINVAL, "leading dimension smaller than the path length");
        if (flags && ldf < p->nedges) midbf::fail(MIDBF_EINVAL, "flag leading dimension smaller than the edge count");
        if (D && (!flags || ldD < p->nedges + 1)) midbf::fail(MIDBF_EINVAL, "D needs flags and ldD >= edges + 1");
        if (!(tau > 0.0)) midbf::fail(MIDBF_EINVAL, "tau must be positive");
        int dev = 0;
        RCK(cudaGetDevice(&dev));
        if (dev != p->device) midbf::fail(MIDBF_EINVAL, "the current device is not the device of this path");
        const char* ub = reinterpret_cast<const char*>(u);
        const char* vb = reinterpret_cast<const char*>(v);
        const size_t vbytes = ((size_t)(nvec > 0 ? nvec - 1 : 0) * ldv + p->n) * sizeof(double);
        const size_t ubytes = ((size_t)(nvec > 0 ? nvec - 1 : 0) * ldu + p->n) * sizeof(double);
        if (nvec > 0 && ub < vb + vbytes && vb < ub + ubytes) midbf::fail(MIDBF_EINVAL, "u and v overlap");
        midbf::launch_recover(*p, nvec, u, ldu, v, ldv, tau, flags, ldf, D, ldD, nD, static_cast<cudaStream_t>(stream));
        return MIDBF_OK;
    } catch (const midbf::Error& e) {
        midbf::set_last_error(e.what());
        return e.code;
    }
}

}  // extern "C"
