// Internal host-side data structures of the MIDBF library.
//
// A plan is the factor product of eq. (finishIDBF) of Sec. 3.5 held as a list
// of stages in forward order (V stages, the middle factor S, U stages).  Each
// stage is a list of blocks with explicit position maps between vector
// spaces: stage s reads the output space of stage s-1 (the user input for the
// first stage) and writes its own output space (the user output for the last
// stage).
//
//  * V block: its input (the "wide" side, m entries) is gathered, and each of
//    its interpolative decompositions (sub-blocks) writes k entries of the
//    output (the "narrow" side): out_c = in[skel_c] + T_c in[red_c]
//    (Sec. 3.2, V = [I T] Lambda^T).
//  * U block: the narrow side is its input (k entries per sub-block), the wide
//    side its output: out = sum_c U_c in_c with U_c = Lambda [I T_c]^T.
//  * S block: out = K(xidx, widx) in, entries kernel values (Sec. 3.5).
#pragma once

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/midbf.h"

namespace midbf {

using cplx = std::complex<double>;

enum StageKind { KIND_V = 0, KIND_S = 1, KIND_U = 2 };

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

[[noreturn]] inline void fail(int code, const std::string& msg) { throw Error(code, msg); }

struct Sub {
    int32_t k = 0;               // rows of the ID (narrow entries)
    int32_t m = 0;               // wide size (block input for V, output for U)
    std::vector<int32_t> skel;   // k positions in [0, m)
    std::vector<int32_t> red;    // m - k positions
    std::vector<cplx> T;         // k x (m - k), row-major (FP64 storage)
    std::vector<std::complex<float>> Tf;   // the same in FP32 (params.store_fp32); then T is empty
    size_t t_size() const { return Tf.empty() ? T.size() : Tf.size(); }
    cplx t(size_t i) const { return Tf.empty() ? T[i] : cplx(Tf[i].real(), Tf[i].imag()); }
    // keep T in FP32 only
    void to_fp32() {
        Tf.resize(T.size());
        for (size_t i = 0; i < T.size(); ++i) Tf[i] = std::complex<float>((float)T[i].real(), (float)T[i].imag());
        std::vector<cplx>().swap(T);
    }
};

struct Block {
    std::vector<int64_t> in_idx;   // positions in the input space
    std::vector<int64_t> out_idx;  // positions in the output space
    std::vector<Sub> subs;         // V / U blocks
    std::vector<int64_t> xidx;     // S blocks: X point of each row
    std::vector<int64_t> widx;     // S blocks: Omega point of each column
};

struct Stage {
    int32_t kind = KIND_V;
    int32_t in_space = -1;   // -1: user input vector
    int32_t out_user = 0;    // 1: output space is the user output vector
    int64_t out_len = 0;
    std::vector<Block> blocks;
};

// Phase function over index pairs (rows in X, columns in Omega).
struct Phase {
    int family = 0;
    int d = 2;
    int64_t nx = 0, nw = 0;
    std::vector<double> X, W;   // row-major coordinates
    int r = 0;                  // low-rank terms (family LOWRANK)
    std::vector<double> U, V;   // row-major nx x r, nw x r

    double eval_xy(const double* x, const double* w) const;
    double operator()(int64_t i, int64_t j) const {
        if (family == MIDBF_PHASE_LOWRANK) {
            double s = 0.0;
            const double* u = &U[(size_t)i * r];
            const double* v = &V[(size_t)j * r];
            for (int t = 0; t < r; ++t) s += u[t] * v[t];
            return s;
        }
        return eval_xy(&X[(size_t)i * d], &W[(size_t)j * d]);
    }
    // K(xi[a], wj[b]) into out[a * sx + b * sw] for a < na, b < nb: the same
    // formulas as kernel(), with the parts that depend on one point only
    // (the FIO coefficients c_k(x), |xi|, ...) evaluated once per point.
    void kernel_block(const int64_t* xi, size_t na, const int64_t* wj, size_t nb, cplx* out, size_t sx,
                      size_t sw) const;
    // exp(2 pi i Phi), Phi reduced modulo one first.
    cplx kernel(int64_t i, int64_t j) const {
        double p = (*this)(i, j);
        p -= std::nearbyint(p);
        double s, c;
        sincos(2.0 * M_PI * p, &s, &c);
        return cplx(c, s);
    }
};

struct Plan {
    bool released = false;   // ID coefficients handed to a device plan (midbf_dplan_create_ex)
    int d = 2, L = 0, delta = 1, nsteps = 0;
    double tol = 0.0;
    Phase phase;
    std::vector<Stage> stages;
    int64_t nx() const { return phase.nx; }
    int64_t nw() const { return phase.nw; }
};

// plan.cpp
std::vector<uint8_t> plan_serialize(const Plan& p);
std::unique_ptr<Plan> plan_deserialize(const uint8_t* buf, size_t len);
void plan_validate(const Plan& p);
void plan_stats(const Plan& p, midbf_stats* st);

// phase.cpp
void phase_check(const Phase& ph);

// build.cpp
std::unique_ptr<Plan> build_plan(const Phase& ph, const midbf_params& prm);

// recover.cpp
// device = true: every vector recovery of Algorithm 4 (the detection along the
// root row and column, and each piece of Algorithm 6) runs on the current CUDA
// device (recover_gpu.cu); the results are the same bit for bit.
std::unique_ptr<Phase> recover_phase(int d, int64_t nx, const double* X, int64_t nw, const double* W,
                                     const midbf_access& acc, int r, int q, double tau, int max_disc,
                                     uint64_t seed, midbf_recover_info* info, bool device = false);

// recover_gpu.cu: Algorithm 4 on the device.  device_recover_along recovers the
// host vectors vs[k] (start values in place) from the observations us[k]
// along the edges E of a path piece rooted at root; device_detect returns D
// (the path root, then the flagged children in path order) for u along P.
void device_recover_along(int64_t n, const std::vector<std::pair<int64_t, int64_t>>& E, int64_t root,
                          const std::vector<const double*>& us, const std::vector<double*>& vs);
std::vector<int64_t> device_detect(const std::vector<double>& u, const std::vector<std::pair<int64_t, int64_t>>& P,
                                   double tau);

// qr.cpp: column interpolative decomposition of a dense column-major matrix
struct IdResult {
    std::vector<int32_t> skel, red;
    std::vector<cplx> T;     // k x (n - k) row-major
    std::vector<double> rdiag;
};
// A is ms x n column-major (lda = ms); overwritten.
IdResult column_id(std::vector<cplx>& A, int ms, int n, double tol, int kmax);

void set_last_error(const std::string& s);

// build_gpu.cu: batched column IDs on the current CUDA device.
struct IdRequest {
    const std::vector<int64_t>* cols;   // decomposed point indices (n)
    std::vector<int64_t> samples;       // sample point indices on the other side (ns)
    bool cols_x;                        // decomposed points are X points
};
struct IdReply {
    int k = 0;
    std::vector<int32_t> skel, red;
    std::vector<cplx> T;                // k x (n - k) row-major
    std::vector<std::complex<float>> Tf;   // the same in FP32 (fp32 requested; then T is empty)
};
struct GpuIdContext;
std::unique_ptr<GpuIdContext, void (*)(GpuIdContext*)> gpu_id_context(const Phase& ph);
void gpu_id_batch(GpuIdContext& ctx, const std::vector<IdRequest>& reqs, double tol, int kmax,
                  std::vector<IdReply>& out, bool fp32 = false);

}  // namespace midbf
