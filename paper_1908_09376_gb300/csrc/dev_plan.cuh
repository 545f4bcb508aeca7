// Device plans and the launcher interface shared by the translation units of
// the device library: device.cu (plan upload, the apply, the autotuner, the
// C ABI) and the kernel launchers launch_rc.cu (interpolation stages, SIMT),
// launch_s.cu (middle factor, SIMT), launch_tc.cu (tensor cores) and
// batched.cu (many instances).  Splitting the launchers lets their kernel
// instantiations compile in parallel.
#pragma once

#include <algorithm>
#include <array>
#include <cstdio>
#include <functional>
#include <map>
#include <mutex>
#include <numeric>
#include <set>
#include <thread>
#include <tuple>
#include <type_traits>
#include <vector>

#include "internal.hpp"
#include "kernels.cuh"
#include "tc.cuh"

namespace midbf_gpu {

using namespace midbf;
using namespace midbf_dev;

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) fail(MIDBF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

constexpr int kRangeC = 64;   // output entries per pattern-C item
static_assert(kRangeC <= midbf_dev::kCgOut, "the column GEMM takes at most kCgOut outputs per item");
constexpr size_t kSmemCap = 200 * 1024;  // dynamic shared memory budget per CTA

struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
};

// The middle factor and the interpolation stage next to it (forward: S then
// the first U stage; adjoint: that U stage's adjoint then S's) can overlap:
// their blocks fall into groups such that each U block reads only outputs of
// S blocks in its own group, so the two stages run chunk by chunk, chunk k of
// the second stage on a side stream after chunk k of the first.  Work items
// of the two stages are stored grouped by chunk, and ck_* hold the item
// offsets of every chunk (kMaxChunks at most).
constexpr int kMaxChunks = 8;
constexpr int kDefaultChunks = 4;   // chunks prepared at creation and used by default

struct DevStageBase {
    int kind = KIND_V;
    int64_t in_len = 0, out_len = 0;
    bool out_user = false, in_user = false;
    int nchunks = 0;   // 0: the stage is not split
    int ck_r[kMaxChunks + 1] = {}, ck_c[kMaxChunks + 1] = {}, ck_c1[kMaxChunks + 1] = {};
    int ck_rows[kMaxChunks + 1] = {}, ck_rows4[kMaxChunks + 1] = {}, ck_cols[kMaxChunks + 1] = {},
        ck_cols4[kMaxChunks + 1] = {};
};

template <class R>
struct DevStage : DevStageBase {
    // ID stages (and stored S)
    bool id = false;
    IdStage<R> ids{};
    IdStage<R> ids1{};   // same data, items for the one-RHS pattern-C kernel
    int n_items_r = 0, n_items_c = 0, n_items_c1 = 0, rt = 1;
    int range_c1 = kRangeC1;   // outputs per one-RHS column item (smaller for stages of few wide blocks)
    int row_cl = 1;            // CTAs per cluster of the one-RHS row pattern by default (1: no cluster)
    int n_subs = 0, max_k = 0;          // interpolative decompositions of the stage, their largest rank
    int max_nred = 0, max_narrow = 0, max_nsub = 1;
    int n_blocks = 0, max_m = 0;        // blocks of an ID stage, their largest wide size
    // on-the-fly S
    SStage<R> ss{};
    SSide<R> srows{}, scols{};
    const int2* items_rows = nullptr;   // 64-row items (RT = 2)
    const int2* items_cols = nullptr;
    const int2* items_rows4 = nullptr;  // 128-row items (RT = 4)
    const int2* items_cols4 = nullptr;
    int n_items_rows = 0, n_items_cols = 0, n_items_rows4 = 0, n_items_cols4 = 0, rt_rows = 1, rt_cols = 1;
    int n4_rows_stage = 0, n4_cols_stage = 0;   // 128-row items of the whole stage (item-size rule)
    bool s_dist = false;                // square-root term in the distance form (DISTANCE phase)
    bool s_df = false;                  // accurate phase: double-FP32 (MIDBF_S_ONTHEFLY_DF)
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

// Compile-time phase shape of an on-the-fly middle factor: the distance form
// in both precisions; FP32 fixes the shapes of the other workload families,
// FP64 takes the general one.
template <class R>
inline int s_shape(const DevStage<R>& ds) {
    if (ds.s_dist) return kShapeDistance;
    return sizeof(R) == 4 ? phase_shape_code(ds.ss.P, ds.ss.Q) : 0;
}

}  // namespace midbf_gpu

struct midbf_dplan {
    int precision = MIDBF_FP32;   // storage: MIDBF_FP32 (also for the BF16 modes) or MIDBF_FP64
    int tc_mode = 0;              // 0: SIMT only; 1: BF16 tensor cores; 2: BF16 + refinement
    int* d_status = nullptr;      // device status word written by bounded waits
    int s_mode = MIDBF_S_ONTHEFLY;
    int device = 0;
    void* noalloc_scratch = nullptr;   // device address of midbf_apply_noalloc's scratch array
    std::string noalloc_err;           // why the lookup failed, when it did
    // overlap of the middle factor with its neighbouring U stage (see DevStageBase):
    // s_stage = index of the middle factor (-1: none); chunks_built = chunks prepared
    // at creation (0: none); chunks = chunks_built while the overlap is on, else 0.
    // Plans with chunks give the U stage's internal output space a third workspace
    // vector, since the stage before the middle factor reads the ping-pong buffer it
    // would otherwise write.
    int s_stage = -1;
    int chunks = 0;
    int chunks_built = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_ck[midbf_gpu::kMaxChunks] = {};
    mutable std::mutex pipe_mu;        // one overlapped apply of this plan issued at a time
    int64_t nx = 0, nw = 0;
    int64_t max_space = 0;        // longest internal vector space
    size_t factor_bytes = 0, index_bytes = 0;
    size_t pad_bytes = 0;   // of factor_bytes: the zero padding of the T columns (not algorithmic)
    size_t tc_image_bytes = 0;    // dense BF16 tile images (tensor-core modes)
    int max_tc_chunks = 0;        // most B-image chunks of one tensor-core stage launch
    std::vector<void*> allocs;
    std::vector<midbf_gpu::DevStage<float>> st32;
    std::vector<midbf_gpu::DevStage<double>> st64;
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
        for (cudaEvent_t e : ev_ck)
            if (e) cudaEventDestroy(e);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side) cudaStreamDestroy(side);
        if (d_status) cudaFree(d_status);
        for (void* p : allocs) cudaFree(p);
    }
};

namespace midbf_gpu {

// Raise a kernel's dynamic shared-memory limit to the library's cap (device.cu).
void set_smem_ptr(const void* kernel, size_t bytes);

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

// A forced RHS tile (from the autotuner) is taken when it is one of the
// compiled tiles and fits the shared-memory budget; otherwise pick_nr decides.
template <class R>
int forced_or_pick(int force, int nrhs, const std::function<size_t(int)>& smem) {
    const int cap = sizeof(R) == 4 ? 16 : 8;
    if (force > 0 && force <= cap && (force & (force - 1)) == 0 && smem(force) <= kSmemCap) return force;
    return pick_nr<R>(nrhs, smem);
}

// Grid of a persistent SIMT launch (device.cu).
int grid_for(const void* kernel, size_t smem, int nitems, bool persist);
int sm_count();
void launch_wait_selftest(int* status, int ctas, cudaStream_t s);

constexpr int kNarrowK = 48;      // one RHS: the narrow-ID kernels for stages whose ranks are all <= this
constexpr int kNarrowRed = 128;   // and (row pattern) whose IDs have at most this many redundant columns
constexpr int kNarrowWarps = 32;  // and (row pattern) at least this many IDs (one warp each) per SM
constexpr int kClusterCtasPerSm = 6;  // one RHS, row pattern: clusters when a stage has fewer items per SM
constexpr int kGemmMinRhs = 32;       // FP32 ID stages: the GEMM forms from this many RHS on
constexpr int kSGemmMinRhs = 128;     // FP32 middle factor on the fly: the GEMM form from this many RHS on
constexpr int kWarpBlocksPerSm = 16;  // narrow column pattern: a warp per block from this many blocks per SM
constexpr size_t kWarpBlockSmem = 64 * 1024;   // and while a CTA's 8 blocks fit this much shared memory
constexpr int kMaxRowCluster = 8;     // CTAs per cluster (the portable limit)
constexpr int kTcMinRhs = 16;     // tensor cores for the middle factor from this many RHS on
constexpr int kTcBlkMinRhs = 16;  // and for the V / U stages


// SIMT RHS tile named by a choice (0: none).
inline bool whole_choice(int choice) {   // a choice that takes no MIDBF_CHOICE_PERSIST bit
    return choice == MIDBF_CHOICE_TENSOR || choice == MIDBF_CHOICE_NARROW || choice == MIDBF_CHOICE_CLUSTER ||
           choice == MIDBF_CHOICE_GEMM;
}

// Whether a launch takes a register-tiled GEMM form (FP32 only): the middle
// factor made on the fly with the FP32 phase (k_s_gemm), or an ID stage or
// the stored middle factor in the row pattern (k_r_gemm) or the column
// pattern (k_c_gemm).  Asked for (MIDBF_CHOICE_GEMM), or by default: the row
// pattern from kGemmMinRhs RHS on; the column pattern from kGemmMinRhs RHS
// on when its IDs have 64 redundant columns or more (the tile has 64 column
// slots; on the 64-RHS FIO2D plan a stage of ~16 redundant columns per ID ran
// 1.5x slower than the SIMT tiles); the middle factor made on the fly from
// kSGemmMinRhs RHS on (at 64 RHS the 16-RHS SIMT tile, which makes every
// entry four times, was 7% faster).
template <class R>
inline bool use_gemm(const DevStage<R>& ds, int nrhs, int choice, bool row_pattern) {
    if (sizeof(R) != 4 || (!ds.id && ds.s_df)) return false;
    if (choice == MIDBF_CHOICE_GEMM) return true;
    if (choice != MIDBF_CHOICE_DEFAULT) return false;
    if (!ds.id) return nrhs >= kSGemmMinRhs;
    return nrhs >= kGemmMinRhs && (row_pattern || ds.max_nred >= 64);
}

inline int choice_tile(int choice) {
    const int base = whole_choice(choice) ? 0 : (choice & ~MIDBF_CHOICE_PERSIST);
    return base >= 1 && base <= 16 ? base : 0;
}

inline bool valid_choice(int choice) {
    if (whole_choice(choice)) return true;
    const int base = choice & ~MIDBF_CHOICE_PERSIST;
    return base == MIDBF_CHOICE_DEFAULT || base == MIDBF_CHOICE_COLUMN1 || base == 1 || base == 2 || base == 4 ||
           base == 8 || base == 16;
}

// Whether a one-RHS ID-stage launch takes the narrow-ID kernels: asked for
// (MIDBF_CHOICE_NARROW), or by default when every rank is at most kNarrowK
// and, for the row pattern (a warp walks all the redundant columns of its ID
// alone), every ID has at most kNarrowRed redundant columns and the stage has
// at least kNarrowWarps IDs per SM; never for a stage prepared for the
// overlap (those launch chunks of items).  Measured on one GB300: the
// paper-grid plan of Example 1 at n = 1024 (ranks ~11, ~33 redundant
// columns, 16,384 IDs per stage) runs its stages in about half the time;
// Example 2's leaf IDs (rank 44, 468 redundant columns) ran 5x slower in the
// row pattern, with too few warps for the serial column walk, and so did the
// n = 256 paper-grid plan (1,024 IDs per stage: 7 warps per SM) by 3-4x.
template <class R>
inline bool use_narrow(const DevStage<R>& ds, int nrhs, int choice, bool row_pattern) {
    if (nrhs != 1 || !ds.id || ds.nchunks != 0 || ds.max_k > 64) return false;
    if (choice == MIDBF_CHOICE_NARROW) return true;
    return choice == MIDBF_CHOICE_DEFAULT && ds.max_k <= kNarrowK &&
           (!row_pattern || (ds.max_nred <= kNarrowRed && ds.n_subs >= kNarrowWarps * sm_count()));
}

// Cluster size of the one-RHS row pattern for a stage of n_items row items
// whose IDs have at most max_nred redundant columns: 1 when the stage has
// kClusterCtasPerSm items per SM or more, else enough CTAs per item to reach
// that, at most kMaxRowCluster and with ~4 columns per warp at least.  Fixed
// per stage when the plan is made, so every launch of the stage (whole, by
// chunks, or in a batch) splits the columns alike.
inline int row_cluster_size(int n_items, int max_nred) {
    const int target = kClusterCtasPerSm * sm_count();
    if (n_items <= 0 || n_items >= target) return 1;
    int cl = std::min(kMaxRowCluster, (target + n_items - 1) / n_items);
    while (cl > 1 && max_nred < 4 * kWarps * cl) --cl;
    return cl;
}

// The cluster size of a one-RHS row-pattern launch of stage ds under a choice:
// the stage's default size, at least 2 when asked for (MIDBF_CHOICE_CLUSTER),
// 1 under any other choice.
template <class R>
inline int row_cluster_for(const DevStage<R>& ds, int choice) {
    if (choice == MIDBF_CHOICE_CLUSTER) return std::max(2, ds.row_cl);
    return choice == MIDBF_CHOICE_DEFAULT ? ds.row_cl : 1;
}

// Internal vectors of the workspace: the two ping-pong vectors, and a third
// one when the middle factor overlaps its U stage.
inline int vec_buffers(const midbf_dplan* dp) { return dp->chunks_built > 1 ? 3 : 2; }

// Bytes of the workspace's internal vectors, rounded up to 256.
inline size_t vec_workspace_bytes(const midbf_dplan* dp, int nrhs) {
    const size_t ce = dp->precision == MIDBF_FP32 ? 8 : 16;
    const size_t b = (size_t)vec_buffers(dp) * (size_t)std::max<int64_t>(dp->max_space, 1) * (size_t)nrhs * ce;
    return (b + 255) / 256 * 256;
}

inline size_t tc_bimg_bytes(const midbf_dplan* dp, int nrhs) {
    if (!dp->tc_mode || dp->max_tc_chunks == 0) return 0;
    const int Rpad = (std::min(nrhs, kTcR) + 15) & ~15;
    const size_t b = (size_t)dp->max_tc_chunks * tc_bimg_elems(Rpad, dp->tc_mode == 2) * 2;
    return (b + 255) / 256 * 256;
}

// Choice recorded by the autotuner (or midbf_set_choice) for this RHS count,
// stage and direction; MIDBF_CHOICE_DEFAULT when there is none (device.cu).
int tuned_choice(const midbf_dplan* dp, int nrhs, int sidx, bool adjoint);

// ---- kernel launchers (defined in the launcher units for float and double)
template <class R>
void launch_r(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, bool conj, cudaStream_t s, int force = 0,
              bool persist = false);
template <class R>
void launch_c(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, bool conj, cudaStream_t s, int force = 0,
              bool persist = false);
template <class R>
void launch_r_narrow(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, bool conj, cudaStream_t s);
template <class R>
void launch_r_cluster(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, bool conj, int cl, cudaStream_t s);
template <class R>
void launch_c_narrow(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, bool conj, cudaStream_t s);
template <class R>
void launch_s(const DevStage<R>& ds, VecRef<R> src, VecRef<R> dst, int nrhs, bool adjoint, cudaStream_t s,
              int force = 0, bool persist = false);
void launch_s_gemm(const DevStage<float>& ds, VecRef<float> src, VecRef<float> dst, int nrhs, bool adjoint,
                   cudaStream_t s);
void launch_c_gemm(const DevStage<float>& ds, VecRef<float> src, VecRef<float> dst, int nrhs, bool conj,
                   cudaStream_t s);
void launch_r_gemm(const DevStage<float>& ds, VecRef<float> src, VecRef<float> dst, int nrhs, bool conj,
                   cudaStream_t s);
void launch_tc(const DevStage<float>& ds, VecRef<float> src, VecRef<float> dst, int nrhs, bool adjoint, bool refine,
               __nv_bfloat16* bimg, int* status, cudaStream_t s);
void launch_blk_tc(const DevStage<float>& ds, int o, VecRef<float> src, VecRef<float> dst, int nrhs, bool refine,
                   __nv_bfloat16* bimg, int* status, cudaStream_t s);
size_t instance_workspace(const midbf_dplan* dp, int nrhs);
template <class R>
int run_batched(int count, const midbf_dplan* const* dps, const int* adjoint, const void* const* in,
                const int64_t* ldin, void* const* out, const int64_t* ldout, const int* nrhs, cudaStream_t s,
                char* ws, bool dry = false);

}  // namespace midbf_gpu
