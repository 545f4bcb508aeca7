/*
 * midbf.h - C ABI of the GB300 MIDBF library.
 *
 * The library applies the multidimensional interpolative decomposition
 * butterfly factorization (MIDBF) of K(x, xi) = exp(2 pi i Phi(x, xi)) and of
 * its adjoint to vectors on one GPU (Chen, Zhang, Ho, Yang, "Multidimensional
 * Phase Recovery and Interpolative Decomposition Butterfly Factorization").
 * The calls follow the paper's statement of the problem (Sec. 1, eq. (1)):
 *
 *   1. a phase Phi: a closed form (Scenario 1 of Table 1), a low-rank factor
 *      pair Psi = U V^T, or one recovered from a few rows and columns of K
 *      (Scenario 2, Algorithm 7);
 *   2. midbf_build: the butterfly factors from kernel samples (Sec. 3);
 *   3. midbf_dplan_create + midbf_apply: g = K f or f = K^H g on the GPU.
 *
 * Conventions for every function:
 *   - Return value: MIDBF_OK (0) or a negative MIDBF_E* code.  On failure a
 *     human-readable message is available from midbf_last_error() (per
 *     thread) and no output handle is written.
 *   - Handles (midbf_phase, midbf_plan, midbf_dplan) are owned by the caller
 *     after creation and released with the matching *_destroy call.  Host
 *     arrays passed in are copied; the library keeps no pointer to them.
 *   - Indices are 0-based.  Coordinates are row-major (n x d) doubles.
 *   - Complex vectors are interleaved (re, im) pairs: double (complex128) for
 *     MIDBF_FP64, float (complex64) for MIDBF_FP32.  Multiple right-hand sides
 *     are stored column-major: entry p of RHS r at offset r * ld + p.
 *   - Nothing here falls back to the CPU: apply calls need a CUDA device and
 *     fail with MIDBF_ECUDA when none is present.
 */
#ifndef MIDBF_H
#define MIDBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MIDBF_OK          0
#define MIDBF_EINVAL     -1   /* bad argument, size or handle                 */
#define MIDBF_ENOMEM     -2   /* host or device allocation failed             */
#define MIDBF_ECUDA      -3   /* a CUDA runtime call failed / no device        */
#define MIDBF_ECALLBACK  -4   /* a caller-supplied access callback failed      */
#define MIDBF_ERANK      -5   /* a rank cap was hit before the tolerance       */
#define MIDBF_ERECOVERY  -6   /* phase recovery could not proceed              */
#define MIDBF_ETIMEOUT   -7   /* a device-side bounded wait gave up            */
#define MIDBF_EINTERNAL  -8   /* inconsistent plan or internal error           */
#define MIDBF_EFORMAT    -9   /* malformed plan file                           */

/* ---- phase families (Scenario 1 closed forms) -------------------------- */
#define MIDBF_PHASE_FIO2D       1 /* x.xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2), Sec. 4 Example 1 */
#define MIDBF_PHASE_FIO3D       2 /* x.xi + sqrt(sum c_k^2 xi_k^2), c_k=(2+sin2pi x_k cos2pi x_{k+1})/16 */
#define MIDBF_PHASE_FIO2D_JUMP  3 /* FIO2D + 0.5 |xi| sign(x1 - 0.5), sign(0) = +1 */
#define MIDBF_PHASE_DOT         4 /* x.xi (Fourier, Sec. 4 Example 2)              */
#define MIDBF_PHASE_ZERO        5 /* 0 (rank-one K)                                */
#define MIDBF_PHASE_SEPARABLE   6 /* sum_k sin(2 pi x_k) + 0.05 sum_k xi_k^2        */
#define MIDBF_PHASE_LOWRANK     7 /* Psi(i, j) = sum_t U[i,t] V[j,t] (Algorithm 7)  */
#define MIDBF_PHASE_DISTANCE    8 /* |x - xi|_2: the Helmholtz phase h |x - xi| of
                                     Sec. 4 Example 3 with h folded into the points */

/* ---- apply precisions -------------------------------------------------- */
#define MIDBF_FP64  0   /* plain form: complex128 data and arithmetic          */
#define MIDBF_FP32  1   /* mixed form: complex64 data and arithmetic           */
#define MIDBF_BF16  2   /* complex64 data; with 16 or more right-hand sides the
                           middle factor runs on the tensor cores (tcgen05, BF16
                           operands, FP32 accumulation)                        */
#define MIDBF_REFINE 16 /* flag for MIDBF_BF16: split operands into BF16 hi + lo
                           and add the refinement products A_hi B_lo + A_lo B_hi */

/* ---- middle-factor modes ----------------------------------------------- */
#define MIDBF_S_ONTHEFLY 0  /* S entries exp(2 pi i Phi) generated in the kernel */
#define MIDBF_S_STORED   1  /* S entries precomputed once at dplan creation      */
#define MIDBF_S_ONTHEFLY_DF 2 /* on the fly with the accurate phase (MIDBF_FP32 plans,
                           inner-product phases): the phase of every entry in
                           double-FP32 arithmetic (TwoSum / TwoProduct error-free
                           transformations), so its rounding no longer grows with
                           the phase's magnitude; about 3x the middle factor's
                           arithmetic.  Not taken by midbf_apply_batched.       */

typedef struct midbf_phase midbf_phase;  /* phase function over (X, Omega)   */
typedef struct midbf_plan midbf_plan;    /* host butterfly factors (immutable) */
typedef struct midbf_dplan midbf_dplan;  /* device-resident copy of a plan    */

/* Thread-local description of the last failure on this thread ("" if none). */
const char* midbf_last_error(void);

/* Library version string. */
const char* midbf_version(void);

/* ---- phases -------------------------------------------------------------
 * midbf_phase_closed_form: Phi of one of the MIDBF_PHASE_* closed forms over
 * the point sets X (nx x d) and W (nw x d), d = 2 or 3.  FIO2D/FIO2D_JUMP need
 * d = 2, FIO3D needs d = 3.  For h |x - xi| pass h X and h W with DISTANCE.
 * Errors: MIDBF_EINVAL.
 */
int midbf_phase_closed_form(int family, int d, int64_t nx, const double* X,
                            int64_t nw, const double* W, midbf_phase** out);

/* midbf_phase_lowrank: Psi(i, j) = sum_t U[i*r + t] V[j*r + t] (U nx x r,
 * V nw x r, row-major), the output form of Algorithm 7 (Sec. 2.3).  X and W
 * are still required: the butterfly trees are built over them. */
int midbf_phase_lowrank(int d, int64_t nx, const double* X, int64_t nw, const double* W,
                        int r, const double* U, const double* V, midbf_phase** out);

/* Indirect access to K (Scenario 2 of Table 1): rows_fn writes K(idx[c], :)
 * for c < cnt into out[c * nw + j] (interleaved complex128); cols_fn writes
 * K(:, idx[c]) into out[c * nx + i].  Return 0 on success, nonzero to abort
 * (reported as MIDBF_ECALLBACK). */
typedef int (*midbf_rows_fn)(void* user, const int64_t* idx, int64_t cnt, double* out);
typedef struct {
    midbf_rows_fn rows_fn;
    midbf_rows_fn cols_fn;
    void* user;
} midbf_access;

typedef struct {
    int64_t rows_requested;   /* rows fetched through rows_fn                  */
    int64_t cols_requested;   /* columns fetched through cols_fn               */
    int64_t disc_rows;        /* |D_r| - 1: discontinuities found along X      */
    int64_t disc_cols;        /* |D_c| - 1                                      */
    double tau;               /* detection threshold finally used              */
    int64_t mismatches;       /* recovered rows and columns disagreeing (Lemma 3.2) */
} midbf_recover_info;

/* midbf_phase_recover: Algorithm 7 (with Algorithms 1, 4, 5, 6).  Samples
 * r*q rows and columns (index 0 plus seeded random ones), recovers them along
 * Euclidean-MST recovery paths of X and W (Def. 3.3), and factors the result
 * with the restricted randomized SVD into a rank-r phase.  tau: initial
 * discontinuity threshold (paper: 1/4), raised by 1/40 while more than
 * max_disc discontinuities are found, at most to 1/2.  info may be NULL.
 * Errors: MIDBF_EINVAL, MIDBF_ECALLBACK (a callback failed, or returned a
 * non-finite or zero value, which has no phase), MIDBF_ERECOVERY. */
int midbf_phase_recover(int d, int64_t nx, const double* X, int64_t nw, const double* W,
                        const midbf_access* acc, int r, int q, double tau, int max_disc,
                        uint64_t seed, midbf_phase** out, midbf_recover_info* info);

/* midbf_phase_recover with flags.  MIDBF_RECOVER_DEVICE: every vector
 * recovery of Algorithm 4 - the detection of discontinuities along the root
 * column and root row, and the recovery of the sampled rows and columns
 * along each piece of Algorithm 6 - runs on the current CUDA device
 * (midbf_recover_vectors); the recovery paths (Algorithm 5) and the
 * factorization (Algorithm 1) stay on the host.  The result is the same bit
 * for bit as with flags = 0.  Errors as midbf_phase_recover, MIDBF_EINVAL for
 * unknown flags, and MIDBF_ECUDA / MIDBF_ENOMEM from the device. */
#define MIDBF_RECOVER_DEVICE 1
int midbf_phase_recover_ex(int d, int64_t nx, const double* X, int64_t nw, const double* W,
                           const midbf_access* acc, int r, int q, double tau, int max_disc,
                           uint64_t seed, int flags, midbf_phase** out, midbf_recover_info* info);

/* ---- vector recovery on the GPU (Algorithm 4, Sec. 2.3) -------------------
 * Algorithm 4 fixes, along a recovery path (Def. 3.3), the unwrapped value of
 * each child from its parent's, v(ed) = u(ed) - round(u(ed) - v(bg)) (round
 * half away from zero), and flags ed when |v(ed) - v(bg)| >= tau; D is the
 * path root followed by the flagged children in path order.
 *
 * midbf_rpath_create: a path (or a piece of one, as Partition2 cuts it) over
 * n points, on the current device.  edges: nedges (parent, child) pairs,
 * row-major int64, host memory, copied; every parent must be root or the
 * child of an earlier edge, and no node may be a child twice.  The edges are
 * cut into runs of consecutive edges whose parents were all fixed by earlier
 * runs (one run per depth for a breadth-first path); midbf_rpath_info reports
 * their number.  Errors: MIDBF_EINVAL (bad sizes or edges, n >= 2^31),
 * MIDBF_ECUDA (no device), MIDBF_ENOMEM. */
typedef struct midbf_rpath midbf_rpath;
int midbf_rpath_create(int64_t n, int64_t nedges, const int64_t* edges, int64_t root, midbf_rpath** out);
void midbf_rpath_destroy(midbf_rpath* p);
int midbf_rpath_info(const midbf_rpath* p, int64_t* n, int64_t* nedges, int* nruns);

/* midbf_recover_vectors: Algorithm 4 along the path for nvec vectors at once
 * (one CTA per vector, the runs one after the other), asynchronous on stream
 * (a cudaStream_t).  Device arrays: u (nvec x n, leading dimension ldu) the
 * observed values modulo one; v (ldv) holds the start values (at least at the
 * root) on entry and the recovered values on exit (entries not reached by
 * the edges keep their start values); u and v must not overlap.  flags
 * (optional, uint8, nvec x nedges, ldf): 1 where the edge's child is flagged
 * at tau.  D (optional, needs flags; int64, ldD >= nedges + 1) and nD
 * (optional, int64 per vector): the flagged set D of each vector and its
 * length.  Every edge performs the FP64 operations of the sequential loop,
 * so v, flags and D equal a sequential run of Algorithm 4 bit for bit.
 * Errors: MIDBF_EINVAL (bad arguments, or the current device is not the
 * path's), MIDBF_ECUDA. */
int midbf_recover_vectors(const midbf_rpath* p, int nvec, const double* u, int64_t ldu, double* v, int64_t ldv,
                          double tau, uint8_t* flags, int64_t ldf, int64_t* D, int64_t ldD, int64_t* nD,
                          void* stream);

/* Evaluate Phi at n index pairs (ix[c], iw[c]) into out[c] (host, FP64). */
int midbf_phase_eval(const midbf_phase* ph, int64_t n, const int64_t* ix, const int64_t* iw,
                     double* out);

/* Rank r of a low-rank phase (0 for closed forms); copies U, V when not NULL. */
int midbf_phase_factors(const midbf_phase* ph, int* r, double* U, double* V);

void midbf_phase_destroy(midbf_phase* ph);

/* ---- construction (Sec. 3) ------------------------------------------------
 * Parameters of midbf_build.  midbf_params_default fills the paper's choices
 * (Sec. 4: eps = 1e-9, n0 = 8^d, t = 5) adjusted as documented: t = 2 with the
 * sample regrown to t * k_eps rows, kest = 30 (2D) / 80 (3D). */
typedef struct {
    double tol;        /* relative ID tolerance eps (Sec. 3.6)                  */
    int n0;            /* target points per leaf; depth L = round(log_b(N/n0))  */
    double t;          /* oversampling: sample >= t * k_eps rows (Sec. 3.2)     */
    int kest;          /* initial rank estimate k                               */
    int kmax;          /* rank cap, 0 = none (cap reached -> still succeeds)    */
    uint64_t seed;     /* seed of the random top-up of Mock-Chebyshev samples   */
    int nthreads;      /* host threads, 0 = all cores                           */
    int use_box;       /* 1: use boxX/boxW as the tree domains, 0: tight cubes  */
    double boxX[4];    /* lo[0..d-1], side (at index d)                         */
    double boxW[4];
    int device_ids;    /* 1: kernel samples and pivoted QRs on the current CUDA
                          device (FP64), 0: on the host threads               */
    int store_fp32;    /* 1: keep the ID coefficients T of the built plan in
                          complex FP32 on the host (half the memory; the QRs
                          still run in FP64, and T's rounding, 6e-8 relative,
                          is far below the ID tolerance); export writes FP64.
                          0: complex FP64                                      */
} midbf_params;

int midbf_params_default(int d, midbf_params* p);

/* Build the butterfly factors of K = exp(2 pi i Phi) over the phase's point
 * sets.  Host FP64 (pivoted QRs and kernel samples).  Errors: MIDBF_EINVAL,
 * MIDBF_ENOMEM. */
int midbf_build(const midbf_phase* ph, const midbf_params* p, midbf_plan** out);

/* Serialize a plan into the level-program file format; *buf is allocated with
 * malloc and released by the caller with midbf_free. */
int midbf_plan_export(const midbf_plan* plan, void** buf, size_t* len);

/* Read a plan file (from this library or any writer of the same format).
 * The plan is validated (every index in range, every output written once).
 * Errors: MIDBF_EFORMAT, MIDBF_ENOMEM. */
int midbf_plan_import(const void* buf, size_t len, midbf_plan** out);

typedef struct {
    int d, L, delta, nsteps, nstages;
    int64_t nx, nw;
    int64_t nblocks;         /* blocks over all stages                         */
    int64_t nsubs;           /* interpolative decompositions                   */
    int64_t t_entries;       /* stored interpolation entries (T parts)         */
    int64_t skel_entries;    /* identity (skeleton) entries, not stored        */
    int64_t s_entries;       /* middle-factor entries (generated or stored)    */
    int64_t index_entries;   /* gather/scatter position entries                */
    int max_rank;
    double mean_rank;
} midbf_stats;

int midbf_plan_stats(const midbf_plan* plan, midbf_stats* st);

/* Ranks k of the interpolative decompositions of one stage (stage index in
 * [0, nstages)), or of every V/U stage with stage = -1, in plan order:
 * writes min(count, cap) ranks to ranks (may be NULL with cap = 0) and the
 * total number of decompositions to *count.  The middle factor holds none.
 * Errors: MIDBF_EINVAL. */
int midbf_plan_ranks(const midbf_plan* plan, int stage, int32_t* ranks, int64_t cap, int64_t* count);
void midbf_plan_destroy(midbf_plan* plan);
void midbf_free(void* p);

/* ---- device plans and the apply ----------------------------------------
 * midbf_dplan_create: copy a plan to the current CUDA device in one precision
 * (MIDBF_FP64, MIDBF_FP32, or MIDBF_BF16 [| MIDBF_REFINE]) and middle-factor
 * mode.  Allocates device memory
 * (cudaMalloc) and synchronizes the device; call before any stream capture.
 * Errors: MIDBF_EINVAL, MIDBF_ENOMEM, MIDBF_ECUDA. */
int midbf_dplan_create(const midbf_plan* plan, int precision, int s_mode, midbf_dplan** out);

/* midbf_dplan_create with flags.  MIDBF_DPLAN_CONSUME: release each stage's
 * ID coefficients from the host plan as soon as they are on the device, so
 * that host memory falls while the plan is uploaded (plans of ~1e10 entries
 * do not fit twice).  The plan keeps its structure and statistics, but
 * midbf_plan_export and further device plans from it then fail with
 * MIDBF_EINVAL.  Errors as midbf_dplan_create, and MIDBF_EINVAL for unknown
 * flags or an already consumed plan. */
#define MIDBF_DPLAN_CONSUME 1
/* MIDBF_DPLAN_OVERLAP: prepare the overlap of the middle factor with the U
 * stage after it (see midbf_dplan_set_overlap below) and switch it on. */
#define MIDBF_DPLAN_OVERLAP 2
int midbf_dplan_create_ex(midbf_plan* plan, int precision, int s_mode, int flags, midbf_dplan** out);
void midbf_dplan_destroy(midbf_dplan* dp);

/* Device-side status of a plan's kernels: MIDBF_OK, or MIDBF_ETIMEOUT when a
 * bounded wait inside a tensor-core kernel gave up (its results are then
 * invalid).  Reading synchronizes the device; reset = 1 clears the word. */
int midbf_dplan_status(const midbf_dplan* dp, int reset, int* status);

/* Failure-detection self-test of the bounded waits (no GPU fault involved):
 * launches ctas (1..1024) one-thread CTAs on stream (a cudaStream_t) that
 * each wait, with the tensor-core kernels' bounded wait (2 s limit), on an
 * mbarrier nothing arrives on.  Each gives up, sets the plan's status word to
 * MIDBF_ETIMEOUT and exits; midbf_dplan_status then reads MIDBF_ETIMEOUT and
 * the context stays usable.  Asynchronous.  The status word is the plan's:
 * tensor-core applies of the same plan in flight meanwhile would see it set
 * and give up, so run the self-test alone.  Errors: MIDBF_EINVAL (bad
 * arguments, or the stream is being recorded into a graph). */
int midbf_wait_selftest(midbf_dplan* dp, int ctas, void* stream);

/* Bytes of device workspace midbf_apply needs for nrhs right-hand sides. */
int midbf_workspace_size(const midbf_dplan* dp, int nrhs, size_t* bytes);

/* Device bytes held by the plan's factors and index maps (for roofline use):
 * bytes the apply must stream once per call, per direction. */
int midbf_dplan_bytes(const midbf_dplan* dp, size_t* factor_bytes, size_t* index_bytes);

/* midbf_apply: out = K in (adjoint = 0; in has nw entries, out nx) or
 * out = K^H in (adjoint = 1; in nx, out nw), for nrhs right-hand sides.  The
 * forward apply is the factor product of eq. (finishIDBF) (Sec. 3.5),
 * U^L ... U^h S^h V^h ... V^L applied right to left to f, which approximates
 * the sum g(x_i) = sum_j exp(2 pi i Phi(x_i, xi_j)) f(xi_j) of eq. (1); the
 * adjoint applies the conjugate transposes of the same factors in reverse
 * order, (V^L)^H ... (S^h)^H ... (U^L)^H.  Runs on the CUDA stream `stream` (cudaStream_t, NULL = legacy default stream).
 * in/out are device pointers with leading dimensions ldin/ldout (>= vector
 * length); they must not overlap.  workspace: device memory of at least
 * midbf_workspace_size bytes, owned by the caller, not shared between calls
 * in flight.  Asynchronous: argument errors are returned immediately; device
 * faults surface through later CUDA calls.  Allocates nothing.
 * Errors: MIDBF_EINVAL, MIDBF_ECUDA. */
int midbf_apply(const midbf_dplan* dp, int adjoint, const void* in, int64_t ldin,
                void* out, int64_t ldout, int nrhs, void* stream,
                void* workspace, size_t workspace_bytes);

/* midbf_apply_host: as midbf_apply with HOST in/out buffers (ideally pinned):
 * copies in to the device, applies, copies out back, all on `stream`, then
 * synchronizes the stream.  The workspace must hold
 * midbf_workspace_size + (nx + nw) * nrhs complex entries. */
int midbf_apply_host(const midbf_dplan* dp, int adjoint, const void* in_host, void* out_host,
                     int nrhs, void* stream, void* workspace, size_t workspace_bytes);

/* ---- batched apply (many uneven instances) -------------------------------
 * midbf_apply_batched: count independent applies of possibly different plans,
 * directions (adjoint[i]) and numbers of right-hand sides (nrhs[i]), issued
 * together on one stream.  Level index q of every instance goes into one
 * group of launches (forward instances run their stage q, adjoint instances
 * their stage ns-1-q), so the number of launches grows with the number of
 * levels and kernel variants, not with count; a one-RHS instance's stage
 * that the single-instance apply runs on the narrow-ID or cluster kernels
 * gets that launch of its own, so every output equals the single-instance
 * apply's (tuned SIMT tiles included) bit for bit.  All dplans must share one
 * precision and device; in[i]/out[i] are device vectors with leading
 * dimensions ldin[i]/ldout[i] as in midbf_apply; no two instances may share
 * an output.  workspace: device memory of midbf_batched_workspace_size bytes.
 * Errors: MIDBF_EINVAL, MIDBF_ECUDA. */
int midbf_batched_workspace_size(int count, const midbf_dplan* const* dps, const int* nrhs, size_t* bytes);
/* Number of kernel launches midbf_apply_batched issues for these instances,
 * directions and RHS counts (no device work).  Errors: MIDBF_EINVAL. */
int midbf_batched_launches(int count, const midbf_dplan* const* dps, const int* adjoint, const int* nrhs,
                           int* launches);
int midbf_apply_batched(int count, const midbf_dplan* const* dps, const int* adjoint,
                        const void* const* in, const int64_t* ldin, void* const* out,
                        const int64_t* ldout, const int* nrhs, void* stream,
                        void* workspace, size_t workspace_bytes);

/* ---- overlap of the middle factor with its neighbouring stage ------------
 * The middle factor S (Sec. 3.5) is bound by arithmetic (its entries are
 * made on the fly), the U stage after it by memory.  Each U block reads the
 * outputs of a few S blocks only, and these blocks fall into independent
 * groups; midbf_dplan_create_ex with MIDBF_DPLAN_OVERLAP deals the groups
 * into (up to 4) chunks.  With the overlap on, an apply on the SIMT kernels
 * runs S and that U stage chunk by chunk: forward, chunk
 * k of S on the caller's stream and chunk k of U, after an event, on a side
 * stream of the plan; adjoint, U's adjoint chunk first and S's adjoint chunk
 * on the side stream.  The side stream forks from the caller's stream before
 * the pair and joins it after, so the apply stays ordered on the caller's
 * stream and can be recorded into a graph.  Results are the same bit for bit
 * as with the overlap off.  The overlap is skipped while profiling is on
 * (midbf_dplan_profile times each stage alone) and for stages on the tensor
 * cores.  Applies of one plan from several host threads are serialized while
 * they issue the overlapped pair.  Plans with chunks need a third internal
 * vector in the workspace (midbf_workspace_size includes it).  Measured on
 * one GB300 at n = 256, one RHS, the overlap is slower (2.00 ms per forward
 * + adjoint step against 1.85 ms): each chunk's launch leaves a partial wave
 * of CTAs, and S and U do not co-reside enough to win it back, so plans are
 * created without it.
 * midbf_dplan_set_overlap: enable = 1 on (if the plan has chunks), 0 off.
 * midbf_dplan_overlap: the chunk count in force (0: off).  EINVAL on null
 * arguments. */
int midbf_dplan_set_overlap(midbf_dplan* dp, int enable);
int midbf_dplan_overlap(const midbf_dplan* dp, int* chunks);

/* ---- CUDA graphs ----------------------------------------------------------
 * A sequence of midbf_apply / midbf_apply_batched calls issued on one
 * stream can be recorded once and replayed with one
 * launch: midbf_capture_begin(stream), the apply calls on that stream, then
 * midbf_capture_end(stream, &graph); midbf_graph_launch(graph, s) replays
 * the whole sequence on any stream s of the same device, any number of
 * times.  A replay reads and writes the very buffers and workspaces named
 * in the recorded calls, with the same nrhs: their contents may change
 * between replays, their addresses may not, and they must stay allocated
 * while the graph exists.  The apply calls issue no allocation,
 * synchronization or host copy, so they record as kernel nodes only
 * (midbf_apply_host cannot be recorded; it returns MIDBF_EINVAL while its
 * stream records).  Profiling (midbf_dplan_profile) must be off for every
 * plan applied while recording.  The recording is thread-local: other
 * threads keep their ordinary CUDA behaviour.
 * Errors: MIDBF_EINVAL for a null or legacy-default stream, a null output,
 * or midbf_capture_end without a recording in progress; MIDBF_ECUDA when
 * CUDA refuses the capture or the instantiation (the recording is then
 * ended and discarded). */
typedef struct midbf_graph midbf_graph;
int midbf_capture_begin(void* stream);
int midbf_capture_end(void* stream, midbf_graph** graph);
int midbf_graph_launch(const midbf_graph* graph, void* stream);
void midbf_graph_destroy(midbf_graph* graph);

/* ---- kernel choices and the autotuner ------------------------------------
 * Every stage of an apply runs one kernel variant.  By default the library
 * picks it by fixed rules: the tensor-core kernels in the MIDBF_BF16 modes
 * from 16 RHS on; in FP32 the GEMM forms (MIDBF_CHOICE_GEMM) from 32 RHS on
 * as described beside that constant; for one RHS the narrow-ID and cluster
 * kernels as described beside theirs; else the SIMT kernel with the smallest
 * RHS tile that covers nrhs (at most 16 in FP32, 8 in FP64) and fits shared
 * memory, one CTA per work item.  A choice per (nrhs, stage, direction)
 * overrides the rules:
 *   MIDBF_CHOICE_DEFAULT  the rules;
 *   1, 2, 4, 8, 16        the SIMT kernel with this RHS tile (taken when it
 *                         fits shared memory; else the rules' tile);
 *   MIDBF_CHOICE_COLUMN1  the one-RHS column kernel of a U stage forward or a
 *                         V stage adjoint (nrhs = 1 only; else the rules);
 *   any of the above | MIDBF_CHOICE_PERSIST
 *                         the same SIMT kernel launched persistent: as many
 *                         CTAs as are resident on the GPU at once, each
 *                         looping over the level's work items;
 *   MIDBF_CHOICE_TENSOR   the tensor-core kernel (BF16 modes only; else the
 *                         rules);
 *   MIDBF_CHOICE_NARROW, MIDBF_CHOICE_CLUSTER, MIDBF_CHOICE_GEMM
 *                         below (each falls back to the rules where it does
 *                         not apply).
 * midbf_autotune times every applicable variant of every stage in both
 * directions for nrhs right-hand sides on `stream` and records the fastest;
 * later applies with that nrhs use it (midbf_apply_batched uses the tuned
 * choices too, launching the narrow, cluster and GEMM ones per instance).  It allocates and frees temporary device vectors, waits for the
 * stream, and must not run concurrently with applies of the same dplan or
 * while the stream records a graph.  midbf_set_choice records a choice by
 * hand, midbf_get_choice reads the one in force.  stage: index in forward
 * order (0 .. midbf_stage_info's count - 1).
 * Errors: MIDBF_EINVAL (bad arguments or an unknown choice), MIDBF_ENOMEM,
 * MIDBF_ECUDA, MIDBF_ETIMEOUT (a tensor-core wait gave up while tuning). */
#define MIDBF_CHOICE_DEFAULT 0
#define MIDBF_CHOICE_COLUMN1 32
#define MIDBF_CHOICE_PERSIST 256
#define MIDBF_CHOICE_TENSOR 1024
#define MIDBF_CHOICE_NARROW 64   /* one RHS, every rank <= 64: a warp per ID (rows) or
                                    a lane per column (columns); the default for
                                    stages whose ranks are all <= 48 (and, for
                                    the rows, whose IDs have <= 128 redundant
                                    columns and number >= 32 per SM) */
#define MIDBF_CHOICE_GEMM 512    /* FP32: register-tiled complex GEMMs, 4 x 4
                                    micro-tiles per thread, RHS in tiles of 64:
                                    the middle factor made on the fly (each
                                    64 x 32 tile of S made once into shared
                                    memory; the default from 128 RHS on with
                                    the FP32 phase) and the row and column
                                    patterns of ID stages and of the stored
                                    middle factor (T copied into shared memory;
                                    the default from 32 RHS on, the column
                                    pattern when its IDs have >= 64 redundant
                                    columns) */
#define MIDBF_CHOICE_CLUSTER 128 /* one RHS, a V stage forward or a U stage adjoint:
                                    a thread-block cluster of up to 8 CTAs per
                                    work item, splitting its columns, the partial
                                    sums added through distributed shared memory
                                    in a fixed order; the default for such stages
                                    with fewer than 6 work items per SM */
int midbf_autotune(midbf_dplan* dp, int nrhs, void* stream);
int midbf_set_choice(midbf_dplan* dp, int nrhs, int stage, int adjoint, int choice);
int midbf_get_choice(const midbf_dplan* dp, int nrhs, int stage, int adjoint, int* choice);

/* Number of kernel launches one forward midbf_apply with nrhs right-hand
 * sides issues (for launch accounting): one per stage, two (pack, multiply)
 * per group of 256 RHS for a stage on the tensor cores.  EINVAL on a null
 * argument or nrhs <= 0. */
int midbf_apply_launches(const midbf_dplan* dp, int nrhs, int* launches);

/* Per-stage timing for measurement: with enable = 1, every later midbf_apply
 * on this dplan records a CUDA event on its stream before and after each
 * stage launch (calls must then not overlap).  midbf_stage_times waits for
 * the events of the most recent apply and writes up to max_stages durations
 * in milliseconds, in launch order, with the stage kind (0 = V, 1 = S, 2 = U)
 * and the number of algorithmic bytes the stage streams (factor entries,
 * index maps, input and output vectors) per right-hand side batch. */
int midbf_dplan_profile(midbf_dplan* dp, int enable);
int midbf_stage_times(const midbf_dplan* dp, int max_stages, float* ms, int* kinds, double* bytes,
                      int* n_stages);

/* Size of every stage, in forward order, for flop counts: the stage kind,
 * the complex entries of the method's factor (the T entries of the
 * interpolative decompositions V = [I T] Lambda^T of Sec. 3.2, or rows x
 * columns of the middle-factor blocks of Sec. 3.5) and of the dense blocks
 * (identity parts included; the blocks the tensor-core modes multiply).
 * Writes up to max_stages entries of each non-null array and the stage count
 * to *n_stages.  Host-only; no device work.  EINVAL on a null plan or count. */
int midbf_stage_info(const midbf_dplan* dp, int max_stages, int* kinds, int64_t* entries, int64_t* dense,
                     int* n_stages);

/* Measured arithmetic rates of the current device (for rooflines of the
 * kernels bound by arithmetic): FP32 fused multiply-adds per second (eight
 * independent chains per thread), SFU operations per second (chains of
 * rsqrt.approx) and, when dfma_per_s is not NULL, FP64 fused multiply-adds
 * per second; all over every SM, best of three timed launches on stream.
 * Allocates a small device buffer and synchronizes.  The paper has no
 * counterpart: this is measurement support.  Errors: MIDBF_EINVAL,
 * MIDBF_ECUDA. */
int midbf_pipe_rates(void* stream, double* fma_per_s, double* sfu_per_s, double* dfma_per_s);

/* midbf_apply_noalloc: midbf_apply for callers that cannot allocate device
 * memory when they apply the operator - for example a service whose GPU
 * memory is entirely owned by another allocator, or a latency-bound loop in
 * which cudaMalloc would synchronize the device.  It takes no workspace:
 * the intermediate vectors live in one scratch array of
 * midbf_noalloc_scratch_bytes() bytes (32 MiB) that the library holds in the
 * device memory of every GPU that loads it, until the process exits.  It
 * calls no cudaMalloc, cudaFree or allocating library routine.
 *   - Arguments and layout are those of midbf_apply; dp's device must be the
 *     current device.
 *   - The argument checks are those of midbf_apply (MIDBF_EINVAL for a null
 *     pointer, nrhs <= 0, a short leading dimension, overlapping in/out,
 *     vectors of 2^31 entries or more, or profiling on while the stream
 *     records a graph).
 *   - Plans whose workspace for nrhs right-hand sides (midbf_workspace_size)
 *     exceeds the scratch size are rejected with MIDBF_EINVAL and a message
 *     saying how many bytes they need.
 *   - The scratch array's device address is looked up (cudaGetSymbolAddress)
 *     when the device plan is created, with its device current, and kept in
 *     the plan; like the plan's other device memory it belongs to that
 *     device's context and does not survive cudaDeviceReset.  If the lookup
 *     failed, this call returns MIDBF_ECUDA with the reason.
 *   - All calls share the array and a call overwrites the previous call's
 *     contents (nothing in it needs to start at zero); calls that overlap on
 *     the GPU (different streams, unordered host threads) race on it and
 *     give wrong results.
 * The paper has no counterpart to this call: it is an allocation policy of
 * this library, not a step of the method. */
int midbf_apply_noalloc(const midbf_dplan* dp, int adjoint, const void* in, int64_t ldin,
                        void* out, int64_t ldout, int nrhs, void* stream);
size_t midbf_noalloc_scratch_bytes(void);

#ifdef __cplusplus
}
#endif
#endif /* MIDBF_H */
