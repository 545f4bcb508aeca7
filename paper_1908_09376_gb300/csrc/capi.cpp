// C ABI entry points for phases, plans and construction (host side).
#include <cstdlib>
#include <thread>

#include "internal.hpp"

using namespace midbf;

namespace midbf {
namespace {
thread_local std::string g_last_error;
}
void set_last_error(const std::string& s) { g_last_error = s; }
}  // namespace midbf

namespace {

template <class F>
int guarded(F&& f) {
    try {
        set_last_error("");
        f();
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

Phase* as_phase(midbf_phase* p) { return reinterpret_cast<Phase*>(p); }
const Phase* as_phase(const midbf_phase* p) { return reinterpret_cast<const Phase*>(p); }
const Plan* as_plan(const midbf_plan* p) { return reinterpret_cast<const Plan*>(p); }

void check_points(int d, int64_t nx, const double* X, int64_t nw, const double* W) {
    if (d != 2 && d != 3) fail(MIDBF_EINVAL, "d must be 2 or 3");
    if (nx <= 0 || nw <= 0 || !X || !W) fail(MIDBF_EINVAL, "empty or null point set");
    if (nx >= (1LL << 31) || nw >= (1LL << 31)) fail(MIDBF_EINVAL, "point sets larger than 2^31");
}

}  // namespace

extern "C" {

const char* midbf_last_error(void) { return g_last_error.c_str(); }

const char* midbf_version(void) { return "midbf-gb300 0.1"; }

void midbf_free(void* p) { std::free(p); }

int midbf_phase_closed_form(int family, int d, int64_t nx, const double* X, int64_t nw, const double* W,
                            midbf_phase** out) {
    return guarded([&] {
        if (!out) fail(MIDBF_EINVAL, "null output handle");
        check_points(d, nx, X, nw, W);
        if (family == MIDBF_PHASE_LOWRANK) fail(MIDBF_EINVAL, "use midbf_phase_lowrank for low-rank phases");
        auto ph = std::make_unique<Phase>();
        ph->family = family;
        ph->d = d;
        ph->nx = nx;
        ph->nw = nw;
        ph->X.assign(X, X + nx * d);
        ph->W.assign(W, W + nw * d);
        phase_check(*ph);
        *out = reinterpret_cast<midbf_phase*>(ph.release());
    });
}

int midbf_phase_lowrank(int d, int64_t nx, const double* X, int64_t nw, const double* W, int r, const double* U,
                        const double* V, midbf_phase** out) {
    return guarded([&] {
        if (!out || !U || !V) fail(MIDBF_EINVAL, "null argument");
        check_points(d, nx, X, nw, W);
        if (r <= 0 || r > 64) fail(MIDBF_EINVAL, "rank must be in [1, 64]");
        auto ph = std::make_unique<Phase>();
        ph->family = MIDBF_PHASE_LOWRANK;
        ph->d = d;
        ph->nx = nx;
        ph->nw = nw;
        ph->X.assign(X, X + nx * d);
        ph->W.assign(W, W + nw * d);
        ph->r = r;
        ph->U.assign(U, U + nx * r);
        ph->V.assign(V, V + nw * r);
        phase_check(*ph);
        *out = reinterpret_cast<midbf_phase*>(ph.release());
    });
}

int midbf_phase_recover_ex(int d, int64_t nx, const double* X, int64_t nw, const double* W,
                           const midbf_access* acc, int r, int q, double tau, int max_disc, uint64_t seed,
                           int flags, midbf_phase** out, midbf_recover_info* info) {
    return guarded([&] {
        if (!out || !acc || !acc->rows_fn || !acc->cols_fn) fail(MIDBF_EINVAL, "null argument");
        if (flags & ~MIDBF_RECOVER_DEVICE) fail(MIDBF_EINVAL, "unknown flags");
        check_points(d, nx, X, nw, W);
        if (r <= 0 || q <= 0 || (int64_t)r * q > std::min(nx, nw)) fail(MIDBF_EINVAL, "bad rank / oversampling");
        if (!(tau > 0.0 && tau <= 0.5)) fail(MIDBF_EINVAL, "tau must be in (0, 1/2]");
        if ((flags & MIDBF_RECOVER_DEVICE) && (nx >= (int64_t(1) << 31) || nw >= (int64_t(1) << 31)))
            fail(MIDBF_EINVAL, "device recovery needs fewer than 2^31 points");
        auto ph = recover_phase(d, nx, X, nw, W, *acc, r, q, tau, max_disc, seed, info,
                                (flags & MIDBF_RECOVER_DEVICE) != 0);
        *out = reinterpret_cast<midbf_phase*>(ph.release());
    });
}

int midbf_phase_recover(int d, int64_t nx, const double* X, int64_t nw, const double* W, const midbf_access* acc,
                        int r, int q, double tau, int max_disc, uint64_t seed, midbf_phase** out,
                        midbf_recover_info* info) {
    return midbf_phase_recover_ex(d, nx, X, nw, W, acc, r, q, tau, max_disc, seed, 0, out, info);
}

int midbf_phase_eval(const midbf_phase* ph, int64_t n, const int64_t* ix, const int64_t* iw, double* out) {
    return guarded([&] {
        if (!ph || (n > 0 && (!ix || !iw || !out)) || n < 0) fail(MIDBF_EINVAL, "bad argument");
        const Phase& p = *as_phase(ph);
        for (int64_t c = 0; c < n; ++c) {
            if (ix[c] < 0 || ix[c] >= p.nx || iw[c] < 0 || iw[c] >= p.nw) fail(MIDBF_EINVAL, "index out of range");
            out[c] = p(ix[c], iw[c]);
        }
    });
}

int midbf_phase_factors(const midbf_phase* ph, int* r, double* U, double* V) {
    return guarded([&] {
        if (!ph || !r) fail(MIDBF_EINVAL, "null argument");
        const Phase& p = *as_phase(ph);
        *r = p.family == MIDBF_PHASE_LOWRANK ? p.r : 0;
        if (*r && U) std::copy(p.U.begin(), p.U.end(), U);
        if (*r && V) std::copy(p.V.begin(), p.V.end(), V);
    });
}

void midbf_phase_destroy(midbf_phase* ph) { delete as_phase(ph); }

int midbf_params_default(int d, midbf_params* p) {
    return guarded([&] {
        if (!p || (d != 2 && d != 3)) fail(MIDBF_EINVAL, "bad argument");
        std::memset(p, 0, sizeof(*p));
        p->tol = 1e-9;
        p->n0 = d == 2 ? 64 : 512;
        p->t = 2.0;
        p->kest = d == 2 ? 30 : 80;
        p->kmax = 0;
        p->seed = 0;
        p->nthreads = 0;
        p->use_box = 0;
    });
}

int midbf_build(const midbf_phase* ph, const midbf_params* p, midbf_plan** out) {
    return guarded([&] {
        if (!ph || !p || !out) fail(MIDBF_EINVAL, "null argument");
        if (!(p->tol > 0.0 && p->tol < 1.0)) fail(MIDBF_EINVAL, "tol must be in (0, 1)");
        if (p->n0 <= 0 || !(p->t >= 1.0) || p->kest <= 0 || p->kmax < 0) fail(MIDBF_EINVAL, "bad parameters");
        if (p->use_box) {
            const int d = as_phase(ph)->d;
            for (const double* box : {p->boxX, p->boxW}) {
                for (int k = 0; k < d; ++k)
                    if (!std::isfinite(box[k])) fail(MIDBF_EINVAL, "non-finite box corner");
                if (!(std::isfinite(box[d]) && box[d] > 0.0)) fail(MIDBF_EINVAL, "box side must be positive");
            }
        }
        auto pl = build_plan(*as_phase(ph), *p);
        *out = reinterpret_cast<midbf_plan*>(pl.release());
    });
}

int midbf_plan_export(const midbf_plan* plan, void** buf, size_t* len) {
    return guarded([&] {
        if (!plan || !buf || !len) fail(MIDBF_EINVAL, "null argument");
        std::vector<uint8_t> v = plan_serialize(*as_plan(plan));
        void* p = std::malloc(v.size());
        if (!p) fail(MIDBF_ENOMEM, "malloc failed");
        std::memcpy(p, v.data(), v.size());
        *buf = p;
        *len = v.size();
    });
}

int midbf_plan_import(const void* buf, size_t len, midbf_plan** out) {
    return guarded([&] {
        if (!buf || !out) fail(MIDBF_EINVAL, "null argument");
        auto pl = plan_deserialize(static_cast<const uint8_t*>(buf), len);
        *out = reinterpret_cast<midbf_plan*>(pl.release());
    });
}

int midbf_plan_stats(const midbf_plan* plan, midbf_stats* st) {
    return guarded([&] {
        if (!plan || !st) fail(MIDBF_EINVAL, "null argument");
        plan_stats(*as_plan(plan), st);
    });
}

int midbf_plan_ranks(const midbf_plan* plan, int stage, int32_t* ranks, int64_t cap, int64_t* count) {
    return guarded([&] {
        if (!plan || !count || cap < 0 || (cap > 0 && !ranks)) fail(MIDBF_EINVAL, "null argument");
        const Plan& pl = *as_plan(plan);
        if (stage < -1 || stage >= (int)pl.stages.size()) fail(MIDBF_EINVAL, "stage index out of range");
        int64_t n = 0;
        for (size_t q = 0; q < pl.stages.size(); ++q) {
            if (stage >= 0 && (int)q != stage) continue;
            const Stage& st = pl.stages[q];
            if (st.kind == KIND_S) continue;
            for (const Block& b : st.blocks)
                for (const Sub& sb : b.subs) {
                    if (n < cap) ranks[n] = sb.k;
                    ++n;
                }
        }
        *count = n;
    });
}

void midbf_plan_destroy(midbf_plan* plan) { delete reinterpret_cast<Plan*>(plan); }

}  // extern "C"
