// Level-program file format (read/write), plan validation and statistics.
//
// Layout (little-endian; the oracle has an independent reader/writer):
//   char[8] "MIDBFPL1"; i32 d, L, delta, nsteps; i64 nx, nw; f64 tol;
//   i32 family, r; f64 X[nx*d], W[nw*d]; if r > 0: f64 U[nx*r], V[nw*r];
//   i32 nstages; per stage: i32 kind, in_space, out_user, pad; i64 out_len,
//   nblocks; per block: i64 nin, nout, in_idx[nin], out_idx[nout];
//   S: i64 xidx[nout], widx[nin]; V/U: i32 nsub, pad; per sub: i32 k, m,
//   i32 skel[k], red[m-k], c128 T[k*(m-k)] row-major.
#include <algorithm>

#include "internal.hpp"

namespace midbf {

namespace {

struct Writer {
    std::vector<uint8_t> b;
    template <class T>
    void put(const T& v) {
        const uint8_t* p = reinterpret_cast<const uint8_t*>(&v);
        b.insert(b.end(), p, p + sizeof(T));
    }
    template <class T>
    void put_vec(const std::vector<T>& v) {
        const uint8_t* p = reinterpret_cast<const uint8_t*>(v.data());
        b.insert(b.end(), p, p + sizeof(T) * v.size());
    }
};

struct Reader {
    const uint8_t* p;
    size_t len, pos = 0;
    template <class T>
    T get() {
        if (pos + sizeof(T) > len) fail(MIDBF_EFORMAT, "truncated plan file");
        T v;
        std::memcpy(&v, p + pos, sizeof(T));
        pos += sizeof(T);
        return v;
    }
    template <class T>
    void get_vec(std::vector<T>& v, int64_t n) {
        if (n < 0 || (uint64_t)n > (len - pos) / sizeof(T)) fail(MIDBF_EFORMAT, "truncated plan file");
        v.resize((size_t)n);
        std::memcpy(v.data(), p + pos, sizeof(T) * (size_t)n);
        pos += sizeof(T) * (size_t)n;
    }
};

const char kMagic[8] = {'M', 'I', 'D', 'B', 'F', 'P', 'L', '1'};

}  // namespace

std::vector<uint8_t> plan_serialize(const Plan& pl) {
    if (pl.released) fail(MIDBF_EINVAL, "the plan's coefficients were released by a consuming upload");
    Writer w;
    for (char c : kMagic) w.put(c);
    w.put<int32_t>(pl.d);
    w.put<int32_t>(pl.L);
    w.put<int32_t>(pl.delta);
    w.put<int32_t>(pl.nsteps);
    w.put<int64_t>(pl.phase.nx);
    w.put<int64_t>(pl.phase.nw);
    w.put<double>(pl.tol);
    w.put<int32_t>(pl.phase.family);
    w.put<int32_t>(pl.phase.family == MIDBF_PHASE_LOWRANK ? pl.phase.r : 0);
    w.put_vec(pl.phase.X);
    w.put_vec(pl.phase.W);
    if (pl.phase.family == MIDBF_PHASE_LOWRANK) {
        w.put_vec(pl.phase.U);
        w.put_vec(pl.phase.V);
    }
    w.put<int32_t>((int32_t)pl.stages.size());
    for (const Stage& st : pl.stages) {
        w.put<int32_t>(st.kind);
        w.put<int32_t>(st.in_space);
        w.put<int32_t>(st.out_user);
        w.put<int32_t>(0);
        w.put<int64_t>(st.out_len);
        w.put<int64_t>((int64_t)st.blocks.size());
        for (const Block& bk : st.blocks) {
            w.put<int64_t>((int64_t)bk.in_idx.size());
            w.put<int64_t>((int64_t)bk.out_idx.size());
            w.put_vec(bk.in_idx);
            w.put_vec(bk.out_idx);
            if (st.kind == KIND_S) {
                w.put_vec(bk.xidx);
                w.put_vec(bk.widx);
                continue;
            }
            w.put<int32_t>((int32_t)bk.subs.size());
            w.put<int32_t>(0);
            for (const Sub& s : bk.subs) {
                w.put<int32_t>(s.k);
                w.put<int32_t>(s.m);
                w.put_vec(s.skel);
                w.put_vec(s.red);
                if (s.Tf.empty()) {
                    w.put_vec(s.T);
                } else {
                    std::vector<cplx> t64(s.Tf.size());
                    for (size_t i = 0; i < t64.size(); ++i) t64[i] = s.t(i);
                    w.put_vec(t64);
                }
            }
        }
    }
    return std::move(w.b);
}

std::unique_ptr<Plan> plan_deserialize(const uint8_t* buf, size_t len) {
    Reader rd{buf, len};
    for (char c : kMagic)
        if (rd.get<char>() != c) fail(MIDBF_EFORMAT, "not a MIDBF plan file");
    auto pl = std::make_unique<Plan>();
    pl->d = rd.get<int32_t>();
    pl->L = rd.get<int32_t>();
    pl->delta = rd.get<int32_t>();
    pl->nsteps = rd.get<int32_t>();
    Phase& ph = pl->phase;
    ph.d = pl->d;
    ph.nx = rd.get<int64_t>();
    ph.nw = rd.get<int64_t>();
    pl->tol = rd.get<double>();
    ph.family = rd.get<int32_t>();
    ph.r = rd.get<int32_t>();
    if (ph.d != 2 && ph.d != 3) fail(MIDBF_EFORMAT, "bad dimension in plan file");
    if (ph.nx <= 0 || ph.nw <= 0 || ph.r < 0) fail(MIDBF_EFORMAT, "bad sizes in plan file");
    rd.get_vec(ph.X, ph.nx * ph.d);
    rd.get_vec(ph.W, ph.nw * ph.d);
    if (ph.r > 0) {
        rd.get_vec(ph.U, ph.nx * ph.r);
        rd.get_vec(ph.V, ph.nw * ph.r);
    }
    int32_t nst = rd.get<int32_t>();
    if (nst <= 0 || nst > 4096) fail(MIDBF_EFORMAT, "bad stage count");
    pl->stages.resize(nst);
    for (Stage& st : pl->stages) {
        st.kind = rd.get<int32_t>();
        st.in_space = rd.get<int32_t>();
        st.out_user = rd.get<int32_t>();
        rd.get<int32_t>();
        st.out_len = rd.get<int64_t>();
        int64_t nb = rd.get<int64_t>();
        if (st.kind < 0 || st.kind > 2 || nb < 0 || nb > (int64_t)len) fail(MIDBF_EFORMAT, "bad stage header");
        st.blocks.resize((size_t)nb);
        for (Block& bk : st.blocks) {
            int64_t nin = rd.get<int64_t>(), nout = rd.get<int64_t>();
            rd.get_vec(bk.in_idx, nin);
            rd.get_vec(bk.out_idx, nout);
            if (st.kind == KIND_S) {
                rd.get_vec(bk.xidx, nout);
                rd.get_vec(bk.widx, nin);
                continue;
            }
            int32_t nsub = rd.get<int32_t>();
            rd.get<int32_t>();
            if (nsub < 0 || nsub > 64) fail(MIDBF_EFORMAT, "bad sub-block count");
            bk.subs.resize(nsub);
            for (Sub& s : bk.subs) {
                s.k = rd.get<int32_t>();
                s.m = rd.get<int32_t>();
                if (s.k < 0 || s.m < s.k) fail(MIDBF_EFORMAT, "bad sub-block shape");
                rd.get_vec(s.skel, s.k);
                rd.get_vec(s.red, (int64_t)s.m - s.k);
                rd.get_vec(s.T, (int64_t)s.k * (s.m - s.k));
            }
        }
    }
    if (rd.pos != len) fail(MIDBF_EFORMAT, "trailing bytes in plan file");
    phase_check(ph);
    plan_validate(*pl);
    return pl;
}

// Every position in range, every output written exactly once, every
// skeleton/redundant set a partition of the wide side, T finite.
void plan_validate(const Plan& pl) {
    const int64_t nx = pl.phase.nx, nw = pl.phase.nw;
    int64_t in_len = nw;
    for (size_t s = 0; s < pl.stages.size(); ++s) {
        const Stage& st = pl.stages[s];
        const bool last = s + 1 == pl.stages.size();
        if ((bool)st.out_user != last) fail(MIDBF_EFORMAT, "only the last stage writes the user vector");
        if (st.in_space != (int32_t)s - 1) fail(MIDBF_EFORMAT, "stages must chain in order");
        if (last && st.out_len != nx) fail(MIDBF_EFORMAT, "last stage must write nx entries");
        if (st.out_len < 0 || st.out_len > ((int64_t)1 << 31)) fail(MIDBF_EFORMAT, "stage too long");
        std::vector<uint8_t> written((size_t)st.out_len, 0), read((size_t)in_len, 0);
        for (const Block& bk : st.blocks) {
            for (int64_t v : bk.in_idx) {
                if (v < 0 || v >= in_len) fail(MIDBF_EFORMAT, "input position out of range");
                if (read[(size_t)v]++) fail(MIDBF_EFORMAT, "input position read twice");
            }
            for (int64_t v : bk.out_idx) {
                if (v < 0 || v >= st.out_len) fail(MIDBF_EFORMAT, "output position out of range");
                if (written[(size_t)v]++) fail(MIDBF_EFORMAT, "output position written twice");
            }
            if (st.kind == KIND_S) {
                if (bk.xidx.size() != bk.out_idx.size() || bk.widx.size() != bk.in_idx.size())
                    fail(MIDBF_EFORMAT, "S block point lists do not match its size");
                for (int64_t v : bk.xidx)
                    if (v < 0 || v >= nx) fail(MIDBF_EFORMAT, "S row point out of range");
                for (int64_t v : bk.widx)
                    if (v < 0 || v >= nw) fail(MIDBF_EFORMAT, "S column point out of range");
                continue;
            }
            const int64_t wide = st.kind == KIND_V ? (int64_t)bk.in_idx.size() : (int64_t)bk.out_idx.size();
            const int64_t narrow = st.kind == KIND_V ? (int64_t)bk.out_idx.size() : (int64_t)bk.in_idx.size();
            int64_t ksum = 0;
            for (const Sub& sb : bk.subs) {
                if (sb.m != wide) fail(MIDBF_EFORMAT, "sub-block width differs from its block");
                std::vector<uint8_t> seen((size_t)sb.m, 0);
                for (int32_t v : sb.skel) {
                    if (v < 0 || v >= sb.m || seen[v]++) fail(MIDBF_EFORMAT, "bad skeleton set");
                }
                for (int32_t v : sb.red) {
                    if (v < 0 || v >= sb.m || seen[v]++) fail(MIDBF_EFORMAT, "bad redundant set");
                }
                if (sb.t_size() != (size_t)sb.k * (size_t)(sb.m - sb.k)) fail(MIDBF_EFORMAT, "T has the wrong size");
                for (size_t i = 0; i < sb.t_size(); ++i) {
                    const cplx z = sb.t(i);
                    if (!std::isfinite(z.real()) || !std::isfinite(z.imag())) fail(MIDBF_EFORMAT, "non-finite T");
                }
                ksum += sb.k;
            }
            if (ksum != narrow) fail(MIDBF_EFORMAT, "sub-block ranks do not add up to the narrow side");
        }
        for (uint8_t w : written)
            if (!w) fail(MIDBF_EFORMAT, "an output position is never written");
        for (uint8_t r : read)
            if (!r) fail(MIDBF_EFORMAT, "an input position is never read (the adjoint would leave it unset)");
        in_len = st.out_len;
    }
}

void plan_stats(const Plan& pl, midbf_stats* st) {
    std::memset(st, 0, sizeof(*st));
    st->d = pl.d;
    st->L = pl.L;
    st->delta = pl.delta;
    st->nsteps = pl.nsteps;
    st->nstages = (int)pl.stages.size();
    st->nx = pl.phase.nx;
    st->nw = pl.phase.nw;
    double ranks = 0.0;
    for (const Stage& s : pl.stages) {
        st->nblocks += (int64_t)s.blocks.size();
        for (const Block& b : s.blocks) {
            st->index_entries += (int64_t)(b.in_idx.size() + b.out_idx.size());
            if (s.kind == KIND_S) {
                st->s_entries += (int64_t)b.xidx.size() * (int64_t)b.widx.size();
                continue;
            }
            for (const Sub& sb : b.subs) {
                st->nsubs++;
                st->t_entries += (int64_t)sb.k * (int64_t)(sb.m - sb.k);
                st->skel_entries += sb.k;
                st->max_rank = std::max(st->max_rank, (int)sb.k);
                ranks += sb.k;
            }
        }
    }
    st->mean_rank = st->nsubs ? ranks / (double)st->nsubs : 0.0;
}

}  // namespace midbf
