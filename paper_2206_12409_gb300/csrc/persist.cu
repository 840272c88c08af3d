// Persistence of a context's operator (Sec. VI: the compressed coupling
// matrices are computed once and reused).  vsie_save writes the body grid, the
// materials, the frequency, the options, every operator part of vsie_parts and
// the port table to a versioned little-endian binary file; vsie_load reads it
// back and recreates the context through vsie_create (no set-up integrals are
// recomputed).  Arrays are stored with their element counts, which vsie_load
// checks against the counts the header implies.
#include "vsie_internal.h"

#include <cmath>
#include <cstdio>
#include <memory>

namespace vsie {

static const char kMagic[8] = {'V', 'S', 'I', 'E', 'O', 'P', 'S', '1'};
constexpr uint32_t kVersion = 3;   // 3: vsie_options with the H-matrix and GEMM fields

struct FileCloser {
    void operator()(FILE* f) const { if (f) fclose(f); }
};
using File = std::unique_ptr<FILE, FileCloser>;

static void put(FILE* f, const void* p, size_t bytes) {
    if (bytes && fwrite(p, 1, bytes, f) != bytes) throw Error(VSIE_EINVAL, "write failed");
}
template <typename T> static void put_val(FILE* f, const T& v) { put(f, &v, sizeof(T)); }
// element count, then the elements
template <typename T> static void put_arr(FILE* f, const T* p, int64_t n) {
    put_val(f, n);
    if (n > 0 && !p) throw Error(VSIE_EINVAL, "missing operator part");
    put(f, p, (size_t)n * sizeof(T));
}

static void get(FILE* f, void* p, size_t bytes) {
    if (bytes && fread(p, 1, bytes, f) != bytes) throw Error(VSIE_EINVAL, "truncated or unreadable operator file");
}
template <typename T> static T get_val(FILE* f) {
    T v;
    get(f, &v, sizeof(T));
    return v;
}
template <typename T> static std::vector<T> get_arr(FILE* f, int64_t expect) {
    const int64_t n = get_val<int64_t>(f);
    if (n != expect) throw Error(VSIE_EINVAL, "operator file: array size mismatch");
    std::vector<T> v((size_t)n);
    get(f, v.data(), (size_t)n * sizeof(T));
    return v;
}

}  // namespace vsie

using namespace vsie;

extern "C" {

vsie_status vsie_save(const vsie_ctx* ctx_c, const char* path) {
    if (!ctx_c) { set_global_err("null context"); return VSIE_EINVAL; }
    vsie_ctx* ctx = const_cast<vsie_ctx*>(ctx_c);
    Ctx& c = *reinterpret_cast<Ctx*>(ctx);
    try {
        if (!path) throw Error(VSIE_EINVAL, "null path");
        vsie_parts P{};
        const vsie_status st = vsie_get_parts(ctx, &P);
        if (st != VSIE_OK) return st;
        File f(fopen(path, "wb"));
        if (!f) throw Error(VSIE_EINVAL, std::string("cannot open ") + path + " for writing");
        FILE* fp = f.get();
        put(fp, kMagic, sizeof(kMagic));
        put_val(fp, kVersion);
        vsie_grid g{};
        for (int i = 0; i < 3; ++i) { g.n[i] = c.nb[i]; g.origin[i] = c.origin[i]; }
        g.h = c.h;
        put_val(fp, g);
        put_val(fp, c.freq);
        put_val(fp, c.opts);
        put_arr(fp, c.eps_r.data(), c.n_b);
        put_arr(fp, c.sigma.data(), c.n_b);
        put_val(fp, P.m_f);
        put_val(fp, P.m_n);
        put_val(fp, P.stencil);
        const int64_t s3 = (int64_t)P.stencil * P.stencil * P.stencil;
        if (P.m_n > 0) {
            put_arr(fp, P.W, 2 * (int64_t)P.m_n * 3 * s3);
            put_arr(fp, P.base, 3 * (int64_t)P.m_n);
            put_val(fp, P.pre_nnz);
            if (P.pre_nnz > 0) {
                put_arr(fp, P.pre_rowptr, 3 * c.n_b + 1);
                put_arr(fp, P.pre_col, P.pre_nnz);
                put_arr(fp, P.pre_val, 2 * P.pre_nnz);
            }
            put_arr(fp, P.Znn, 2 * (int64_t)P.m_n * P.m_n);
        }
        if (P.m_f > 0) {
            put_arr(fp, P.Zff, 2 * (int64_t)P.m_f * P.m_f);
            put_val(fp, P.aca_rank);
            if (P.aca_rank > 0 && P.m_n > 0) {
                put_arr(fp, P.U, 2 * (int64_t)P.m_n * P.aca_rank);
                put_arr(fp, P.V, 2 * (int64_t)P.m_f * P.aca_rank);
            }
            put_val(fp, P.tt_rank);
            for (int a = 0; a < 3; ++a) {
                const int64_t r1 = P.tt_rank[a][0], r2 = P.tt_rank[a][1], r3 = P.tt_rank[a][2];
                if (r1 == 0) continue;
                put_arr(fp, P.tt_core[a][0], 2 * (int64_t)c.nb[0] * r1);
                put_arr(fp, P.tt_core[a][1], 2 * r1 * c.nb[1] * r2);
                put_arr(fp, P.tt_core[a][2], 2 * r2 * c.nb[2] * r3);
                put_arr(fp, P.tt_core[a][3], 2 * r3 * (int64_t)P.m_f);
            }
        }
        put_arr(fp, c.port_row.data(), (int64_t)c.port_row.size());
        put_arr(fp, c.port_len.data(), (int64_t)c.port_len.size());
        if (fflush(fp) != 0) throw Error(VSIE_EINVAL, "write failed");
    } catch (const Error& e) {
        c.err = e.msg;
        return e.st;
    }
    return VSIE_OK;
}

vsie_status vsie_load(const char* path, vsie_ctx** out) {
    if (!out) { set_global_err("null output pointer"); return VSIE_EINVAL; }
    *out = nullptr;
    try {
        if (!path) throw Error(VSIE_EINVAL, "null path");
        File f(fopen(path, "rb"));
        if (!f) throw Error(VSIE_EINVAL, std::string("cannot open ") + path);
        FILE* fp = f.get();
        char magic[8];
        get(fp, magic, sizeof(magic));
        if (memcmp(magic, kMagic, sizeof(kMagic)) != 0) throw Error(VSIE_EINVAL, "not a vsie operator file");
        if (get_val<uint32_t>(fp) != kVersion) throw Error(VSIE_EINVAL, "unsupported operator file version");
        const vsie_grid g = get_val<vsie_grid>(fp);
        if (g.n[0] <= 0 || g.n[1] <= 0 || g.n[2] <= 0) throw Error(VSIE_EINVAL, "operator file: bad grid");
        const double freq = get_val<double>(fp);
        const vsie_options o = get_val<vsie_options>(fp);
        const int64_t nb = (int64_t)g.n[0] * g.n[1] * g.n[2];
        const std::vector<double> eps_r = get_arr<double>(fp, nb), sigma = get_arr<double>(fp, nb);
        vsie_parts P{};
        P.m_f = get_val<int32_t>(fp);
        P.m_n = get_val<int32_t>(fp);
        P.stencil = get_val<int32_t>(fp);
        if (P.m_f < 0 || P.m_n < 0 || P.stencil < 0 || P.stencil > 16)
            throw Error(VSIE_EINVAL, "operator file: bad part sizes");
        const int64_t s3 = (int64_t)P.stencil * P.stencil * P.stencil;
        std::vector<double> W, pre_val, Znn, Zff, U, V, tt[3][4];
        std::vector<int32_t> base, pre_col;
        std::vector<int64_t> pre_row;
        if (P.m_n > 0) {
            W = get_arr<double>(fp, 2 * (int64_t)P.m_n * 3 * s3);
            base = get_arr<int32_t>(fp, 3 * (int64_t)P.m_n);
            P.pre_nnz = get_val<int64_t>(fp);
            if (P.pre_nnz < 0) throw Error(VSIE_EINVAL, "operator file: bad precorrection size");
            if (P.pre_nnz > 0) {
                pre_row = get_arr<int64_t>(fp, 3 * nb + 1);
                pre_col = get_arr<int32_t>(fp, P.pre_nnz);
                pre_val = get_arr<double>(fp, 2 * P.pre_nnz);
            }
            Znn = get_arr<double>(fp, 2 * (int64_t)P.m_n * P.m_n);
            P.W = W.data();
            P.base = base.data();
            P.pre_rowptr = pre_row.empty() ? nullptr : pre_row.data();
            P.pre_col = pre_col.empty() ? nullptr : pre_col.data();
            P.pre_val = pre_val.empty() ? nullptr : pre_val.data();
            P.Znn = Znn.data();
        }
        if (P.m_f > 0) {
            Zff = get_arr<double>(fp, 2 * (int64_t)P.m_f * P.m_f);
            P.Zff = Zff.data();
            P.aca_rank = get_val<int32_t>(fp);
            if (P.aca_rank < 0) throw Error(VSIE_EINVAL, "operator file: bad ACA rank");
            if (P.aca_rank > 0 && P.m_n > 0) {
                U = get_arr<double>(fp, 2 * (int64_t)P.m_n * P.aca_rank);
                V = get_arr<double>(fp, 2 * (int64_t)P.m_f * P.aca_rank);
                P.U = U.data();
                P.V = V.data();
            }
            get(fp, P.tt_rank, sizeof(P.tt_rank));
            for (int a = 0; a < 3; ++a) {
                const int64_t r1 = P.tt_rank[a][0], r2 = P.tt_rank[a][1], r3 = P.tt_rank[a][2];
                if (r1 < 0 || r2 < 0 || r3 < 0) throw Error(VSIE_EINVAL, "operator file: bad TT ranks");
                if (r1 == 0) continue;
                tt[a][0] = get_arr<double>(fp, 2 * (int64_t)g.n[0] * r1);
                tt[a][1] = get_arr<double>(fp, 2 * r1 * g.n[1] * r2);
                tt[a][2] = get_arr<double>(fp, 2 * r2 * g.n[2] * r3);
                tt[a][3] = get_arr<double>(fp, 2 * r3 * (int64_t)P.m_f);
                for (int q = 0; q < 4; ++q) P.tt_core[a][q] = tt[a][q].data();
            }
        }
        const int64_t np = get_val<int64_t>(fp);
        if (np < 0 || np > (int64_t)P.m_f + P.m_n) throw Error(VSIE_EINVAL, "operator file: bad port table");
        std::vector<int64_t> port_row((size_t)np);
        get(fp, port_row.data(), (size_t)np * sizeof(int64_t));
        const std::vector<double> port_len = get_arr<double>(fp, np);
        // ports drive surface unknowns only: a row outside [0, m_f + m_n) or a
        // length that is not a finite positive number would make vsie_rhs_ports
        // write outside the right-hand side or scale it by garbage
        for (int64_t q = 0; q < np; ++q) {
            if (port_row[q] < 0 || port_row[q] >= (int64_t)P.m_f + P.m_n)
                throw Error(VSIE_EINVAL, "operator file: port row outside the surface unknowns");
            if (!std::isfinite(port_len[q]) || !(port_len[q] > 0))
                throw Error(VSIE_EINVAL, "operator file: port edge length must be finite and positive");
        }
        vsie_ctx* ctx = nullptr;
        const vsie_status st = vsie_create(&g, eps_r.data(), sigma.data(), freq, &o, &P, &ctx);
        if (st != VSIE_OK) return st;
        Ctx* c = reinterpret_cast<Ctx*>(ctx);
        c->port_row = port_row;
        c->port_len = port_len;
        *out = ctx;
    } catch (const Error& e) {
        set_global_err(e.msg);
        return e.st;
    }
    return VSIE_OK;
}

}  // extern "C"
