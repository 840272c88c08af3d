// C ABI of libvsie: context creation from operator parts, the matvec entry point
// and bookkeeping (see include/vsie.h for the contract of each call).
#include "vsie_internal.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>

namespace vsie {

static std::mutex g_err_mu;
static std::string g_err;   // last context-less error

void set_global_err(const std::string& m) {
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_err = m;
}

void* dalloc(Ctx& c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(VSIE_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                     cudaGetErrorString(e));
    }
    c.allocs.push_back(p);
    return p;
}

template <typename T>
static T* upload(Ctx& c, const T* h, size_t n) {
    T* d = (T*)dalloc(c, n * sizeof(T));
    if (n) VSIE_CUDA(cudaMemcpy(d, h, n * sizeof(T), cudaMemcpyHostToDevice));
    return d;
}

bool fft_factor(int L, FFTPlan& pl, int max_radix) {
    pl = FFTPlan();
    pl.L = L;
    if (L < 1) return false;
    int n = L, p2 = 0;
    while (n % 2 == 0) { n /= 2; ++p2; }
    std::vector<int> r;
    if (max_radix >= 16)
        while (p2 >= 4) { r.push_back(16); p2 -= 4; }
    while (p2 >= 3) { r.push_back(8); p2 -= 3; }
    if (p2 == 2) r.push_back(4);
    if (p2 == 1) r.push_back(2);
    for (int q : {3, 5, 7})
        while (n % q == 0) { r.push_back(q); n /= q; }
    if (n != 1 || (int)r.size() > kMaxStages) return false;
    pl.nst = (int)r.size();
    int ns = 1;
    for (int i = 0; i < pl.nst; ++i) {
        pl.rad[i] = r[i];
        pl.ns[i] = ns;
        pl.nsmagic[i] = magic_div((uint32_t)ns);
        pl.twstep[i] = L / (ns * r[i]);
        ns *= r[i];
    }
    return true;
}

int next_smooth(int n) {
    for (int m = std::max(n, 1);; ++m) {
        int k = m;
        for (int q : {2, 3, 5, 7})
            while (k % q == 0) k /= q;
        if (k == 1) return m;
    }
}

// ------------------------------------------------------------------ parts upload
template <typename R>
static std::vector<cx<R>> convert(const std::complex<double>* h, size_t n) {
    std::vector<cx<R>> out(n);
    for (size_t i = 0; i < n; ++i) {
        out[i].x = (R)h[i].real();
        out[i].y = (R)h[i].imag();
    }
    return out;
}

template <typename R>
static cx<R>* up_c(Ctx& c, const std::vector<std::complex<double>>& h) {
    auto v = convert<R>(h.data(), h.size());
    return upload(c, v.data(), v.size());
}

// Work buffers of the convolution: [chunk][3][n3][n2][L1] and
// [chunk][3][n3][L2][L1] complex values.  The right-hand sides of one matvec are
// processed in groups of `chunk` so that the buffers stay within kConvWorkBudget
// bytes (a 1 mm head grid needs 2.1 GB per FP32 right-hand side).
constexpr size_t kConvWorkBudget = 16ull << 30;

static size_t conv_elems_A(const Ctx& c) { return 3 * (size_t)c.ne[2] * c.ne[1] * c.L[0]; }
static size_t conv_elems_B(const Ctx& c) { return 3 * (size_t)c.ne[2] * c.L[1] * c.L[0]; }

static int conv_chunk(const Ctx& c, size_t cs) {
    const size_t per = (conv_elems_A(c) + conv_elems_B(c)) * cs;
    const int most = (int)std::max<size_t>(1, std::min<size_t>((size_t)c.max_rhs, kConvWorkBudget / per));
    const int groups = (c.max_rhs + most - 1) / most;
    return (c.max_rhs + groups - 1) / groups;      // equal groups
}
static size_t conv_offB(const Ctx& c, size_t cs, int chunk) {
    return ((size_t)chunk * conv_elems_A(c) * cs + 255) / 256 * 256;
}
static size_t conv_bytes(const Ctx& c, size_t cs) {
    const int ch = conv_chunk(c, cs);
    return conv_offB(c, cs, ch) + (size_t)ch * conv_elems_B(c) * cs;
}

template <typename R>
static void prepare_precision(Ctx& c) {
    OpData<R>& d = data<R>(c);
    using C = cx<R>;
    build_spectra<R>(c);
    // body diagonal h^3 / chi (0 on vacuum)
    {
        std::vector<C> dv(c.n_b);
        for (int64_t v = 0; v < c.n_b; ++v) {
            const std::complex<double> chi(c.eps_r[v] - 1.0, -c.sigma[v] / (c.omega * kEps0));
            std::complex<double> di = 0.0;
            if (chi != std::complex<double>(0.0, 0.0)) di = c.h * c.h * c.h / chi;
            dv[v].x = (R)di.real();
            dv[v].y = (R)di.imag();
        }
        d.dinv = upload(c, dv.data(), dv.size());
    }
    if (c.m_n > 0) {
        d.W = up_c<R>(c, c.hW);
        // scatter CSR values: reorder W into the (b, active voxel) rows
        std::vector<C> sv(c.sc_nnz);
        for (int64_t e = 0; e < c.sc_nnz; ++e) {
            const std::complex<double> w = c.hW[c.sc_src[e]];
            sv[e].x = (R)w.real();
            sv[e].y = (R)w.imag();
        }
        d.sc_val = upload(c, sv.data(), sv.size());
        if (c.pre_nnz > 0) {
            d.pre_val = up_c<R>(c, c.hPreValRows);
            d.preT_val = up_c<R>(c, c.hPreValT);
        }
        d.Znn = up_c<R>(c, c.hZnn);
        const size_t sa = std::max<size_t>((size_t)3 * c.nact * c.max_rhs, 1);
        d.gc = (C*)dalloc(c, sa * sizeof(C));
        d.cc = (C*)dalloc(c, sa * sizeof(C));
    }
    if (c.m_f > 0) {
        if (c.dZff_in) {
            if (sizeof(R) == 8) {
                d.Zff = (cx<R>*)c.dZff_in;
            } else {
                d.Zff = (cx<R>*)dalloc(c, (size_t)c.m_f * c.m_f * sizeof(cx<R>));
                convert_to_f32(c.dZff_in, (float2*)d.Zff, (size_t)c.m_f * c.m_f);
            }
        } else {
            d.Zff = up_c<R>(c, c.hZff);
        }
        // FP32: row-panel storage for the streamed product (gemm_panel)
        if constexpr (sizeof(R) == 4) d.Zff = to_panel(c, d.Zff, c.m_f, c.m_f);
        if (c.aca_rank > 0 && c.m_n > 0) {
            d.U = up_c<R>(c, c.hU);
            d.V = up_c<R>(c, c.hV);
        }
        for (int a = 0; a < 3; ++a) {
            if (c.tt_rank[a][0] == 0) continue;
            for (int q = 0; q < 3; ++q) d.G[a][q] = up_c<R>(c, c.hTT[a][q]);
            // G4 (r3 x m_f) stored transposed as m_f x r3
            const int r3 = c.tt_rank[a][2];
            std::vector<std::complex<double>> t((size_t)c.m_f * r3);
            for (int i = 0; i < r3; ++i)
                for (int m = 0; m < c.m_f; ++m) t[m + (size_t)c.m_f * i] = c.hTT[a][3][i + (size_t)r3 * m];
            d.G[a][3] = up_c<R>(c, t);
        }
    }
    // workspaces: the convolution's two work buffers for `chunk` right-hand sides
    // inside the shared allocation (sized in init_ctx)
    const size_t p = c.max_rhs;
    d.chunk = conv_chunk(c, sizeof(C));
    d.bufA = (C*)c.conv_work;
    d.bufB = (C*)((char*)c.conv_work + conv_offB(c, sizeof(C), d.chunk));
    int r1 = 1, r2 = 1, r3 = 1;
    for (int a = 0; a < 3; ++a) {
        r1 = std::max(r1, c.tt_rank[a][0]);
        r2 = std::max(r2, c.tt_rank[a][1]);
        r3 = std::max(r3, c.tt_rank[a][2]);
    }
    const size_t k1 = std::max<size_t>(std::max(r3, c.aca_rank), 1) * p;
    d.t1 = (C*)dalloc(c, k1 * sizeof(C));
    d.t2 = (C*)dalloc(c, (size_t)r2 * c.nb[2] * p * sizeof(C));
    d.t3 = (C*)dalloc(c, (size_t)r1 * c.nb[1] * c.nb[2] * p * sizeof(C));
    d.splitk_elems = std::max<size_t>((size_t)4 * 1024 * 1024, (size_t)2 * std::max(c.m_f, 1) * p * 8);
    d.splitk = (C*)dalloc(c, d.splitk_elems * sizeof(C));
    conv_set_attrs<R>();
    VSIE_CUDA(cudaDeviceSynchronize());
    conv_autotune<R>(c);
    d.ready = true;
}

// Build the precision-independent index structures and host copies.
static void init_ctx(Ctx& c, const vsie_grid* body, const double* eps_r, const double* sigma,
                     double freq, const vsie_options* opts, const vsie_parts* parts) {
    if (!body || !eps_r || !sigma) throw Error(VSIE_EINVAL, "null body grid or material map");
    if (!(freq > 0) || !std::isfinite(freq)) throw Error(VSIE_EINVAL, "frequency must be > 0");
    if (!(body->h > 0)) throw Error(VSIE_EINVAL, "voxel size h must be > 0");
    for (int i = 0; i < 3; ++i)
        if (body->n[i] < 1) throw Error(VSIE_EINVAL, "body grid dimensions must be >= 1");
    vsie_options o{};
    if (opts) o = *opts;
    c.opts = o;
    for (int i = 0; i < 3; ++i) {
        c.nb[i] = body->n[i];
        c.ne[i] = o.ext_n[i] > 0 ? o.ext_n[i] : body->n[i];
        c.off[i] = o.ext_n[i] > 0 ? o.ext_offset[i] : 0;
        if (c.off[i] < 0 || c.off[i] + c.nb[i] > c.ne[i])
            throw Error(VSIE_EINVAL, "body grid does not fit in the extended grid");
        c.origin[i] = body->origin[i];
    }
    c.h = body->h;
    c.freq = freq;
    c.omega = 2.0 * M_PI * freq;
    c.k0 = c.omega / kC0;
    c.n_b = (int64_t)c.nb[0] * c.nb[1] * c.nb[2];
    c.n_e = (int64_t)c.ne[0] * c.ne[1] * c.ne[2];
    c.max_rhs = o.max_rhs > 0 ? o.max_rhs : 16;
    c.precisions = o.precisions > 0 ? o.precisions : 3;
    for (int i = 0; i < 3; ++i) {
        c.L[i] = next_smooth(2 * c.ne[i] - 1);
        c.Lh[i] = c.L[i] / 2 + 1;
        if (!fft_factor(c.L[i], c.plan[i], 8) || !fft_factor(c.L[i], c.plan16[i], 16))
            throw Error(VSIE_EUNSUPPORTED, "FFT length");
    }
    // half-length plans of the third axis (Z pass), twiddles read from the L3 table
    if (c.L[2] % 2 == 0 && fft_factor(c.L[2] / 2, c.plan3h, 8) && fft_factor(c.L[2] / 2, c.plan3h16, 16)) {
        for (int s2 = 0; s2 < c.plan3h.nst; ++s2) c.plan3h.twstep[s2] *= 2;
        for (int s2 = 0; s2 < c.plan3h16.nst; ++s2) c.plan3h16.twstep[s2] *= 2;
    } else {
        c.plan3h = FFTPlan();
        c.plan3h16 = FFTPlan();
    }
    c.eps_r.assign(eps_r, eps_r + c.n_b);
    c.sigma.assign(sigma, sigma + c.n_b);
    for (int64_t v = 0; v < c.n_b; ++v)
        if (!std::isfinite(c.eps_r[v]) || !std::isfinite(c.sigma[v]))
            throw Error(VSIE_EINVAL, "non-finite material value");
    std::vector<uint8_t> mask(c.n_b);
    for (int64_t v = 0; v < c.n_b; ++v) mask[v] = (c.eps_r[v] != 1.0 || c.sigma[v] != 0.0) ? 1 : 0;
    c.mask = upload(c, mask.data(), mask.size());

    // parts
    c.m_f = parts ? parts->m_f : 0;
    c.m_n = parts ? parts->m_n : 0;
    if (c.m_f < 0 || c.m_n < 0) throw Error(VSIE_EINVAL, "negative part sizes");
    c.N = (int64_t)c.m_f + c.m_n + 3 * c.n_b;
    c.s = parts && parts->stencil > 0 ? parts->stencil : 3;
    const int s = c.s, s3 = s * s * s;
    std::vector<int32_t> flags((size_t)c.ne[1] * c.ne[2], 0);
    // bit 1: the line crosses the body grid; bit 4: it holds a material voxel (its
    // x-forward transform can be non-zero); bit 2 (below): coil grid points
    for (int i3 = 0; i3 < c.nb[2]; ++i3)
        for (int i2 = 0; i2 < c.nb[1]; ++i2) {
            int32_t& f = flags[(i2 + c.off[1]) + (size_t)c.ne[1] * (i3 + c.off[2])];
            f |= 1;
            const size_t b0 = (size_t)c.nb[0] * (i2 + (size_t)c.nb[1] * i3);
            for (int i1 = 0; i1 < c.nb[0]; ++i1)
                if (mask[b0 + i1]) {
                    f |= 4;
                    break;
                }
        }
    std::vector<int32_t> lptr((size_t)c.ne[1] * c.ne[2] + 1, 0), li1, lci;
    if (c.m_n > 0) {
        if (!parts->W || !parts->base || !parts->Znn)
            throw Error(VSIE_EINVAL, "near parts: W, base and Znn are required");
        const std::complex<double>* W = reinterpret_cast<const std::complex<double>*>(parts->W);
        c.hW.assign(W, W + (size_t)c.m_n * 3 * s3);
        c.hBase.assign(parts->base, parts->base + (size_t)c.m_n * 3);
        // active voxels
        std::vector<int64_t> vox((size_t)c.m_n * s3);
        for (int n = 0; n < c.m_n; ++n) {
            const int* b = &c.hBase[(size_t)n * 3];
            for (int i = 0; i < 3; ++i)
                if (b[i] < 0 || b[i] + s > c.ne[i])
                    throw Error(VSIE_EINVAL, "pFFT stencil leaves the extended grid");
            for (int q = 0; q < s3; ++q) {
                const int qx = q % s, qy = (q / s) % s, qz = q / (s * s);
                vox[(size_t)n * s3 + q] =
                    (b[0] + qx) + (int64_t)c.ne[0] * ((b[1] + qy) + (int64_t)c.ne[1] * (b[2] + qz));
            }
        }
        std::vector<int64_t> act(vox);
        std::sort(act.begin(), act.end());
        act.erase(std::unique(act.begin(), act.end()), act.end());
        c.nact = (int64_t)act.size();
        std::vector<int32_t> cidx(vox.size());
        for (size_t e = 0; e < vox.size(); ++e)
            cidx[e] = (int32_t)(std::lower_bound(act.begin(), act.end(), vox[e]) - act.begin());
        c.W_cidx = upload(c, cidx.data(), cidx.size());
        // scatter CSR: rows (b, c) = b * nact + c, entries (n, index into W)
        const int64_t nrows = 3 * c.nact;
        std::vector<int32_t> cnt(nrows + 1, 0);
        for (int n = 0; n < c.m_n; ++n)
            for (int b = 0; b < 3; ++b)
                for (int q = 0; q < s3; ++q) cnt[b * c.nact + cidx[(size_t)n * s3 + q] + 1]++;
        for (int64_t r = 0; r < nrows; ++r) cnt[r + 1] += cnt[r];
        c.sc_nnz = cnt[nrows];
        std::vector<int32_t> col(c.sc_nnz);
        c.sc_src.assign(c.sc_nnz, 0);
        std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
        for (int n = 0; n < c.m_n; ++n)
            for (int b = 0; b < 3; ++b)
                for (int q = 0; q < s3; ++q) {
                    const int64_t r = b * c.nact + cidx[(size_t)n * s3 + q];
                    const int32_t at = fill[r]++;
                    col[at] = n;
                    c.sc_src[at] = (int64_t)n * 3 * s3 + b * s3 + q;
                }
        c.sc_ptr = upload(c, cnt.data(), cnt.size());
        c.sc_col = upload(c, col.data(), col.size());
        // per-line lists of active voxels
        std::vector<std::vector<std::pair<int32_t, int32_t>>> lines((size_t)c.ne[1] * c.ne[2]);
        for (int64_t a = 0; a < c.nact; ++a) {
            const int64_t v = act[a];
            const int i1 = v % c.ne[0];
            const int64_t lin = v / c.ne[0];
            lines[lin].push_back({i1, (int32_t)a});
            flags[lin] |= 2;
        }
        for (size_t l = 0; l < lines.size(); ++l) {
            lptr[l + 1] = lptr[l] + (int32_t)lines[l].size();
            for (auto& pr : lines[l]) {
                li1.push_back(pr.first);
                lci.push_back(pr.second);
            }
        }
        c.hZnn.assign(reinterpret_cast<const std::complex<double>*>(parts->Znn),
                      reinterpret_cast<const std::complex<double>*>(parts->Znn) +
                          (size_t)c.m_n * c.m_n);
        // precorrection
        c.pre_nnz = parts->pre_nnz;
        if (c.pre_nnz > 0) {
            if (!parts->pre_rowptr || !parts->pre_col || !parts->pre_val)
                throw Error(VSIE_EINVAL, "precorrection CSR arrays are required when nnz > 0");
            const int64_t nr = 3 * c.n_b;
            const int64_t* rp = parts->pre_rowptr;
            if (rp[0] != 0 || rp[nr] != c.pre_nnz)
                throw Error(VSIE_EINVAL, "precorrection row pointer inconsistent with nnz");
            const std::complex<double>* pv =
                reinterpret_cast<const std::complex<double>*>(parts->pre_val);
            c.hPreRow.assign(rp, rp + nr + 1);
            c.hPreCol.assign(parts->pre_col, parts->pre_col + c.pre_nnz);
            c.hPreVal.assign(pv, pv + c.pre_nnz);
            std::vector<int32_t> rows;
            std::vector<int64_t> ptr{0};
            std::vector<int32_t> pc;
            c.hPreValRows.clear();
            for (int64_t r = 0; r < nr; ++r) {
                if (rp[r + 1] < rp[r]) throw Error(VSIE_EINVAL, "precorrection rows not sorted");
                if (rp[r + 1] == rp[r]) continue;
                rows.push_back((int32_t)r);
                for (int64_t q = rp[r]; q < rp[r + 1]; ++q) {
                    if (parts->pre_col[q] < 0 || parts->pre_col[q] >= c.m_n)
                        throw Error(VSIE_EINVAL, "precorrection column out of range");
                    pc.push_back(parts->pre_col[q]);
                    c.hPreValRows.push_back(pv[q]);
                }
                ptr.push_back((int64_t)pc.size());
            }
            c.pre_nr = (int64_t)rows.size();
            c.pre_rows = upload(c, rows.data(), rows.size());
            c.pre_ptr = upload(c, ptr.data(), ptr.size());
            c.pre_col = upload(c, pc.data(), pc.size());
            // transpose: rows = RWG, cols = body unknown index
            std::vector<std::vector<std::pair<int32_t, std::complex<double>>>> tr(c.m_n);
            for (int64_t r = 0; r < nr; ++r)
                for (int64_t q = rp[r]; q < rp[r + 1]; ++q) tr[parts->pre_col[q]].push_back({(int32_t)r, pv[q]});
            std::vector<int32_t> trows, tcol;
            std::vector<int64_t> tptr{0};
            c.hPreValT.clear();
            for (int n = 0; n < c.m_n; ++n) {
                if (tr[n].empty()) continue;
                trows.push_back(n);
                for (auto& pr : tr[n]) {
                    tcol.push_back(pr.first);
                    c.hPreValT.push_back(pr.second);
                }
                tptr.push_back((int64_t)tcol.size());
            }
            c.preT_nr = (int64_t)trows.size();
            c.preT_rows = upload(c, trows.data(), trows.size());
            c.preT_ptr = upload(c, tptr.data(), tptr.size());
            c.preT_col = upload(c, tcol.data(), tcol.size());
        }
    }
    c.line_ptr = upload(c, lptr.data(), lptr.size());
    c.line_i1 = upload(c, li1.data(), li1.size());
    c.line_cidx = upload(c, lci.data(), lci.size());
    c.body_lines = upload(c, flags.data(), flags.size());
    if (c.m_f > 0) {
        if (!c.dZff_in) {
            if (!parts->Zff) throw Error(VSIE_EINVAL, "far parts: Zff is required");
            const auto* Z = reinterpret_cast<const std::complex<double>*>(parts->Zff);
            c.hZff.assign(Z, Z + (size_t)c.m_f * c.m_f);
        }
        c.aca_rank = parts->aca_rank;
        if (c.aca_rank > 0 && c.m_n > 0) {
            if (!parts->U || !parts->V) throw Error(VSIE_EINVAL, "ACA factors missing");
            const auto* U = reinterpret_cast<const std::complex<double>*>(parts->U);
            const auto* V = reinterpret_cast<const std::complex<double>*>(parts->V);
            c.hU.assign(U, U + (size_t)c.m_n * c.aca_rank);
            c.hV.assign(V, V + (size_t)c.m_f * c.aca_rank);
        } else {
            c.aca_rank = 0;
        }
        for (int a = 0; a < 3; ++a) {
            const int r1 = parts->tt_rank[a][0], r2 = parts->tt_rank[a][1], r3 = parts->tt_rank[a][2];
            c.tt_rank[a][0] = r1;
            c.tt_rank[a][1] = r2;
            c.tt_rank[a][2] = r3;
            if (r1 == 0) continue;
            if (r2 <= 0 || r3 <= 0) throw Error(VSIE_EINVAL, "TT ranks must be positive");
            const size_t sz[4] = {(size_t)c.nb[0] * r1, (size_t)r1 * c.nb[1] * r2,
                                  (size_t)r2 * c.nb[2] * r3, (size_t)r3 * c.m_f};
            for (int q = 0; q < 4; ++q) {
                if (!parts->tt_core[a][q]) throw Error(VSIE_EINVAL, "TT core missing");
                const auto* G = reinterpret_cast<const std::complex<double>*>(parts->tt_core[a][q]);
                c.hTT[a][q].assign(G, G + sz[q]);
            }
        }
    }
    {
        size_t need = 0;
        if (c.precisions & 2) need = std::max(need, conv_bytes(c, sizeof(float2)));
        if (c.precisions & 1) need = std::max(need, conv_bytes(c, sizeof(double2)));
        c.conv_work = dalloc(c, need);
        c.conv_work_bytes = need;
    }
    if (c.precisions & 2) prepare_precision<float>(c);
    if (c.precisions & 1) prepare_precision<double>(c);
    VSIE_CUDA(cudaDeviceSynchronize());
}

template <typename R>
static void matvec_impl(Ctx& c, int p, const void* X, int64_t ldx, void* Y, int64_t ldy,
                        cudaStream_t st) {
    const cx<R>* x = (const cx<R>*)X;
    cx<R>* y = (cx<R>*)Y;
    surface_pre<R>(c, p, x, ldx, st);
    conv_apply<R>(c, p, x, ldx, y, ldy, st);
    surface_apply<R>(c, p, x, ldx, y, ldy, st);
    apply_loads<R>(c, p, x, ldx, y, ldy, st);
}

template <typename R>
void matvec_internal(Ctx& c, int p, const cx<R>* X, int64_t ldx, cx<R>* Y, int64_t ldy,
                     cudaStream_t st) {
    matvec_impl<R>(c, p, X, ldx, Y, ldy, st);
}
template void matvec_internal<float>(Ctx&, int, const float2*, int64_t, float2*, int64_t, cudaStream_t);
template void matvec_internal<double>(Ctx&, int, const double2*, int64_t, double2*, int64_t, cudaStream_t);

vsie_status fail(Ctx* c, const Error& e) {
    if (c) c->err = e.msg;
    else set_global_err(e.msg);
    return e.st;
}

void destroy_ctx(Ctx* c) {
    if (!c) return;
    for (int g = 0; g < PG_N; ++g)
        for (auto& e : c->prof.ev[g]) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    for (void* p : c->allocs) cudaFree(p);
    delete c;
}

// vsie_get_parts: host views of the operator parts (Zff copied from the device
// when the set-up produced it there).
static void fill_parts(Ctx& c, vsie_parts& p) {
    if (c.hm.on)
        throw Error(VSIE_EUNSUPPORTED, "the far-far block is hierarchical; its dense form is not kept");
    p = vsie_parts{};
    p.m_f = c.m_f;
    p.m_n = c.m_n;
    p.stencil = c.s;
    if (c.m_n > 0) {
        p.W = reinterpret_cast<const double*>(c.hW.data());
        p.base = c.hBase.data();
        p.pre_nnz = c.pre_nnz;
        if (c.pre_nnz > 0) {
            p.pre_rowptr = c.hPreRow.data();
            p.pre_col = c.hPreCol.data();
            p.pre_val = reinterpret_cast<const double*>(c.hPreVal.data());
        }
        p.Znn = reinterpret_cast<const double*>(c.hZnn.data());
    }
    if (c.m_f > 0) {
        if (c.hZff.empty()) {
            c.hZff_copy.resize((size_t)c.m_f * c.m_f);
            VSIE_CUDA(cudaMemcpy(c.hZff_copy.data(), c.f64.ready ? (const void*)c.f64.Zff : (const void*)c.dZff_in,
                                 c.hZff_copy.size() * sizeof(double2), cudaMemcpyDeviceToHost));
            p.Zff = reinterpret_cast<const double*>(c.hZff_copy.data());
        } else {
            p.Zff = reinterpret_cast<const double*>(c.hZff.data());
        }
        p.aca_rank = c.aca_rank;
        if (c.aca_rank > 0) {
            p.U = reinterpret_cast<const double*>(c.hU.data());
            p.V = reinterpret_cast<const double*>(c.hV.data());
        }
        for (int a = 0; a < 3; ++a) {
            for (int q = 0; q < 3; ++q) p.tt_rank[a][q] = c.tt_rank[a][q];
            for (int q = 0; q < 4; ++q)
                p.tt_core[a][q] = c.tt_rank[a][0] ? reinterpret_cast<const double*>(c.hTT[a][q].data()) : nullptr;
        }
    }
}

vsie_status create_from_parts_impl(const vsie_grid* body, const double* eps_r,
                                   const double* sigma, double freq, const vsie_options* opts,
                                   const vsie_parts* parts, double2* dZff, Ctx** out) {
    if (!out) { set_global_err("null output pointer"); return VSIE_EINVAL; }
    *out = nullptr;
    Ctx* c = new (std::nothrow) Ctx();
    if (!c) { set_global_err("host allocation failed"); return VSIE_ENOMEM; }
    try {
        VSIE_CUDA(cudaGetDevice(&c->device));
        c->dZff_in = dZff;
        init_ctx(*c, body, eps_r, sigma, freq, opts, parts);
    } catch (const Error& e) {
        set_global_err(e.msg);
        destroy_ctx(c);
        return e.st;
    } catch (const std::bad_alloc&) {
        set_global_err("host allocation failed");
        destroy_ctx(c);
        return VSIE_ENOMEM;
    }
    *out = c;
    return VSIE_OK;
}

vsie_status create_from_parts(const vsie_grid* body, const double* eps_r, const double* sigma,
                              double freq, const vsie_options* opts, const vsie_parts* parts,
                              vsie_ctx** out) {
    if (!out) { set_global_err("null output pointer"); return VSIE_EINVAL; }
    Ctx* c = nullptr;
    const vsie_status st = create_from_parts_impl(body, eps_r, sigma, freq, opts, parts, nullptr, &c);
    *out = reinterpret_cast<vsie_ctx*>(c);
    return st;
}

}  // namespace vsie

using namespace vsie;

extern "C" {

const char* vsie_last_error(const vsie_ctx* ctx) {
    if (ctx) return reinterpret_cast<const Ctx*>(ctx)->err.c_str();
    std::lock_guard<std::mutex> lk(g_err_mu);
    static thread_local std::string copy;
    copy = g_err;
    return copy.c_str();
}

const char* vsie_version(void) { return "libvsie 0.1 (sm_103a)"; }

vsie_status vsie_create(const vsie_grid* body, const double* eps_r, const double* sigma,
                        double freq_hz, const vsie_options* opts, const vsie_parts* parts,
                        vsie_ctx** out) {
    return create_from_parts(body, eps_r, sigma, freq_hz, opts, parts, out);
}

vsie_status vsie_sizes(const vsie_ctx* ctx, int64_t* N, int64_t* m_f, int64_t* m_n, int64_t* n_b) {
    if (!ctx) { set_global_err("null context"); return VSIE_EINVAL; }
    const Ctx* c = reinterpret_cast<const Ctx*>(ctx);
    if (N) *N = c->N;
    if (m_f) *m_f = c->m_f;
    if (m_n) *m_n = c->m_n;
    if (n_b) *n_b = c->n_b;
    return VSIE_OK;
}

vsie_status vsie_matvec(vsie_ctx* ctx, int32_t p, const void* X, int64_t ldx, void* Y,
                        int64_t ldy, int32_t precision, vsie_stream stream) {
    if (!ctx) { set_global_err("null context"); return VSIE_EINVAL; }
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    try {
        if (!X || !Y) throw Error(VSIE_EINVAL, "null X or Y");
        if (p < 1 || p > c->max_rhs) throw Error(VSIE_EINVAL, "p outside [1, max_rhs]");
        if (ldx < c->N || ldy < c->N) throw Error(VSIE_EINVAL, "leading dimension < N");
        const size_t es = precision == VSIE_C128 ? 16 : 8;
        const char* xb = (const char*)X;
        const char* yb = (const char*)Y;
        const size_t xl = ((size_t)(p - 1) * ldx + c->N) * es, yl = ((size_t)(p - 1) * ldy + c->N) * es;
        if (!(xb + xl <= yb || yb + yl <= xb)) throw Error(VSIE_EINVAL, "X and Y overlap");
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        if (precision == VSIE_C128) {
            if (!c->f64.ready) throw Error(VSIE_EUNSUPPORTED, "context built without C128");
            matvec_impl<double>(*c, p, X, ldx, Y, ldy, st);
        } else if (precision == VSIE_C64) {
            if (!c->f32.ready) throw Error(VSIE_EUNSUPPORTED, "context built without C64");
            matvec_impl<float>(*c, p, X, ldx, Y, ldy, st);
        } else {
            throw Error(VSIE_EINVAL, "unknown precision");
        }
    } catch (const Error& e) {
        return fail(c, e);
    }
    return VSIE_OK;
}

vsie_status vsie_get_parts(vsie_ctx* ctx, vsie_parts* parts) {
    if (!ctx || !parts) { set_global_err("null context or output"); return VSIE_EINVAL; }
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    try {
        fill_parts(*c, *parts);
    } catch (const Error& e) {
        return fail(c, e);
    }
    return VSIE_OK;
}

vsie_status vsie_profile(vsie_ctx* ctx, int32_t enable) {
    if (!ctx) { set_global_err("null context"); return VSIE_EINVAL; }
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (enable) {
        cudaDeviceSynchronize();
        for (int g = 0; g < PG_N; ++g) {
            for (auto& e : c->prof.ev[g]) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
            c->prof.ev[g].clear();
            c->prof.launches[g] = 0;
            c->prof.alg_bytes[g] = 0;
        }
    }
    c->prof.on = enable != 0;
    return VSIE_OK;
}

vsie_status vsie_profile_query(vsie_ctx* ctx, int32_t group, double* ms, int64_t* launches,
                               double* alg_bytes) {
    if (!ctx) { set_global_err("null context"); return VSIE_EINVAL; }
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (group < -1 || group >= PG_N) { c->err = "unknown profiling group"; return VSIE_EINVAL; }
    if (group == -1) {
        int64_t s = 0;
        for (int g = 0; g < PG_N; ++g) s += c->prof.launches[g];
        if (launches) *launches = s;
        if (ms) *ms = 0;
        if (alg_bytes) *alg_bytes = 0;
        return VSIE_OK;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) { c->err = "device error"; return VSIE_ECUDA; }
    double t = 0;
    for (auto& e : c->prof.ev[group]) {
        float f = 0;
        if (cudaEventElapsedTime(&f, e.first, e.second) == cudaSuccess) t += f;
    }
    if (ms) *ms = t;
    if (launches) *launches = c->prof.launches[group];
    if (alg_bytes) *alg_bytes = c->prof.alg_bytes[group];
    return VSIE_OK;
}

void vsie_destroy(vsie_ctx* ctx) { destroy_ctx(reinterpret_cast<Ctx*>(ctx)); }

}  // extern "C"
