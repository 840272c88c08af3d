// vsie_setup: the hybrid-VSIE operator from geometry (Sec. III).
//
//  * RWG functions of the near (coil) and far (shield, bore) meshes (Sec. II.B);
//  * pFFT projection of each near RWG onto an s^3 voxel stencil: Tikhonov least
//    squares matching of the fields h^3 Gop(r - r_q) w_q of the stencil's voxel
//    currents to the RWG field Gop f_n on a collocation sphere (Sec. II.C, III);
//  * precorrection on near (material voxel, RWG) pairs: direct 8 x 6-point
//    coupling minus the grid's prediction (Sec. IV.C quadrature);
//  * near block with the grid part folded out: Znn~ = Z_nn - (-P^T K_grid P),
//    where P^T K_grid P is applied by this library's own FP64 matvec;
//  * far blocks: Z_ff dense; U V^H = ACA(Z_cc^fn) (Zhao et al. 2005);
//  * TT of the far coupling Z_cb^{f,chi} (1 x 1-point entries) per component:
//    matrix cross (ACA with partial pivoting, entries evaluated on the GPU) on
//    the (voxel | far RWG) unfolding, orthonormalisation of the RWG factor, and
//    truncated TT-SVD of the voxel factor over (n1, n2, n3, k) (Sec. II.D).
#include "setup.h"
#include "hostla.h"
#include "hmatrix.h"

#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <chrono>
#include <cstdio>
#include <random>
#include <cstdlib>

namespace vsie {

using hla::cd;

// Phase timing of the set-up, printed to stderr when the environment variable
// VSIE_TRACE is set.
struct PhaseTimer {
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    const bool on = std::getenv("VSIE_TRACE") != nullptr;
    void mark(const char* what) {
        if (!on) return;
        cudaDeviceSynchronize();
        const auto t = std::chrono::steady_clock::now();
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        fprintf(stderr, "[vsie setup] %-28s %8.3f s  (device free %.1f GB)\n", what,
                std::chrono::duration<double>(t - t0).count(), fr / 1e9);
        t0 = t;
    }
};

vsie_status create_from_parts_impl(const vsie_grid* body, const double* eps_r,
                                   const double* sigma, double freq, const vsie_options* opts,
                                   const vsie_parts* parts, double2* dZff, Ctx** out);
template <typename R>
void matvec_internal(Ctx& c, int p, const cx<R>* X, int64_t ldx, cx<R>* Y, int64_t ldy,
                     cudaStream_t st);
void destroy_ctx(Ctx* c);

// ------------------------------------------------------------------ meshes
MeshHost build_rwg(const vsie_mesh& mesh) {
    if (mesh.nverts < 3 || mesh.ntris < 1 || !mesh.xyz || !mesh.tri)
        throw Error(VSIE_EINVAL, "mesh needs vertices and triangles");
    MeshHost h;
    h.xyz.assign(mesh.xyz, mesh.xyz + 3 * (size_t)mesh.nverts);
    h.tri.assign(mesh.tri, mesh.tri + 3 * (size_t)mesh.ntris);
    h.ntris = mesh.ntris;
    for (int v : h.tri)
        if (v < 0 || v >= mesh.nverts) throw Error(VSIE_EINVAL, "triangle vertex out of range");
    for (double x : h.xyz)
        if (!std::isfinite(x)) throw Error(VSIE_EINVAL, "non-finite vertex coordinate");
    const int nt = mesh.ntris;
    h.area.resize(nt);
    h.centroid.resize(3 * (size_t)nt);
    h.normal.resize(3 * (size_t)nt);
    h.diam.resize(nt);
    for (int t = 0; t < nt; ++t) {
        const double* P[3];
        for (int k = 0; k < 3; ++k) P[k] = &h.xyz[3 * (size_t)h.tri[3 * t + k]];
        double e1[3], e2[3], cr[3];
        for (int d = 0; d < 3; ++d) {
            e1[d] = P[1][d] - P[0][d];
            e2[d] = P[2][d] - P[0][d];
        }
        cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
        cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
        cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
        const double n2 = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        if (!(n2 > 0)) throw Error(VSIE_EINVAL, "degenerate triangle");
        h.area[t] = 0.5 * n2;
        double dmax = 0;
        for (int k = 0; k < 3; ++k) {
            double s = 0;
            for (int d = 0; d < 3; ++d) {
                const double q = P[(k + 1) % 3][d] - P[k][d];
                s += q * q;
            }
            dmax = std::max(dmax, std::sqrt(s));
        }
        h.diam[t] = dmax;
        for (int d = 0; d < 3; ++d) {
            h.normal[3 * t + d] = cr[d] / n2;
            h.centroid[3 * t + d] = (P[0][d] + P[1][d] + P[2][d]) / 3.0;
        }
    }
    // interior edges: (min, max) vertex pair shared by exactly two triangles
    std::map<std::pair<int, int>, std::vector<std::pair<int, int>>> emap;
    for (int t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) {
            const int a = h.tri[3 * t + (k + 1) % 3], b = h.tri[3 * t + (k + 2) % 3];
            emap[{std::min(a, b), std::max(a, b)}].push_back({t, h.tri[3 * t + k]});
        }
    std::map<std::pair<int, int>, int> index;
    for (auto& kv : emap) {
        if (kv.second.size() > 2) throw Error(VSIE_EINVAL, "non-manifold edge (more than 2 triangles)");
        if (kv.second.size() != 2) continue;
        auto pr = kv.second;
        std::sort(pr.begin(), pr.end());
        index[kv.first] = h.m++;
        h.tplus.push_back(pr[0].first);
        h.vplus.push_back(pr[0].second);
        h.tminus.push_back(pr[1].first);
        h.vminus.push_back(pr[1].second);
        const double* A = &h.xyz[3 * (size_t)kv.first.first];
        const double* B = &h.xyz[3 * (size_t)kv.first.second];
        h.len.push_back(std::sqrt((A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) +
                                  (A[2] - B[2]) * (A[2] - B[2])));
    }
    if (h.m == 0) throw Error(VSIE_EINVAL, "mesh has no interior edges");
    for (int p = 0; p < mesh.nports; ++p) {
        const int a = mesh.ports[2 * p], b = mesh.ports[2 * p + 1];
        auto it = index.find({std::min(a, b), std::max(a, b)});
        if (it == index.end()) throw Error(VSIE_EINVAL, "port is not an interior edge");
        h.ports.push_back(it->second);
    }
    return h;
}

template <typename T>
static T* up(Ctx& c, const std::vector<T>& v) {
    T* d = (T*)dalloc(c, v.size() * sizeof(T));
    if (!v.empty()) VSIE_CUDA(cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return d;
}

MeshDev upload_mesh(Ctx& c, const MeshHost& h) {
    MeshDev d;
    d.xyz = up(c, h.xyz);
    d.tri = up(c, h.tri);
    d.area = up(c, h.area);
    d.centroid = up(c, h.centroid);
    d.normal = up(c, h.normal);
    d.diam = up(c, h.diam);
    d.tplus = up(c, h.tplus);
    d.tminus = up(c, h.tminus);
    d.vplus = up(c, h.vplus);
    d.vminus = up(c, h.vminus);
    d.len = up(c, h.len);
    d.ntris = h.ntris;
    d.m = h.m;
    return d;
}

// ------------------------------------------------------------------ host physics
// (k0^2 I + grad grad) g at R (closed form), times h^3; self term at R = 0.
static void voxel_kernel_host(int dx, int dy, int dz, double h, double k0, cd T[3][3]) {
    if (dx == 0 && dy == 0 && dz == 0) {
        const double a = std::cbrt(3.0 / (4.0 * M_PI)) * h;
        const cd s = (2.0 / 3.0) * cd(1.0, k0 * a) * std::exp(cd(0.0, -k0 * a)) - 1.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) T[i][j] = i == j ? s : 0.0;
        return;
    }
    const double r[3] = {h * dx, h * dy, h * dz};
    const double R = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    const cd g = std::exp(cd(0.0, -k0 * R)) / (4.0 * M_PI * R);
    const double kR = k0 * R;
    const cd A = g / (R * R) * cd(kR * kR - 1.0, -kR);
    const cd B = g / (R * R) * cd(3.0 - kR * kR, 3.0 * kR);
    const double h3 = h * h * h;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[i][j] = h3 * ((i == j ? A : 0.0) + B * (r[i] / R) * (r[j] / R));
}

static void dyad_host(const double r[3], double k0, cd D[3][3]) {
    const double R = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    const cd g = std::exp(cd(0.0, -k0 * R)) / (4.0 * M_PI * R);
    const double kR = k0 * R;
    const cd A = g / (R * R) * cd(kR * kR - 1.0, -kR);
    const cd B = g / (R * R) * cd(3.0 - kR * kR, 3.0 * kR);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) D[i][j] = (i == j ? A : 0.0) + B * (r[i] / R) * (r[j] / R);
}

// ------------------------------------------------------------------ device helpers
// max |x_i| over i with used[i] == 0, and sum |x_i|^2; per-block partials
__global__ void k_absmax(const double2* __restrict__ x, int64_t n, const uint8_t* __restrict__ used,
                         double* __restrict__ bv, int64_t* __restrict__ bi, double* __restrict__ bs) {
    __shared__ double sv[256];
    __shared__ int64_t si[256];
    __shared__ double ss[256];
    double v = -1.0, s = 0.0;
    int64_t idx = -1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double a = x[i].x * x[i].x + x[i].y * x[i].y;
        s += a;
        if ((!used || !used[i]) && a > v) { v = a; idx = i; }
    }
    sv[threadIdx.x] = v;
    si[threadIdx.x] = idx;
    ss[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const int o = threadIdx.x + w;
            if (sv[o] > sv[threadIdx.x] || (sv[o] == sv[threadIdx.x] && si[o] >= 0 &&
                                             (si[threadIdx.x] < 0 || si[o] < si[threadIdx.x]))) {
                sv[threadIdx.x] = sv[o];
                si[threadIdx.x] = si[o];
            }
            ss[threadIdx.x] += ss[o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        bv[blockIdx.x] = sv[0];
        bi[blockIdx.x] = si[0];
        bs[blockIdx.x] = ss[0];
    }
}

struct Scratch {
    Ctx c;   // owns the set-up's temporary device allocations
    double* bv = nullptr;
    int64_t* bi = nullptr;
    double* bs = nullptr;
    Scratch() {
        // split-K workspace of the set-up's GEMMs (Gram matrices of the TT factors
        // reduce over ~10^7 columns at the 1 mm head grid)
        c.f64.splitk_elems = (size_t)4 << 20;
        c.f64.splitk = (double2*)dalloc(c, c.f64.splitk_elems * sizeof(double2));
    }
    ~Scratch() {
        for (void* p : c.allocs) cudaFree(p);
    }
};

// argmax over unused entries (first index on ties) and squared 2-norm
static void absmax(Scratch& S, const double2* x, int64_t n, const uint8_t* used, int64_t& imax,
                   double& nrm2) {
    const int nbk = 256;
    if (!S.bv) {
        S.bv = (double*)dalloc(S.c, nbk * sizeof(double));
        S.bi = (int64_t*)dalloc(S.c, nbk * sizeof(int64_t));
        S.bs = (double*)dalloc(S.c, nbk * sizeof(double));
    }
    double* bv = S.bv;
    int64_t* bi = S.bi;
    double* bs = S.bs;
    k_absmax<<<nbk, 256>>>(x, n, used, bv, bi, bs);
    VSIE_CUDA(cudaGetLastError());
    double hv[nbk], hs[nbk];
    int64_t hi[nbk];
    VSIE_CUDA(cudaMemcpy(hv, bv, sizeof(hv), cudaMemcpyDeviceToHost));
    VSIE_CUDA(cudaMemcpy(hi, bi, sizeof(hi), cudaMemcpyDeviceToHost));
    VSIE_CUDA(cudaMemcpy(hs, bs, sizeof(hs), cudaMemcpyDeviceToHost));
    double best = -1.0;
    imax = -1;
    nrm2 = 0.0;
    for (int b = 0; b < nbk; ++b) {
        nrm2 += hs[b];
        if (hi[b] >= 0 && (hv[b] > best || (hv[b] == best && hi[b] < imax))) {
            best = hv[b];
            imax = hi[b];
        }
    }
}

__global__ void k_scale_col(double2* x, int64_t n, double2 s) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = cmul(x[i], s);
}

__global__ void k_to_f32(const double2* __restrict__ a, float2* __restrict__ b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

void convert_to_f32(const double2* a, float2* b, size_t n) {
    k_to_f32<<<2048, 256>>>(a, b, n);
    VSIE_CUDA(cudaGetLastError());
}

static inline double2 d2(cd z) { return make_double2(z.real(), z.imag()); }
static inline cd cdv(double2 z) { return cd(z.x, z.y); }

// ------------------------------------------------------------------ ACA
// Partial-pivoting ACA of an m x n matrix whose rows/columns are written into
// device buffers by callbacks; Z ~= U V^H with U (m x k) and V (n x k) kept on
// the device (capacity kmax columns each).  Stops when ||u_k|| ||v_k|| <=
// tol ||Z_k||_F with ||Z_k||_F updated recursively (Zhao et al. 2005).  All
// vector work runs on the GPU; the host only handles scalars.
struct AcaResult {
    int k = 0;
    std::vector<int64_t> rows, cols;   // pivot row / column of each cross
};

__global__ void k_conj_scale(double2* x, int64_t n, double2 s) {
    // x = conj(x * s)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 t = cmul(x[i], s);
        x[i] = make_double2(t.x, -t.y);
    }
}

template <typename RowF, typename ColF>
static AcaResult aca_device(Scratch& S, int64_t m, int64_t n, double tol, int kmax, RowF get_row,
                            ColF get_col, double2* Ud, double2* Vd) {
    // Vd columns hold conj(v_k) (so that Z ~= U V^H); the residual row uses
    // v_k = conj(Vd[:, k]).
    AcaResult out;
    uint8_t* used_r = (uint8_t*)dalloc(S.c, m);
    uint8_t* used_c = (uint8_t*)dalloc(S.c, n);
    VSIE_CUDA(cudaMemset(used_r, 0, m));
    VSIE_CUDA(cudaMemset(used_c, 0, n));
    double2* col = (double2*)dalloc(S.c, m * sizeof(double2));
    double2* row = (double2*)dalloc(S.c, n * sizeof(double2));
    double2* coef = (double2*)dalloc(S.c, (size_t)std::max(kmax, 1) * sizeof(double2));
    double2* dots = (double2*)dalloc(S.c, (size_t)std::max(kmax, 1) * sizeof(double2));
    double2* dots2 = (double2*)dalloc(S.c, (size_t)std::max(kmax, 1) * sizeof(double2));
    int64_t i = 0;
    double norm2 = 0.0;
    int k = 0;
    const double2 one = make_double2(1, 0), zero = make_double2(0, 0), mone = make_double2(-1, 0);
    const uint8_t one_b = 1;
    for (int it = 0; it < kmax && k < kmax; ++it) {
        VSIE_CUDA(cudaMemcpy(used_r + i, &one_b, 1, cudaMemcpyHostToDevice));
        get_row(i, row);
        if (k > 0) {
            // row -= sum_l U[i, l] v_l,  v_l = conj(Vd[:, l]):
            //   conj(row) -= Vd[:, :k] conj(U[i, :k])
            VSIE_CUDA(cudaMemcpy2D(coef, sizeof(double2), Ud + i, m * sizeof(double2),
                                   sizeof(double2), k, cudaMemcpyDeviceToDevice));
            k_conj_scale<<<64, 256>>>(row, n, one);             // row <- conj(row)
            k_conj_scale<<<1, 256>>>(coef, k, one);             // coef <- conj(U[i, :])
            cgemm<double>(S.c, OP_N, (int)n, 1, k, mone, Vd, n, 0, coef, k, 0, one, row, n, 0, 1,
                          nullptr, nullptr, 0);
            k_conj_scale<<<64, 256>>>(row, n, one);             // back to row
            VSIE_CUDA(cudaGetLastError());
        }
        int64_t jm;
        double rn2;
        absmax(S, row, n, used_c, jm, rn2);
        double2 piv = make_double2(0, 0);
        if (jm >= 0) VSIE_CUDA(cudaMemcpy(&piv, row + jm, sizeof(double2), cudaMemcpyDeviceToHost));
        if (jm < 0 || (piv.x == 0.0 && piv.y == 0.0)) {
            // zero residual row: try the next unused row
            std::vector<uint8_t> ur(m);
            VSIE_CUDA(cudaMemcpy(ur.data(), used_r, m, cudaMemcpyDeviceToHost));
            int64_t q = 0;
            while (q < m && ur[q]) ++q;
            if (q == m) break;
            i = q;
            continue;
        }
        VSIE_CUDA(cudaMemcpy(used_c + jm, &one_b, 1, cudaMemcpyHostToDevice));
        out.rows.push_back(i);
        out.cols.push_back(jm);
        // v = row / piv, stored conjugated in Vd[:, k]
        const cd ip = 1.0 / cdv(piv);
        VSIE_CUDA(cudaMemcpy(Vd + (size_t)n * k, row, n * sizeof(double2), cudaMemcpyDeviceToDevice));
        k_conj_scale<<<64, 256>>>(Vd + (size_t)n * k, n, d2(ip));
        // residual column: col -= U[:, :k] v[jm, :k],  v_l[jm] = conj(Vd[jm, l])
        get_col(jm, col);
        if (k > 0) {
            VSIE_CUDA(cudaMemcpy2D(coef, sizeof(double2), Vd + jm, n * sizeof(double2),
                                   sizeof(double2), k, cudaMemcpyDeviceToDevice));
            k_conj_scale<<<1, 256>>>(coef, k, one);
            cgemm<double>(S.c, OP_N, (int)m, 1, k, mone, Ud, m, 0, coef, k, 0, one, col, m, 0, 1,
                          nullptr, nullptr, 0);
        }
        VSIE_CUDA(cudaGetLastError());
        int64_t inext;
        double nu2;
        absmax(S, col, m, used_r, inext, nu2);
        int64_t dummy;
        double nv2;
        absmax(S, Vd + (size_t)n * k, n, nullptr, dummy, nv2);
        double cross = 0.0;
        if (k > 0) {
            // (u_l^H u)(v_l^H v) with v = conj(Vd): v_l^H v = conj(Vd_l^H Vd_k)
            cgemm<double>(S.c, OP_H, k, 1, (int)m, one, Ud, m, 0, col, m, 0, zero, dots, k, 0, 1,
                          nullptr, nullptr, 0);
            cgemm<double>(S.c, OP_H, k, 1, (int)n, one, Vd, n, 0, Vd + (size_t)n * k, n, 0, zero,
                          dots2, k, 0, 1, nullptr, nullptr, 0);
            std::vector<double2> a(k), b(k);
            VSIE_CUDA(cudaMemcpy(a.data(), dots, k * sizeof(double2), cudaMemcpyDeviceToHost));
            VSIE_CUDA(cudaMemcpy(b.data(), dots2, k * sizeof(double2), cudaMemcpyDeviceToHost));
            for (int l = 0; l < k; ++l) cross += 2.0 * std::real(cdv(a[l]) * std::conj(cdv(b[l])));
        }
        VSIE_CUDA(cudaMemcpy(Ud + (size_t)m * k, col, m * sizeof(double2), cudaMemcpyDeviceToDevice));
        ++k;
        norm2 += cross + nu2 * nv2;
        if (std::sqrt(nu2 * nv2) <= tol * std::sqrt(std::max(norm2, 0.0))) break;
        if (inext < 0) break;
        i = inext;
    }
    out.k = k;
    return out;
}

// ------------------------------------------------------------------ truncated factorisation
// A (m x c, device, ld m) ~= Lf (m x r) Rf (r x c) with orthonormal Lf, keeping
// the smallest r whose discarded Frobenius energy is <= delta^2.
struct Factor {
    int r = 0;
    double2* L = nullptr;   // device m x r
    double2* R = nullptr;   // device r x c
};

static double frob2(Scratch& S, const double2* A, int64_t n) {
    int64_t im;
    double s;
    absmax(S, A, n, nullptr, im, s);
    return s;
}

static int rank_from(const std::vector<double>& lam, double total2, double delta2) {
    double kept = 0.0;
    const int n = (int)lam.size();
    for (int r = 0; r <= n; ++r) {
        if (total2 - kept <= delta2) return std::max(r, 1);
        if (r < n) kept += std::max(lam[r], 0.0);
    }
    return -1;   // not enough captured energy
}

static Factor truncate(Scratch& S, const double2* A, int m, int c, double delta2, uint64_t seed) {
    const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
    const double tot = frob2(S, A, (int64_t)m * c);
    Factor F;
    if (m <= 512 || c <= 512) {
        const bool left = m <= c;
        const int q = left ? m : c;
        double2* G = (double2*)dalloc(S.c, (size_t)q * q * sizeof(double2));
        if (left) cgemm2<double>(S.c, OP_N, OP_H, m, m, c, one, A, m, 0, A, m, 0, zero, G, m, 0, 1, nullptr, nullptr, 0);
        else cgemm<double>(S.c, OP_H, c, c, m, one, A, m, 0, A, m, 0, zero, G, c, 0, 1, nullptr, nullptr, 0);
        std::vector<double2> hg((size_t)q * q);
        VSIE_CUDA(cudaMemcpy(hg.data(), G, hg.size() * sizeof(double2), cudaMemcpyDeviceToHost));
        std::vector<cd> H(hg.size());
        for (size_t i = 0; i < hg.size(); ++i) H[i] = cdv(hg[i]);
        // symmetrise
        for (int j = 0; j < q; ++j)
            for (int i = 0; i < j; ++i) {
                const cd a = 0.5 * (H[i + (size_t)q * j] + std::conj(H[j + (size_t)q * i]));
                H[i + (size_t)q * j] = a;
                H[j + (size_t)q * i] = std::conj(a);
            }
        std::vector<double> w;
        std::vector<cd> V;
        hla::herm_eig(q, H, w, V);
        int r = rank_from(w, tot, delta2);
        if (r < 0) r = q;
        r = std::min(r, q);
        while (r > 1 && !(w[r - 1] > 1e-300)) --r;
        F.r = r;
        F.L = (double2*)dalloc(S.c, (size_t)m * r * sizeof(double2));
        F.R = (double2*)dalloc(S.c, (size_t)r * c * sizeof(double2));
        if (left) {
            std::vector<double2> hv((size_t)m * r);
            for (int k = 0; k < r; ++k)
                for (int i = 0; i < m; ++i) hv[i + (size_t)m * k] = d2(V[i + (size_t)m * k]);
            VSIE_CUDA(cudaMemcpy(F.L, hv.data(), hv.size() * sizeof(double2), cudaMemcpyHostToDevice));
            cgemm<double>(S.c, OP_H, r, c, m, one, F.L, m, 0, A, m, 0, zero, F.R, r, 0, 1, nullptr, nullptr, 0);
        } else {
            // right singular vectors Vr (c x r): L = A Vr diag(1/s), R = diag(s) Vr^H
            std::vector<double2> hv((size_t)c * r), hr((size_t)r * c);
            for (int k = 0; k < r; ++k) {
                const double s = std::sqrt(std::max(w[k], 0.0));
                for (int i = 0; i < c; ++i) {
                    hv[i + (size_t)c * k] = d2(V[i + (size_t)c * k] / s);
                    hr[k + (size_t)r * i] = d2(s * std::conj(V[i + (size_t)c * k]));
                }
            }
            double2* Vd = (double2*)dalloc(S.c, hv.size() * sizeof(double2));
            VSIE_CUDA(cudaMemcpy(Vd, hv.data(), hv.size() * sizeof(double2), cudaMemcpyHostToDevice));
            cgemm<double>(S.c, OP_N, m, r, c, one, A, m, 0, Vd, c, 0, zero, F.L, m, 0, 1, nullptr, nullptr, 0);
            VSIE_CUDA(cudaMemcpy(F.R, hr.data(), hr.size() * sizeof(double2), cudaMemcpyHostToDevice));
        }
        return F;
    }
    // randomized range finder with one power iteration, adaptive sample size
    std::mt19937_64 gen(seed);
    std::normal_distribution<double> N01;
    for (int s0 = 64;; s0 *= 2) {
        s0 = std::min(s0, std::min(m, c));
        std::vector<double2> om((size_t)c * s0);
        for (auto& z : om) z = make_double2(N01(gen), N01(gen));
        double2* Om = (double2*)dalloc(S.c, om.size() * sizeof(double2));
        VSIE_CUDA(cudaMemcpy(Om, om.data(), om.size() * sizeof(double2), cudaMemcpyHostToDevice));
        double2* Y = (double2*)dalloc(S.c, (size_t)m * s0 * sizeof(double2));
        double2* Zt = (double2*)dalloc(S.c, (size_t)c * s0 * sizeof(double2));
        cgemm<double>(S.c, OP_N, m, s0, c, one, A, m, 0, Om, c, 0, zero, Y, m, 0, 1, nullptr, nullptr, 0);
        cgemm<double>(S.c, OP_H, c, s0, m, one, A, m, 0, Y, m, 0, zero, Zt, c, 0, 1, nullptr, nullptr, 0);
        cgemm<double>(S.c, OP_N, m, s0, c, one, A, m, 0, Zt, c, 0, zero, Y, m, 0, 1, nullptr, nullptr, 0);
        std::vector<double2> hy((size_t)m * s0);
        VSIE_CUDA(cudaMemcpy(hy.data(), Y, hy.size() * sizeof(double2), cudaMemcpyDeviceToHost));
        std::vector<cd> Yh(hy.size());
        for (size_t i = 0; i < hy.size(); ++i) Yh[i] = cdv(hy[i]);
        const std::vector<cd> Q = hla::qr_q(m, s0, Yh);
        for (size_t i = 0; i < Q.size(); ++i) hy[i] = d2(Q[i]);
        VSIE_CUDA(cudaMemcpy(Y, hy.data(), hy.size() * sizeof(double2), cudaMemcpyHostToDevice));
        double2* B = (double2*)dalloc(S.c, (size_t)s0 * c * sizeof(double2));
        cgemm<double>(S.c, OP_H, s0, c, m, one, Y, m, 0, A, m, 0, zero, B, s0, 0, 1, nullptr, nullptr, 0);
        Factor Fb = truncate(S, B, s0, c, delta2, seed + 1);   // s0 <= 512: Gram path
        // captured energy check: ||A||^2 - ||B||^2 must be within delta2 for the rank found
        const double capt = frob2(S, B, (int64_t)s0 * c);
        if (tot - capt > delta2 && s0 < std::min(m, c) && s0 < 512) continue;
        F.r = Fb.r;
        F.L = (double2*)dalloc(S.c, (size_t)m * F.r * sizeof(double2));
        cgemm<double>(S.c, OP_N, m, F.r, s0, one, Y, m, 0, Fb.L, s0, 0, zero, F.L, m, 0, 1, nullptr, nullptr, 0);
        F.R = Fb.R;
        return F;
    }
}

// In-place inverse of a small n x n FP64 complex matrix on the device (LU).
static void invert_f64(Scratch& S, double2* A, int n) {
    cusolverDnHandle_t h = nullptr;
    if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) throw Error(VSIE_ECUDA, "cusolverDnCreate");
    int lwork = 0;
    cusolverDnZgetrf_bufferSize(h, n, n, (cuDoubleComplex*)A, n, &lwork);
    cuDoubleComplex* work = (cuDoubleComplex*)dalloc(S.c, (size_t)std::max(lwork, 1) * sizeof(double2));
    int* ipiv = (int*)dalloc(S.c, (size_t)n * sizeof(int));
    int* info = (int*)dalloc(S.c, sizeof(int));
    double2* B = (double2*)dalloc(S.c, (size_t)n * n * sizeof(double2));
    std::vector<double2> I((size_t)n * n, make_double2(0, 0));
    for (int i = 0; i < n; ++i) I[i + (size_t)n * i] = make_double2(1, 0);
    VSIE_CUDA(cudaMemcpy(B, I.data(), I.size() * sizeof(double2), cudaMemcpyHostToDevice));
    const bool ok = cusolverDnZgetrf(h, n, n, (cuDoubleComplex*)A, n, work, ipiv, info) == CUSOLVER_STATUS_SUCCESS &&
                    cusolverDnZgetrs(h, CUBLAS_OP_N, n, n, (cuDoubleComplex*)A, n, ipiv, (cuDoubleComplex*)B, n, info) == CUSOLVER_STATUS_SUCCESS;
    cusolverDnDestroy(h);
    if (!ok) throw Error(VSIE_ECUDA, "skeleton core inversion failed");
    VSIE_CUDA(cudaMemcpy(A, B, (size_t)n * n * sizeof(double2), cudaMemcpyDeviceToDevice));
}

static std::vector<cd> to_host(const double2* d, size_t n) {
    std::vector<double2> h(n);
    if (n) VSIE_CUDA(cudaMemcpy(h.data(), d, n * sizeof(double2), cudaMemcpyDeviceToHost));
    std::vector<cd> o(n);
    for (size_t i = 0; i < n; ++i) o[i] = cdv(h[i]);
    return o;
}

// ------------------------------------------------------------------ set-up driver
struct Built {
    std::vector<cd> W, pre_val, Znn, U, V, tt[3][4];
    std::vector<cd> Znn_direct;   // Z_nn = -K_nn itself (the near-near block of the operator)
    std::vector<int32_t> base, pre_col;
    std::vector<int64_t> pre_row;
    int aca_rank = 0;
    int tt_rank[3][3] = {{0}};
    double2* dZff = nullptr;   // device, owned by the scratch until handed over
};

static void setup_impl(const vsie_grid* body, const double* eps_r, const double* sigma,
                       const vsie_mesh* coil, const vsie_mesh* shield, double freq,
                       const vsie_options* opts_in, Ctx** out) {
    if (!body || !eps_r || !sigma) throw Error(VSIE_EINVAL, "null body grid or material map");
    if (!(freq > 0) || !std::isfinite(freq)) throw Error(VSIE_EINVAL, "frequency must be > 0");
    vsie_options o{};
    if (opts_in) o = *opts_in;
    const int s = o.stencil > 0 ? o.stencil : 3;
    if (s % 2 == 0) throw Error(VSIE_EINVAL, "pFFT stencil must be odd");
    const int nearr = o.near_radius > 0 ? o.near_radius : s + 1;
    const double rfac = o.colloc_rfac > 0 ? o.colloc_rfac : 2.0;
    const double tt_tol = o.tt_tol > 0 ? o.tt_tol : 1e-6;
    const double aca_tol = o.aca_tol > 0 ? o.aca_tol : 1e-6;
    const double omega = 2.0 * M_PI * freq, k0 = omega / kC0;
    const double h = body->h;
    int nb[3], ne[3], off[3];
    for (int i = 0; i < 3; ++i) {
        nb[i] = body->n[i];
        ne[i] = o.ext_n[i] > 0 ? o.ext_n[i] : nb[i];
        off[i] = o.ext_n[i] > 0 ? o.ext_offset[i] : 0;
        if (nb[i] < 1 || off[i] < 0 || off[i] + nb[i] > ne[i])
            throw Error(VSIE_EINVAL, "body grid does not fit in the extended grid");
    }
    if (!(h > 0)) throw Error(VSIE_EINVAL, "voxel size h must be > 0");
    const int64_t n_b = (int64_t)nb[0] * nb[1] * nb[2];
    double eorig[3];
    for (int i = 0; i < 3; ++i) eorig[i] = body->origin[i] - h * off[i];
    std::vector<uint8_t> mat(n_b);
    for (int64_t v = 0; v < n_b; ++v) mat[v] = (eps_r[v] != 1.0 || sigma[v] != 0.0) ? 1 : 0;

    Scratch S;
    VSIE_CUDA(cudaGetDevice(&S.c.device));
    PhaseTimer T;
    Built B;
    MeshHost mh_c, mh_s;
    MeshDev md_c, md_s;
    const bool has_c = coil && coil->ntris > 0, has_s = shield && shield->ntris > 0;
    if (has_c) { mh_c = build_rwg(*coil); md_c = upload_mesh(S.c, mh_c); }
    if (has_s) { mh_s = build_rwg(*shield); md_s = upload_mesh(S.c, mh_s); }
    const int m_n = has_c ? mh_c.m : 0, m_f = has_s ? mh_s.m : 0;
    T.mark("meshes");
    const int s3 = s * s * s;
    const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
    GridDev gb;
    for (int i = 0; i < 3; ++i) { gb.n[i] = nb[i]; gb.origin[i] = body->origin[i]; }
    gb.h = h;

    if (has_c) {
        // --- pFFT projection
        const int Nc = 6 * s3;
        std::vector<double> col(3 * (size_t)Nc);
        const double rad = rfac * s * h / 2.0;
        for (int k = 0; k < Nc; ++k) {
            const double z = 1.0 - (2.0 * k + 1.0) / Nc;
            const double rr = std::sqrt(std::max(0.0, 1.0 - z * z));
            const double ph = k * M_PI * (3.0 - std::sqrt(5.0));
            col[3 * k] = rad * rr * std::cos(ph);
            col[3 * k + 1] = rad * rr * std::sin(ph);
            col[3 * k + 2] = rad * z;
        }
        const int hs = (s - 1) / 2;
        std::vector<cd> A((size_t)3 * Nc * 3 * s3);
        for (int q = 0; q < s3; ++q) {
            const int qx = q % s - hs, qy = (q / s) % s - hs, qz = q / (s * s) - hs;
            for (int cI = 0; cI < Nc; ++cI) {
                const double r[3] = {col[3 * cI] - h * qx, col[3 * cI + 1] - h * qy,
                                     col[3 * cI + 2] - h * qz};
                cd D[3][3];
                dyad_host(r, k0, D);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        A[(a * Nc + cI) + (size_t)(3 * Nc) * (b * s3 + q)] = h * h * h * D[a][b];
            }
        }
        const std::vector<cd> X = hla::tikhonov_pinv(3 * Nc, 3 * s3, A, 1e-10);   // 3s3 x 3Nc
        // stencil centres and RWG fields at the collocation points
        std::vector<int> ic(3 * (size_t)m_n);
        std::vector<double> ctr(3 * (size_t)m_n);
        B.base.resize(3 * (size_t)m_n);
        for (int n = 0; n < m_n; ++n)
            for (int d = 0; d < 3; ++d) {
                const double cn = 0.5 * (mh_c.centroid[3 * mh_c.tplus[n] + d] +
                                         mh_c.centroid[3 * mh_c.tminus[n] + d]);
                const int i = (int)std::nearbyint((cn - eorig[d]) / h);
                if (i - hs < 0 || i + hs >= ne[d])
                    throw Error(VSIE_EINVAL, "pFFT stencil leaves the extended grid");
                ic[3 * n + d] = i;
                ctr[3 * n + d] = eorig[d] + h * i;
                B.base[3 * n + d] = i - hs;
            }
        double* dcol = up(S.c, col);
        double* dctr = up(S.c, ctr);
        double2* E = (double2*)dalloc(S.c, (size_t)3 * Nc * m_n * sizeof(double2));
        field_points(md_c, Nc, dcol, m_n, nullptr, dctr, k0, E);
        std::vector<double2> hX((size_t)3 * s3 * 3 * Nc);
        for (size_t i = 0; i < hX.size(); ++i) hX[i] = d2(X[i]);
        double2* dX = (double2*)dalloc(S.c, hX.size() * sizeof(double2));
        VSIE_CUDA(cudaMemcpy(dX, hX.data(), hX.size() * sizeof(double2), cudaMemcpyHostToDevice));
        double2* dW = (double2*)dalloc(S.c, (size_t)3 * s3 * m_n * sizeof(double2));
        cgemm<double>(S.c, OP_N, 3 * s3, m_n, 3 * Nc, one, dX, 3 * s3, 0, E, 3 * Nc, 0, zero, dW,
                      3 * s3, 0, 1, nullptr, nullptr, 0);
        B.W = to_host(dW, (size_t)3 * s3 * m_n);   // column n = row n of W (3 s3 per RWG)
        T.mark("pFFT projection");

        // --- precorrection on near pairs
        std::vector<std::vector<std::pair<int32_t, cd>>> rows(3 * (size_t)n_b);
        for (int n = 0; n < m_n; ++n) {
            int lo[3], hi[3];
            bool any = true;
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::max(ic[3 * n + d] - off[d] - nearr, 0);
                hi[d] = std::min(ic[3 * n + d] - off[d] + nearr, nb[d] - 1);
                if (hi[d] < lo[d]) any = false;
            }
            if (!any) continue;
            std::vector<int64_t> vox;
            for (int z = lo[2]; z <= hi[2]; ++z)
                for (int y = lo[1]; y <= hi[1]; ++y)
                    for (int x = lo[0]; x <= hi[0]; ++x) {
                        const int64_t v = x + (int64_t)nb[0] * (y + (int64_t)nb[1] * z);
                        if (mat[v]) vox.push_back(v);
                    }
            if (vox.empty()) continue;
            const int nv = (int)vox.size();
            int64_t* dv = up(S.c, vox);
            double2* Kd = (double2*)dalloc(S.c, (size_t)3 * nv * sizeof(double2));
            const int ncol = n;
            int* dcolp = up(S.c, std::vector<int>{ncol});
            coupling_block(md_c, gb, nv, dv, 1, dcolp, k0, true, 1.0, Kd, nv, nv);
            const std::vector<cd> kd = to_host(Kd, (size_t)3 * nv);
            const cd* w = &B.W[(size_t)3 * s3 * n];
            for (int iv = 0; iv < nv; ++iv) {
                const int64_t v = vox[iv];
                const int px = (int)(v % nb[0]) + off[0], py = (int)((v / nb[0]) % nb[1]) + off[1],
                          pz = (int)(v / ((int64_t)nb[0] * nb[1])) + off[2];
                cd kg[3] = {0.0, 0.0, 0.0};
                for (int q = 0; q < s3; ++q) {
                    const int qx = B.base[3 * n] + q % s, qy = B.base[3 * n + 1] + (q / s) % s,
                              qz = B.base[3 * n + 2] + q / (s * s);
                    cd T[3][3];
                    voxel_kernel_host(px - qx, py - qy, pz - qz, h, k0, T);
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) kg[a] += T[a][b] * w[b * s3 + q];
                }
                const double h3 = h * h * h;
                for (int a = 0; a < 3; ++a) {
                    const cd S_ = kd[(size_t)a * nv + iv] - h3 * kg[a];
                    rows[(size_t)a * n_b + v].push_back({n, -S_});
                }
            }
        }
        B.pre_row.assign(3 * (size_t)n_b + 1, 0);
        for (size_t r = 0; r < rows.size(); ++r) {
            std::sort(rows[r].begin(), rows[r].end(),
                      [](const std::pair<int32_t, cd>& x, const std::pair<int32_t, cd>& y) { return x.first < y.first; });
            B.pre_row[r + 1] = B.pre_row[r] + (int64_t)rows[r].size();
            for (auto& e : rows[r]) {
                B.pre_col.push_back(e.first);
                B.pre_val.push_back(e.second);
            }
        }

        T.mark("precorrection");
        // --- direct near block and the grid part P^T K P: Znn~ = Z_nn - (-h^3 P^T T P),
        // the grid part summed directly over stencil pairs (it equals the grid
        // convolution exactly; see ptkp_add)
        double2* Knn = (double2*)dalloc(S.c, (size_t)m_n * m_n * sizeof(double2));
        efie_block(md_c, md_c, true, m_n, nullptr, m_n, nullptr, k0, -1.0, Knn, m_n);
        B.Znn_direct = to_host(Knn, (size_t)m_n * m_n);
        {
            int* dbase = up(S.c, B.base);
            const double a = std::cbrt(3.0 / (4.0 * M_PI)) * h;
            const cd sv = (2.0 / 3.0) * cd(1.0, k0 * a) * std::exp(cd(0.0, -k0 * a)) - 1.0;
            ptkp_add(m_n, s, dW, dbase, h, k0, d2(sv), Knn, m_n);
        }
        std::vector<cd> Znn = to_host(Knn, (size_t)m_n * m_n);
        B.Znn = std::move(Znn);
        T.mark("near block");
    }

    if (has_s) {
        // --- far-far dense block (device, FP64)
        B.dZff = (double2*)dalloc(S.c, (size_t)m_f * m_f * sizeof(double2));
        efie_block(md_s, md_s, true, m_f, nullptr, m_f, nullptr, k0, -1.0, B.dZff, m_f);
        T.mark("far-far block");
        // --- near-far block by ACA
        if (has_c) {
            double2* Zfn = (double2*)dalloc(S.c, (size_t)m_n * m_f * sizeof(double2));
            efie_block(md_c, md_s, false, m_n, nullptr, m_f, nullptr, k0, -1.0, Zfn, m_n);
            const int kmax = std::min(m_n, m_f);
            double2* Ud = (double2*)dalloc(S.c, (size_t)m_n * std::max(kmax, 1) * sizeof(double2));
            double2* Vd = (double2*)dalloc(S.c, (size_t)m_f * std::max(kmax, 1) * sizeof(double2));
            auto row = [&](int64_t i, double2* dst) {
                VSIE_CUDA(cudaMemcpy2D(dst, sizeof(double2), Zfn + i, m_n * sizeof(double2),
                                       sizeof(double2), m_f, cudaMemcpyDeviceToDevice));
            };
            auto colf = [&](int64_t j, double2* dst) {
                VSIE_CUDA(cudaMemcpy(dst, Zfn + (size_t)m_n * j, m_n * sizeof(double2),
                                     cudaMemcpyDeviceToDevice));
            };
            AcaResult ar = aca_device(S, m_n, m_f, aca_tol, kmax, row, colf, Ud, Vd);
            B.aca_rank = ar.k;
            B.U = to_host(Ud, (size_t)m_n * ar.k);
            B.V = to_host(Vd, (size_t)m_f * ar.k);
            T.mark("near-far ACA");
        }
        // --- TT of the far coupling, per component.  Cross approximation: ACA on a
        // sub-sample of the voxels (every `st`-th voxel per axis, ends included)
        // picks the pivot voxels I and far RWG J; the skeleton
        //   Z ~= Z[:, J] Z[I, J]^-1 Z[I, :]
        // is then formed over all voxels (U = Z[:, J], V^H = Z[I, J]^-1 Z[I, :]).
        int stv = 1;
        while ((int64_t)((nb[0] + stv - 1) / stv) * ((nb[1] + stv - 1) / stv) * ((nb[2] + stv - 1) / stv) > 32768) ++stv;
        std::vector<int> axis_idx[3];
        for (int d = 0; d < 3; ++d) {
            for (int i = 0; i < nb[d]; i += stv) axis_idx[d].push_back(i);
            if (axis_idx[d].back() != nb[d] - 1) axis_idx[d].push_back(nb[d] - 1);
        }
        std::vector<int64_t> sub;
        for (int z : axis_idx[2])
            for (int y : axis_idx[1])
                for (int x : axis_idx[0]) sub.push_back(x + (int64_t)nb[0] * (y + (int64_t)nb[1] * z));
        const int64_t ns = (int64_t)sub.size();
        int64_t* dsub = up(S.c, sub);
        const int kmax = (int)std::min<int64_t>({(int64_t)m_f, ns, (int64_t)2048});
        int64_t* dvox1 = (int64_t*)dalloc(S.c, sizeof(int64_t));
        int* dcol1 = (int*)dalloc(S.c, sizeof(int));
        for (int a = 0; a < 3; ++a) {
            Scratch L;   // per-component temporaries, freed at the end of the iteration
            double2* rowbuf = (double2*)dalloc(L.c, (size_t)m_f * sizeof(double2));
            double2* colbuf = (double2*)dalloc(L.c, (size_t)ns * sizeof(double2));
            double2* Usub = (double2*)dalloc(L.c, (size_t)ns * kmax * sizeof(double2));
            double2* Vall = (double2*)dalloc(L.c, (size_t)m_f * kmax * sizeof(double2));
            auto row = [&](int64_t i, double2* dst) {
                const int64_t v = sub[i];
                VSIE_CUDA(cudaMemcpy(dvox1, &v, sizeof(int64_t), cudaMemcpyHostToDevice));
                coupling_block(md_s, gb, 1, dvox1, m_f, nullptr, k0, false, -1.0, rowbuf, 1, m_f, a);
                VSIE_CUDA(cudaMemcpy(dst, rowbuf, m_f * sizeof(double2), cudaMemcpyDeviceToDevice));
            };
            auto colf = [&](int64_t j, double2* dst) {
                const int jj = (int)j;
                VSIE_CUDA(cudaMemcpy(dcol1, &jj, sizeof(int), cudaMemcpyHostToDevice));
                coupling_block(md_s, gb, (int)ns, dsub, 1, dcol1, k0, false, -1.0, colbuf, ns, ns, a);
                VSIE_CUDA(cudaMemcpy(dst, colbuf, ns * sizeof(double2), cudaMemcpyDeviceToDevice));
            };
            // the ACA stopping test is a heuristic that can overshoot its tolerance by a
            // few times; tol / 10 leaves the TT-SVD half of the budget
            AcaResult ar = aca_device(L, ns, m_f, tt_tol / 10, kmax, row, colf, Usub, Vall);
            const int k = ar.k;
            T.mark("TT cross (ACA)");
            // skeleton over all voxels
            std::vector<int> J(ar.cols.begin(), ar.cols.end());
            std::vector<int64_t> Ivox(k);
            for (int l = 0; l < k; ++l) Ivox[l] = sub[ar.rows[l]];
            int* dJ = up(L.c, J);
            int64_t* dI = up(L.c, Ivox);
            double2* Ud = (double2*)dalloc(L.c, (size_t)n_b * k * sizeof(double2));      // Z[:, J]
            coupling_block(md_s, gb, (int)n_b, nullptr, k, dJ, k0, false, -1.0, Ud, n_b, 0, a);
            double2* Ra = (double2*)dalloc(L.c, (size_t)k * m_f * sizeof(double2));      // Z[I, :]
            coupling_block(md_s, gb, k, dI, m_f, nullptr, k0, false, -1.0, Ra, k, 0, a);
            // core Z[I, J] (k x k) = columns J of Ra, then its inverse
            double2* Sk = (double2*)dalloc(L.c, (size_t)k * k * sizeof(double2));
            for (int l = 0; l < k; ++l)
                VSIE_CUDA(cudaMemcpy(Sk + (size_t)k * l, Ra + (size_t)k * J[l], k * sizeof(double2),
                                     cudaMemcpyDeviceToDevice));
            invert_f64(L, Sk, k);
            // V = (Z[I,J]^-1 Z[I,:])^H = Ra^H Sk^-H   (m_f x k)
            cgemm2<double>(L.c, OP_H, OP_H, m_f, k, k, one, Ra, k, 0, Sk, k, 0, zero, Vall, m_f, 0, 1,
                           nullptr, nullptr, 0);
            T.mark("TT skeleton");
            // orthonormalise V (m_f x k) by Cholesky QR, twice: V = Q R; U' = U R^H.
            // U' overwrites Z[:, J] in place, in row chunks (n_b k values of FP64
            // complex are ~40 GB at the 1 mm head grid: no second copy is made)
            double2* Vd = Vall;
            double2* Up = Ud;
            const int64_t chunk = std::min<int64_t>(n_b, std::max<int64_t>(m_f, (int64_t)1 << 20));
            double2* Gk = (double2*)dalloc(L.c, (size_t)k * k * sizeof(double2));
            double2* Rk = (double2*)dalloc(L.c, (size_t)k * k * sizeof(double2));
            double2* Tq = (double2*)dalloc(L.c, (size_t)std::max<int64_t>(chunk, m_f) * k * sizeof(double2));
            for (int pass = 0; pass < 2; ++pass) {
                cgemm<double>(L.c, OP_H, k, k, m_f, one, Vd, m_f, 0, Vd, m_f, 0, zero, Gk, k, 0, 1, nullptr, nullptr, 0);
                std::vector<cd> G = to_host(Gk, (size_t)k * k);
                for (int j = 0; j < k; ++j)
                    for (int i = 0; i < j; ++i) {
                        const cd v = 0.5 * (G[i + (size_t)k * j] + std::conj(G[j + (size_t)k * i]));
                        G[i + (size_t)k * j] = v;
                        G[j + (size_t)k * i] = std::conj(v);
                    }
                std::vector<cd> R = hla::cholesky_upper(k, G);
                if (R.empty()) throw Error(VSIE_EUNSUPPORTED, "far coupling cross factors are rank deficient");
                const std::vector<cd> Ri = hla::upper_inv(k, R);
                std::vector<double2> hr((size_t)k * k), hri((size_t)k * k);
                for (size_t i = 0; i < hr.size(); ++i) { hr[i] = d2(R[i]); hri[i] = d2(Ri[i]); }
                VSIE_CUDA(cudaMemcpy(Rk, hri.data(), hri.size() * sizeof(double2), cudaMemcpyHostToDevice));
                cgemm<double>(L.c, OP_N, m_f, k, k, one, Vd, m_f, 0, Rk, k, 0, zero, Tq, m_f, 0, 1, nullptr, nullptr, 0);
                VSIE_CUDA(cudaMemcpy(Vd, Tq, (size_t)m_f * k * sizeof(double2), cudaMemcpyDeviceToDevice));
                VSIE_CUDA(cudaMemcpy(Rk, hr.data(), hr.size() * sizeof(double2), cudaMemcpyHostToDevice));
                for (int64_t r0 = 0; r0 < n_b; r0 += chunk) {
                    const int rows = (int)std::min<int64_t>(chunk, n_b - r0);
                    cgemm2<double>(L.c, OP_N, OP_H, rows, k, k, one, Up + r0, n_b, 0, Rk, k, 0, zero, Tq, rows, 0, 1,
                                   nullptr, nullptr, 0);
                    VSIE_CUDA(cudaMemcpy2D(Up + r0, n_b * sizeof(double2), Tq, rows * sizeof(double2),
                                           rows * sizeof(double2), k, cudaMemcpyDeviceToDevice));
                }
            }
            // truncated TT-SVD of U' over (n1, n2, n3, k)
            const double tot = frob2(L, Up, n_b * k);
            const double delta2 = (tt_tol * 0.5) * (tt_tol * 0.5) * tot / 3.0;
            Factor f1 = truncate(L, Up, nb[0], (int)((int64_t)nb[1] * nb[2] * k), delta2, 11 + a);
            const int r1 = f1.r;
            Factor f2 = truncate(L, f1.R, r1 * nb[1], nb[2] * k, delta2, 23 + a);
            const int r2 = f2.r;
            Factor f3 = truncate(L, f2.R, r2 * nb[2], k, delta2, 37 + a);
            const int r3 = f3.r;
            // G4 = H4 Q_V^H  (r3 x m_f)
            double2* G4 = (double2*)dalloc(L.c, (size_t)r3 * m_f * sizeof(double2));
            cgemm2<double>(L.c, OP_N, OP_H, r3, m_f, k, one, f3.R, r3, 0, Vd, m_f, 0, zero, G4, r3, 0, 1, nullptr, nullptr, 0);
            B.tt_rank[a][0] = r1;
            B.tt_rank[a][1] = r2;
            B.tt_rank[a][2] = r3;
            B.tt[a][0] = to_host(f1.L, (size_t)nb[0] * r1);
            B.tt[a][1] = to_host(f2.L, (size_t)r1 * nb[1] * r2);
            B.tt[a][2] = to_host(f3.L, (size_t)r2 * nb[2] * r3);
            B.tt[a][3] = to_host(G4, (size_t)r3 * m_f);
            T.mark("TT-SVD");
        }
    }
    VSIE_CUDA(cudaDeviceSynchronize());

    // --- final context
    vsie_parts P{};
    P.m_f = m_f;
    P.m_n = m_n;
    P.stencil = s;
    if (m_n > 0) {
        P.W = reinterpret_cast<const double*>(B.W.data());
        P.base = B.base.data();
        P.pre_nnz = (int64_t)B.pre_col.size();
        P.pre_rowptr = B.pre_row.data();
        P.pre_col = B.pre_col.data();
        P.pre_val = reinterpret_cast<const double*>(B.pre_val.data());
        P.Znn = reinterpret_cast<const double*>(B.Znn.data());
    }
    if (m_f > 0) {
        P.aca_rank = B.aca_rank;
        P.U = reinterpret_cast<const double*>(B.U.data());
        P.V = reinterpret_cast<const double*>(B.V.data());
        for (int a = 0; a < 3; ++a) {
            for (int q = 0; q < 3; ++q) P.tt_rank[a][q] = B.tt_rank[a][q];
            for (int q = 0; q < 4; ++q) P.tt_core[a][q] = reinterpret_cast<const double*>(B.tt[a][q].data());
        }
    }
    if (T.on)
        fprintf(stderr, "[vsie setup] m_f %d m_n %d aca rank %d tt ranks %d,%d,%d | %d,%d,%d | %d,%d,%d\n", m_f, m_n,
                P.aca_rank, P.tt_rank[0][0], P.tt_rank[0][1], P.tt_rank[0][2], P.tt_rank[1][0], P.tt_rank[1][1],
                P.tt_rank[1][2], P.tt_rank[2][0], P.tt_rank[2][1], P.tt_rank[2][2]);
    vsie_options fo = o;
    fo.stencil = s;
    Ctx* c = nullptr;
    vsie_status st = create_from_parts_impl(body, eps_r, sigma, freq, &fo, &P, B.dZff, &c);
    if (st != VSIE_OK) throw Error(st, "context creation from the set-up parts failed");
    T.mark("context");
    if (B.dZff) {   // the context now owns the far-far block
        auto& al = S.c.allocs;
        al.erase(std::remove(al.begin(), al.end(), (void*)B.dZff), al.end());
        c->allocs.push_back(B.dZff);
    }
    c->hZnn_direct = std::move(B.Znn_direct);
    // hierarchical far-far block: cluster tree over the far RWG functions (centres:
    // midpoints of the two triangle centroids; supports: boxes of both triangles)
    const bool want_hm = has_s && c->f32.ready && c->f64.ready &&
                         (o.far_hmatrix > 0 || (o.far_hmatrix == 0 && m_f >= 8192));
    if (want_hm) {
        try {
            std::vector<double> cen(3 * (size_t)m_f), slo(3 * (size_t)m_f), shi(3 * (size_t)m_f);
            for (int i = 0; i < m_f; ++i) {
                for (int d = 0; d < 3; ++d) {
                    cen[3 * i + d] = 0.5 * (mh_s.centroid[3 * mh_s.tplus[i] + d] + mh_s.centroid[3 * mh_s.tminus[i] + d]);
                    slo[3 * i + d] = 1e300;
                    shi[3 * i + d] = -1e300;
                }
                for (int t : {mh_s.tplus[i], mh_s.tminus[i]})
                    for (int k = 0; k < 3; ++k)
                        for (int d = 0; d < 3; ++d) {
                            const double x = mh_s.xyz[3 * (size_t)mh_s.tri[3 * t + k] + d];
                            slo[3 * i + d] = std::min(slo[3 * i + d], x);
                            shi[3 * i + d] = std::max(shi[3 * i + d], x);
                        }
            }
            const int leaf = o.hm_leaf > 0 ? std::min(o.hm_leaf, 256) : 128;
            const double eta = o.hm_eta > 0 ? o.hm_eta : 1.0;
            const HmPlan plan = hm_plan(m_f, cen.data(), slo.data(), shi.data(), leaf, eta);
            hm_build(*c, plan, B.dZff, m_f, aca_tol);
        } catch (...) {
            destroy_ctx(c);
            throw;
        }
        T.mark("far-far H-matrix");
    }
    if (c->f32.ready && c->f64.ready) {
        try {
            build_block_precond(*c);
        } catch (...) {
            destroy_ctx(c);
            throw;
        }
        T.mark("block preconditioner");
    }
    if (c->hm.on) {
        // the dense far-far block (FP64, and its FP32 panels) served the ACA and the
        // preconditioner's factorisation; the product uses the H-matrix from now on
        auto release = [&](void* ptr) {
            auto& al = c->allocs;
            al.erase(std::remove(al.begin(), al.end(), ptr), al.end());
            cudaFree(ptr);
        };
        release(c->f32.Zff);
        release(c->f64.Zff);
        c->f32.Zff = nullptr;
        c->f64.Zff = nullptr;
        c->dZff_in = nullptr;
    }
    // RWG geometry for the plane-wave right-hand side (far first, then near)
    {
        std::vector<double> geo;
        geo.reserve((size_t)26 * (m_f + m_n));
        for (const MeshHost* mh : {&mh_s, &mh_c}) {
            for (int i = 0; i < mh->m; ++i) {
                const int tt[2] = {mh->tplus[i], mh->tminus[i]}, vv[2] = {mh->vplus[i], mh->vminus[i]};
                for (int hf = 0; hf < 2; ++hf) {
                    for (int k = 0; k < 3; ++k)
                        for (int d = 0; d < 3; ++d) geo.push_back(mh->xyz[3 * (size_t)mh->tri[3 * tt[hf] + k] + d]);
                    for (int d = 0; d < 3; ++d) geo.push_back(mh->xyz[3 * (size_t)vv[hf] + d]);
                    geo.push_back((hf == 0 ? 0.5 : -0.5) * mh->len[i]);
                }
            }
        }
        if (!geo.empty()) {
            try {
                c->rwg_geo = up(*c, geo);
            } catch (...) {
                destroy_ctx(c);
                throw;
            }
        }
    }
    // ports: far ports first, then coil ports
    for (int e : mh_s.ports) {
        c->port_row.push_back(e);
        c->port_len.push_back(mh_s.len[e]);
    }
    for (int e : mh_c.ports) {
        c->port_row.push_back((int64_t)m_f + e);
        c->port_len.push_back(mh_c.len[e]);
    }
    *out = c;
}

}  // namespace vsie

using namespace vsie;

extern "C" vsie_status vsie_setup(const vsie_grid* body, const double* eps_r, const double* sigma,
                                  const vsie_mesh* coil, const vsie_mesh* shield, double freq_hz,
                                  const vsie_options* opts, vsie_ctx** out) {
    if (!out) return VSIE_EINVAL;
    *out = nullptr;
    try {
        Ctx* c = nullptr;
        setup_impl(body, eps_r, sigma, coil, shield, freq_hz, opts, &c);
        *out = reinterpret_cast<vsie_ctx*>(c);
        return VSIE_OK;
    } catch (const Error& e) {
        set_global_err(e.msg);
        return e.st;
    } catch (const std::bad_alloc&) {
        set_global_err("host allocation failed");
        return VSIE_ENOMEM;
    }
}
