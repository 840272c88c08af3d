// Port network of the conductors (Sec. IV.B and V: the coil ports, their tuning
// and matching loads, and the network parameters that characterise the array).
//
//  * vsie_set_loads: a lumped impedance Z_L in series with port edge m.  Its
//    voltage drop -Z_L I_m, with I_m = j_m l_m the current through the edge,
//    enters the delta-gap row i omega eps0 (V - Z_L I_m) l_m; moved to the left
//    it adds i omega eps0 Z_L l_m^2 to the operator's diagonal entry (m, m).
//    The matvec applies it as a diagonal term on the loaded rows (both
//    precisions); the block preconditioner is left as built.
//  * vsie_port_network: from the solutions for each port driven by 1 V in turn
//    (the others shorted), the current through port edge i for excitation j is
//    I_ij = j_i l_i, so Y = I (siemens), Z = Y^-1 and S = (Z - z0)(Z + z0)^-1.
#include "vsie_internal.h"

#include <algorithm>
#include <cmath>
#include <complex>

namespace vsie {

template <typename R>
__global__ void k_load_diag(int nl, int p, const int64_t* __restrict__ rows, const cx<R>* __restrict__ d,
                            const cx<R>* __restrict__ X, int64_t ldx, cx<R>* __restrict__ Y, int64_t ldy) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nl * p) return;
    const int i = e % nl, j = e / nl;
    const int64_t r = rows[i];
    cx<R>* y = Y + (size_t)j * ldy + r;
    cfma(*y, d[i], X[(size_t)j * ldx + r]);
}

template <typename R>
void apply_loads(Ctx& c, int p, const cx<R>* X, int64_t ldx, cx<R>* Y, int64_t ldy, cudaStream_t st) {
    if (c.nloads == 0) return;
    const cx<R>* d = sizeof(R) == 8 ? (const cx<R>*)c.load_d64 : (const cx<R>*)c.load_d32;
    const int tot = c.nloads * p;
    ProfScope ps(c, PG_SURF, st);
    prof_count(c, 1);
    k_load_diag<R><<<(tot + 127) / 128, 128, 0, st>>>(c.nloads, p, c.load_rows, d, X, ldx, Y, ldy);
    VSIE_CUDA(cudaGetLastError());
}
template void apply_loads<float>(Ctx&, int, const float2*, int64_t, float2*, int64_t, cudaStream_t);
template void apply_loads<double>(Ctx&, int, const double2*, int64_t, double2*, int64_t, cudaStream_t);

// I_ij = x_j[row_i] l_i (current through port edge i for the drive of port j)
__global__ void k_port_currents(int n, const int64_t* __restrict__ rows, const double* __restrict__ len,
                                const double2* __restrict__ X, int64_t ldx, double2* __restrict__ I) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int i = e % n, j = e / n;
    const double2 x = X[(size_t)j * ldx + rows[i]];
    I[e] = make_double2(x.x * len[i], x.y * len[i]);
}

// one column: port edge m_i driven by the complex voltage v_i
__global__ void k_drive_entries(int n, const int64_t* __restrict__ rows, const double2* __restrict__ b,
                                double2* __restrict__ B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) B[rows[i]] = b[i];
}

template <typename T> struct TmpBuf {
    T* p = nullptr;
    explicit TmpBuf(size_t n) { VSIE_CUDA(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T))); }
    ~TmpBuf() { if (p) cudaFree(p); }
    TmpBuf(const TmpBuf&) = delete;
    TmpBuf& operator=(const TmpBuf&) = delete;
};

// Gauss-Jordan inverse with partial pivoting of a small complex matrix
// (column-major); false if singular.
static bool small_inverse(int n, std::vector<std::complex<double>>& A) {
    std::vector<std::complex<double>> B((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) B[i + (size_t)n * i] = 1.0;
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (std::abs(A[i + (size_t)n * k]) > std::abs(A[piv + (size_t)n * k])) piv = i;
        if (!(std::abs(A[piv + (size_t)n * k]) > 0)) return false;
        if (piv != k)
            for (int j = 0; j < n; ++j) {
                std::swap(A[k + (size_t)n * j], A[piv + (size_t)n * j]);
                std::swap(B[k + (size_t)n * j], B[piv + (size_t)n * j]);
            }
        const std::complex<double> ip = 1.0 / A[k + (size_t)n * k];
        for (int j = 0; j < n; ++j) {
            A[k + (size_t)n * j] *= ip;
            B[k + (size_t)n * j] *= ip;
        }
        for (int i = 0; i < n; ++i) {
            if (i == k) continue;
            const std::complex<double> f = A[i + (size_t)n * k];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                A[i + (size_t)n * j] -= f * A[k + (size_t)n * j];
                B[i + (size_t)n * j] -= f * B[k + (size_t)n * j];
            }
        }
    }
    A = B;
    return true;
}

static void put(double* out, const std::vector<std::complex<double>>& M) {
    if (!out) return;
    for (size_t i = 0; i < M.size(); ++i) {
        out[2 * i] = M[i].real();
        out[2 * i + 1] = M[i].imag();
    }
}

}  // namespace vsie

using namespace vsie;

extern "C" vsie_status vsie_set_loads(vsie_ctx* ctx, int32_t nloads, const int32_t* ports, const double* z_load) {
    if (!ctx) { set_global_err("null context"); return VSIE_EINVAL; }
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    try {
        if (nloads < 0 || (nloads > 0 && (!ports || !z_load))) throw Error(VSIE_EINVAL, "bad load list");
        std::vector<int64_t> rows(nloads);
        std::vector<double2> d64(nloads);
        std::vector<float2> d32(nloads);
        for (int i = 0; i < nloads; ++i) {
            const int q = ports[i];
            if (q < 0 || q >= (int)c->port_row.size()) throw Error(VSIE_EINVAL, "load port index out of range");
            for (int k = 0; k < i; ++k)
                if (ports[k] == q) throw Error(VSIE_EINVAL, "a port carries at most one load");
            if (!std::isfinite(z_load[2 * i]) || !std::isfinite(z_load[2 * i + 1]))
                throw Error(VSIE_EINVAL, "non-finite load impedance");
            const double l = c->port_len[q];
            const std::complex<double> zl(z_load[2 * i], z_load[2 * i + 1]);
            const std::complex<double> d = std::complex<double>(0.0, c->omega * kEps0) * zl * (l * l);
            rows[i] = c->port_row[q];
            d64[i] = make_double2(d.real(), d.imag());
            d32[i] = make_float2((float)d.real(), (float)d.imag());
        }
        VSIE_CUDA(cudaDeviceSynchronize());
        auto release = [&](void* p) {
            if (!p) return;
            auto& al = c->allocs;
            al.erase(std::remove(al.begin(), al.end(), p), al.end());
            cudaFree(p);
        };
        release(c->load_rows);
        release(c->load_d64);
        release(c->load_d32);
        c->load_rows = nullptr;
        c->load_d64 = nullptr;
        c->load_d32 = nullptr;
        c->nloads = 0;
        if (nloads > 0) {
            c->load_rows = (int64_t*)dalloc(*c, nloads * sizeof(int64_t));
            c->load_d64 = (double2*)dalloc(*c, nloads * sizeof(double2));
            c->load_d32 = (float2*)dalloc(*c, nloads * sizeof(float2));
            VSIE_CUDA(cudaMemcpy(c->load_rows, rows.data(), nloads * sizeof(int64_t), cudaMemcpyHostToDevice));
            VSIE_CUDA(cudaMemcpy(c->load_d64, d64.data(), nloads * sizeof(double2), cudaMemcpyHostToDevice));
            VSIE_CUDA(cudaMemcpy(c->load_d32, d32.data(), nloads * sizeof(float2), cudaMemcpyHostToDevice));
            c->nloads = nloads;
        }
    } catch (const Error& e) {
        c->err = e.msg;
        return e.st;
    }
    return VSIE_OK;
}

extern "C" vsie_status vsie_port_network(vsie_ctx* ctx, int32_t nports, const int32_t* ports, const void* X,
                                         int64_t ldx, double z0, double* Y, double* Z, double* S) {
    if (!ctx) { set_global_err("null context"); return VSIE_EINVAL; }
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    try {
        if (nports < 1 || !ports || !X) throw Error(VSIE_EINVAL, "need ports and their solutions");
        if (ldx < c->N) throw Error(VSIE_EINVAL, "leading dimension < N");
        if (!(z0 > 0) || !std::isfinite(z0)) throw Error(VSIE_EINVAL, "reference impedance must be > 0");
        const int n = nports;
        std::vector<int64_t> hrow(n);
        std::vector<double> hlen(n);
        for (int i = 0; i < n; ++i) {
            const int q = ports[i];
            if (q < 0 || q >= (int)c->port_row.size()) throw Error(VSIE_EINVAL, "port index out of range");
            hrow[i] = c->port_row[q];
            hlen[i] = c->port_len[q];
        }
        // gather I_ij = x_j[row_i] l_i on the device, one copy back
        TmpBuf<int64_t> drow(n);
        TmpBuf<double> dlen(n);
        TmpBuf<double2> dI((size_t)n * n);
        VSIE_CUDA(cudaMemcpy(drow.p, hrow.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice));
        VSIE_CUDA(cudaMemcpy(dlen.p, hlen.data(), n * sizeof(double), cudaMemcpyHostToDevice));
        k_port_currents<<<(n * n + 127) / 128, 128>>>(n, drow.p, dlen.p, (const double2*)X, ldx, dI.p);
        VSIE_CUDA(cudaGetLastError());
        std::vector<std::complex<double>> I((size_t)n * n);
        VSIE_CUDA(cudaMemcpy(I.data(), dI.p, (size_t)n * n * sizeof(double2), cudaMemcpyDeviceToHost));
        put(Y, I);
        std::vector<std::complex<double>> Zm = I;
        if (!small_inverse(n, Zm)) throw Error(VSIE_EBREAKDOWN, "singular admittance matrix");
        put(Z, Zm);
        if (S) {
            std::vector<std::complex<double>> P = Zm, Q = Zm;
            for (int i = 0; i < n; ++i) {
                P[i + (size_t)n * i] -= z0;
                Q[i + (size_t)n * i] += z0;
            }
            if (!small_inverse(n, Q)) throw Error(VSIE_EBREAKDOWN, "singular Z + z0");
            std::vector<std::complex<double>> Sm((size_t)n * n, 0.0);
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j)
                    for (int k = 0; k < n; ++k) Sm[i + (size_t)n * j] += P[i + (size_t)n * k] * Q[k + (size_t)n * j];
            put(S, Sm);
        }
    } catch (const Error& e) {
        c->err = e.msg;
        return e.st;
    }
    return VSIE_OK;
}

extern "C" vsie_status vsie_rhs_drive(vsie_ctx* ctx, int32_t nports, const int32_t* ports, const double* v,
                                      void* B, vsie_stream stream) {
    if (!ctx) { set_global_err("null context"); return VSIE_EINVAL; }
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    try {
        if (!B || nports < 1 || !ports || !v) throw Error(VSIE_EINVAL, "need B, ports and voltages");
        std::vector<int64_t> hrow(nports);
        std::vector<double2> hb(nports);
        for (int i = 0; i < nports; ++i) {
            const int q = ports[i];
            if (q < 0 || q >= (int)c->port_row.size()) throw Error(VSIE_EINVAL, "port index out of range");
            for (int k = 0; k < i; ++k)
                if (ports[k] == q) throw Error(VSIE_EINVAL, "a port is listed twice");
            if (!std::isfinite(v[2 * i]) || !std::isfinite(v[2 * i + 1])) throw Error(VSIE_EINVAL, "non-finite voltage");
            // i omega eps0 V l: i (a + i b) = -b + i a
            const double s = c->omega * kEps0 * c->port_len[q];
            hrow[i] = c->port_row[q];
            hb[i] = make_double2(-s * v[2 * i + 1], s * v[2 * i]);
        }
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        TmpBuf<int64_t> drow(nports);
        TmpBuf<double2> db(nports);
        VSIE_CUDA(cudaMemcpy(drow.p, hrow.data(), nports * sizeof(int64_t), cudaMemcpyHostToDevice));
        VSIE_CUDA(cudaMemcpy(db.p, hb.data(), nports * sizeof(double2), cudaMemcpyHostToDevice));
        VSIE_CUDA(cudaMemsetAsync(B, 0, c->N * sizeof(double2), st));
        k_drive_entries<<<(nports + 127) / 128, 128, 0, st>>>(nports, drow.p, db.p, (double2*)B);
        VSIE_CUDA(cudaGetLastError());
        VSIE_CUDA(cudaStreamSynchronize(st));   // the staging buffers are freed on return
    } catch (const Error& e) {
        c->err = e.msg;
        return e.st;
    }
    return VSIE_OK;
}
