// K7 and the solver: restarted GMRES for p right-hand sides at once (Sec. III.A:
// GMRES with restart; Saad and Schultz 1986), each RHS with its own Krylov space
// and one shared multi-RHS matvec per iteration.
//
// Both modes apply the block preconditioner of precond.cu on the right
// (A M y = b, x = M y) unless precond = 1.
//  mode 0 (plain FP64): GMRES(m), FP64 matvec, FP64 basis, classical
//         Gram-Schmidt with one re-orthogonalisation pass (CGS2), Givens
//         rotations, true residual recomputed at every restart.
//  mode 1 (mixed): iterative refinement.  The outer loop forms the FP64
//         residual r = b - Z x with the FP64 matvec; the inner solve is
//         GMRES(m) on the FP32 operator with an FP32 basis and FP32
//         Gram-Schmidt arithmetic (CGS), to the loose inner tolerance; its
//         correction is widened and added to the FP64 iterate.  Dot products
//         sum in FP32 per thread and in FP64 across threads and blocks; the
//         Hessenberg matrix and the Givens rotations are FP64 on the host.
// The Krylov basis is stored [i][c][n] (basis index, RHS, row), N rows each.
// Dot products use a fixed two-stage reduction (deterministic results).
#include "vsie_internal.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <cmath>
#include <complex>

namespace vsie {

template <typename R>
void matvec_internal(Ctx& c, int p, const cx<R>* X, int64_t ldx, cx<R>* Y, int64_t ldy,
                     cudaStream_t st);

constexpr int kDotGroup = 8;     // basis vectors per dot-product group
constexpr int kDotBlocks = 152;  // row chunks per (column, group): one per SM

// Vector loads of the FP32 kernels move two complex values (one float4); the
// FP64 kernels one (double2).  Every p x N block below has a leading dimension
// ld >= N; the FP32 paths need ld even (16-byte aligned rows).
template <typename R> struct Pack;
template <> struct Pack<float> { using T = float4; static constexpr int K = 2; };
template <> struct Pack<double> { using T = double2; static constexpr int K = 1; };

// conj(v) . x summed over the complex values of one pack, accumulated into a
template <typename T, typename A>
__device__ __forceinline__ void pack_dot(A& a, const T& v, const T& x);
template <>
__device__ __forceinline__ void pack_dot<float4, float2>(float2& a, const float4& v, const float4& x) {
    a.x += v.x * x.x + v.y * x.y + v.z * x.z + v.w * x.w;
    a.y += v.x * x.y - v.y * x.x + v.z * x.w - v.w * x.z;
}
template <>
__device__ __forceinline__ void pack_dot<double2, double2>(double2& a, const double2& v, const double2& x) {
    a.x += v.x * x.x + v.y * x.y;
    a.y += v.x * x.y - v.y * x.x;
}
// s += v * h for each complex value of the pack
__device__ __forceinline__ void pack_fma(float4& s, const float4& v, float2 h) {
    s.x += v.x * h.x - v.y * h.y;
    s.y += v.x * h.y + v.y * h.x;
    s.z += v.z * h.x - v.w * h.y;
    s.w += v.z * h.y + v.w * h.x;
}
__device__ __forceinline__ void pack_fma(double2& s, const double2& v, double2 h) {
    s.x += v.x * h.x - v.y * h.y;
    s.y += v.x * h.y + v.y * h.x;
}
__device__ __forceinline__ void pack_sub(float4& t, const float4& s, float sg) {
    t.x += sg * s.x; t.y += sg * s.y; t.z += sg * s.z; t.w += sg * s.w;
}
__device__ __forceinline__ void pack_sub(double2& t, const double2& s, double sg) {
    t.x += sg * s.x; t.y += sg * s.y;
}

// partial[(blk * p + c) * nvec + i] = sum_{n in chunk} conj(V_i[c][n]) w[c][n]
// V_i[c] = V + (i p + c) ld.  Per-thread sums in R, the warp and block sums in
// FP64.  Chunks are whole packs; block 0 adds the odd last row.
template <typename R>
__global__ void __launch_bounds__(256)
k_block_dot(const cx<R>* __restrict__ V, int nvec, int64_t N, int64_t ld, int p,
            const cx<R>* __restrict__ w, int64_t ldw, double2* __restrict__ partial) {
    using T = typename Pack<R>::T;
    constexpr int PK = Pack<R>::K;
    const int c = blockIdx.y;
    const int g0 = blockIdx.z * kDotGroup;
    const int ng = min(kDotGroup, nvec - g0);
    const int64_t NP = N / PK;
    const int64_t chunk = (NP + gridDim.x - 1) / gridDim.x;
    const int64_t n0 = blockIdx.x * chunk, n1 = min(NP, n0 + chunk);
    cx<R> acc[kDotGroup];
#pragma unroll
    for (int g = 0; g < kDotGroup; ++g) acc[g] = mk<cx<R>>(0, 0);
    const T* wc = reinterpret_cast<const T*>(w + (size_t)c * ldw);
    for (int64_t n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
        const T x = wc[n];
        T v[kDotGroup];
#pragma unroll
        for (int g = 0; g < kDotGroup; ++g)
            if (g < ng) v[g] = reinterpret_cast<const T*>(V + ((size_t)(g0 + g) * p + c) * ld)[n];
#pragma unroll
        for (int g = 0; g < kDotGroup; ++g)
            if (g < ng) pack_dot(acc[g], v[g], x);
    }
    if (PK == 2 && (N & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        const cx<R> x = w[(size_t)c * ldw + N - 1];
        for (int g = 0; g < ng; ++g) {
            const cx<R> v = V[((size_t)(g0 + g) * p + c) * ld + N - 1];
            acc[g].x += v.x * x.x + v.y * x.y;
            acc[g].y += v.x * x.y - v.y * x.x;
        }
    }
    __shared__ double2 red[kDotGroup][8];
#pragma unroll
    for (int g = 0; g < kDotGroup; ++g) {
        double rx = acc[g].x, ry = acc[g].y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rx += __shfl_down_sync(0xffffffffu, rx, o);
            ry += __shfl_down_sync(0xffffffffu, ry, o);
        }
        if ((threadIdx.x & 31) == 0) red[g][threadIdx.x >> 5] = make_double2(rx, ry);
    }
    __syncthreads();
    if (threadIdx.x < ng) {
        double2 s = make_double2(0, 0);
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s = cadd(s, red[threadIdx.x][q]);
        partial[((size_t)blockIdx.x * p + c) * nvec + g0 + threadIdx.x] = s;
    }
}

__global__ void k_reduce_dots(const double2* __restrict__ partial, int nblk, int p, int nvec,
                              double2* __restrict__ h) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p * nvec) return;
    double2 s = make_double2(0, 0);
    for (int b = 0; b < nblk; ++b) s = cadd(s, partial[(size_t)b * p * nvec + e]);
    h[e] = s;   // h[c * nvec + i]
}

// w[c][n] += sgn * sum_i V_i[c][n] * h[c * nvec + i]   (h in FP64, rounded to R)
// grid (blocks, p); dynamic shared memory: nvec complex values of R
template <typename R>
__global__ void __launch_bounds__(256)
k_basis_update(const cx<R>* __restrict__ V, int nvec, int64_t N, int64_t ld, int p,
               const double2* __restrict__ h, double sgn, cx<R>* __restrict__ w, int64_t ldw) {
    using T = typename Pack<R>::T;
    constexpr int PK = Pack<R>::K;
    extern __shared__ __align__(16) unsigned char kb_smem[];
    cx<R>* hs = reinterpret_cast<cx<R>*>(kb_smem);
    const int c = blockIdx.y;
    for (int i = threadIdx.x; i < nvec; i += blockDim.x)
        hs[i] = mk<cx<R>>((R)h[c * nvec + i].x, (R)h[c * nvec + i].y);
    __syncthreads();
    const int64_t NP = N / PK;
    T* wc = reinterpret_cast<T*>(w + (size_t)c * ldw);
    const T* Vc = reinterpret_cast<const T*>(V + (size_t)c * ld);
    const size_t vstride = (size_t)p * ld / PK;   // packs between basis vectors
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < NP;
         n += (int64_t)gridDim.x * blockDim.x) {
        T s;
        memset(&s, 0, sizeof(T));
        int i = 0;
        for (; i + 8 <= nvec; i += 8) {
            T v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = Vc[(size_t)(i + u) * vstride + n];
#pragma unroll
            for (int u = 0; u < 8; ++u) pack_fma(s, v[u], hs[i + u]);
        }
        for (; i < nvec; ++i) pack_fma(s, Vc[(size_t)i * vstride + n], hs[i]);
        T t = wc[n];
        pack_sub(t, s, (R)sgn);
        wc[n] = t;
    }
    if (PK == 2 && (N & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        cx<R> s = mk<cx<R>>(0, 0);
        for (int i = 0; i < nvec; ++i) cfma(s, V[((size_t)i * p + c) * ld + N - 1], hs[i]);
        cx<R>& t = w[(size_t)c * ldw + N - 1];
        t.x += (R)sgn * s.x;
        t.y += (R)sgn * s.y;
    }
}

// dst[c][n] = src[c][n] * scale[c]  (scale complex, FP64, rounded to R)
template <typename R>
__global__ void k_scale_cols(const cx<R>* __restrict__ src, int64_t lds, int64_t N, int p,
                             const double2* __restrict__ scale, cx<R>* __restrict__ dst, int64_t ldd) {
    const int64_t tot = N * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = e / N;
        const int64_t n = e - (int64_t)c * N;
        dst[(size_t)c * ldd + n] = cmul(src[(size_t)c * lds + n], mk<cx<R>>((R)scale[c].x, (R)scale[c].y));
    }
}

template <typename R>
__global__ void k_sub(const cx<R>* __restrict__ a, int64_t lda, const cx<R>* __restrict__ b,
                      int64_t ldb, int64_t N, int p, cx<R>* __restrict__ out, int64_t ldo) {
    const int64_t tot = N * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = e / N;
        const int64_t n = e - (int64_t)c * N;
        out[(size_t)c * ldo + n] = csub(a[(size_t)c * lda + n], b[(size_t)c * ldb + n]);
    }
}

__global__ void k_narrow(const double2* __restrict__ a, int64_t lda, int64_t N, int p,
                         float2* __restrict__ b, int64_t ldb) {
    const int64_t tot = N * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = e / N;
        const int64_t n = e - (int64_t)c * N;
        const double2 v = a[(size_t)c * lda + n];
        b[(size_t)c * ldb + n] = make_float2((float)v.x, (float)v.y);
    }
}

// b[c][n] = a[c][n]  (FP32 to FP64)
__global__ void k_widen_to(const float2* __restrict__ a, int64_t lda, int64_t N, int p,
                           double2* __restrict__ b, int64_t ldb) {
    const int64_t tot = N * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = e / N;
        const int64_t n = e - (int64_t)c * N;
        const float2 v = a[(size_t)c * lda + n];
        b[(size_t)c * ldb + n] = make_double2(v.x, v.y);
    }
}

// X[c][n] += a[c][n]  (a FP32, X FP64)
__global__ void k_add_widen(const float2* __restrict__ a, int64_t lda, int64_t N, int p,
                            double2* __restrict__ X, int64_t ldx) {
    const int64_t tot = N * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = e / N;
        const int64_t n = e - (int64_t)c * N;
        const float2 v = a[(size_t)c * lda + n];
        double2& x = X[(size_t)c * ldx + n];
        x.x += v.x;
        x.y += v.y;
    }
}

static int nblk(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); }

template <typename R>
struct Krylov {
    Ctx& c;
    int p;
    int64_t N;
    int64_t ld;        // leading dimension of every p x N block (even)
    int m;
    cx<R>* V;          // (m+1) x p x ld
    cx<R>* w;          // p x ld
    double2* h;        // p x (m+1)
    double2* part;     // kDotBlocks x p x (m+1)
    double2* scl;      // p
    cudaStream_t st;

    // h[c][i] = V_i^H w for i < nvec (device h), copied to host hh
    void dots(int nvec, std::vector<std::complex<double>>& hh) {
        ProfScope ps(c, PG_KRYLOV, st);
        prof_count(c, 2);
        dim3 g(kDotBlocks, p, (nvec + kDotGroup - 1) / kDotGroup);
        k_block_dot<R><<<g, 256, 0, st>>>(V, nvec, N, ld, p, w, ld, part);
        k_reduce_dots<<<(p * nvec + 255) / 256, 256, 0, st>>>(part, kDotBlocks, p, nvec, h);
        VSIE_CUDA(cudaGetLastError());
        hh.resize((size_t)p * nvec);
        VSIE_CUDA(cudaMemcpyAsync(hh.data(), h, hh.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
        VSIE_CUDA(cudaStreamSynchronize(st));
    }
    // squared norms of the columns of w
    void norms(std::vector<double>& nn) {
        ProfScope ps(c, PG_KRYLOV, st);
        prof_count(c, 2);
        // w against itself: treat w as a one-vector basis
        dim3 g(kDotBlocks, p, 1);
        k_block_dot<R><<<g, 256, 0, st>>>(w, 1, N, ld, p, w, ld, part);
        k_reduce_dots<<<(p + 255) / 256, 256, 0, st>>>(part, kDotBlocks, p, 1, h);
        VSIE_CUDA(cudaGetLastError());
        std::vector<double2> t(p);
        VSIE_CUDA(cudaMemcpyAsync(t.data(), h, p * sizeof(double2), cudaMemcpyDeviceToHost, st));
        VSIE_CUDA(cudaStreamSynchronize(st));
        nn.resize(p);
        for (int c2 = 0; c2 < p; ++c2) nn[c2] = t[c2].x;
    }
    // tgt (p x N, leading dimension ld) += sgn B hh, B = V unless given
    void update(int nvec, const std::vector<std::complex<double>>& hh, double sgn, cx<R>* tgt,
                const cx<R>* B = nullptr) {
        ProfScope ps(c, PG_KRYLOV, st);
        prof_count(c, 1);
        VSIE_CUDA(cudaMemcpyAsync(h, hh.data(), (size_t)p * nvec * sizeof(double2), cudaMemcpyHostToDevice, st));
        const int64_t packs = N / Pack<R>::K;
        const int bx = (int)std::max<int64_t>(1, std::min<int64_t>((packs + 255) / 256, 1216));
        k_basis_update<R><<<dim3(bx, p), 256, (size_t)nvec * sizeof(cx<R>), st>>>(B ? B : V, nvec, N, ld,
                                                                                 p, h, sgn, tgt, ld);
        VSIE_CUDA(cudaGetLastError());
    }
    void scale_into(const cx<R>* src, const std::vector<std::complex<double>>& s, cx<R>* dst) {
        ProfScope ps(c, PG_KRYLOV, st);
        prof_count(c, 1);
        VSIE_CUDA(cudaMemcpyAsync(scl, s.data(), p * sizeof(double2), cudaMemcpyHostToDevice, st));
        k_scale_cols<R><<<nblk(N * p), 256, 0, st>>>(src, ld, N, p, scl, dst, ld);
        VSIE_CUDA(cudaGetLastError());
    }
    cx<R>* basis(int i) { return V + (size_t)i * p * ld; }
};

using cdd = std::complex<double>;

// One restarted GMRES(m) solve of A e = r (A applied through `apply`, FP64 in
// and out) for all p columns, relative tolerance tol with respect to
// ||r||; returns the correction in e (p x N, leading dimension K.ld).  iters[c] accumulates the
// iterations until column c met its tolerance.
// Flexible variant (Zb != nullptr): z_j = prec(v_j) is kept in Zb, w = A z_j
// and the correction is Zb y (Saad 1993); `apply` is then the plain operator.
template <typename R, typename Apply, typename Prec>
static void gmres_core(Krylov<R>& K, const cx<R>* r, double tol, int maxit, bool cgs2, Apply apply,
                       Prec prec, cx<R>* Zb, cx<R>* e, std::vector<int>& iters,
                       std::vector<double>& relres_est, int& nmatvec) {
    const int p = K.p;
    const int64_t N = K.N, ld = K.ld;
    const int m = K.m;
    VSIE_CUDA(cudaMemsetAsync(e, 0, (size_t)ld * p * sizeof(cx<R>), K.st));
    // residual of the current correction: starts as r
    cx<R>* res = K.w;
    VSIE_CUDA(cudaMemcpyAsync(res, r, (size_t)ld * p * sizeof(cx<R>), cudaMemcpyDeviceToDevice, K.st));
    std::vector<double> nr0;
    K.norms(nr0);
    std::vector<double> beta0(p);
    for (int c = 0; c < p; ++c) beta0[c] = std::sqrt(nr0[c]);
    std::vector<bool> done(p, false);
    for (int c = 0; c < p; ++c)
        if (!(beta0[c] > 0)) done[c] = true;
    relres_est.assign(p, 0.0);
    int total = 0;
    while (total < maxit) {
        // residual norms of this cycle
        std::vector<double> nr;
        K.norms(nr);
        std::vector<double> beta(p);
        bool all = true;
        for (int c = 0; c < p; ++c) {
            beta[c] = std::sqrt(nr[c]);
            if (!std::isfinite(beta[c])) throw Error(VSIE_EBREAKDOWN, "non-finite residual");
            if (beta0[c] > 0 && beta[c] <= tol * beta0[c]) done[c] = true;
            relres_est[c] = beta0[c] > 0 ? beta[c] / beta0[c] : 0.0;
            all = all && done[c];
        }
        if (all) break;
        // v0 = res / beta
        std::vector<cdd> sc(p);
        for (int c = 0; c < p; ++c) sc[c] = beta[c] > 0 ? 1.0 / beta[c] : 0.0;
        K.scale_into(res, sc, K.basis(0));
        std::vector<std::vector<cdd>> H(p, std::vector<cdd>((size_t)(m + 1) * m, 0.0));
        std::vector<std::vector<cdd>> cs(p, std::vector<cdd>(m)), sn(p, std::vector<cdd>(m));
        std::vector<std::vector<cdd>> g(p, std::vector<cdd>(m + 1, 0.0));
        for (int c = 0; c < p; ++c) g[c][0] = beta[c];
        std::vector<bool> cyc_done(done);
        int j = 0;
        for (; j < m && total < maxit; ++j) {
            if (Zb) {
                cx<R>* zj = Zb + (size_t)j * p * ld;
                prec(K.basis(j), zj);   // z_j = M_j v_j
                apply(zj, K.w);         // w = A z_j
            } else {
                apply(K.basis(j), K.w);   // w = A v_j
            }
            ++nmatvec;
            std::vector<cdd> hh, hh2;
            K.dots(j + 1, hh);
            K.update(j + 1, hh, -1.0, K.w);
            if (cgs2) {
                K.dots(j + 1, hh2);
                K.update(j + 1, hh2, -1.0, K.w);
                for (size_t q = 0; q < hh.size(); ++q) hh[q] += hh2[q];
            }
            std::vector<double> nw;
            K.norms(nw);
            std::vector<cdd> inv(p);
            ++total;
            for (int c = 0; c < p; ++c) {
                const double hn = std::sqrt(nw[c]);
                if (!std::isfinite(hn)) throw Error(VSIE_EBREAKDOWN, "non-finite Arnoldi vector");
                std::vector<cdd>& Hc = H[c];
                for (int i = 0; i <= j; ++i) Hc[i + (size_t)(m + 1) * j] = hh[(size_t)c * (j + 1) + i];
                Hc[j + 1 + (size_t)(m + 1) * j] = hn;
                inv[c] = hn > 1e-300 * std::max(beta0[c], 1e-300) ? 1.0 / hn : 0.0;
                // apply previous rotations to the new column
                // rotations G_i = [[conj(c), conj(s)], [-s, c]] (unitary), the same
                // form as the new rotation below
                for (int i = 0; i < j; ++i) {
                    const cdd a = Hc[i + (size_t)(m + 1) * j], b = Hc[i + 1 + (size_t)(m + 1) * j];
                    Hc[i + (size_t)(m + 1) * j] = std::conj(cs[c][i]) * a + std::conj(sn[c][i]) * b;
                    Hc[i + 1 + (size_t)(m + 1) * j] = -sn[c][i] * a + cs[c][i] * b;
                }
                const cdd a = Hc[j + (size_t)(m + 1) * j], b = Hc[j + 1 + (size_t)(m + 1) * j];
                const double den = std::sqrt(std::norm(a) + std::norm(b));
                if (den == 0.0) { cs[c][j] = 1.0; sn[c][j] = 0.0; }
                else { cs[c][j] = a / den; sn[c][j] = b / den; }
                Hc[j + (size_t)(m + 1) * j] = std::conj(cs[c][j]) * a + std::conj(sn[c][j]) * b;
                Hc[j + 1 + (size_t)(m + 1) * j] = 0.0;
                g[c][j + 1] = -sn[c][j] * g[c][j];
                g[c][j] = std::conj(cs[c][j]) * g[c][j];
                const double est = std::abs(g[c][j + 1]) / (beta0[c] > 0 ? beta0[c] : 1.0);
                if (!cyc_done[c]) {
                    iters[c]++;
                    relres_est[c] = est;
                    if (est <= tol || inv[c] == 0.0) cyc_done[c] = true;
                }
            }
            bool all2 = true;
            for (int c = 0; c < p; ++c) all2 = all2 && cyc_done[c];
            if (j + 1 < m) K.scale_into(K.w, inv, K.basis(j + 1));
            if (all2) { ++j; break; }
        }
        // y = H^-1 g (upper triangular, k = j columns); e += V y
        const int k = j;
        std::vector<cdd> Y((size_t)p * k, 0.0);
        for (int c = 0; c < p; ++c) {
            if (done[c]) continue;
            for (int i = k - 1; i >= 0; --i) {
                cdd s = g[c][i];
                for (int q = i + 1; q < k; ++q) s -= H[c][i + (size_t)(m + 1) * q] * Y[(size_t)c * k + q];
                const cdd d = H[c][i + (size_t)(m + 1) * i];
                Y[(size_t)c * k + i] = d != 0.0 ? s / d : 0.0;
            }
        }
        K.update(k, Y, 1.0, e, Zb);
        // true residual of the correction: res = r - A e
        apply(e, K.w);
        ++nmatvec;
        k_sub<R><<<nblk(N * p), 256, 0, K.st>>>(r, ld, K.w, ld, N, p, K.w, ld);
        VSIE_CUDA(cudaGetLastError());
        for (int c = 0; c < p; ++c) done[c] = done[c] || cyc_done[c];
        // (loop re-evaluates the true residual norms at the top)
    }
    std::vector<double> nr;
    K.norms(nr);
    for (int c = 0; c < p; ++c) relres_est[c] = beta0[c] > 0 ? std::sqrt(nr[c]) / beta0[c] : 0.0;
}

vsie_status solve_impl(Ctx& c, int p, const double2* B, int64_t ldb, double2* X, int64_t ldx,
                       double tol, const vsie_solve_opts* o_in, vsie_solve_info* info,
                       cudaStream_t st) {
    vsie_solve_opts o{};
    if (o_in) o = *o_in;
    const int m = o.restart > 0 ? o.restart : 50;
    const int maxit = o.maxit > 0 ? o.maxit : 2000;
    const double inner_tol = o.inner_tol > 0 ? o.inner_tol : 1e-4;
    const int max_outer = o.max_outer > 0 ? o.max_outer : 20;
    if (!(tol > 0)) throw Error(VSIE_EINVAL, "tol must be > 0");
    if (p < 1 || p > c.max_rhs) throw Error(VSIE_EINVAL, "p outside [1, max_rhs]");
    if (ldb < c.N || ldx < c.N) throw Error(VSIE_EINVAL, "leading dimension < N");
    if (!c.f64.ready) throw Error(VSIE_EUNSUPPORTED, "vsie_solve needs the C128 operator");
    if (o.mode == 1 && !c.f32.ready) throw Error(VSIE_EUNSUPPORTED, "mode 1 needs the C64 operator");
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t N = c.N;
    const int64_t L = (N + 63) / 64 * 64;   // padded leading dimension of the work blocks
    const size_t pN = (size_t)p * L;
    // workspace (kept in the context between solves): the basis in the
    // precision of the mode, four FP64 and five FP32 p x N blocks, dot scratch
    if (o.precond < 0 || o.precond > 2) throw Error(VSIE_EINVAL, "precond must be 0, 1 or 2");
    const bool use_pc = o.precond != 1;
    const bool flex = o.precond == 2;   // learned body preconditioner: flexible GMRES
    if (flex && !c.net) throw Error(VSIE_EINVAL, "precond = 2 needs a network (vsie_net_attach)");
    if (flex && !c.f32.ready) throw Error(VSIE_EUNSUPPORTED, "precond = 2 needs the C64 operator");
    if (use_pc) build_block_precond(c);
    // basis (and, for flexible GMRES, the preconditioned basis) in the mode's precision
    const size_t basis_bytes = (size_t)(m + 1) * pN * (o.mode == 0 ? sizeof(double2) : sizeof(float2)) *
                               (flex ? 2 : 1);
    const size_t need = basis_bytes + 5 * pN * sizeof(double2) + 5 * pN * sizeof(float2) +
                        ((size_t)kDotBlocks * p * (m + 1) + (size_t)p * (m + 1) + p) * sizeof(double2) +
                        16 * 256;   // slack for the 256-byte alignment of each slice below
    if (c.kr_bytes < need) {
        if (c.kr_V) {
            auto& al = c.allocs;
            al.erase(std::remove(al.begin(), al.end(), (void*)c.kr_V), al.end());
            cudaFree(c.kr_V);
            c.kr_V = nullptr;
            c.kr_bytes = 0;
        }
        c.kr_V = (double2*)dalloc(c, need);
        c.kr_bytes = need;
    }
    char* base = (char*)c.kr_V;
    auto take = [&](size_t bytes) { char* q = base; base += (bytes + 255) / 256 * 256; return q; };
    void* Vb = take(basis_bytes);
    void* Zbb = flex ? (void*)((char*)Vb + basis_bytes / 2) : nullptr;
    double2* w64 = (double2*)take(pN * sizeof(double2));
    double2* r64 = (double2*)take(pN * sizeof(double2));
    double2* e64 = (double2*)take(pN * sizeof(double2));
    double2* Ax = (double2*)take(pN * sizeof(double2));
    double2* z64 = (double2*)take(pN * sizeof(double2));
    float2* w32 = (float2*)take(pN * sizeof(float2));
    float2* r32 = (float2*)take(pN * sizeof(float2));
    float2* e32 = (float2*)take(pN * sizeof(float2));
    float2* t32 = (float2*)take(pN * sizeof(float2));
    float2* z32 = (float2*)take(pN * sizeof(float2));
    double2* part = (double2*)take((size_t)kDotBlocks * p * (m + 1) * sizeof(double2));
    double2* hbuf = (double2*)take((size_t)p * (m + 1) * sizeof(double2));
    double2* scl = (double2*)take((size_t)p * sizeof(double2));
    Krylov<double> K64{c, p, N, L, m, o.mode == 0 ? (double2*)Vb : nullptr, w64, hbuf, part, scl, st};
    Krylov<float> K32{c, p, N, L, m, o.mode == 0 ? nullptr : (float2*)Vb, w32, hbuf, part, scl, st};
    int mv64 = 0, mv32 = 0, outer = 0;
    std::vector<int> iters(p, 0);
    std::vector<double> est;
    // ||b|| per column
    VSIE_CUDA(cudaMemcpy2DAsync(r64, L * sizeof(double2), B, ldb * sizeof(double2),
                                N * sizeof(double2), p, cudaMemcpyDeviceToDevice, st));
    VSIE_CUDA(cudaMemcpyAsync(w64, r64, pN * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    std::vector<double> bn2;
    K64.norms(bn2);
    std::vector<double> bn(p);
    for (int q = 0; q < p; ++q) {
        bn[q] = std::sqrt(bn2[q]);
        if (!std::isfinite(bn[q])) throw Error(VSIE_EBREAKDOWN, "non-finite right-hand side");
    }
    auto apply64 = [&](const double2* in, double2* out) {
        matvec_internal<double>(c, p, in, L, out, L, st);
    };
    // right-preconditioned operators A M (FP64) and A32 M32 (FP32)
    auto apply64_pc = [&](const double2* in, double2* out) {
        if (!use_pc) { apply64(in, out); return; }
        apply_block_precond<double>(c, p, in, L, z64, L, st);
        apply64(z64, out);
    };
    auto apply32_pc = [&](const float2* in, float2* out) {
        const float2* src = in;
        if (use_pc) {
            apply_block_precond<float>(c, p, in, L, t32, L, st);
            src = t32;
        }
        matvec_internal<float>(c, p, src, L, out, L, st);
    };
    // flexible GMRES: plain operators and the learned preconditioner
    auto apply32 = [&](const float2* in, float2* out) { matvec_internal<float>(c, p, in, L, out, L, st); };
    auto prec32 = [&](const float2* in, float2* out) { apply_learned_precond(c, p, in, L, out, L, st); };
    auto prec64 = [&](const double2* in, double2* out) {
        k_narrow<<<nblk(N * p), 256, 0, st>>>(in, L, N, p, t32, L);
        apply_learned_precond(c, p, t32, L, z32, L, st);
        k_widen_to<<<nblk(N * p), 256, 0, st>>>(z32, L, N, p, out, L);
        VSIE_CUDA(cudaGetLastError());
    };
    auto noprec32 = [](const float2*, float2*) {};
    auto noprec64 = [](const double2*, double2*) {};
    // x = 0
    VSIE_CUDA(cudaMemset2DAsync(X, ldx * sizeof(double2), 0, N * sizeof(double2), p, st));
    std::vector<double> relres(p, 1.0);
    bool have_res = false;
    if (o.mode == 0) {
        int cnt = 0;
        if (flex)
            gmres_core(K64, r64, tol, maxit, true, apply64, prec64, (double2*)Zbb, e64, iters, est, cnt);
        else
            gmres_core(K64, r64, tol, maxit, true, apply64_pc, noprec64, (double2*)nullptr, e64, iters,
                       est, cnt);
        mv64 += cnt;
        // x = M e (flexible: e is already the solution)
        const double2* xs = e64;
        if (use_pc && !flex) {
            apply_block_precond<double>(c, p, e64, L, z64, L, st);
            xs = z64;
        }
        VSIE_CUDA(cudaMemcpy2DAsync(X, ldx * sizeof(double2), xs, L * sizeof(double2),
                                    N * sizeof(double2), p, cudaMemcpyDeviceToDevice, st));
    } else {
        for (outer = 0; outer < max_outer; ++outer) {
            // r = b - Z64 x  (x = 0 on the first pass: r = b, no matvec)
            if (outer == 0) {
                VSIE_CUDA(cudaMemcpy2DAsync(r64, L * sizeof(double2), B, ldb * sizeof(double2),
                                            N * sizeof(double2), p, cudaMemcpyDeviceToDevice, st));
            } else {
                VSIE_CUDA(cudaMemcpy2DAsync(e64, L * sizeof(double2), X, ldx * sizeof(double2),
                                            N * sizeof(double2), p, cudaMemcpyDeviceToDevice, st));
                apply64(e64, Ax);
                ++mv64;
                k_sub<double><<<nblk(N * p), 256, 0, st>>>(B, ldb, Ax, L, N, p, r64, L);
                VSIE_CUDA(cudaGetLastError());
            }
            VSIE_CUDA(cudaMemcpyAsync(w64, r64, pN * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            std::vector<double> rn2;
            K64.norms(rn2);
            if (c.tc_err) {   // a bounded wait of the tensor-core preconditioner kernel ran out
                int e = 0;
                VSIE_CUDA(cudaMemcpy(&e, c.tc_err, sizeof(int), cudaMemcpyDeviceToHost));
                if (e) {
                    VSIE_CUDA(cudaMemset(c.tc_err, 0, sizeof(int)));
                    throw Error(VSIE_ETIMEOUT, "tensor-core far-block kernel: a bounded wait ran out");
                }
            }
            bool conv = true;
            for (int q = 0; q < p; ++q) {
                relres[q] = bn[q] > 0 ? std::sqrt(rn2[q]) / bn[q] : 0.0;
                if (!std::isfinite(relres[q])) throw Error(VSIE_EBREAKDOWN, "non-finite residual");
                conv = conv && relres[q] <= tol;
            }
            have_res = true;   // relres is the true FP64 residual of the current x
            if (conv) break;
            // inner correction to inner_tol (never tighter than the outer target needs)
            double itol = inner_tol;
            double worst = 0;
            for (int q = 0; q < p; ++q) worst = std::max(worst, relres[q]);
            itol = std::max(itol, 0.5 * tol / std::max(worst, 1e-300));
            itol = std::min(itol, 0.5);
            int cnt = 0;
            int budget = maxit;
            for (int q = 0; q < p; ++q) budget = std::min(budget, maxit - iters[q]);
            if (budget <= 0) break;
            k_narrow<<<nblk(N * p), 256, 0, st>>>(r64, L, N, p, r32, L);
            VSIE_CUDA(cudaGetLastError());
            if (flex)
                gmres_core(K32, r32, itol, budget, false, apply32, prec32, (float2*)Zbb, e32, iters, est,
                           cnt);
            else
                gmres_core(K32, r32, itol, budget, false, apply32_pc, noprec32, (float2*)nullptr, e32,
                           iters, est, cnt);
            mv32 += cnt;
            // x += M32 e (flexible: e is already the correction)
            const float2* corr = e32;
            if (use_pc && !flex) {
                apply_block_precond<float>(c, p, e32, L, z32, L, st);
                corr = z32;
            }
            k_add_widen<<<nblk(N * p), 256, 0, st>>>(corr, L, N, p, X, ldx);
            VSIE_CUDA(cudaGetLastError());
            have_res = false;
        }
    }
    // final true FP64 residual (already at hand when the refinement loop stopped
    // right after computing it)
    if (!have_res) {
        VSIE_CUDA(cudaMemcpy2DAsync(e64, L * sizeof(double2), X, ldx * sizeof(double2),
                                    N * sizeof(double2), p, cudaMemcpyDeviceToDevice, st));
        apply64(e64, Ax);
        ++mv64;
        k_sub<double><<<nblk(N * p), 256, 0, st>>>(B, ldb, Ax, L, N, p, w64, L);
        VSIE_CUDA(cudaGetLastError());
        std::vector<double> rn2;
        K64.norms(rn2);
        for (int q = 0; q < p; ++q) relres[q] = bn[q] > 0 ? std::sqrt(rn2[q]) / bn[q] : 0.0;
    }
    bool conv = true;
    for (int q = 0; q < p; ++q) conv = conv && relres[q] <= tol;
    VSIE_CUDA(cudaStreamSynchronize(st));
    if (info) {
        *info = vsie_solve_info{};
        for (int q = 0; q < p && q < 64; ++q) {
            info->iters[q] = iters[q];
            info->relres[q] = relres[q];
        }
        info->outer = outer;
        info->matvecs64 = mv64;
        info->matvecs32 = mv32;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    for (int q = 0; q < p; ++q)
        if (!std::isfinite(relres[q])) throw Error(VSIE_EBREAKDOWN, "non-finite final residual");
    return conv ? VSIE_OK : VSIE_ENOCONV;
}

// delta-gap right-hand sides
__global__ void k_set_entry(double2* B, int64_t ldb, int j, int64_t row, double2 v) {
    B[(size_t)j * ldb + row] = v;
}

}  // namespace vsie

using namespace vsie;

extern "C" {

vsie_status vsie_solve(vsie_ctx* ctx, int32_t p, const void* B, int64_t ldb, void* X, int64_t ldx,
                       double tol, const vsie_solve_opts* opts, vsie_solve_info* info,
                       vsie_stream stream) {
    if (!ctx) { set_global_err("null context"); return VSIE_EINVAL; }
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    try {
        if (!B || !X) throw Error(VSIE_EINVAL, "null B or X");
        const vsie_status st = solve_impl(*c, p, (const double2*)B, ldb, (double2*)X, ldx, tol, opts,
                                          info, reinterpret_cast<cudaStream_t>(stream));
        if (st == VSIE_ENOCONV) c->err = "GMRES reached maxit before the tolerance";
        return st;
    } catch (const Error& e) {
        c->err = e.msg;
        return e.st;
    }
}

vsie_status vsie_solve_batch(int32_t nctx, vsie_ctx* const* ctxs, const int32_t* p, const void* const* B,
                             const int64_t* ldb, void* const* X, const int64_t* ldx, double tol,
                             const vsie_solve_opts* opts, vsie_solve_info* info, vsie_status* status,
                             int32_t nthreads) {
    if (nctx < 0 || (nctx > 0 && (!ctxs || !p || !B || !ldb || !X || !ldx))) {
        set_global_err("null batch arrays or nctx < 0");
        return VSIE_EINVAL;
    }
    if (nctx == 0) return VSIE_OK;
    const bool learned = opts && opts->precond == 2;
    for (int i = 0; i < nctx; ++i)
        for (int k = 0; k < i; ++k) {
            if (ctxs[i] == ctxs[k]) {   // a context is not thread-safe
                set_global_err("a context appears twice in the batch");
                return VSIE_EINVAL;
            }
            if (learned && ctxs[i] && ctxs[k] && reinterpret_cast<Ctx*>(ctxs[i])->net &&
                reinterpret_cast<Ctx*>(ctxs[i])->net == reinterpret_cast<Ctx*>(ctxs[k])->net) {
                set_global_err("contexts of a batch share one network (its buffers are not thread-safe)");
                return VSIE_EINVAL;
            }
        }
    std::vector<vsie_status> st(nctx, VSIE_OK);
    const int nw = std::max(1, std::min<int>(nthreads > 0 ? nthreads : 8, nctx));
    std::atomic<int> next{0};
    auto worker = [&]() {
        cudaStream_t s = nullptr;
        int have_dev = -1;
        for (int i = next++; i < nctx; i = next++) {
            if (!ctxs[i]) { st[i] = VSIE_EINVAL; continue; }
            const int dev = reinterpret_cast<Ctx*>(ctxs[i])->device;
            if (dev != have_dev) {
                if (s) cudaStreamDestroy(s);
                s = nullptr;
                if (cudaSetDevice(dev) != cudaSuccess ||
                    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
                    cudaGetLastError();
                    st[i] = VSIE_ECUDA;
                    have_dev = -1;
                    continue;
                }
                have_dev = dev;
            }
            st[i] = vsie_solve(ctxs[i], p[i], B[i], ldb[i], X[i], ldx[i], tol, opts, info ? &info[i] : nullptr,
                               reinterpret_cast<vsie_stream>(s));
        }
        if (s) cudaStreamDestroy(s);
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < nw; ++w) pool.emplace_back(worker);
    worker();
    for (auto& t : pool) t.join();
    vsie_status first = VSIE_OK;
    for (int i = 0; i < nctx; ++i) {
        if (status) status[i] = st[i];
        if (first == VSIE_OK && st[i] != VSIE_OK) first = st[i];
    }
    return first;
}

vsie_status vsie_rhs_ports(vsie_ctx* ctx, int32_t nports, const int32_t* ports, double V, void* B,
                           int64_t ldb, vsie_stream stream) {
    if (!ctx) { set_global_err("null context"); return VSIE_EINVAL; }
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    try {
        if (!B || (nports > 0 && !ports)) throw Error(VSIE_EINVAL, "null B or port list");
        if (ldb < c->N) throw Error(VSIE_EINVAL, "leading dimension < N");
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        VSIE_CUDA(cudaMemset2DAsync(B, ldb * sizeof(double2), 0, c->N * sizeof(double2), nports, st));
        for (int j = 0; j < nports; ++j) {
            const int q = ports[j];
            if (q < 0 || q >= (int)c->port_row.size()) throw Error(VSIE_EINVAL, "port index out of range");
            const std::complex<double> v(0.0, c->omega * kEps0 * V * c->port_len[q]);
            k_set_entry<<<1, 1, 0, st>>>((double2*)B, ldb, j, c->port_row[q], make_double2(v.real(), v.imag()));
        }
        VSIE_CUDA(cudaGetLastError());
    } catch (const Error& e) {
        c->err = e.msg;
        return e.st;
    }
    return VSIE_OK;
}

}  // extern "C"
