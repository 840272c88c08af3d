// Block preconditioner for the hybrid-VSIE system (right preconditioning of
// the GMRES of Sec. III.A):
//   M = blockdiag( Z_ff^-1, Z_nn^-1, D_b^-1 ),
// the inverses of the far-far and near-near surface blocks of Eq. (hvsie)
// (dense; the EFIE blocks are what keeps restarted GMRES from converging) and
// the inverse diagonal of the body block, h^3 (1/chi - self term), on material
// voxels (identity on vacuum voxels).
//
// Set-up: Z_nn is the direct near block when vsie_setup provides it, else it is
// read off this context's own FP32 matvec applied to unit vectors on the near
// unknowns; both blocks are inverted once in FP32 by LU
// (cuSOLVER getrf/getrs, set-up only).  The FP64 copies used by the FP64 solver
// are the widened FP32 inverses (M only has to be a fixed operator).
// Application (every GMRES iteration): two dense complex GEMMs and one
// elementwise body kernel, all in this library's own kernels.
#include "vsie_internal.h"

#include <cusolverDn.h>

#include <algorithm>

namespace vsie {

template <typename R>
void matvec_internal(Ctx& c, int p, const cx<R>* X, int64_t ldx, cx<R>* Y, int64_t ldy,
                     cudaStream_t st);

#define VSIE_CUSOLVER(call)                                                                \
    do {                                                                                   \
        cusolverStatus_t s_ = (call);                                                      \
        if (s_ != CUSOLVER_STATUS_SUCCESS)                                                 \
            throw Error(VSIE_ECUDA, std::string(#call) + " failed: " + std::to_string(s_)); \
    } while (0)

__global__ void k_identity_c(float2* A, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n;
         e += (int64_t)gridDim.x * blockDim.x)
        A[e] = make_float2((e % n) == (e / n) ? 1.f : 0.f, 0.f);
}

__global__ void k_f32_widen(const float2* a, double2* b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        b[i] = make_double2(a[i].x, a[i].y);
}

// R[m * ldr + k] = A[m + lda * k] (32 x 32 tiles through shared memory)
__global__ void k_transpose32(const float2* __restrict__ A, int64_t lda, int n, float2* __restrict__ R, int64_t ldr) {
    __shared__ float2 t[32][33];
    const int k0 = blockIdx.x * 32, m0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int m = m0 + threadIdx.x, k = k0 + j;
        if (m < n && k < n) t[j][threadIdx.x] = A[(size_t)m + (size_t)lda * k];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int m = m0 + j, k = k0 + threadIdx.x;
        if (m < n && k < n) R[(size_t)m * ldr + k] = t[threadIdx.x][j];
    }
}

__global__ void k_unit_cols(float2* X, int64_t N, int p, int64_t row0) {
    // column j gets 1 at row0 + j (the rest was zeroed)
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < p) X[(size_t)j * N + row0 + j] = make_float2(1.f, 0.f);
}

// In-place inverse of an n x n FP32 complex matrix A (device, column-major).
static void invert_f32(Ctx& c, float2* A, int n) {
    cusolverDnHandle_t h = nullptr;
    VSIE_CUSOLVER(cusolverDnCreate(&h));
    float2* B = nullptr;
    int* ipiv = nullptr;
    int* info = nullptr;
    cuComplex* work = nullptr;
    try {
        int lwork = 0;
        VSIE_CUSOLVER(cusolverDnCgetrf_bufferSize(h, n, n, (cuComplex*)A, n, &lwork));
        if (cudaMalloc(&work, (size_t)std::max(lwork, 1) * sizeof(cuComplex)) != cudaSuccess ||
            cudaMalloc(&ipiv, (size_t)n * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&info, sizeof(int)) != cudaSuccess ||
            cudaMalloc(&B, (size_t)n * n * sizeof(float2)) != cudaSuccess)
            throw Error(VSIE_ENOMEM, "preconditioner factorisation workspace");
        VSIE_CUSOLVER(cusolverDnCgetrf(h, n, n, (cuComplex*)A, n, work, ipiv, info));
        int hinfo = 0;
        VSIE_CUDA(cudaMemcpy(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost));
        if (hinfo != 0) throw Error(VSIE_EBREAKDOWN, "singular surface block in the preconditioner");
        k_identity_c<<<2048, 256>>>(B, n);
        VSIE_CUDA(cudaGetLastError());
        VSIE_CUSOLVER(cusolverDnCgetrs(h, CUBLAS_OP_N, n, n, (cuComplex*)A, n, ipiv, (cuComplex*)B, n, info));
        VSIE_CUDA(cudaMemcpy(A, B, (size_t)n * n * sizeof(float2), cudaMemcpyDeviceToDevice));
        VSIE_CUDA(cudaDeviceSynchronize());
    } catch (...) {
        cudaFree(B); cudaFree(ipiv); cudaFree(info); cudaFree(work);
        cusolverDnDestroy(h);
        throw;
    }
    cudaFree(B); cudaFree(ipiv); cudaFree(info); cudaFree(work);
    cusolverDnDestroy(h);
}

void build_block_precond(Ctx& c) {
    if (c.pc_ready) return;
    if (!c.f32.ready || !c.f64.ready)
        throw Error(VSIE_EUNSUPPORTED, "the block preconditioner needs both precisions");
    // body: inverse diagonal of Z_bb
    {
        const double a = std::cbrt(3.0 / (4.0 * M_PI)) * c.h;
        const std::complex<double> self =
            (2.0 / 3.0) * std::complex<double>(1.0, c.k0 * a) * std::exp(std::complex<double>(0.0, -c.k0 * a)) - 1.0;
        std::vector<double2> d64(c.n_b);
        std::vector<float2> d32(c.n_b);
        const double h3 = c.h * c.h * c.h;
        for (int64_t v = 0; v < c.n_b; ++v) {
            const std::complex<double> chi(c.eps_r[v] - 1.0, -c.sigma[v] / (c.omega * kEps0));
            std::complex<double> di = 1.0;
            if (chi != std::complex<double>(0.0, 0.0)) di = 1.0 / (h3 * (1.0 / chi - self));
            d64[v] = make_double2(di.real(), di.imag());
            d32[v] = make_float2((float)di.real(), (float)di.imag());
        }
        c.f64.pc_bdiag = (double2*)dalloc(c, c.n_b * sizeof(double2));
        c.f32.pc_bdiag = (float2*)dalloc(c, c.n_b * sizeof(float2));
        VSIE_CUDA(cudaMemcpy(c.f64.pc_bdiag, d64.data(), c.n_b * sizeof(double2), cudaMemcpyHostToDevice));
        VSIE_CUDA(cudaMemcpy(c.f32.pc_bdiag, d32.data(), c.n_b * sizeof(float2), cudaMemcpyHostToDevice));
    }
    if (c.m_f > 0) {
        const size_t nn = (size_t)c.m_f * c.m_f;
        float2* A = (float2*)dalloc(c, nn * sizeof(float2));
        if (!c.f32.Zff) throw Error(VSIE_EUNSUPPORTED, "the dense far-far block is no longer held");
        from_panel(c.f32.Zff, c.m_f, c.m_f, A);     // the FP32 Z_ff is stored in row panels
        invert_f32(c, A, c.m_f);
        if (!c.hm.on) {   // with the hierarchical block only the FP32 (mixed) solves apply it
            c.f64.pc_Zffi = (double2*)dalloc(c, nn * sizeof(double2));
            k_f32_widen<<<2048, 256>>>(A, c.f64.pc_Zffi, nn);
            VSIE_CUDA(cudaGetLastError());
        }
        if (c.opts.dense_gemm == 0) {
            // row-major copy for the tensor-core kernel (even row pitch for TMA)
            const int mf = c.m_f;
            const int64_t ld = (mf + 1) / 2 * 2;
            float2* R = (float2*)dalloc(c, (size_t)mf * ld * sizeof(float2));
            VSIE_CUDA(cudaMemset(R, 0, (size_t)mf * ld * sizeof(float2)));
            dim3 tg((mf + 31) / 32, (mf + 31) / 32);
            k_transpose32<<<tg, dim3(32, 8)>>>(A, mf, mf, R, ld);
            VSIE_CUDA(cudaGetLastError());
            VSIE_CUDA(cudaDeviceSynchronize());
            auto& al = c.allocs;
            al.erase(std::remove(al.begin(), al.end(), (void*)A), al.end());
            cudaFree(A);
            if (!tc_make_map(c.pc_map, R, mf, mf, ld))
                throw Error(VSIE_ECUDA, "cannot encode the TMA tensor map of the far-block inverse");
            if (!c.tc_err) {
                c.tc_err = (int*)dalloc(c, sizeof(int));
                VSIE_CUDA(cudaMemset(c.tc_err, 0, sizeof(int)));
            }
            // B' workspace: 2048 floats per 16 complex k
            c.pc_bprep_elems = (size_t)((2 * (size_t)mf + 31) / 32) * 2048;
            c.pc_bprep = (float*)dalloc(c, c.pc_bprep_elems * sizeof(float));
            int dev = 0, nsm = 0;
            VSIE_CUDA(cudaGetDevice(&dev));
            VSIE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
            if (nsm > 0) c.num_sms = nsm;
            c.f32.pc_Zffi = R;
            c.pc_ld = ld;
            c.pc_tc = true;
        } else {
            c.f32.pc_Zffi = to_panel(c, A, c.m_f, c.m_f);   // frees A
        }
    }
    if (c.m_n > 0 && c.hZnn_direct.size() == (size_t)c.m_n * c.m_n) {
        // the set-up's direct near block Z_nn = -K_nn: the near-near block of the
        // operator (the grid part folded out of Znn~ is added back by the grid)
        const size_t nn = (size_t)c.m_n * c.m_n;
        std::vector<float2> h32(nn);
        for (size_t i = 0; i < nn; ++i)
            h32[i] = make_float2((float)c.hZnn_direct[i].real(), (float)c.hZnn_direct[i].imag());
        std::vector<std::complex<double>>().swap(c.hZnn_direct);
        float2* A = (float2*)dalloc(c, nn * sizeof(float2));
        VSIE_CUDA(cudaMemcpy(A, h32.data(), nn * sizeof(float2), cudaMemcpyHostToDevice));
        invert_f32(c, A, c.m_n);
        c.f32.pc_Znni = A;
        c.f64.pc_Znni = (double2*)dalloc(c, nn * sizeof(double2));
        k_f32_widen<<<2048, 256>>>(A, c.f64.pc_Znni, nn);
        VSIE_CUDA(cudaGetLastError());
    } else if (c.m_n > 0) {
        const int mn = c.m_n;
        const size_t nn = (size_t)mn * mn;
        float2* A = (float2*)dalloc(c, nn * sizeof(float2));
        // columns of Z_nn from the FP32 operator applied to unit vectors
        const int p = c.max_rhs;
        float2* X = nullptr;
        float2* Y = nullptr;
        if (cudaMalloc(&X, (size_t)c.N * p * sizeof(float2)) != cudaSuccess ||
            cudaMalloc(&Y, (size_t)c.N * p * sizeof(float2)) != cudaSuccess) {
            cudaFree(X);
            throw Error(VSIE_ENOMEM, "preconditioner set-up vectors");
        }
        try {
            for (int c0 = 0; c0 < mn; c0 += p) {
                const int pc = std::min(p, mn - c0);
                VSIE_CUDA(cudaMemset(X, 0, (size_t)c.N * p * sizeof(float2)));
                k_unit_cols<<<1, 64>>>(X, c.N, pc, (int64_t)c.m_f + c0);
                matvec_internal<float>(c, pc, X, c.N, Y, c.N, 0);
                VSIE_CUDA(cudaMemcpy2D(A + (size_t)mn * c0, mn * sizeof(float2), Y + c.m_f,
                                       c.N * sizeof(float2), mn * sizeof(float2), pc,
                                       cudaMemcpyDeviceToDevice));
            }
            VSIE_CUDA(cudaDeviceSynchronize());
        } catch (...) {
            cudaFree(X);
            cudaFree(Y);
            throw;
        }
        cudaFree(X);
        cudaFree(Y);
        invert_f32(c, A, mn);
        c.f32.pc_Znni = A;
        c.f64.pc_Znni = (double2*)dalloc(c, nn * sizeof(double2));
        k_f32_widen<<<2048, 256>>>(A, c.f64.pc_Znni, nn);
        VSIE_CUDA(cudaGetLastError());
    }
    VSIE_CUDA(cudaDeviceSynchronize());
    c.pc_ready = true;
}

template <typename R>
__global__ void k_body_diag(const cx<R>* __restrict__ X, int64_t ldx, const cx<R>* __restrict__ d,
                            int64_t nb, int p, int64_t off, cx<R>* __restrict__ Y, int64_t ldy) {
    const int64_t tot = 3 * nb * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = e / (3 * nb);
        const int64_t r = e - (int64_t)j * 3 * nb;
        const int64_t v = r % nb;
        Y[(size_t)j * ldy + off + r] = cmul(X[(size_t)j * ldx + off + r], d[v]);
    }
}

void apply_far_inverse32(Ctx& c, int p, const float2* X, int64_t ldx, float2* Y, int64_t ldy, cudaStream_t st) {
    if (c.pc_tc) tc_gemm(c, c.pc_map, c.m_f, p, c.m_f, X, ldx, Y, ldy, st);   // tensor cores
    else gemm_panel(c, c.m_f, p, c.m_f, c.f32.pc_Zffi, X, ldx, Y, ldy, st);   // SIMT row panels
}

// Y = M X (X, Y: N x p, leading dimensions ldx, ldy; must not overlap)
template <typename R>
void apply_block_precond(Ctx& c, int p, const cx<R>* X, int64_t ldx, cx<R>* Y, int64_t ldy,
                         cudaStream_t st) {
    OpData<R>& d = data<R>(c);
    ProfScope ps(c, PG_PRECOND, st);
    prof_count(c, 1);
    const cx<R> one = mk<cx<R>>(1, 0), zero = mk<cx<R>>(0, 0);
    if (c.m_f > 0) {
        if (!d.pc_Zffi)
            throw Error(VSIE_EUNSUPPORTED, "no FP64 far-block inverse (hierarchical Z_ff): use the mixed solve");
        if constexpr (sizeof(R) == 4)
            apply_far_inverse32(c, p, X, ldx, Y, ldy, st);
        else
            cgemm<R>(c, OP_N, c.m_f, p, c.m_f, one, d.pc_Zffi, c.m_f, 0, X, ldx, 0, zero, Y, ldy, 0, 1,
                     nullptr, nullptr, st);
    }
    if (c.m_n > 0)
        cgemm<R>(c, OP_N, c.m_n, p, c.m_n, one, d.pc_Znni, c.m_n, 0, X + c.m_f, ldx, 0, zero,
                 Y + c.m_f, ldy, 0, 1, nullptr, nullptr, st);
    const int64_t tot = 3 * c.n_b * p;
    k_body_diag<R><<<(int)std::min<int64_t>((tot + 255) / 256, 152 * 16), 256, 0, st>>>(
        X, ldx, d.pc_bdiag, c.n_b, p, (int64_t)c.m_f + c.m_n, Y, ldy);
    VSIE_CUDA(cudaGetLastError());
}

template void apply_block_precond<float>(Ctx&, int, const float2*, int64_t, float2*, int64_t, cudaStream_t);
template void apply_block_precond<double>(Ctx&, int, const double2*, int64_t, double2*, int64_t, cudaStream_t);

}  // namespace vsie
