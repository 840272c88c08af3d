// Surface blocks of the hybrid-VSIE matvec (Eq. hvsie_disc):
//   K2  pFFT projection (P x_n onto the coil-active voxels of the extended grid),
//       gather form: one output per (active voxel, component, RHS), no atomics;
//   K3  pFFT interpolation y_n = -P^T c (c: convolution on active voxels);
//   K4  precorrection y_b += Pre x_n and y_n += Pre^T (M x_b) (two CSR forms);
//   K6  y_n += Znn x_n + U (V^H x_f),  y_f = Z_ff x_f + conj(V) (U^T x_n);
//   K5  y_b += M TT(x_f) by Eq. (mvp), y_f += sum_chi TT_chi^T (M x_b,chi) by
//       Eq. (tmvp), each a chain of contractions: the first core against the
//       body by k_tt_g1 / k_tt_g1t (masked, all RHS in one launch), the others
//       by the GEMM kernels of gemm.cu.
// The FP32 dense Z_ff is stored in row panels and applied by gemm_panel; a
// hierarchical Z_ff (hmatrix.cu) replaces both dense products.
#include "hmatrix.h"

namespace vsie {

template <typename R>
__global__ void k_scatter(int64_t nrows, int p, const int32_t* __restrict__ ptr,
                          const int32_t* __restrict__ col, const cx<R>* __restrict__ val,
                          const cx<R>* __restrict__ X, int64_t ldx, int64_t xoff,
                          cx<R>* __restrict__ gc) {
    // rows are (b, c) = b * nact + c; output gc[(j * 3 + b) * nact + c] = gc[j * nrows + row]
    const int64_t tot = nrows * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e % nrows;
        const int j = e / nrows;
        const cx<R>* x = X + (size_t)j * ldx + xoff;
        cx<R> s = czero<cx<R>>();
        for (int q = ptr[row]; q < ptr[row + 1]; ++q) cfma(s, val[q], x[col[q]]);
        gc[(size_t)j * nrows + row] = s;
    }
}

template <typename R>
__global__ void k_gather(int m_n, int p, int s3, int64_t nact, const cx<R>* __restrict__ W,
                         const int32_t* __restrict__ cidx, const cx<R>* __restrict__ cc,
                         cx<R>* __restrict__ Y, int64_t ldy, int64_t yoff) {
    const int64_t tot = (int64_t)m_n * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int n = e % m_n;
        const int j = e / m_n;
        cx<R> s = czero<cx<R>>();
        for (int b = 0; b < 3; ++b) {
            const cx<R>* cb = cc + ((size_t)j * 3 + b) * nact;
            const cx<R>* w = W + (size_t)n * 3 * s3 + b * s3;
            const int32_t* ci = cidx + (size_t)n * s3;
            for (int q = 0; q < s3; ++q) cfma(s, w[q], cb[ci[q]]);
        }
        Y[(size_t)j * ldy + yoff + n] = make_neg(s);
    }
}

// Row-compressed CSR SpMV: y[rows[r]] += sum val * x[col]; optional row mask
// (rows of vacuum voxels are left untouched) and optional column mask.
template <typename R>
__global__ void k_spmv_add(int64_t nr, int p, const int32_t* __restrict__ rows,
                           const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                           const cx<R>* __restrict__ val, const cx<R>* __restrict__ X,
                           int64_t ldx, int64_t xoff, cx<R>* __restrict__ Y, int64_t ldy,
                           int64_t yoff, const uint8_t* __restrict__ rowmask, int64_t rowmod,
                           const uint8_t* __restrict__ colmask, int64_t colmod) {
    const int64_t tot = nr * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e % nr;
        const int j = e / nr;
        const int64_t row = rows[r];
        if (rowmask && !rowmask[row % rowmod]) continue;
        const cx<R>* x = X + (size_t)j * ldx + xoff;
        cx<R> s = czero<cx<R>>();
        for (int64_t q = ptr[r]; q < ptr[r + 1]; ++q) {
            const int32_t cidx = col[q];
            if (colmask && !colmask[cidx % colmod]) continue;
            cfma(s, val[q], x[cidx]);
        }
        cx<R>* y = Y + (size_t)j * ldy + yoff + row;
        *y = cadd(*y, s);
    }
}

static inline int nblk(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); }

// First TT core against the body (Eq. (mvp), last step, and Eq. (tmvp), first
// step), all p right-hand sides, material voxels only.  G1 is n1 x r1
// (column-major), a body column is the n1 voxels i1 of one (i2, i3).
constexpr int kG1Cols = 8;    // columns per CTA, forward
constexpr int kG1tCols = 28;  // columns per CTA, transposed (r1 x 28 <= 256 outputs: one round for r1 <= 9)

// y[j][i1 + n1 col] += sum_r G1[i1 + n1 r] t3[j][r + r1 col]   (mask[i1 + n1 col] != 0)
template <typename R>
__global__ void __launch_bounds__(256)
k_tt_g1(const cx<R>* __restrict__ G1, int n1, int r1, int ncol, const cx<R>* __restrict__ t3, int64_t st3,
        const uint8_t* __restrict__ mask, cx<R>* __restrict__ Y, int64_t ldy) {
    extern __shared__ __align__(16) unsigned char g1_smem[];
    cx<R>* g = reinterpret_cast<cx<R>*>(g1_smem);
    for (int i = threadIdx.x; i < n1 * r1; i += blockDim.x) g[i] = G1[i];
    __syncthreads();
    const int j = blockIdx.y, col0 = blockIdx.x * kG1Cols;
    const cx<R>* t = t3 + (size_t)j * st3;
    cx<R>* y = Y + (size_t)j * ldy;
    for (int e = threadIdx.x; e < n1 * kG1Cols; e += blockDim.x) {
        const int i1 = e % n1, col = col0 + e / n1;
        if (col >= ncol) break;
        const size_t v = (size_t)i1 + (size_t)n1 * col;
        if (!mask[v]) continue;
        cx<R> acc = mk<cx<R>>(0, 0);
        const cx<R>* tc = t + (size_t)r1 * col;
        for (int r = 0; r < r1; ++r) cfma(acc, g[i1 + n1 * r], tc[r]);
        y[v] = cadd(y[v], acc);
    }
}

// z[j][r + r1 col] = sum_i1 G1[i1 + n1 r] x[j][i1 + n1 col]   (x read as 0 where mask == 0)
// shared memory: G1 transposed with row stride n1 + 1, then the x columns with
// stride n1 + 1 (conflict-free reads across r and across columns)
template <typename R>
__global__ void __launch_bounds__(256)
k_tt_g1t(const cx<R>* __restrict__ G1, int n1, int r1, int ncol, const cx<R>* __restrict__ X, int64_t ldx,
         const uint8_t* __restrict__ mask, cx<R>* __restrict__ Z, int64_t sz) {
    extern __shared__ __align__(16) unsigned char g1_smem[];
    cx<R>* gt = reinterpret_cast<cx<R>*>(g1_smem);          // r1 x (n1 + 1)
    cx<R>* xs = gt + (size_t)r1 * (n1 + 1);                  // kG1tCols x (n1 + 1)
    const int j = blockIdx.y, col0 = blockIdx.x * kG1tCols;
    for (int i = threadIdx.x; i < n1 * r1; i += blockDim.x) {
        const int i1 = i % n1, r = i / n1;
        gt[r * (n1 + 1) + i1] = G1[i];
    }
    const cx<R>* x = X + (size_t)j * ldx;
    for (int e = threadIdx.x; e < n1 * kG1tCols; e += blockDim.x) {
        const int i1 = e % n1, c = e / n1, col = col0 + c;
        cx<R> v = mk<cx<R>>(0, 0);
        if (col < ncol) {
            const size_t q = (size_t)i1 + (size_t)n1 * col;
            if (mask[q]) v = x[q];
        }
        xs[c * (n1 + 1) + i1] = v;
    }
    __syncthreads();
    cx<R>* z = Z + (size_t)j * sz;
    for (int e = threadIdx.x; e < r1 * kG1tCols; e += blockDim.x) {
        const int r = e % r1, c = e / r1, col = col0 + c;
        if (col >= ncol) break;
        cx<R> acc = mk<cx<R>>(0, 0);
        const cx<R>* gr = gt + (size_t)r * (n1 + 1);
        const cx<R>* xc = xs + (size_t)c * (n1 + 1);
        for (int i1 = 0; i1 < n1; ++i1) cfma(acc, gr[i1], xc[i1]);
        z[(size_t)r + (size_t)r1 * col] = acc;
    }
}

template <typename R>
static size_t g1t_smem(int n1, int r1) { return ((size_t)r1 + kG1tCols) * (n1 + 1) * sizeof(cx<R>); }

template <typename R>
void surface_pre(Ctx& c, int p, const cx<R>* X, int64_t ldx, cudaStream_t st) {
    OpData<R>& d = data<R>(c);
    if (c.m_n == 0 || c.nact == 0) return;
    ProfScope ps(c, PG_PFFT, st);
    prof_count(c, 1);
    const int64_t nrows = 3 * c.nact;
    k_scatter<R><<<nblk(nrows * p), 256, 0, st>>>(nrows, p, c.sc_ptr, c.sc_col, d.sc_val, X, ldx,
                                                  (int64_t)c.m_f, d.gc);
    VSIE_CUDA(cudaGetLastError());
}

template <typename R>
void surface_apply(Ctx& c, int p, const cx<R>* X, int64_t ldx, cx<R>* Y, int64_t ldy,
                   cudaStream_t st) {
    using C = cx<R>;
    OpData<R>& d = data<R>(c);
    const C one = mk<C>(1, 0), zero = mk<C>(0, 0);
    const int64_t xb = (int64_t)c.m_f + c.m_n;
    const int mf = c.m_f, mn = c.m_n;
    if (mn > 0) {
        const int s3 = c.s * c.s * c.s;
        {
        ProfScope ps(c, PG_PFFT, st);
        prof_count(c, 1);
        k_gather<R><<<nblk((int64_t)mn * p), 256, 0, st>>>(mn, p, s3, c.nact, d.W, c.W_cidx, d.cc,
                                                           Y, ldy, (int64_t)mf);
        VSIE_CUDA(cudaGetLastError());
        }
        ProfScope ps(c, PG_SURF, st);
        cgemm<R>(c, OP_N, mn, p, mn, one, d.Znn, mn, 0, X + mf, ldx, 0, one, Y + mf, ldy, 0, 1,
                 nullptr, nullptr, st);
        if (c.pre_nnz > 0) {
            ProfScope ps2(c, PG_PRECORR, st);
            prof_count(c, 2);
            k_spmv_add<R><<<nblk(c.pre_nr * p), 256, 0, st>>>(
                c.pre_nr, p, c.pre_rows, c.pre_ptr, c.pre_col, d.pre_val, X, ldx, (int64_t)mf, Y,
                ldy, xb, c.mask, c.n_b, nullptr, 1);
            k_spmv_add<R><<<nblk(c.preT_nr * p), 256, 0, st>>>(
                c.preT_nr, p, c.preT_rows, c.preT_ptr, c.preT_col, d.preT_val, X, ldx, xb, Y, ldy,
                (int64_t)mf, nullptr, 1, c.mask, c.n_b);
            VSIE_CUDA(cudaGetLastError());
        }
    }
    if (mf > 0) {
        {
        ProfScope ps(c, PG_SURF, st);
        if (c.hm.on)
            hm_apply<R>(c, p, X, ldx, Y, ldy, st);                    // hierarchical Z_ff
        else if constexpr (sizeof(R) == 4)
            gemm_panel(c, mf, p, mf, d.Zff, X, ldx, Y, ldy, st);   // FP32 Z_ff in row panels
        else
            cgemm<R>(c, OP_N, mf, p, mf, one, d.Zff, mf, 0, X, ldx, 0, zero, Y, ldy, 0, 1, nullptr,
                     nullptr, st);
        if (mn > 0 && c.aca_rank > 0) {
            const int k = c.aca_rank;
            // t = V^H x_f (k x p); y_n += U t
            cgemm<R>(c, OP_H, k, p, mf, one, d.V, mf, 0, X, ldx, 0, zero, d.t1, k, 0, 1, nullptr,
                     nullptr, st);
            cgemm<R>(c, OP_N, mn, p, k, one, d.U, mn, 0, d.t1, k, 0, one, Y + mf, ldy, 0, 1,
                     nullptr, nullptr, st);
            // t = U^T x_n; y_f += conj(V) t
            cgemm<R>(c, OP_T, k, p, mn, one, d.U, mn, 0, X + mf, ldx, 0, zero, d.t1, k, 0, 1,
                     nullptr, nullptr, st);
            cgemm<R>(c, OP_R, mf, p, k, one, d.V, mf, 0, d.t1, k, 0, one, Y, ldy, 0, 1, nullptr,
                     nullptr, st);
        }
        }
        // tensor trains of the far coupling, one per component
        ProfScope pst(c, PG_TT, st);
        const int n1 = c.nb[0], n2 = c.nb[1], n3 = c.nb[2];
        for (int a = 0; a < 3; ++a) {
            const int r1 = c.tt_rank[a][0], r2 = c.tt_rank[a][1], r3 = c.tt_rank[a][2];
            if (r1 == 0) continue;
            C* const* G = d.G[a];
            const int64_t boff = xb + (int64_t)a * c.n_b;
            // Eq. (mvp): y = G4 x_f; y = G3 y; Y = G2 Y; Y = G1 Y (masked accumulate)
            cgemm<R>(c, OP_T, r3, p, mf, one, G[3], mf, 0, X, ldx, 0, zero, d.t1, r3, 0, 1,
                     nullptr, nullptr, st);
            cgemm<R>(c, OP_N, r2 * n3, p, r3, one, G[2], (int64_t)r2 * n3, 0, d.t1, r3, 0, zero,
                     d.t2, (int64_t)r2 * n3, 0, 1, nullptr, nullptr, st);
            cgemm<R>(c, OP_N, r1 * n2, n3 * p, r2, one, G[1], (int64_t)r1 * n2, 0, d.t2, r2, 0,
                     zero, d.t3, (int64_t)r1 * n2, 0, 1, nullptr, nullptr, st);
            const int ncol = n2 * n3;
            const size_t sm1 = (size_t)n1 * r1 * sizeof(C), sm2 = g1t_smem<R>(n1, r1);
            const bool fused = sm1 <= 200 * 1024 && sm2 <= 200 * 1024;
            if (fused && (sm1 > 48 * 1024 || sm2 > 48 * 1024)) {
                VSIE_CUDA(cudaFuncSetAttribute(k_tt_g1<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)sm1));
                VSIE_CUDA(cudaFuncSetAttribute(k_tt_g1t<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)sm2));
            }
            if (fused) {
                k_tt_g1<R><<<dim3((ncol + kG1Cols - 1) / kG1Cols, p), 256, sm1, st>>>(
                    G[0], n1, r1, ncol, d.t3, (int64_t)r1 * ncol, c.mask, Y + boff, ldy);
                VSIE_CUDA(cudaGetLastError());
                prof_count(c, 1);
            } else {
                cgemm<R>(c, OP_N, n1, n2 * n3, r1, one, G[0], n1, 0, d.t3, r1,
                         (int64_t)r1 * n2 * n3, one, Y + boff, n1, ldy, p, nullptr, c.mask, st);
            }
            // Eq. (tmvp): Z1 = G1^T (M x_b); Z2 = G2^T Z1; Z3 = G3^T Z2; y_f += G4^T Z3
            if (fused) {
                k_tt_g1t<R><<<dim3((ncol + kG1tCols - 1) / kG1tCols, p), 256, sm2, st>>>(
                    G[0], n1, r1, ncol, X + boff, ldx, c.mask, d.t3, (int64_t)r1 * ncol);
                VSIE_CUDA(cudaGetLastError());
                prof_count(c, 1);
            } else {
                cgemm<R>(c, OP_T, r1, n2 * n3, n1, one, G[0], n1, 0, X + boff, n1, ldx, zero, d.t3,
                         r1, (int64_t)r1 * n2 * n3, p, c.mask, nullptr, st);
            }
            cgemm<R>(c, OP_T, r2, n3 * p, r1 * n2, one, G[1], (int64_t)r1 * n2, 0, d.t3,
                     (int64_t)r1 * n2, 0, zero, d.t2, r2, 0, 1, nullptr, nullptr, st);
            cgemm<R>(c, OP_T, r3, p, r2 * n3, one, G[2], (int64_t)r2 * n3, 0, d.t2,
                     (int64_t)r2 * n3, 0, zero, d.t1, r3, 0, 1, nullptr, nullptr, st);
            cgemm<R>(c, OP_N, mf, p, r3, one, G[3], mf, 0, d.t1, r3, 0, one, Y, ldy, 0, 1, nullptr,
                     nullptr, st);
        }
    }
}

template void surface_pre<float>(Ctx&, int, const float2*, int64_t, cudaStream_t);
template void surface_pre<double>(Ctx&, int, const double2*, int64_t, cudaStream_t);
template void surface_apply<float>(Ctx&, int, const float2*, int64_t, float2*, int64_t,
                                   cudaStream_t);
template void surface_apply<double>(Ctx&, int, const double2*, int64_t, double2*, int64_t,
                                    cudaStream_t);

}  // namespace vsie
