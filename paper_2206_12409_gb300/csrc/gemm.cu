// Complex GEMM used by the surface blocks (K6: Z_ff, Znn, U V^H and conj(V) U^T)
// and the TT chain (K5: Eq. mvp and Eq. tmvp are sequences of small-K
// contractions).  Column-major; C_b = alpha op(A_b) B_b + beta C_b.
// cgemm2 picks the kernel by shape:
//   k_gemm_ip     op(A) in {T, H}, few columns of A, long K (inner products);
//   k_gemm_ts     op(A) in {N, R}, many rows, N <= 16 (one thread per row);
//   k_cgemm       everything else: tiles of BM x BN outputs, BK = 16 staged
//                 through shared memory;
// and gemm_panel applies the FP32 far block stored in row panels.  Split-K
// partial sums go to a workspace and are reduced in a fixed order (the result
// does not depend on scheduling).  Optional masks: maskB zeroes B elements,
// maskC leaves masked C elements untouched.
#include "vsie_internal.h"

#include <algorithm>

namespace vsie {

constexpr int BK = 16;

template <typename R, int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__(256)
k_cgemm(int opA, int opB, int M, int N, int K, cx<R> alpha, const cx<R>* __restrict__ A, int64_t lda,
        int64_t sA, const cx<R>* __restrict__ B, int64_t ldb, int64_t sB, cx<R> beta,
        cx<R>* __restrict__ C, int64_t ldc, int64_t sC, int batch, int splits,
        const uint8_t* __restrict__ maskB, const uint8_t* __restrict__ maskC,
        cx<R>* __restrict__ ws) {
    using Cx = cx<R>;
    constexpr int TX = BM / TM, TY = BN / TN;
    static_assert(TX * TY == 256, "256 threads");
    __shared__ Cx As[BK][BM + 1];
    __shared__ Cx Bs[BK][BN + 1];
    const int bz = blockIdx.z;
    const int b = bz % batch, sp = bz / batch;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const Cx* Ab = A + (size_t)b * sA;
    const Cx* Bb = B + (size_t)b * sB;
    const int ktiles = (K + BK - 1) / BK;
    const int per = (ktiles + splits - 1) / splits;
    const int kt0 = sp * per, kt1 = min(ktiles, kt0 + per);
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    Cx acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = czero<Cx>();
    const bool trans = (opA == OP_T || opA == OP_H);
    const bool conj = (opA == OP_H || opA == OP_R);
    for (int kt = kt0; kt < kt1; ++kt) {
        const int k0 = kt * BK;
        for (int e = tid; e < BM * BK; e += 256) {
            int m, k;
            if (trans) { k = e % BK; m = e / BK; } else { m = e % BM; k = e / BM; }
            const int gm = m0 + m, gk = k0 + k;
            Cx v = czero<Cx>();
            if (gm < M && gk < K) {
                v = trans ? Ab[(size_t)gk + (size_t)gm * lda] : Ab[(size_t)gm + (size_t)gk * lda];
                if (conj) v.y = -v.y;
            }
            As[k][m] = v;
        }
        for (int e = tid; e < BK * BN; e += 256) {
            const int k = e % BK, n = e / BK;
            const int gk = k0 + k, gn = n0 + n;
            Cx v = czero<Cx>();
            if (gk < K && gn < N) {
                if (opB == OP_N) v = Bb[(size_t)gk + (size_t)gn * ldb];
                else v = Bb[(size_t)gn + (size_t)gk * ldb];
                if (opB == OP_H) v.y = -v.y;
                if (maskB && !maskB[(size_t)gk + (size_t)K * gn]) v = czero<Cx>();
            }
            Bs[k][n] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            Cx a[TM], bb[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[k][tx + i * TX];
#pragma unroll
            for (int j = 0; j < TN; ++j) bb[j] = Bs[k][ty + j * TY];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) cfma(acc[i][j], a[i], bb[j]);
        }
        __syncthreads();
    }
    if (splits > 1) {
        Cx* w = ws + ((size_t)sp * batch + b) * (size_t)M * N;
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int gm = m0 + tx + i * TX, gn = n0 + ty + j * TY;
                if (gm < M && gn < N) w[(size_t)gm + (size_t)M * gn] = acc[i][j];
            }
        return;
    }
    Cx* Cb = C + (size_t)b * sC;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int gm = m0 + tx + i * TX, gn = n0 + ty + j * TY;
            if (gm >= M || gn >= N) continue;
            if (maskC && !maskC[(size_t)gm + (size_t)M * gn]) continue;
            Cx* cp = Cb + (size_t)gm + (size_t)gn * ldc;
            Cx r = cmul(alpha, acc[i][j]);
            if (beta.x != 0 || beta.y != 0) cfma(r, beta, *cp);
            *cp = r;
        }
}

template <typename R>
__global__ void k_splitk_reduce(int M, int N, int batch, int splits, cx<R> alpha,
                                const cx<R>* __restrict__ ws, cx<R> beta, cx<R>* __restrict__ C,
                                int64_t ldc, int64_t sC, const uint8_t* __restrict__ maskC) {
    using Cx = cx<R>;
    const size_t tot = (size_t)batch * M * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot;
         e += (size_t)gridDim.x * blockDim.x) {
        const int b = e / ((size_t)M * N);
        const size_t r = e - (size_t)b * M * N;
        const int gm = r % M, gn = r / M;
        if (maskC && !maskC[(size_t)gm + (size_t)M * gn]) continue;
        Cx s = czero<Cx>();
        for (int sp = 0; sp < splits; ++sp) s = cadd(s, ws[((size_t)sp * batch + b) * M * N + r]);
        Cx* cp = C + (size_t)b * sC + gm + (size_t)gn * ldc;
        Cx out = cmul(alpha, s);
        if (beta.x != 0 || beta.y != 0) cfma(out, beta, *cp);
        *cp = out;
    }
}

// Tall-skinny product C = alpha op(A) B (+ beta C) for op(A) in {N, R}, N <= NB
// right-hand sides and large M: one thread per row of C keeps all N
// accumulators in registers and streams its row of A (coalesced across the
// threads of a CTA, KU loads in flight); B is staged through shared memory one
// K-chunk at a time.  This is the shape of the dense surface blocks and of the
// block preconditioner (M, K ~ m_f, N = p): HBM-bound on reading A once.
template <typename R, int NB>
__global__ void __launch_bounds__(256)
k_gemm_ts(int conjA, int M, int N, int K, const cx<R>* __restrict__ A, int64_t lda,
          const cx<R>* __restrict__ B, int64_t ldb, int splits, cx<R>* __restrict__ ws,
          cx<R> alpha, cx<R> beta, cx<R>* __restrict__ C, int64_t ldc) {
    using Cx = cx<R>;
    constexpr int KC = 64, KU = 8;
    __shared__ Cx Bs[KC][NB];
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int sp = blockIdx.y;
    const int kper = (((K + splits - 1) / splits) + KC - 1) / KC * KC;
    const int k0 = sp * kper, k1 = min(K, k0 + kper);
    Cx acc[NB];
#pragma unroll
    for (int n = 0; n < NB; ++n) acc[n] = czero<Cx>();
    for (int kc = k0; kc < k1; kc += KC) {
        const int kn = min(KC, k1 - kc);
        __syncthreads();
        for (int e = threadIdx.x; e < KC * NB; e += blockDim.x) {
            const int kk = e / NB, n = e - kk * NB;
            Bs[kk][n] = (kk < kn && n < N) ? B[(size_t)(kc + kk) + (size_t)n * ldb] : czero<Cx>();
        }
        __syncthreads();
        if (m < M) {
            const Cx* Ap = A + (size_t)m + (size_t)kc * lda;
            for (int kk0 = 0; kk0 < kn; kk0 += KU) {
                Cx a[KU];
#pragma unroll
                for (int u = 0; u < KU; ++u) {
                    a[u] = (kk0 + u < kn) ? Ap[(size_t)(kk0 + u) * lda] : czero<Cx>();
                    if (conjA) a[u].y = -a[u].y;
                }
#pragma unroll
                for (int u = 0; u < KU; ++u)
#pragma unroll
                    for (int n = 0; n < NB; ++n) cfma(acc[n], a[u], Bs[kk0 + u][n]);
            }
        }
    }
    if (m >= M) return;
    if (splits > 1) {
        Cx* w = ws + (size_t)sp * M * N;
#pragma unroll
        for (int n = 0; n < NB; ++n)
            if (n < N) w[(size_t)m + (size_t)M * n] = acc[n];
        return;
    }
#pragma unroll
    for (int n = 0; n < NB; ++n) {
        if (n >= N) break;
        Cx* cp = C + (size_t)m + (size_t)n * ldc;
        Cx r = cmul(alpha, acc[n]);
        if (beta.x != 0 || beta.y != 0) cfma(r, beta, *cp);
        *cp = r;
    }
}

template <typename R, int NB>
static void launch_ts(Ctx& c, bool conjA, int M, int N, int K, cx<R> alpha, const cx<R>* A,
                      int64_t lda, const cx<R>* B, int64_t ldb, cx<R> beta, cx<R>* C, int64_t ldc,
                      cudaStream_t st) {
    OpData<R>& d = data<R>(c);
    const int mb = (M + 255) / 256;
    int splits = std::max(1, std::min((4 * 152 + mb - 1) / mb, K / 256));
    while (splits > 1 && (size_t)splits * M * N > d.splitk_elems) --splits;
    dim3 g(mb, splits);
    prof_count(c, splits > 1 ? 2 : 1);
    k_gemm_ts<R, NB><<<g, 256, 0, st>>>(conjA ? 1 : 0, M, N, K, A, lda, B, ldb, splits, d.splitk,
                                        alpha, beta, C, ldc);
    if (splits > 1) {
        const size_t tot = (size_t)M * N;
        const int blocks = (int)std::min<size_t>((tot + 255) / 256, 4096);
        k_splitk_reduce<R><<<blocks, 256, 0, st>>>(M, N, 1, splits, alpha, d.splitk, beta, C, ldc,
                                                   0, nullptr);
    }
    VSIE_CUDA(cudaGetLastError());
}

template <typename R, int BM, int BN, int TM, int TN>
static void launch1(Ctx& c, GemmOp opA, GemmOp opB, int M, int N, int K, cx<R> alpha, const cx<R>* A,
                    int64_t lda, int64_t sA, const cx<R>* B, int64_t ldb, int64_t sB, cx<R> beta,
                    cx<R>* C, int64_t ldc, int64_t sC, int batch, const uint8_t* maskB,
                    const uint8_t* maskC, cudaStream_t st);

// Column tiles go to gridDim.y (at most 65535): wider products run in column
// chunks (a TT factor over a 1 mm head grid has ~10^7 columns).
template <typename R, int BM, int BN, int TM, int TN>
static void launch(Ctx& c, GemmOp opA, GemmOp opB, int M, int N, int K, cx<R> alpha, const cx<R>* A,
                   int64_t lda, int64_t sA, const cx<R>* B, int64_t ldb, int64_t sB, cx<R> beta,
                   cx<R>* C, int64_t ldc, int64_t sC, int batch, const uint8_t* maskB,
                   const uint8_t* maskC, cudaStream_t st) {
    const int maxN = 65535 * BN;
    for (int n0 = 0; n0 < N; n0 += maxN) {
        const int nn = std::min(maxN, N - n0);
        const cx<R>* Bc = opB == OP_N ? B + (size_t)n0 * ldb : B + n0;
        launch1<R, BM, BN, TM, TN>(c, opA, opB, M, nn, K, alpha, A, lda, sA, Bc, ldb, sB, beta,
                                   C + (size_t)n0 * ldc, ldc, sC, batch,
                                   maskB ? maskB + (size_t)n0 * K : nullptr,
                                   maskC ? maskC + (size_t)n0 * M : nullptr, st);
    }
}

template <typename R, int BM, int BN, int TM, int TN>
static void launch1(Ctx& c, GemmOp opA, GemmOp opB, int M, int N, int K, cx<R> alpha, const cx<R>* A,
                    int64_t lda, int64_t sA, const cx<R>* B, int64_t ldb, int64_t sB, cx<R> beta,
                    cx<R>* C, int64_t ldc, int64_t sC, int batch, const uint8_t* maskB,
                    const uint8_t* maskC, cudaStream_t st) {
    OpData<R>& d = data<R>(c);
    const int tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
    const int ktiles = (K + BK - 1) / BK;
    const long tiles = (long)tm * tn * batch;
    int splits = 1;
    if (tiles < 2 * 152 && ktiles >= 8) {
        splits = (int)((2 * 152 + tiles - 1) / tiles);
        splits = std::min(splits, ktiles / 4);
        splits = std::max(splits, 1);
        const size_t need = (size_t)splits * batch * M * N;
        while (splits > 1 && need > d.splitk_elems) {
            --splits;
        }
        if ((size_t)splits * batch * M * N > d.splitk_elems) splits = 1;
    }
    dim3 g(tm, tn, batch * splits);
    prof_count(c, splits > 1 ? 2 : 1);
    k_cgemm<R, BM, BN, TM, TN><<<g, 256, 0, st>>>(opA, opB, M, N, K, alpha, A, lda, sA, B, ldb, sB,
                                                  beta, C, ldc, sC, batch, splits, maskB, maskC,
                                                  d.splitk);
    if (splits > 1) {
        const size_t tot = (size_t)batch * M * N;
        const int blocks = (int)std::min<size_t>((tot + 255) / 256, 4096);
        k_splitk_reduce<R><<<blocks, 256, 0, st>>>(M, N, batch, splits, alpha, d.splitk, beta, C,
                                                   ldc, sC, maskC);
    }
    VSIE_CUDA(cudaGetLastError());
}

// Inner-product shape C = alpha op(A) B (+ beta C) for op(A) in {T, H}, A stored
// K x M column-major with few columns (M <= 512), long K, N <= NB: a CTA owns
// IPC columns of A and one K split, its threads stride over K (coalesced reads
// of the A columns and of B), and the sums reduce by warp shuffles.
template <typename R, int NB, int IPC>
__global__ void __launch_bounds__(256)
k_gemm_ip(int conjA, int M, int N, int K, const cx<R>* __restrict__ A, int64_t lda,
          const cx<R>* __restrict__ B, int64_t ldb, int splits, cx<R>* __restrict__ ws, cx<R> alpha,
          cx<R> beta, cx<R>* __restrict__ C, int64_t ldc) {
    using Cx = cx<R>;
    const int i0 = blockIdx.x * IPC, sp = blockIdx.y;
    const int kper = (K + splits - 1) / splits;
    const int k0 = sp * kper, k1 = min(K, k0 + kper);
    Cx acc[IPC][NB];
#pragma unroll
    for (int q = 0; q < IPC; ++q)
#pragma unroll
        for (int n = 0; n < NB; ++n) acc[q][n] = czero<Cx>();
    for (int m = k0 + threadIdx.x; m < k1; m += blockDim.x) {
        Cx a[IPC];
#pragma unroll
        for (int q = 0; q < IPC; ++q) {
            a[q] = i0 + q < M ? A[(size_t)m + (size_t)(i0 + q) * lda] : czero<Cx>();
            if (conjA) a[q].y = -a[q].y;
        }
#pragma unroll
        for (int n = 0; n < NB; ++n) {
            if (n >= N) break;
            const Cx b = B[(size_t)m + (size_t)n * ldb];
#pragma unroll
            for (int q = 0; q < IPC; ++q) cfma(acc[q][n], a[q], b);
        }
    }
    __shared__ Cx red[IPC][NB][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < IPC; ++q)
#pragma unroll
        for (int n = 0; n < NB; ++n) {
            if (n >= N) break;
            auto vx = acc[q][n].x, vy = acc[q][n].y;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                vx += __shfl_down_sync(0xffffffffu, vx, o);
                vy += __shfl_down_sync(0xffffffffu, vy, o);
            }
            if (lane == 0) { red[q][n][wid].x = vx; red[q][n][wid].y = vy; }
        }
    __syncthreads();
    for (int e = threadIdx.x; e < IPC * N; e += blockDim.x) {
        const int q = e / N, n = e - q * N;
        const int i = i0 + q;
        if (i >= M) continue;
        Cx s = czero<Cx>();
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = cadd(s, red[q][n][w]);
        if (splits > 1) {
            ws[(size_t)sp * M * N + i + (size_t)M * n] = s;
        } else {
            Cx* cp = C + i + (size_t)n * ldc;
            Cx r = cmul(alpha, s);
            if (beta.x != 0 || beta.y != 0) cfma(r, beta, *cp);
            *cp = r;
        }
    }
}

template <typename R>
static void launch_ip(Ctx& c, bool conjA, int M, int N, int K, cx<R> alpha, const cx<R>* A, int64_t lda,
                      const cx<R>* B, int64_t ldb, cx<R> beta, cx<R>* C, int64_t ldc, cudaStream_t st) {
    OpData<R>& d = data<R>(c);
    // columns per CTA: 64 accumulator words per thread at most
    const int ipc = N <= 8 ? (sizeof(R) == 4 ? 4 : 2) : (sizeof(R) == 4 ? 2 : 1);
    const int mb = (M + ipc - 1) / ipc;
    int splits = std::max(1, std::min((2 * 152 + mb - 1) / mb, K / 512));
    while (splits > 1 && (size_t)splits * M * N > d.splitk_elems) --splits;
    dim3 g(mb, splits);
    prof_count(c, splits > 1 ? 2 : 1);
    const int cj = conjA ? 1 : 0;
    if (N <= 8) {
        if (sizeof(R) == 4) k_gemm_ip<R, 8, 4><<<g, 256, 0, st>>>(cj, M, N, K, A, lda, B, ldb, splits, d.splitk, alpha, beta, C, ldc);
        else k_gemm_ip<R, 8, 2><<<g, 256, 0, st>>>(cj, M, N, K, A, lda, B, ldb, splits, d.splitk, alpha, beta, C, ldc);
    } else {
        if (sizeof(R) == 4) k_gemm_ip<R, 16, 2><<<g, 256, 0, st>>>(cj, M, N, K, A, lda, B, ldb, splits, d.splitk, alpha, beta, C, ldc);
        else k_gemm_ip<R, 16, 1><<<g, 256, 0, st>>>(cj, M, N, K, A, lda, B, ldb, splits, d.splitk, alpha, beta, C, ldc);
    }
    if (splits > 1) {
        const size_t tot = (size_t)M * N;
        const int blocks = (int)std::min<size_t>((tot + 255) / 256, 4096);
        k_splitk_reduce<R><<<blocks, 256, 0, st>>>(M, N, 1, splits, alpha, d.splitk, beta, C, ldc, 0, nullptr);
    }
    VSIE_CUDA(cudaGetLastError());
}

template <typename R>
void cgemm2(Ctx& c, GemmOp opA, GemmOp opB, int M, int N, int K, cx<R> alpha, const cx<R>* A,
            int64_t lda, int64_t sA, const cx<R>* B, int64_t ldb, int64_t sB, cx<R> beta, cx<R>* C,
            int64_t ldc, int64_t sC, int batch, const uint8_t* maskB, const uint8_t* maskC,
            cudaStream_t st) {
    if (M <= 0 || N <= 0 || batch <= 0) return;
    if (K <= 0) {
        // C = beta C
        if (beta.x == 1 && beta.y == 0) return;
    }
    if (batch == 1 && opB == OP_N && (opA == OP_T || opA == OP_H) && !maskB && !maskC &&
        M <= 8192 && K >= 1024 && N <= 16) {
        launch_ip<R>(c, opA == OP_H, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
        return;
    }
    if (batch == 1 && opB == OP_N && (opA == OP_N || opA == OP_R) && !maskB && !maskC &&
        M >= 1024 && N <= 16) {
        if (N <= 8)
            launch_ts<R, 8>(c, opA == OP_R, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
        else
            launch_ts<R, 16>(c, opA == OP_R, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
        return;
    }
    if (N <= 8)
        launch<R, 128, 8, 4, 1>(c, opA, opB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC,
                                batch, maskB, maskC, st);
    else if (N <= 16)
        launch<R, 64, 16, 2, 2>(c, opA, opB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC,
                                batch, maskB, maskC, st);
    else
        launch<R, 64, 64, 4, 4>(c, opA, opB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC,
                                batch, maskB, maskC, st);
}

template <typename R>
void cgemm(Ctx& c, GemmOp opA, int M, int N, int K, cx<R> alpha, const cx<R>* A, int64_t lda,
           int64_t sA, const cx<R>* B, int64_t ldb, int64_t sB, cx<R> beta, cx<R>* C,
           int64_t ldc, int64_t sC, int batch, const uint8_t* maskB, const uint8_t* maskC,
           cudaStream_t st) {
    cgemm2<R>(c, opA, OP_N, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch,
              maskB, maskC, st);
}

template void cgemm2<double>(Ctx&, GemmOp, GemmOp, int, int, int, double2, const double2*,
                             int64_t, int64_t, const double2*, int64_t, int64_t, double2,
                             double2*, int64_t, int64_t, int, const uint8_t*, const uint8_t*,
                             cudaStream_t);
template void cgemm2<float>(Ctx&, GemmOp, GemmOp, int, int, int, float2, const float2*,
                            int64_t, int64_t, const float2*, int64_t, int64_t, float2,
                            float2*, int64_t, int64_t, int, const uint8_t*, const uint8_t*,
                            cudaStream_t);
template void cgemm<float>(Ctx&, GemmOp, int, int, int, float2, const float2*, int64_t, int64_t,
                           const float2*, int64_t, int64_t, float2, float2*, int64_t, int64_t,
                           int, const uint8_t*, const uint8_t*, cudaStream_t);
template void cgemm<double>(Ctx&, GemmOp, int, int, int, double2, const double2*, int64_t,
                            int64_t, const double2*, int64_t, int64_t, double2, double2*,
                            int64_t, int64_t, int, const uint8_t*, const uint8_t*,
                            cudaStream_t);

// ------------------------------------------------------------------ row panels
// Dense FP32 blocks that are streamed every iteration (Z_ff and its inverse) are
// stored as row panels: element (m, k) at ((m / 256) K + k) 256 + m % 256, so a
// CTA that owns 256 rows reads one contiguous stretch of memory.  Rows past M
// in the last panel are zero.
constexpr int kPanel = 256;

size_t panel_elems(int M, int K) { return (size_t)((M + kPanel - 1) / kPanel) * kPanel * (size_t)K; }

__global__ void k_to_panel(const float2* __restrict__ A, int64_t lda, int M, int K, float2* __restrict__ P) {
    const int mp = (M + kPanel - 1) / kPanel;
    const size_t n = (size_t)mp * kPanel * K;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i % kPanel);
        const size_t t = i / kPanel;
        const int k = (int)(t % K), pn = (int)(t / K);
        const int m = pn * kPanel + r;
        P[i] = m < M ? A[(size_t)m + (size_t)k * lda] : make_float2(0.f, 0.f);
    }
}

__global__ void k_from_panel(const float2* __restrict__ P, int M, int K, float2* __restrict__ A, int64_t lda) {
    const size_t n = (size_t)M * K;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(i % M), k = (int)(i / M);
        A[(size_t)m + (size_t)k * lda] = P[((size_t)(m / kPanel) * K + k) * kPanel + m % kPanel];
    }
}

// Partial products of C = P B over one K split, one thread per row, N <= NB
// columns, with the three-multiplication complex product (Gauss):
//   (a + ib)(c + id) = [c(a + b) - b(c + d)] + i [c(a + b) + a(d - c)],
// the B-side sums c, d - c, c + d staged in shared memory once per K chunk.
template <int NB>
__global__ void __launch_bounds__(256)
k_gemm_panel(int M, int N, int K, const float2* __restrict__ P, const float2* __restrict__ B, int64_t ldb,
             int splits, float2* __restrict__ ws, float2* __restrict__ C, int64_t ldc) {
    constexpr int KC = 64, KU = 8;
    __shared__ float Bs[KC][3][NB];
    const int m = blockIdx.x * kPanel + threadIdx.x;
    const int sp = blockIdx.y;
    const int kper = (((K + splits - 1) / splits) + KC - 1) / KC * KC;
    const int k0 = sp * kper, k1 = min(K, k0 + kper);
    float s1[NB], s2[NB], s3[NB];
#pragma unroll
    for (int n = 0; n < NB; ++n) { s1[n] = 0.f; s2[n] = 0.f; s3[n] = 0.f; }
    const float2* Ab = P + (size_t)blockIdx.x * K * kPanel + threadIdx.x;
    for (int kc = k0; kc < k1; kc += KC) {
        const int kn = min(KC, k1 - kc);
        __syncthreads();
        for (int e = threadIdx.x; e < KC * NB; e += blockDim.x) {
            const int kk = e / NB, n = e - kk * NB;
            const float2 b = (kk < kn && n < N) ? B[(size_t)(kc + kk) + (size_t)n * ldb] : make_float2(0.f, 0.f);
            Bs[kk][0][n] = b.x;
            Bs[kk][1][n] = b.y - b.x;
            Bs[kk][2][n] = b.x + b.y;
        }
        __syncthreads();
        const float2* Ap = Ab + (size_t)kc * kPanel;
        for (int kk0 = 0; kk0 < kn; kk0 += KU) {
            float2 a[KU];
#pragma unroll
            for (int u = 0; u < KU; ++u)
                a[u] = (kk0 + u < kn) ? Ap[(size_t)(kk0 + u) * kPanel] : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < KU; ++u) {
                const float sa = a[u].x + a[u].y;
#pragma unroll
                for (int n = 0; n < NB; ++n) {
                    s1[n] = fmaf(sa, Bs[kk0 + u][0][n], s1[n]);
                    s2[n] = fmaf(a[u].x, Bs[kk0 + u][1][n], s2[n]);
                    s3[n] = fmaf(a[u].y, Bs[kk0 + u][2][n], s3[n]);
                }
            }
        }
    }
    if (m >= M) return;
    if (splits == 1) {
#pragma unroll
        for (int n = 0; n < NB; ++n)
            if (n < N) C[(size_t)m + (size_t)n * ldc] = make_float2(s1[n] - s3[n], s1[n] + s2[n]);
        return;
    }
    float2* w = ws + (size_t)sp * M * N;
#pragma unroll
    for (int n = 0; n < NB; ++n)
        if (n < N) w[(size_t)m + (size_t)M * n] = make_float2(s1[n] - s3[n], s1[n] + s2[n]);
}

void gemm_panel(Ctx& c, int M, int N, int K, const float2* P, const float2* B, int64_t ldb, float2* C,
                int64_t ldc, cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    OpData<float>& d = data<float>(c);
    const int mb = (M + kPanel - 1) / kPanel;
    for (int n0 = 0; n0 < N; n0 += 16) {
        const int nn = std::min(16, N - n0);
        int splits = std::max(1, std::min(16, K / 256));
        while (splits > 1 && (size_t)splits * M * nn > d.splitk_elems) --splits;
        dim3 g(mb, splits);
        prof_count(c, splits > 1 ? 2 : 1);
        if (nn <= 8)
            k_gemm_panel<8><<<g, kPanel, 0, st>>>(M, nn, K, P, B + (size_t)n0 * ldb, ldb, splits, d.splitk,
                                                C + (size_t)n0 * ldc, ldc);
        else
            k_gemm_panel<16><<<g, kPanel, 0, st>>>(M, nn, K, P, B + (size_t)n0 * ldb, ldb, splits, d.splitk,
                                                 C + (size_t)n0 * ldc, ldc);
        if (splits > 1) {
            const size_t tot = (size_t)M * nn;
            const int blocks = (int)std::min<size_t>((tot + 255) / 256, 4096);
            k_splitk_reduce<float><<<blocks, 256, 0, st>>>(M, nn, 1, splits, make_float2(1.f, 0.f), d.splitk,
                                                           make_float2(0.f, 0.f), C + (size_t)n0 * ldc, ldc, 0,
                                                           nullptr);
        }
    }
    VSIE_CUDA(cudaGetLastError());
}

float2* to_panel(Ctx& c, float2* A, int M, int K) {
    float2* P = (float2*)dalloc(c, panel_elems(M, K) * sizeof(float2));
    k_to_panel<<<152 * 16, 256>>>(A, M, M, K, P);
    VSIE_CUDA(cudaGetLastError());
    VSIE_CUDA(cudaDeviceSynchronize());
    auto& al = c.allocs;
    al.erase(std::remove(al.begin(), al.end(), (void*)A), al.end());
    cudaFree(A);
    return P;
}

void from_panel(const float2* P, int M, int K, float2* A) {
    k_from_panel<<<152 * 16, 256>>>(P, M, K, A, M);
    VSIE_CUDA(cudaGetLastError());
}

}  // namespace vsie
