// Dense FP32 complex product C (M x N, N <= 16) = A (M x K) B (K x N) on the
// 5th-generation tensor cores: tcgen05.mma (kind::tf32, M = 128, N = 32, K = 8)
// with the accumulator in tensor memory.  This is the shape of the block
// preconditioner's far-block inverse (M = K = m_f, N = p right-hand sides): a
// matrix streamed once from HBM against a thin operand, so the kernel is built
// to keep HBM busy.
//
// Complex to real: row m of A, read as 2K floats (re, im interleaved), times the
// 2K x 32 real matrix B' with
//   B'[2k][n] = Re B[k][n],  B'[2k+1][n] = -Im B[k][n]          (columns 0..15: Re C)
//   B'[2k][16+n] = Im B[k][n],  B'[2k+1][16+n] = Re B[k][n]     (columns 16..31: Im C)
// gives Re C in columns n and Im C in columns 16 + n.
// Split TF32 (FP32-level accuracy): x = hi + lo with hi = tf32(x) rounded to
// nearest and lo = x - hi; C ~= A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped
// A_lo B_lo term is ~2^-22 relative).
//
// Warp roles (192 threads, one CTA per SM, 5-stage shared-memory ring of 40 KB
// stages; a variant with a 7-stage ring of A tiles and a separate 2-slot ring of
// A_lo tiles measured 15 % slower, the split then waiting on the MMAs):
//   warp 0    one lane issues, per 32-float K chunk, the TMA load of the A tile
//             (128 rows x 128 B, 128-byte swizzle) and a bulk copy of the
//             prepared B' chunk (hi and lo, already swizzled) onto full[s];
//   warps 2-5 split the A tile in place into hi and lo (element-wise, so the
//             swizzle does not matter) and arrive on conv[s]; at the end they
//             read the accumulator out of tensor memory (warp w reads lanes
//             32 (w mod 4) .. +31) and store C;
//   warp 1    one lane issues the 3 x 4 MMAs of a chunk and commits them to
//             empty[s], which frees the stage for the next load.
// B' is written once per call by k_tc_prepB (K/16 chunks of 8 KB).  The K range
// is split over gridDim.y; partial sums go to a workspace and k_tc_reduce adds
// them in a fixed order.  Every mbarrier wait is bounded: a wait that runs out
// sets the error flag, the other roles then run out too, the producer waits
// (bounded) for its copies in flight and the tensor memory is freed.
// A must be stored row-major (K-major): row m at A + m lda, lda complex values,
// lda even (16-byte rows for TMA).
#include "vsie_internal.h"

#include <cuda.h>

namespace vsie {

namespace {
constexpr int TC_BM = 128;                      // rows per CTA: one MMA M
constexpr int TC_BK = 32;                       // floats of the real row view per stage (128 B)
constexpr int TC_NP = 32;                       // real product columns (16 re + 16 im)
constexpr int TC_ST = 5;                        // pipeline stages
constexpr int TC_A_BYTES = TC_BM * TC_BK * 4;   // 16 KB
constexpr int TC_B_BYTES = TC_NP * TC_BK * 4;   // 4 KB
constexpr int TC_STAGE = 2 * TC_A_BYTES + 2 * TC_B_BYTES;   // A hi, A lo, B' hi, B' lo: 40 KB
constexpr int TC_THREADS = 192;
constexpr uint32_t kSpinLimit = 1u << 24;       // bounded mbarrier waits: polls
constexpr uint64_t kWaitNs = 2000000000ull;     // and wall time (2 s)
}  // namespace

struct TcArgs {
    int M, N, K;
    const float* Bp;   // prepared B' chunks [kc][hi 1024 | lo 1024] floats
    float2* C;
    int64_t ldc;
    float2* ws;        // split-K partials [split][n][m]
    int splits, kper;  // k-chunks (of 32 floats) per split
    int* err;          // set when a bounded wait runs out
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait: gives up after kWaitNs of wall time (checked every 256 polls) or
// kSpinLimit polls, whichever comes first
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        if (mbar_try_wait(b, parity)) return true;
        if ((i & 255u) == 255u && globaltimer_ns() - t0 > kWaitNs) return false;
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
// shared memory descriptor, K-major operand with the 128-byte swizzle: start
// address, stride between 8-row groups 1024 B, descriptor version 1
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// B' of chunk kc (16 complex k): 32 rows (n') of 32 floats, K-major with the
// 128-byte swizzle (16-byte unit u of row r stored at unit u ^ (r mod 8)); hi at
// [kc][0, 1024), lo at [kc][1024, 2048).
__global__ void k_tc_prepB(int K, int N, const float2* __restrict__ B, int64_t ldb, int nchunks, float* __restrict__ Bp) {
    const size_t tot = (size_t)nchunks * 1024;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int kc = (int)(e >> 10), r = (int)(e & 1023);
        const int np = r >> 5, f = r & 31;
        const int kk = kc * (TC_BK / 2) + (f >> 1), n = np & 15;
        float v = 0.f;
        if (kk < K && n < N) {
            const float2 b = B[(size_t)kk + (size_t)n * ldb];
            v = np < 16 ? ((f & 1) ? -b.y : b.x) : ((f & 1) ? b.x : b.y);
        }
        const float hi = tf32_rna(v);
        const int off = np * 32 + ((((f >> 2) ^ (np & 7))) << 2) + (f & 3);
        Bp[(size_t)kc * 2048 + off] = hi;
        Bp[(size_t)kc * 2048 + 1024 + off] = v - hi;
    }
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_tcgemm(const __grid_constant__ CUtensorMap tmapA, TcArgs g) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full[TC_ST], conv[TC_ST], empty[TC_ST], done;
    __shared__ uint32_t tmem_base;
    __shared__ int fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_BM;
    const int nk_total = (2 * g.K + TC_BK - 1) / TC_BK;
    const int kc0 = blockIdx.y * g.kper;
    const int nk = min(nk_total, kc0 + g.kper) - kc0;
    if (tid == 0) {
        for (int s = 0; s < TC_ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], 4);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    if (warp == 0) {
        if (lane == 0) {   // producer
            bool bad = false;
            int issued = 0;
            for (int i = 0; i < nk; ++i) {
                const int s = i % TC_ST;
                if (i >= TC_ST && !mbar_wait(&empty[s], ((i / TC_ST) - 1) & 1)) { bad = true; break; }
                unsigned char* st = sm + s * TC_STAGE;
                mbar_expect_tx(&full[s], TC_A_BYTES + 2 * TC_B_BYTES);
                tma_load_2d(st, &tmapA, (kc0 + i) * TC_BK, m0, &full[s]);
                bulk_load(st + 2 * TC_A_BYTES, g.Bp + (size_t)(kc0 + i) * 2048, 2 * TC_B_BYTES, &full[s]);
                issued = i + 1;
            }
            // every copy still in flight lands before the CTA may exit (the
            // latest phase of each stage is the only one that can be pending)
            for (int q = max(0, issued - TC_ST); q < issued; ++q)
                if (!mbar_wait(&full[q % TC_ST], (q / TC_ST) & 1)) bad = true;
            if (bad) atomicExch(&fail, 1);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            // D = F32 (bits 4-5), A = B = TF32 (bits 7-9, 10-12), both K-major, N / 8 (bits 17-22), M / 16 (bits 24-28)
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_NP >> 3) << 17) |
                                   ((uint32_t)(TC_BM >> 4) << 24);
            bool bad = false;
            for (int i = 0; i < nk; ++i) {
                const int s = i % TC_ST;
                if (!mbar_wait(&conv[s], (i / TC_ST) & 1)) { bad = true; break; }
                tc_fence_after();
                const uint32_t ah = smem_u32(sm + s * TC_STAGE), al = ah + TC_A_BYTES;
                const uint32_t bh = ah + 2 * TC_A_BYTES, bl = bh + TC_B_BYTES;
#pragma unroll
                for (int j = 0; j < TC_BK / 8; ++j) {   // K = 8 TF32 (32 bytes) per MMA
                    const uint32_t o = 32u * j;
                    mma_tf32(tmem, sw128_desc(ah + o), sw128_desc(bh + o), idesc, (i > 0 || j > 0) ? 1u : 0u);
                    mma_tf32(tmem, sw128_desc(ah + o), sw128_desc(bl + o), idesc, 1u);
                    mma_tf32(tmem, sw128_desc(al + o), sw128_desc(bh + o), idesc, 1u);
                }
                mma_commit(&empty[s]);
            }
            mma_commit(&done);   // arrives once every MMA issued above has completed
            if (bad) atomicExch(&fail, 1);
        }
        __syncwarp();
    } else {
        // warps 2-5: split the A tile of each stage into hi (in place) and lo
        const int ct = tid - 64;
        bool bad = false;
        for (int i = 0; i < nk; ++i) {
            const int s = i % TC_ST;
            if (!__all_sync(0xffffffffu, mbar_wait(&full[s], (i / TC_ST) & 1))) { bad = true; break; }
            float4* Ahi = reinterpret_cast<float4*>(sm + s * TC_STAGE);
            float4* Alo = reinterpret_cast<float4*>(sm + s * TC_STAGE + TC_A_BYTES);
#pragma unroll
            for (int j = 0; j < TC_A_BYTES / 16 / 128; ++j) {
                const float4 a = Ahi[ct + 128 * j];
                const float4 h = make_float4(tf32_rna(a.x), tf32_rna(a.y), tf32_rna(a.z), tf32_rna(a.w));
                Ahi[ct + 128 * j] = h;
                Alo[ct + 128 * j] = make_float4(a.x - h.x, a.y - h.y, a.z - h.z, a.w - h.w);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&conv[s]);
        }
        if (!__all_sync(0xffffffffu, mbar_wait(&done, 0))) bad = true;
        if (bad && lane == 0) atomicExch(&fail, 1);
    }
    __syncthreads();
    const bool any_bad = fail != 0;
    if (any_bad && tid == 0) atomicExch(g.err, 1);
    tc_fence_after();
    if (!any_bad && warp >= 2) {
        const int q = warp & 3;   // tensor-memory lanes 32 q .. 32 q + 31
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16), r);
        const int m = m0 + q * 32 + lane;
        if (m < g.M) {
            float2* out = g.splits == 1 ? g.C : g.ws + (size_t)blockIdx.y * g.M * g.N;
            const int64_t ld = g.splits == 1 ? g.ldc : g.M;
#pragma unroll
            for (int n = 0; n < 16; ++n)
                if (n < g.N) out[(size_t)m + (size_t)n * ld] = make_float2(__uint_as_float(r[n]), __uint_as_float(r[16 + n]));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}

__global__ void k_tc_reduce(int M, int N, int splits, const float2* __restrict__ ws, float2* __restrict__ C,
                            int64_t ldc) {
    const size_t tot = (size_t)M * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        float2 s = make_float2(0.f, 0.f);
        for (int q = 0; q < splits; ++q) s = cadd(s, ws[(size_t)q * tot + e]);
        const int m = (int)(e % M), n = (int)(e / M);
        C[(size_t)m + (size_t)n * ldc] = s;
    }
}

// ------------------------------------------------------------------ host
bool tc_make_map(void* map, const float2* A, int M, int K, int64_t lda) {
    using Fn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                            const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                            CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Fn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return false;
        fn = (Fn)p;
    }
    if (lda % 2 != 0 || ((uintptr_t)A & 15) != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)2 * K, (cuuint64_t)M};
    const cuuint64_t strides[1] = {(cuuint64_t)lda * sizeof(float2)};
    const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)TC_BM};
    const cuuint32_t es[2] = {1, 1};
    return fn(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)A, dims, strides, box,
              es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void tc_gemm(Ctx& c, const void* map, int M, int N, int K, const float2* B, int64_t ldb, float2* C, int64_t ldc,
             cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    static bool attr = false;
    const int smem = TC_ST * TC_STAGE + 1024;
    if (!attr) {
        VSIE_CUDA(cudaFuncSetAttribute(k_tcgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr = true;
    }
    OpData<float>& d = data<float>(c);
    const int mt = (M + TC_BM - 1) / TC_BM;
    const int nk = (2 * K + TC_BK - 1) / TC_BK;
    if ((size_t)nk * 2048 > c.pc_bprep_elems) throw Error(VSIE_EINVAL, "tensor-core B workspace too small");
    for (int n0 = 0; n0 < N; n0 += 16) {
        const int nn = std::min(16, N - n0);
        // split K so that waves x chunks per CTA (the time, one CTA per SM) is smallest
        int best = 1;
        double best_cost = 1e300;
        for (int sp = 1; sp <= 16 && sp <= std::max(1, nk / 8); ++sp) {
            if (sp > 1 && (size_t)sp * M * nn > d.splitk_elems) break;
            const int kper = (nk + sp - 1) / sp;
            const int spr = (nk + kper - 1) / kper;
            const double cost = (double)((mt * spr + c.num_sms - 1) / c.num_sms) * kper;
            if (cost < best_cost * 0.999) { best_cost = cost; best = sp; }
        }
        const int kper = (nk + best - 1) / best;
        const int splits = (nk + kper - 1) / kper;
        k_tc_prepB<<<(int)std::min<size_t>(((size_t)nk * 1024 + 255) / 256, 8192), 256, 0, st>>>(
            K, nn, B + (size_t)n0 * ldb, ldb, nk, c.pc_bprep);
        TcArgs g{M, nn, K, c.pc_bprep, C + (size_t)n0 * ldc, ldc, d.splitk, splits, kper, c.tc_err};
        CUtensorMap tm;
        memcpy(&tm, map, sizeof(tm));
        k_tcgemm<<<dim3(mt, splits), TC_THREADS, smem, st>>>(tm, g);
        prof_count(c, splits > 1 ? 3 : 2);
        if (splits > 1) {
            const size_t tot = (size_t)M * nn;
            k_tc_reduce<<<(int)std::min<size_t>((tot + 255) / 256, 4096), 256, 0, st>>>(M, nn, splits, d.splitk,
                                                                                      C + (size_t)n0 * ldc, ldc);
        }
    }
    VSIE_CUDA(cudaGetLastError());
}

}  // namespace vsie
