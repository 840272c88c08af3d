// K8: the learned right preconditioner of the body block, a small 3D U-Net
// (not in the paper; it preconditions the body equations of Sec. II.B the way
// Sec. VI suggests a preconditioner for the coupled system should).
//
// Architecture (levels 0..3, channels 16/32/64/64, 3x3x3 convolutions with zero
// "same" padding, ReLU, 2x2x2 average pooling, nearest x2 upsampling, skip
// tensors concatenated after the upsampled ones, a linear 1x1x1 head):
//   e1a 8->16, e1b 16->16 | pool | e2a 16->32, e2b 32->32 | pool |
//   e3a 32->64, e3b 64->64 | pool | ba 64->64, bb 64->64 | up+cat |
//   d3a 128->64, d3b 64->64 | up+cat | d2a 96->32, d2b 32->32 | up+cat |
//   d1a 48->16, d1b 16->16 | head 16->6
// Tensors are FP32, channel-major (C, D, H, W) with W fastest.  Weights are kept
// as FP32 master copies (updated by Adam) and used by the kernels as BF16
// copies in two layouts (forward: [ci][tap][co]; data gradient: the same
// kernel run with [co][flipped tap][ci]).  The 3x3x3 convolutions run on the
// tensor cores (k_conv3_mma), the 1x1x1 head and the weight gradient on the
// FP32 pipes.  Every sum accumulates in FP32; the weight and bias gradients
// reduce over voxel chunks in a fixed order.
// Skip tensors are written by the encoder straight into the channel slice of
// the decoder's concatenation buffer, so no concatenation copies exist.
#include "vsie_internal.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <random>

namespace vsie {

struct LayerDef {
    int ci, co, k;
};
static const LayerDef kLayers[15] = {
    {8, 16, 3},  {16, 16, 3},  {16, 32, 3}, {32, 32, 3}, {32, 64, 3},
    {64, 64, 3}, {64, 64, 3},  {64, 64, 3}, {128, 64, 3}, {64, 64, 3},
    {96, 32, 3}, {32, 32, 3},  {48, 16, 3}, {16, 16, 3}, {16, 6, 1}};
enum { E1A, E1B, E2A, E2B, E3A, E3B, BA, BB, D3A, D3B, D2A, D2B, D1A, D1B, HEAD, NLAYER };

// ------------------------------------------------------------------ kernels
constexpr int TX = 8, TY = 8, TZ = 4;   // output tile of the convolution kernel
constexpr int COT = 8;                  // output channels per thread
constexpr int CIC = 4;                  // input channels staged per round

// y[co][v] = bias[co] + sum_ci sum_t w[ci][t][co] x[ci][v + t - r]  (zero outside),
// then ReLU when relu != 0.  wt: BF16, layout [Ci][K^3][Co].
template <int K>
__global__ void __launch_bounds__(256)
k_conv(const float* __restrict__ x, int Ci, int D, int H, int W, const __nv_bfloat16* __restrict__ wt,
       const float* __restrict__ bias, int Co, int relu, float* __restrict__ y) {
    constexpr int R = K / 2, K3 = K * K * K;
    constexpr int SX = TX + K - 1, SY = TY + K - 1, SZ = TZ + K - 1, SV = SX * SY * SZ;
    __shared__ float s_in[CIC][SV];
    __shared__ __align__(16) float s_w[CIC][K3][COT];
    const int tiles_x = (W + TX - 1) / TX;
    const int x0 = (blockIdx.x % tiles_x) * TX, y0 = (blockIdx.x / tiles_x) * TY;
    const int z0 = blockIdx.y * TZ, co0 = blockIdx.z * COT;
    const int t = threadIdx.x;
    const int tx = t % TX, ty = (t / TX) % TY, tz = t / (TX * TY);
    const size_t V = (size_t)D * H * W;
    float acc[COT];
#pragma unroll
    for (int c = 0; c < COT; ++c) acc[c] = 0.f;
    for (int cb = 0; cb < Ci; cb += CIC) {
        const int nc = min(CIC, Ci - cb);
        __syncthreads();
        for (int e = t; e < CIC * SV; e += 256) {
            const int c = e / SV, r = e - c * SV;
            const int sx = r % SX, sy = (r / SX) % SY, sz = r / (SX * SY);
            const int gx = x0 + sx - R, gy = y0 + sy - R, gz = z0 + sz - R;
            float v = 0.f;
            if (c < nc && gx >= 0 && gx < W && gy >= 0 && gy < H && gz >= 0 && gz < D)
                v = x[(size_t)(cb + c) * V + ((size_t)gz * H + gy) * W + gx];
            s_in[c][r] = v;
        }
        for (int e = t; e < CIC * K3 * COT; e += 256) {
            const int c = e / (K3 * COT), r = e - c * K3 * COT;
            const int tap = r / COT, o = r - tap * COT;
            float v = 0.f;
            if (c < nc && co0 + o < Co)
                v = __bfloat162float(wt[((size_t)(cb + c) * K3 + tap) * Co + co0 + o]);
            s_w[c][tap][o] = v;
        }
        __syncthreads();
        for (int c = 0; c < nc; ++c) {
#pragma unroll
            for (int kz = 0; kz < K; ++kz)
#pragma unroll
                for (int ky = 0; ky < K; ++ky)
#pragma unroll
                    for (int kx = 0; kx < K; ++kx) {
                        const float v = s_in[c][((tz + kz) * SY + ty + ky) * SX + tx + kx];
                        const int tap = (kz * K + ky) * K + kx;
                        const float4 wa = *reinterpret_cast<const float4*>(&s_w[c][tap][0]);
                        const float4 wb = *reinterpret_cast<const float4*>(&s_w[c][tap][4]);
                        acc[0] = fmaf(v, wa.x, acc[0]);
                        acc[1] = fmaf(v, wa.y, acc[1]);
                        acc[2] = fmaf(v, wa.z, acc[2]);
                        acc[3] = fmaf(v, wa.w, acc[3]);
                        acc[4] = fmaf(v, wb.x, acc[4]);
                        acc[5] = fmaf(v, wb.y, acc[5]);
                        acc[6] = fmaf(v, wb.z, acc[6]);
                        acc[7] = fmaf(v, wb.w, acc[7]);
                    }
        }
    }
    const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
    if (gx >= W || gy >= H || gz >= D) return;
    const size_t v = ((size_t)gz * H + gy) * W + gx;
#pragma unroll
    for (int c = 0; c < COT; ++c) {
        const int co = co0 + c;
        if (co >= Co) break;
        float r = acc[c] + (bias ? bias[co] : 0.f);
        if (relu) r = fmaxf(r, 0.f);
        y[(size_t)co * V + v] = r;
    }
}

// Tensor-core form of the 3x3x3 convolution (implicit GEMM on mma.sync
// m16n8k16, BF16 operands, FP32 accumulation):
//   y[co][v] = bias[co] + sum_{ci, tap} w[ci][tap][co] x[ci][v + tap - 1],
// M = 16 output channels per CTA (blockIdx.z), N = an 8 x 8 x 4 voxel tile
// (blockIdx.x over x-y tiles, blockIdx.y over z), K = 16 input channels x 27 taps
// per staged chunk.  The activations are split into two BF16 terms,
// x = hi + lo (hi = bf16(x), lo = bf16(x - hi)), and both are multiplied by the
// BF16 weights, so the products keep about 16 bits of the FP32 activations.
// Warp w owns z-slice w of the tile: 8 rows of 8 voxels = 8 n-tiles.
// Shared memory (dynamic): input hi and lo as [position][16 channels + pad] and
// the weights as [tap][16 co][16 ci + pad], padded so that the fragment loads
// of a warp fall in distinct banks.
constexpr int MC_PAD = 24;                    // BF16 per staged row (16 used)
constexpr int MC_SX = TX + 2, MC_SY = TY + 2, MC_SZ = TZ + 2, MC_SV = MC_SX * MC_SY * MC_SZ;
constexpr size_t kConvMmaSmem = (size_t)(2 * MC_SV + 27 * 16) * MC_PAD * sizeof(__nv_bfloat16);

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(128)
k_conv3_mma(const float* __restrict__ x, int Ci, int D, int H, int W, const __nv_bfloat16* __restrict__ wt,
            const float* __restrict__ bias, int Co, int relu, float* __restrict__ y) {
    extern __shared__ __align__(16) unsigned char mc_smem[];
    __nv_bfloat16* s_hi = reinterpret_cast<__nv_bfloat16*>(mc_smem);
    __nv_bfloat16* s_lo = s_hi + MC_SV * MC_PAD;
    __nv_bfloat16* s_w = s_lo + MC_SV * MC_PAD;          // [27][16 co][MC_PAD]
    const int tiles_x = (W + TX - 1) / TX;
    const int x0 = (blockIdx.x % tiles_x) * TX, y0 = (blockIdx.x / tiles_x) * TY;
    const int z0 = blockIdx.y * TZ, co0 = blockIdx.z * 16;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int g = lane >> 2, t4 = lane & 3;
    const size_t V = (size_t)D * H * W;
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
    for (int cb = 0; cb < Ci; cb += 16) {
        __syncthreads();
        // input halo tile, 16 channels, split into hi and lo
        for (int e = t; e < 16 * MC_SV; e += blockDim.x) {
            const int c = e / MC_SV, r = e - c * MC_SV;
            const int sx = r % MC_SX, sy = (r / MC_SX) % MC_SY, sz = r / (MC_SX * MC_SY);
            const int gx = x0 + sx - 1, gy = y0 + sy - 1, gz = z0 + sz - 1;
            float v = 0.f;
            if (cb + c < Ci && gx >= 0 && gx < W && gy >= 0 && gy < H && gz >= 0 && gz < D)
                v = x[(size_t)(cb + c) * V + ((size_t)gz * H + gy) * W + gx];
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            s_hi[r * MC_PAD + c] = hi;
            s_lo[r * MC_PAD + c] = __float2bfloat16_rn(v - __bfloat162float(hi));
        }
        // weights of this chunk: s_w[tap][o][c] = wt[cb + c][tap][co0 + o]
        for (int e = t; e < 27 * 16 * 16; e += blockDim.x) {
            const int o = e % 16, c = (e / 16) % 16, tap = e / 256;
            __nv_bfloat16 v = __float2bfloat16_rn(0.f);
            if (cb + c < Ci && co0 + o < Co) v = wt[((size_t)(cb + c) * 27 + tap) * Co + co0 + o];
            s_w[(tap * 16 + o) * MC_PAD + c] = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int tap = 0; tap < 27; ++tap) {
            const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
            const __nv_bfloat16* wa = s_w + (size_t)tap * 16 * MC_PAD;
            uint32_t a[4];
            a[0] = *reinterpret_cast<const uint32_t*>(wa + g * MC_PAD + t4 * 2);
            a[1] = *reinterpret_cast<const uint32_t*>(wa + (g + 8) * MC_PAD + t4 * 2);
            a[2] = *reinterpret_cast<const uint32_t*>(wa + g * MC_PAD + t4 * 2 + 8);
            a[3] = *reinterpret_cast<const uint32_t*>(wa + (g + 8) * MC_PAD + t4 * 2 + 8);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                // n-tile j: the row of 8 voxels (x = 0..7) at y = j, z = warp
                const int pos = ((warp + dz) * MC_SY + (j + dy)) * MC_SX + (g + dx);
                const __nv_bfloat16* bh = s_hi + pos * MC_PAD + t4 * 2;
                const __nv_bfloat16* bl = s_lo + pos * MC_PAD + t4 * 2;
                mma_bf16(acc[j], a, *reinterpret_cast<const uint32_t*>(bh),
                         *reinterpret_cast<const uint32_t*>(bh + 8));
                mma_bf16(acc[j], a, *reinterpret_cast<const uint32_t*>(bl),
                         *reinterpret_cast<const uint32_t*>(bl + 8));
            }
        }
    }
    // C fragment: rows g, g + 8 (output channel), columns 2 t4, 2 t4 + 1 (voxel x)
    const int gz = z0 + warp;
    if (gz >= D) return;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int gy = y0 + j;
        if (gy >= H) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int co = co0 + g + (q >= 2 ? 8 : 0);
            const int gx = x0 + t4 * 2 + (q & 1);
            if (co >= Co || gx >= W) continue;
            float r = acc[j][q] + (bias ? bias[co] : 0.f);
            if (relu) r = fmaxf(r, 0.f);
            y[(size_t)co * V + ((size_t)gz * H + gy) * W + gx] = r;
        }
    }
}

// Weight gradient partial sums over one voxel chunk:
// part[chunk][co][ci][t] = sum_{v in chunk} g[co][v] x[ci][v + t - r].
// Block: one input channel ci and WCO output channels; threads over voxels.
constexpr int WCO = 4;
template <int K>
__global__ void __launch_bounds__(256)
k_conv_wgrad(const float* __restrict__ x, int Ci, int D, int H, int W, const float* __restrict__ g,
             int Co, int nchunk, float* __restrict__ part) {
    constexpr int R = K / 2, K3 = K * K * K;
    const int ci = blockIdx.x;
    const int co0 = blockIdx.y * WCO;
    const int chunk = blockIdx.z;
    const size_t V = (size_t)D * H * W;
    const size_t per = (V + nchunk - 1) / nchunk;
    const size_t v0 = (size_t)chunk * per, v1 = min(V, v0 + per);
    float acc[WCO][K3];
#pragma unroll
    for (int o = 0; o < WCO; ++o)
#pragma unroll
        for (int tp = 0; tp < K3; ++tp) acc[o][tp] = 0.f;
    const float* xc = x + (size_t)ci * V;
    for (size_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        const int gx = (int)(v % W), gy = (int)((v / W) % H), gz = (int)(v / ((size_t)W * H));
        float gv[WCO];
#pragma unroll
        for (int o = 0; o < WCO; ++o) gv[o] = (co0 + o < Co) ? g[(size_t)(co0 + o) * V + v] : 0.f;
#pragma unroll
        for (int kz = 0; kz < K; ++kz)
#pragma unroll
            for (int ky = 0; ky < K; ++ky)
#pragma unroll
                for (int kx = 0; kx < K; ++kx) {
                    const int sx = gx + kx - R, sy = gy + ky - R, sz = gz + kz - R;
                    float xv = 0.f;
                    if (sx >= 0 && sx < W && sy >= 0 && sy < H && sz >= 0 && sz < D)
                        xv = __ldg(xc + ((size_t)sz * H + sy) * W + sx);
                    const int tp = (kz * K + ky) * K + kx;
#pragma unroll
                    for (int o = 0; o < WCO; ++o) acc[o][tp] = fmaf(gv[o], xv, acc[o][tp]);
                }
    }
    // block reduction, one (o, tap) at a time through shared memory
    __shared__ float red[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 0; o < WCO; ++o)
#pragma unroll
        for (int tp = 0; tp < K3; ++tp) {
            float s = acc[o][tp];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
            __syncthreads();
            if (lane == 0) red[wid] = s;
            __syncthreads();
            if (threadIdx.x == 0 && co0 + o < Co) {
                float tot = 0.f;
                for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += red[q];
                part[(((size_t)chunk * Co + co0 + o) * Ci + ci) * K3 + tp] = tot;
            }
        }
}

// dw[i] = sum over chunks of part[chunk][i]  (fixed order)
__global__ void k_sum_chunks(const float* __restrict__ part, int nchunk, size_t n, float* __restrict__ out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * n + i];
        out[i] = s;
    }
}

// db[co] = sum_v g[co][v]   (one block per channel)
__global__ void __launch_bounds__(256) k_bias_grad(const float* __restrict__ g, size_t V, float* __restrict__ db) {
    const int co = blockIdx.x;
    float s = 0.f;
    for (size_t v = threadIdx.x; v < V; v += blockDim.x) s += g[(size_t)co * V + v];
    __shared__ float red[8];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += red[q];
        db[co] = tot;
    }
}

// g *= (a > 0)   (ReLU backward from the post-activation tensor)
__global__ void k_relu_mask(float* __restrict__ g, const float* __restrict__ a, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!(a[i] > 0.f)) g[i] = 0.f;
}

// 2x2x2 average pooling: y (C, D/2, H/2, W/2) from x (C, D, H, W)
__global__ void k_pool(const float* __restrict__ x, int C, int D, int H, int W, float* __restrict__ y) {
    const int d = D / 2, h = H / 2, w = W / 2;
    const size_t n = (size_t)C * d * h * w;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int ox = (int)(i % w), oy = (int)((i / w) % h), oz = (int)((i / ((size_t)w * h)) % d);
        const int c = (int)(i / ((size_t)w * h * d));
        const float* xc = x + (size_t)c * D * H * W;
        float s = 0.f;
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx)
                    s += xc[((size_t)(2 * oz + dz) * H + 2 * oy + dy) * W + 2 * ox + dx];
        y[i] = 0.125f * s;
    }
}

// nearest x2 upsampling: y (C, 2d, 2h, 2w) from x (C, d, h, w)
__global__ void k_up(const float* __restrict__ x, int C, int d, int h, int w, float* __restrict__ y) {
    const int D = 2 * d, H = 2 * h, W = 2 * w;
    const size_t n = (size_t)C * D * H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int X = (int)(i % W), Y = (int)((i / W) % H), Z = (int)((i / ((size_t)W * H)) % D);
        const int c = (int)(i / ((size_t)W * H * D));
        y[i] = x[(((size_t)c * d + Z / 2) * h + Y / 2) * w + X / 2];
    }
}

// upsampling backward: gx (C, d, h, w) = sum of the 8 children of gy (C, 2d, 2h, 2w)
__global__ void k_up_bwd(const float* __restrict__ gy, int C, int d, int h, int w, float* __restrict__ gx) {
    const int H = 2 * h, W = 2 * w, D = 2 * d;
    const size_t n = (size_t)C * d * h * w;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int ox = (int)(i % w), oy = (int)((i / w) % h), oz = (int)((i / ((size_t)w * h)) % d);
        const int c = (int)(i / ((size_t)w * h * d));
        const float* g = gy + (size_t)c * D * H * W;
        float s = 0.f;
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx)
                    s += g[((size_t)(2 * oz + dz) * H + 2 * oy + dy) * W + 2 * ox + dx];
        gx[i] = s;
    }
}

// encoder gradient at a skip: g = pool_bwd(gp) + gs, masked by (a > 0)
__global__ void k_pool_bwd_add_mask(const float* __restrict__ gp, const float* __restrict__ gs,
                                    const float* __restrict__ a, int C, int D, int H, int W,
                                    float* __restrict__ g) {
    const size_t n = (size_t)C * D * H * W;
    const int d = D / 2, h = H / 2, w = W / 2;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int X = (int)(i % W), Y = (int)((i / W) % H), Z = (int)((i / ((size_t)W * H)) % D);
        const int c = (int)(i / ((size_t)W * H * D));
        const float v = 0.125f * gp[(((size_t)c * d + Z / 2) * h + Y / 2) * w + X / 2] + gs[i];
        g[i] = a[i] > 0.f ? v : 0.f;
    }
}

// BF16 working copies of one layer's weights w[co][ci][t]:
// wf[ci][t][co] = w[co][ci][t];  wb[co][t][ci] = w[co][ci][K3 - 1 - t]
__global__ void k_make_bf16(const float* __restrict__ w, int Co, int Ci, int K3, __nv_bfloat16* __restrict__ wf,
                            __nv_bfloat16* __restrict__ wb) {
    const size_t n = (size_t)Co * Ci * K3;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int tp = (int)(i % K3), ci = (int)((i / K3) % Ci), co = (int)(i / ((size_t)K3 * Ci));
        const __nv_bfloat16 b = __float2bfloat16_rn(w[i]);
        wf[((size_t)ci * K3 + tp) * Co + co] = b;
        wb[((size_t)co * K3 + (K3 - 1 - tp)) * Ci + ci] = b;
    }
}

// Adam (Kingma and Ba 2015), bias-corrected, in place on FP32 master values
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// mean squared error: dy = 2 (y - t) / n, partial sums of (y - t)^2 per block
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ y, const float* __restrict__ tg, size_t n,
                                             float* __restrict__ dy, double* __restrict__ part) {
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = y[i] - tg[i];
        dy[i] = 2.f * d / (float)n;
        s += (double)d * d;
    }
    __shared__ double red[8];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += red[q];
        part[blockIdx.x] = tot;
    }
}

static int grid1(size_t n) { return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 8)); }

// ------------------------------------------------------------------ the network
struct Net {
    float* w[NLAYER] = {};     // master weights [co][ci][k^3]
    float* b[NLAYER] = {};
    float* gw[NLAYER] = {};
    float* gb[NLAYER] = {};
    float* mw[NLAYER] = {};
    float* vw[NLAYER] = {};
    float* mb[NLAYER] = {};
    float* vb[NLAYER] = {};
    __nv_bfloat16* wf[NLAYER] = {};
    __nv_bfloat16* wb[NLAYER] = {};
    int64_t nparam = 0;
    int adam_t = 0;
    // activations and gradients for the current grid (level-0 dims D, H, W)
    int D = 0, H = 0, W = 0;
    std::vector<void*> bufs;
    float *in0 = nullptr, *a_e1a = nullptr, *cat1 = nullptr, *a_d1a = nullptr, *a_d1b = nullptr, *out = nullptr;
    float *p1 = nullptr, *a_e2a = nullptr, *cat2 = nullptr, *a_d2a = nullptr, *a_d2b = nullptr;
    float *p2 = nullptr, *a_e3a = nullptr, *cat3 = nullptr, *a_d3a = nullptr, *a_d3b = nullptr;
    float *p3 = nullptr, *a_ba = nullptr, *a_bb = nullptr;
    float *g0 = nullptr, *g0b = nullptr, *gcat0 = nullptr;   // level-0 gradient scratch
    float *g1 = nullptr, *g1b = nullptr, *gcat1 = nullptr;
    float *g2 = nullptr, *g2b = nullptr, *gcat2 = nullptr;
    float *g3 = nullptr, *g3b = nullptr;
    float* part = nullptr;     // weight-gradient chunk partials
    size_t part_elems = 0;
    double* lpart = nullptr;   // loss partials
    float* target = nullptr;   // training target (6 x V)
    float* dy = nullptr;       // loss gradient (6 x V)
    std::string err;
    std::vector<void*> pallocs;

    ~Net() {
        free_bufs();
        for (void* p : pallocs) cudaFree(p);
    }
    void free_bufs() {
        for (void* p : bufs) cudaFree(p);
        bufs.clear();
        D = H = W = 0;
    }
    float* fa(size_t n) {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(n, 4) * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            throw Error(VSIE_ENOMEM, "network buffer allocation");
        }
        bufs.push_back(p);
        return (float*)p;
    }
    template <typename T> T* pa(size_t n) {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            throw Error(VSIE_ENOMEM, "network parameter allocation");
        }
        pallocs.push_back(p);
        VSIE_CUDA(cudaMemset(p, 0, std::max<size_t>(n, 1) * sizeof(T)));
        return (T*)p;
    }
    static size_t wsize(int l) {
        const LayerDef& L = kLayers[l];
        return (size_t)L.co * L.ci * L.k * L.k * L.k;
    }
    void alloc_params() {
        nparam = 0;
        for (int l = 0; l < NLAYER; ++l) {
            const size_t nw = wsize(l), nb = kLayers[l].co;
            w[l] = pa<float>(nw); b[l] = pa<float>(nb);
            gw[l] = pa<float>(nw); gb[l] = pa<float>(nb);
            mw[l] = pa<float>(nw); vw[l] = pa<float>(nw);
            mb[l] = pa<float>(nb); vb[l] = pa<float>(nb);
            wf[l] = pa<__nv_bfloat16>(nw); wb[l] = pa<__nv_bfloat16>(nw);
            nparam += (int64_t)(nw + nb);
        }
        lpart = pa<double>(152 * 8);
    }
    void refresh_bf16(cudaStream_t st) {
        for (int l = 0; l < NLAYER; ++l) {
            const LayerDef& L = kLayers[l];
            const size_t n = wsize(l);
            k_make_bf16<<<grid1(n), 256, 0, st>>>(w[l], L.co, L.ci, L.k * L.k * L.k, wf[l], wb[l]);
        }
        VSIE_CUDA(cudaGetLastError());
    }
    void ensure(int d, int h, int ww) {
        if (d % 8 || h % 8 || ww % 8 || d <= 0 || h <= 0 || ww <= 0)
            throw Error(VSIE_EINVAL, "network grid dimensions must be positive multiples of 8");
        if (d == D && h == H && ww == W) return;
        free_bufs();
        const size_t V0 = (size_t)d * h * ww, V1 = V0 / 8, V2 = V1 / 8, V3 = V2 / 8;
        in0 = fa(8 * V0); a_e1a = fa(16 * V0); cat1 = fa(48 * V0); a_d1a = fa(16 * V0); a_d1b = fa(16 * V0);
        out = fa(6 * V0);
        p1 = fa(16 * V1); a_e2a = fa(32 * V1); cat2 = fa(96 * V1); a_d2a = fa(32 * V1); a_d2b = fa(32 * V1);
        p2 = fa(32 * V2); a_e3a = fa(64 * V2); cat3 = fa(128 * V2); a_d3a = fa(64 * V2); a_d3b = fa(64 * V2);
        p3 = fa(64 * V3); a_ba = fa(64 * V3); a_bb = fa(64 * V3);
        g0 = fa(48 * V0); g0b = fa(48 * V0); gcat0 = fa(48 * V0);
        g1 = fa(96 * V1); g1b = fa(96 * V1); gcat1 = fa(96 * V1);
        g2 = fa(128 * V2); g2b = fa(128 * V2); gcat2 = fa(128 * V2);
        g3 = fa(64 * V3); g3b = fa(64 * V3);
        target = fa(6 * V0); dy = fa(6 * V0);
        part_elems = 0;
        for (int l = 0; l < NLAYER; ++l) part_elems = std::max(part_elems, wsize(l));
        part_elems *= kChunks;
        part = fa(part_elems);
        D = d; H = h; W = ww;
    }
    static constexpr int kChunks = 32;

    static void conv3_mma(const float* x, int ci, int d, int h, int ww, const __nv_bfloat16* w,
                          const float* bias, int co, bool relu, float* y, cudaStream_t st) {
        dim3 g(((ww + TX - 1) / TX) * ((h + TY - 1) / TY), (d + TZ - 1) / TZ, (co + 15) / 16);
        k_conv3_mma<<<g, 128, kConvMmaSmem, st>>>(x, ci, d, h, ww, w, bias, co, relu ? 1 : 0, y);
    }
    void conv(int l, const float* x, int d, int h, int ww, float* y, bool relu, cudaStream_t st) {
        const LayerDef& L = kLayers[l];
        if (L.k == 3) {
            conv3_mma(x, L.ci, d, h, ww, wf[l], b[l], L.co, relu, y, st);
            return;
        }
        dim3 g(((ww + TX - 1) / TX) * ((h + TY - 1) / TY), (d + TZ - 1) / TZ, (L.co + COT - 1) / COT);
        k_conv<1><<<g, 256, 0, st>>>(x, L.ci, d, h, ww, wf[l], b[l], L.co, relu ? 1 : 0, y);
    }
    // gradient wrt the layer input: a convolution with the flipped, transposed weights
    void conv_dx(int l, const float* gz, int d, int h, int ww, float* gx, cudaStream_t st) {
        const LayerDef& L = kLayers[l];
        if (L.k == 3) {
            conv3_mma(gz, L.co, d, h, ww, wb[l], nullptr, L.ci, false, gx, st);
            return;
        }
        dim3 g(((ww + TX - 1) / TX) * ((h + TY - 1) / TY), (d + TZ - 1) / TZ, (L.ci + COT - 1) / COT);
        k_conv<1><<<g, 256, 0, st>>>(gz, L.co, d, h, ww, wb[l], nullptr, L.ci, 0, gx);
    }
    void conv_dw(int l, const float* x, const float* gz, int d, int h, int ww, cudaStream_t st) {
        const LayerDef& L = kLayers[l];
        const size_t V = (size_t)d * h * ww;
        const int nch = (int)std::max<size_t>(1, std::min<size_t>(kChunks, V / 256));
        dim3 g(L.ci, (L.co + WCO - 1) / WCO, nch);
        if (L.k == 3)
            k_conv_wgrad<3><<<g, 256, 0, st>>>(x, L.ci, d, h, ww, gz, L.co, nch, part);
        else
            k_conv_wgrad<1><<<g, 256, 0, st>>>(x, L.ci, d, h, ww, gz, L.co, nch, part);
        k_sum_chunks<<<grid1(wsize(l)), 256, 0, st>>>(part, nch, wsize(l), gw[l]);
        k_bias_grad<<<L.co, 256, 0, st>>>(gz, V, gb[l]);
    }

    // forward on in0 (8 x V0) into out (6 x V0)
    void forward(cudaStream_t st) {
        const int d0 = D, h0 = H, w0 = W;
        const int d1 = d0 / 2, h1 = h0 / 2, w1 = w0 / 2, d2 = d1 / 2, h2 = h1 / 2, w2 = w1 / 2;
        const int d3 = d2 / 2, h3 = h2 / 2, w3 = w2 / 2;
        const size_t V0 = (size_t)d0 * h0 * w0, V1 = V0 / 8, V2 = V1 / 8;
        float* s1 = cat1 + 32 * V0;
        float* s2 = cat2 + 64 * V1;
        float* s3 = cat3 + 64 * V2;
        conv(E1A, in0, d0, h0, w0, a_e1a, true, st);
        conv(E1B, a_e1a, d0, h0, w0, s1, true, st);
        k_pool<<<grid1(16 * V1), 256, 0, st>>>(s1, 16, d0, h0, w0, p1);
        conv(E2A, p1, d1, h1, w1, a_e2a, true, st);
        conv(E2B, a_e2a, d1, h1, w1, s2, true, st);
        k_pool<<<grid1(32 * V2), 256, 0, st>>>(s2, 32, d1, h1, w1, p2);
        conv(E3A, p2, d2, h2, w2, a_e3a, true, st);
        conv(E3B, a_e3a, d2, h2, w2, s3, true, st);
        k_pool<<<grid1(64 * (V2 / 8)), 256, 0, st>>>(s3, 64, d2, h2, w2, p3);
        conv(BA, p3, d3, h3, w3, a_ba, true, st);
        conv(BB, a_ba, d3, h3, w3, a_bb, true, st);
        k_up<<<grid1(64 * V2), 256, 0, st>>>(a_bb, 64, d3, h3, w3, cat3);
        conv(D3A, cat3, d2, h2, w2, a_d3a, true, st);
        conv(D3B, a_d3a, d2, h2, w2, a_d3b, true, st);
        k_up<<<grid1(64 * V1), 256, 0, st>>>(a_d3b, 64, d2, h2, w2, cat2);
        conv(D2A, cat2, d1, h1, w1, a_d2a, true, st);
        conv(D2B, a_d2a, d1, h1, w1, a_d2b, true, st);
        k_up<<<grid1(32 * V0), 256, 0, st>>>(a_d2b, 32, d1, h1, w1, cat1);
        conv(D1A, cat1, d0, h0, w0, a_d1a, true, st);
        conv(D1B, a_d1a, d0, h0, w0, a_d1b, true, st);
        conv(HEAD, a_d1b, d0, h0, w0, out, false, st);
        VSIE_CUDA(cudaGetLastError());
    }

    // backward from dy (6 x V0, the gradient of the loss with respect to out);
    // fills gw, gb and, when gin != nullptr, the input gradient (8 x V0)
    void backward(const float* dyp, float* gin, cudaStream_t st) {
        const int d0 = D, h0 = H, w0 = W;
        const int d1 = d0 / 2, h1 = h0 / 2, w1 = w0 / 2, d2 = d1 / 2, h2 = h1 / 2, w2 = w1 / 2;
        const int d3 = d2 / 2, h3 = h2 / 2, w3 = w2 / 2;
        const size_t V0 = (size_t)d0 * h0 * w0, V1 = V0 / 8, V2 = V1 / 8, V3 = V2 / 8;
        float* s1 = cat1 + 32 * V0;
        float* s2 = cat2 + 64 * V1;
        float* s3 = cat3 + 64 * V2;
        // head (linear)
        conv_dw(HEAD, a_d1b, dyp, d0, h0, w0, st);
        conv_dx(HEAD, dyp, d0, h0, w0, g0, st);                        // g(a_d1b), 16 ch
        // d1b
        k_relu_mask<<<grid1(16 * V0), 256, 0, st>>>(g0, a_d1b, 16 * V0);
        conv_dw(D1B, a_d1a, g0, d0, h0, w0, st);
        conv_dx(D1B, g0, d0, h0, w0, g0b, st);                         // g(a_d1a)
        k_relu_mask<<<grid1(16 * V0), 256, 0, st>>>(g0b, a_d1a, 16 * V0);
        conv_dw(D1A, cat1, g0b, d0, h0, w0, st);
        conv_dx(D1A, g0b, d0, h0, w0, gcat0, st);                      // g(cat1), 48 ch
        k_up_bwd<<<grid1(32 * V1), 256, 0, st>>>(gcat0, 32, d1, h1, w1, g1);   // g(a_d2b)
        // d2b, d2a
        k_relu_mask<<<grid1(32 * V1), 256, 0, st>>>(g1, a_d2b, 32 * V1);
        conv_dw(D2B, a_d2a, g1, d1, h1, w1, st);
        conv_dx(D2B, g1, d1, h1, w1, g1b, st);
        k_relu_mask<<<grid1(32 * V1), 256, 0, st>>>(g1b, a_d2a, 32 * V1);
        conv_dw(D2A, cat2, g1b, d1, h1, w1, st);
        conv_dx(D2A, g1b, d1, h1, w1, gcat1, st);                      // g(cat2), 96 ch
        k_up_bwd<<<grid1(64 * V2), 256, 0, st>>>(gcat1, 64, d2, h2, w2, g2);   // g(a_d3b)
        // d3b, d3a
        k_relu_mask<<<grid1(64 * V2), 256, 0, st>>>(g2, a_d3b, 64 * V2);
        conv_dw(D3B, a_d3a, g2, d2, h2, w2, st);
        conv_dx(D3B, g2, d2, h2, w2, g2b, st);
        k_relu_mask<<<grid1(64 * V2), 256, 0, st>>>(g2b, a_d3a, 64 * V2);
        conv_dw(D3A, cat3, g2b, d2, h2, w2, st);
        conv_dx(D3A, g2b, d2, h2, w2, gcat2, st);                      // g(cat3), 128 ch
        k_up_bwd<<<grid1(64 * V3), 256, 0, st>>>(gcat2, 64, d3, h3, w3, g3);   // g(a_bb)
        // bottleneck
        k_relu_mask<<<grid1(64 * V3), 256, 0, st>>>(g3, a_bb, 64 * V3);
        conv_dw(BB, a_ba, g3, d3, h3, w3, st);
        conv_dx(BB, g3, d3, h3, w3, g3b, st);
        k_relu_mask<<<grid1(64 * V3), 256, 0, st>>>(g3b, a_ba, 64 * V3);
        conv_dw(BA, p3, g3b, d3, h3, w3, st);
        conv_dx(BA, g3b, d3, h3, w3, g3, st);                          // g(p3)
        // e3b: pool backward + skip gradient, masked
        k_pool_bwd_add_mask<<<grid1(64 * V2), 256, 0, st>>>(g3, gcat2 + 64 * V2, s3, 64, d2, h2, w2, g2);
        conv_dw(E3B, a_e3a, g2, d2, h2, w2, st);
        conv_dx(E3B, g2, d2, h2, w2, g2b, st);
        k_relu_mask<<<grid1(64 * V2), 256, 0, st>>>(g2b, a_e3a, 64 * V2);
        conv_dw(E3A, p2, g2b, d2, h2, w2, st);
        conv_dx(E3A, g2b, d2, h2, w2, g2, st);                         // g(p2), 32 ch
        k_pool_bwd_add_mask<<<grid1(32 * V1), 256, 0, st>>>(g2, gcat1 + 64 * V1, s2, 32, d1, h1, w1, g1);
        conv_dw(E2B, a_e2a, g1, d1, h1, w1, st);
        conv_dx(E2B, g1, d1, h1, w1, g1b, st);
        k_relu_mask<<<grid1(32 * V1), 256, 0, st>>>(g1b, a_e2a, 32 * V1);
        conv_dw(E2A, p1, g1b, d1, h1, w1, st);
        conv_dx(E2A, g1b, d1, h1, w1, g1, st);                         // g(p1), 16 ch
        k_pool_bwd_add_mask<<<grid1(16 * V0), 256, 0, st>>>(g1, gcat0 + 32 * V0, s1, 16, d0, h0, w0, g0);
        conv_dw(E1B, a_e1a, g0, d0, h0, w0, st);
        conv_dx(E1B, g0, d0, h0, w0, g0b, st);
        k_relu_mask<<<grid1(16 * V0), 256, 0, st>>>(g0b, a_e1a, 16 * V0);
        conv_dw(E1A, in0, g0b, d0, h0, w0, st);
        if (gin) conv_dx(E1A, g0b, d0, h0, w0, gin, st);
        VSIE_CUDA(cudaGetLastError());
    }

    void adam(float lr, cudaStream_t st) {
        ++adam_t;
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float c1 = 1.f - std::pow(b1, (float)adam_t), c2 = 1.f - std::pow(b2, (float)adam_t);
        for (int l = 0; l < NLAYER; ++l) {
            k_adam<<<grid1(wsize(l)), 256, 0, st>>>(w[l], gw[l], mw[l], vw[l], wsize(l), lr, b1, b2, eps, c1, c2);
            k_adam<<<1, 256, 0, st>>>(b[l], gb[l], mb[l], vb[l], kLayers[l].co, lr, b1, b2, eps, c1, c2);
        }
        refresh_bf16(st);
    }

    // loss = mean((out - target)^2); dy = its gradient; returns the loss (syncs)
    double mse(cudaStream_t st) {
        const size_t n = 6 * (size_t)D * H * W;
        const int g = grid1(n);
        k_mse<<<g, 256, 0, st>>>(out, target, n, dy, lpart);
        VSIE_CUDA(cudaGetLastError());
        std::vector<double> hp(g);
        VSIE_CUDA(cudaMemcpyAsync(hp.data(), lpart, g * sizeof(double), cudaMemcpyDeviceToHost, st));
        VSIE_CUDA(cudaStreamSynchronize(st));
        double s = 0;
        for (double v : hp) s += v;
        return s / (double)n;
    }
};

Net* net_of(vsie_net* n) { return reinterpret_cast<Net*>(n); }

// hooks for the solver and trainer (krylov.cu, nettrain.cu)
void net_forward_input(Net& n, cudaStream_t st) { n.forward(st); }
float* net_input(Net& n) { return n.in0; }
float* net_output(Net& n) { return n.out; }
float* net_target(Net& n) { return n.target; }
void net_ensure(Net& n, int d, int h, int w) { n.ensure(d, h, w); }
double net_train_on_target(Net& n, float lr, cudaStream_t st) {
    n.forward(st);
    const double L = n.mse(st);
    n.backward(n.dy, nullptr, st);
    n.adam(lr, st);
    return L;
}

}  // namespace vsie

using namespace vsie;

extern "C" {

vsie_status vsie_net_create(uint64_t seed, vsie_net** out) {
    if (!out) { set_global_err("null output pointer"); return VSIE_EINVAL; }
    *out = nullptr;
    Net* n = nullptr;
    try {
        n = new Net();
        n->alloc_params();
        VSIE_CUDA(cudaFuncSetAttribute(k_conv3_mma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kConvMmaSmem));
        // He-normal initial weights, zero biases
        std::mt19937_64 rng(seed);
        std::normal_distribution<float> nd(0.f, 1.f);
        for (int l = 0; l < NLAYER; ++l) {
            const LayerDef& L = kLayers[l];
            const size_t nw = Net::wsize(l);
            const float sd = std::sqrt(2.f / (float)(L.ci * L.k * L.k * L.k));
            std::vector<float> hw(nw);
            for (auto& v : hw) v = sd * nd(rng);
            VSIE_CUDA(cudaMemcpy(n->w[l], hw.data(), nw * sizeof(float), cudaMemcpyHostToDevice));
        }
        n->refresh_bf16(0);
        VSIE_CUDA(cudaDeviceSynchronize());
    } catch (const Error& e) {
        delete n;
        set_global_err(e.msg);
        return e.st;
    }
    *out = reinterpret_cast<vsie_net*>(n);
    return VSIE_OK;
}

vsie_status vsie_net_num_params(const vsie_net* net, int64_t* n) {
    if (!net || !n) { set_global_err("null argument"); return VSIE_EINVAL; }
    *n = reinterpret_cast<const Net*>(net)->nparam;
    return VSIE_OK;
}

static vsie_status params_io(vsie_net* net, float* host, int64_t n, bool set) {
    if (!net || !host) { set_global_err("null argument"); return VSIE_EINVAL; }
    Net* nt = net_of(net);
    if (n != nt->nparam) { nt->err = "parameter count mismatch"; return VSIE_EINVAL; }
    try {
        int64_t off = 0;
        for (int l = 0; l < NLAYER; ++l) {
            const size_t nw = Net::wsize(l), nb = kLayers[l].co;
            if (set) {
                VSIE_CUDA(cudaMemcpy(nt->w[l], host + off, nw * sizeof(float), cudaMemcpyHostToDevice));
                VSIE_CUDA(cudaMemcpy(nt->b[l], host + off + nw, nb * sizeof(float), cudaMemcpyHostToDevice));
            } else {
                VSIE_CUDA(cudaMemcpy(host + off, nt->w[l], nw * sizeof(float), cudaMemcpyDeviceToHost));
                VSIE_CUDA(cudaMemcpy(host + off + nw, nt->b[l], nb * sizeof(float), cudaMemcpyDeviceToHost));
            }
            off += (int64_t)(nw + nb);
        }
        if (set) {
            nt->refresh_bf16(0);
            VSIE_CUDA(cudaDeviceSynchronize());
        }
    } catch (const Error& e) {
        nt->err = e.msg;
        return e.st;
    }
    return VSIE_OK;
}

vsie_status vsie_net_set_params(vsie_net* net, const float* host, int64_t n) {
    return params_io(net, const_cast<float*>(host), n, true);
}

vsie_status vsie_net_get_params(vsie_net* net, float* host, int64_t n) {
    return params_io(net, host, n, false);
}

vsie_status vsie_net_forward(vsie_net* net, int32_t D, int32_t H, int32_t W, const float* x, float* y,
                             vsie_stream stream) {
    if (!net || !x || !y) { set_global_err("null argument"); return VSIE_EINVAL; }
    Net* nt = net_of(net);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    try {
        nt->ensure(D, H, W);
        const size_t V = (size_t)D * H * W;
        VSIE_CUDA(cudaMemcpyAsync(nt->in0, x, 8 * V * sizeof(float), cudaMemcpyDeviceToDevice, st));
        nt->forward(st);
        VSIE_CUDA(cudaMemcpyAsync(y, nt->out, 6 * V * sizeof(float), cudaMemcpyDeviceToDevice, st));
    } catch (const Error& e) {
        nt->err = e.msg;
        return e.st;
    }
    return VSIE_OK;
}

vsie_status vsie_net_backward(vsie_net* net, int32_t D, int32_t H, int32_t W, const float* x,
                              const float* dy, float* grad_host, float* dx, vsie_stream stream) {
    if (!net || !x || !dy) { set_global_err("null argument"); return VSIE_EINVAL; }
    Net* nt = net_of(net);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    try {
        nt->ensure(D, H, W);
        const size_t V = (size_t)D * H * W;
        VSIE_CUDA(cudaMemcpyAsync(nt->in0, x, 8 * V * sizeof(float), cudaMemcpyDeviceToDevice, st));
        nt->forward(st);
        VSIE_CUDA(cudaMemcpyAsync(nt->dy, dy, 6 * V * sizeof(float), cudaMemcpyDeviceToDevice, st));
        nt->backward(nt->dy, dx, st);
        VSIE_CUDA(cudaStreamSynchronize(st));
        if (grad_host) {
            int64_t off = 0;
            for (int l = 0; l < NLAYER; ++l) {
                const size_t nw = Net::wsize(l), nb = kLayers[l].co;
                VSIE_CUDA(cudaMemcpy(grad_host + off, nt->gw[l], nw * sizeof(float), cudaMemcpyDeviceToHost));
                VSIE_CUDA(cudaMemcpy(grad_host + off + nw, nt->gb[l], nb * sizeof(float), cudaMemcpyDeviceToHost));
                off += (int64_t)(nw + nb);
            }
        }
    } catch (const Error& e) {
        nt->err = e.msg;
        return e.st;
    }
    return VSIE_OK;
}

vsie_status vsie_net_step(vsie_net* net, int32_t D, int32_t H, int32_t W, const float* x,
                          const float* target, double lr, double* loss, vsie_stream stream) {
    if (!net || !x || !target) { set_global_err("null argument"); return VSIE_EINVAL; }
    Net* nt = net_of(net);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    try {
        nt->ensure(D, H, W);
        const size_t V = (size_t)D * H * W;
        VSIE_CUDA(cudaMemcpyAsync(nt->in0, x, 8 * V * sizeof(float), cudaMemcpyDeviceToDevice, st));
        VSIE_CUDA(cudaMemcpyAsync(nt->target, target, 6 * V * sizeof(float), cudaMemcpyDeviceToDevice, st));
        const double L = net_train_on_target(*nt, (float)lr, st);
        if (loss) *loss = L;
        VSIE_CUDA(cudaStreamSynchronize(st));
    } catch (const Error& e) {
        nt->err = e.msg;
        return e.st;
    }
    return VSIE_OK;
}

const char* vsie_net_last_error(const vsie_net* net) {
    return net ? reinterpret_cast<const Net*>(net)->err.c_str() : "null network";
}

void vsie_net_destroy(vsie_net* net) { delete net_of(net); }

}  // extern "C"
