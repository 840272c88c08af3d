// K1: fused FFT convolution of the volume operator on the extended grid
// (Sec. II.B: block-Toeplitz Z_bb applied by FFT; Sec. III: the pFFT grid).
//
// c_a = h^3 sum_b T_ab * g_b with g = E_b M x_b + P x_n on the extended grid
// n = (n1, n2, n3), computed with the circulant embedding of length
// L = (L1, L2, L3) (L_i >= 2 n_i - 1) in five passes over HBM:
//   X-fwd  : g lines along i1 (body values + coil contributions), FFT L1   -> A
//   Y-fwd  : tiles of k1 columns, FFT L2                                   -> B
//   Z      : tiles of k1 pencils at fixed k2, all three components: FFT L3,
//            multiply by the symmetric 3x3 kernel spectrum (octant storage with
//            parity signs), inverse FFT L3, keep the first n3 outputs      -> B
//   Y-inv  : inverse FFT L2, keep the first n2 rows                        -> A
//   X-inv  : inverse FFT L1, epilogue: y_b = M (h^3 x_b / chi - c) + (1 - M) x_b
//            on body lines, and c on coil-active voxels (for P^T c)
// A holds [p][3][n3][n2][L1] and B [p][3][n3][L2][L1]; every pass streams its
// input once and its output once.  Shared memory holds [k][line] tiles.
#include "fft.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>

namespace vsie {

template <typename R>
struct ConvArgs {
    int n1, n2, n3, L1, L2, L3, Lh1, Lh2, Lh3;
    int b1, b2, b3, o1, o2, o3;
    uint32_t L1magic, n2magic;
    int64_t nb, nact;
    const cx<R>* X;
    int64_t ldx, xoff;
    cx<R>* Y;
    int64_t ldy;
    const uint8_t* mask;
    const cx<R>* dinv;
    const int32_t* line_ptr;
    const int32_t* line_i1;
    const int32_t* line_cidx;
    const int32_t* line_flag;
    const cx<R>* gc;
    cx<R>* cc;
    cx<R>* A;
    cx<R>* B;
    const cx<R>* spec;
    const cx<R>* tw1;
    const cx<R>* tw2;
    const cx<R>* tw3;
    FFTPlan pl1, pl2, pl3;
    FFTPlan pl3h;   // length L3 / 2, twiddle steps indexing the L3 table (L3 even)
    int zhalf;      // 1: the Z pass runs on half-length transforms
};

// line flags (per (i2, i3) line of the extended grid): 1 crosses the body grid,
// 2 holds coil grid points, 4 holds a material voxel.  A line without 2 or 4 has a
// zero x-forward transform: the x-forward passes do not store it, the y-forward
// passes read it as zero, and the y-inverse passes do not store it (the x-inverse
// epilogue uses the transform of a line only through bits 2 and 4).
constexpr int kLineLive = 6;

// x / d given magic = magic_div(d); magic 0 encodes d == 1
__device__ __forceinline__ int udiv(int x, uint32_t magic) {
    return magic ? (int)__umulhi((uint32_t)x, magic) : x;
}

template <typename C>
__device__ __forceinline__ void load_tw(C* s, const C* g, int L) {
    for (int i = threadIdx.x; i < L; i += blockDim.x) s[i] = g[i];
}

}  // namespace vsie
#include "conv_reg.cuh"
namespace vsie {

// --------------------------------------------------------------- X forward
template <typename R, int NL>
__global__ void __launch_bounds__(1024) k_xfwd(ConvArgs<R> a) {
    using C = cx<R>;
    constexpr int KS = NL + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + a.L1;
    C* scr = buf + (size_t)a.L1 * KS;
    __shared__ int64_t lbase[NL];   // body voxel index of (q1 = 0) on this line, or -1
    const int comp = blockIdx.y, j = blockIdx.z;
    const int nlines = a.n2 * a.n3;
    const int lin0 = blockIdx.x * NL;
    if (threadIdx.x < NL) {
        const int lin = lin0 + threadIdx.x;
        int64_t b = -1;
        if (lin < nlines) {
            const int i3 = udiv(lin, a.n2magic), i2 = lin - i3 * a.n2;
            const int q2 = i2 - a.o2, q3 = i3 - a.o3;
            if (q2 >= 0 && q2 < a.b2 && q3 >= 0 && q3 < a.b3)
                b = (int64_t)a.b1 * (q2 + (int64_t)a.b2 * q3);
        }
        lbase[threadIdx.x] = b;
    }
    load_tw(tw, a.tw1, a.L1);
    __syncthreads();
    const C* xb = a.X + (size_t)j * a.ldx + a.xoff + (size_t)comp * a.nb;
    constexpr int U = 8;   // independent loads in flight per thread
    const int tot = NL * a.L1;
    for (int e0 = threadIdx.x; e0 < tot; e0 += U * blockDim.x) {
        C v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x;
            v[u] = czero<C>();
            if (e < tot) {
                const int l = udiv(e, a.L1magic), i1 = e - l * a.L1;
                const int q1 = i1 - a.o1;
                const int64_t lb = lbase[l];
                if (lb >= 0 && q1 >= 0 && q1 < a.b1) {
                    const int64_t vb = lb + q1;
                    if (a.mask[vb]) v[u] = xb[vb];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < tot) {
                const int l = udiv(e, a.L1magic), i1 = e - l * a.L1;
                buf[i1 * KS + l] = v[u];
            }
        }
    }
    __syncthreads();
    if (a.nact > 0) {
        const C* g = a.gc + ((size_t)j * 3 + comp) * a.nact;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int l = warp; l < NL; l += blockDim.x >> 5) {
            const int lin = lin0 + l;
            if (lin >= nlines) continue;
            for (int e = a.line_ptr[lin] + lane; e < a.line_ptr[lin + 1]; e += 32) {
                C& t = buf[a.line_i1[e] * KS + l];
                t = cadd(t, g[a.line_cidx[e]]);
            }
        }
        __syncthreads();
    }
    const C* res = fft_pp<false, NL, KS>(buf, scr, a.pl1, tw);
    C* out = a.A + (((size_t)j * 3 + comp) * nlines + lin0) * a.L1;
    const int nvalid = min(NL, nlines - lin0) * a.L1;
    for (int e = threadIdx.x; e < nvalid; e += blockDim.x) {
        const int l = udiv(e, a.L1magic), k = e - l * a.L1;
        if (a.line_flag[lin0 + l] & kLineLive) out[e] = res[k * KS + l];   // zero lines are not stored
    }
}

// --------------------------------------------------------------- Y forward / inverse
template <typename R, int NL, bool INV>
__global__ void __launch_bounds__(1024) k_ypass(ConvArgs<R> a) {
    using C = cx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + a.L2;
    C* scr = buf + (size_t)a.L2 * NL;
    const int k10 = blockIdx.x * NL, i3 = blockIdx.y, ja = blockIdx.z;
    load_tw(tw, a.tw2, a.L2);
    const int nin = INV ? a.L2 : a.n2;     // rows read
    const int nout = INV ? a.n2 : a.L2;    // rows written
    const C* in = INV ? a.B + ((size_t)ja * a.n3 + i3) * a.L2 * a.L1
                      : a.A + ((size_t)ja * a.n3 + i3) * a.n2 * a.L1;
    // rows i2 whose x line is zero: not read (forward), not written (inverse)
    int* rowf = reinterpret_cast<int*>(scr + (size_t)a.L2 * NL);
    for (int i = threadIdx.x; i < a.n2; i += blockDim.x) rowf[i] = a.line_flag[i + a.n2 * i3] & kLineLive;
    __syncthreads();
    constexpr int U = 8;
    const int tot = NL * a.L2;
    for (int e0 = threadIdx.x; e0 < tot; e0 += U * blockDim.x) {
        C v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x;
            const int l = e % NL, row = e / NL;
            const int k1 = k10 + l;
            v[u] = czero<C>();
            if (e < tot && row < nin && k1 < a.L1 && (INV || rowf[row])) v[u] = in[(size_t)row * a.L1 + k1];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < tot) buf[e] = v[u];
        }
    }
    __syncthreads();
    const C* res = fft_pp<INV, NL, NL>(buf, scr, a.pl2, tw);
    C* out = INV ? a.A + ((size_t)ja * a.n3 + i3) * a.n2 * a.L1
                 : a.B + ((size_t)ja * a.n3 + i3) * a.L2 * a.L1;
    for (int e = threadIdx.x; e < NL * nout; e += blockDim.x) {
        const int l = e % NL, row = e / NL;
        const int k1 = k10 + l;
        if (k1 < a.L1 && (!INV || rowf[row])) out[(size_t)row * a.L1 + k1] = res[e];
    }
}

// --------------------------------------------------------------- Z fused
template <typename R, int NL>
__global__ void __launch_bounds__(1024) k_zmul(ConvArgs<R> a) {
    using C = cx<R>;
    constexpr int NLT = 3 * NL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + a.L3;
    C* scr = buf + (size_t)a.L3 * NLT;
    const int k10 = blockIdx.x * NL, j = blockIdx.z;
    // visit k2 and its mirror L2 - k2 back to back (they share spectrum octants)
    const int y = blockIdx.y;
    const int k2 = y == 0 ? 0 : ((y & 1) ? (y + 1) >> 1 : a.L2 - (y >> 1));
    load_tw(tw, a.tw3, a.L3);
    const size_t plane = (size_t)a.L2 * a.L1;
    const C* in = a.B + (size_t)j * 3 * a.n3 * plane + (size_t)k2 * a.L1;
    const size_t cstride = (size_t)a.n3 * plane;
    constexpr int U = 8;
    const int tot = NLT * a.L3;
    for (int e0 = threadIdx.x; e0 < tot; e0 += U * blockDim.x) {
        C v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x;
            const int ln = e % NLT, k3 = e / NLT;
            const int comp = ln / NL, l = ln - comp * NL;
            const int k1 = k10 + l;
            v[u] = czero<C>();
            if (e < tot && k3 < a.n3 && k1 < a.L1) v[u] = in[comp * cstride + (size_t)k3 * plane + k1];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < tot) buf[e] = v[u];
        }
    }
    __syncthreads();
    {
        C* r = fft_pp<false, NLT, NLT>(buf, scr, a.pl3, tw);
        if (r != buf) { scr = buf; buf = r; }
    }
    {
        const size_t oct = (size_t)a.Lh1 * a.Lh2 * a.Lh3;
        const int kk2 = k2 <= a.L2 / 2 ? k2 : a.L2 - k2;
        const R sg2 = k2 <= a.L2 / 2 ? (R)1 : (R)-1;
        for (int e = threadIdx.x; e < NL * a.L3; e += blockDim.x) {
            const int l = e % NL, k3 = e / NL;
            const int k1 = k10 + l;
            if (k1 >= a.L1) continue;
            const int kk1 = k1 <= a.L1 / 2 ? k1 : a.L1 - k1;
            const R sg1 = k1 <= a.L1 / 2 ? (R)1 : (R)-1;
            const int kk3 = k3 <= a.L3 / 2 ? k3 : a.L3 - k3;
            const R sg3 = k3 <= a.L3 / 2 ? (R)1 : (R)-1;
            const size_t o = kk1 + (size_t)a.Lh1 * (kk2 + (size_t)a.Lh2 * kk3);
            const C txx = a.spec[o], tyy = a.spec[oct + o], tzz = a.spec[2 * oct + o];
            const C txy = cscale(a.spec[3 * oct + o], sg1 * sg2);
            const C txz = cscale(a.spec[4 * oct + o], sg1 * sg3);
            const C tyz = cscale(a.spec[5 * oct + o], sg2 * sg3);
            C* px = buf + (size_t)k3 * NLT + l;
            const C x = px[0], yv = px[NL], z = px[2 * NL];
            C ox = cmul(txx, x), oy = cmul(txy, x), oz = cmul(txz, x);
            cfma(ox, txy, yv); cfma(ox, txz, z);
            cfma(oy, tyy, yv); cfma(oy, tyz, z);
            cfma(oz, tyz, yv); cfma(oz, tzz, z);
            px[0] = ox; px[NL] = oy; px[2 * NL] = oz;
        }
    }
    __syncthreads();
    const C* res = fft_pp<true, NLT, NLT>(buf, scr, a.pl3, tw);
    C* out = a.B + (size_t)j * 3 * a.n3 * plane + (size_t)k2 * a.L1;
    for (int e = threadIdx.x; e < NLT * a.n3; e += blockDim.x) {
        const int ln = e % NLT, k3 = e / NLT;
        const int comp = ln / NL, l = ln - comp * NL;
        const int k1 = k10 + l;
        if (k1 < a.L1) out[comp * cstride + (size_t)k3 * plane + k1] = res[e];
    }
}

// --------------------------------------------------------------- Z fused, half length
// For even L3 = 2M (then n3 <= M): with w = exp(-2 pi i / L3) and x zero beyond
// n3, the length-L3 transform splits into X[2k] = FFT_M(x)[k] and
// X[2k+1] = FFT_M(x w^n)[k], and the unnormalised inverse on n < n3 is
// IFFT_M(X_even)[n] + w^-n IFFT_M(X_odd)[n].  The zero half of every line is
// never stored or transformed, and the transforms are half as long.
// Shared memory: the L3 twiddles, then 2 x 3 NL lines of length M (even-part
// lines first) and their ping-pong scratch.
template <typename R, int NL>
__global__ void __launch_bounds__(1024) k_zmul_h(ConvArgs<R> a) {
    using C = cx<R>;
    constexpr int NLT = 3 * NL, NL2 = 2 * NLT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    const int M = a.L3 / 2;
    C* buf = tw + a.L3;
    C* scr = buf + (size_t)M * NL2;
    const int k10 = blockIdx.x * NL, j = blockIdx.z;
    // visit k2 and its mirror L2 - k2 back to back (they share spectrum octants)
    const int y = blockIdx.y;
    const int k2 = y == 0 ? 0 : ((y & 1) ? (y + 1) >> 1 : a.L2 - (y >> 1));
    load_tw(tw, a.tw3, a.L3);
    __syncthreads();
    const size_t plane = (size_t)a.L2 * a.L1;
    const C* in = a.B + (size_t)j * 3 * a.n3 * plane + (size_t)k2 * a.L1;
    const size_t cstride = (size_t)a.n3 * plane;
    constexpr int U = 8;
    const int tot = NLT * M;
    for (int e0 = threadIdx.x; e0 < tot; e0 += U * blockDim.x) {
        C v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x;
            const int ln = e % NLT, k3 = e / NLT;
            const int comp = ln / NL, l = ln - comp * NL;
            const int k1 = k10 + l;
            v[u] = czero<C>();
            if (e < tot && k3 < a.n3 && k1 < a.L1) v[u] = in[comp * cstride + (size_t)k3 * plane + k1];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < tot) {
                const int ln = e % NLT, k3 = e / NLT;
                buf[k3 * NL2 + ln] = v[u];
                buf[k3 * NL2 + NLT + ln] = cmul(v[u], tw[k3]);
            }
        }
    }
    __syncthreads();
    {
        C* r = fft_pp<false, NL2, NL2>(buf, scr, a.pl3h, tw);
        if (r != buf) { scr = buf; buf = r; }
    }
    {
        const size_t oct = (size_t)a.Lh1 * a.Lh2 * a.Lh3;
        const int kk2 = k2 <= a.L2 / 2 ? k2 : a.L2 - k2;
        const R sg2 = k2 <= a.L2 / 2 ? (R)1 : (R)-1;
        for (int e = threadIdx.x; e < NL * a.L3; e += blockDim.x) {
            const int l = e % NL, k3 = e / NL;
            const int k1 = k10 + l;
            if (k1 >= a.L1) continue;
            const int kk1 = k1 <= a.L1 / 2 ? k1 : a.L1 - k1;
            const R sg1 = k1 <= a.L1 / 2 ? (R)1 : (R)-1;
            const int kk3 = k3 <= a.L3 / 2 ? k3 : a.L3 - k3;
            const R sg3 = k3 <= a.L3 / 2 ? (R)1 : (R)-1;
            const size_t o = kk1 + (size_t)a.Lh1 * (kk2 + (size_t)a.Lh2 * kk3);
            const C txx = a.spec[o], tyy = a.spec[oct + o], tzz = a.spec[2 * oct + o];
            const C txy = cscale(a.spec[3 * oct + o], sg1 * sg2);
            const C txz = cscale(a.spec[4 * oct + o], sg1 * sg3);
            const C tyz = cscale(a.spec[5 * oct + o], sg2 * sg3);
            C* px = buf + (size_t)(k3 >> 1) * NL2 + (k3 & 1) * NLT + l;
            const C x = px[0], yv = px[NL], z = px[2 * NL];
            C ox = cmul(txx, x), oy = cmul(txy, x), oz = cmul(txz, x);
            cfma(ox, txy, yv); cfma(ox, txz, z);
            cfma(oy, tyy, yv); cfma(oy, tyz, z);
            cfma(oz, tyz, yv); cfma(oz, tzz, z);
            px[0] = ox; px[NL] = oy; px[2 * NL] = oz;
        }
    }
    __syncthreads();
    const C* res = fft_pp<true, NL2, NL2>(buf, scr, a.pl3h, tw);
    C* out = a.B + (size_t)j * 3 * a.n3 * plane + (size_t)k2 * a.L1;
    for (int e = threadIdx.x; e < NLT * a.n3; e += blockDim.x) {
        const int ln = e % NLT, k3 = e / NLT;
        const int comp = ln / NL, l = ln - comp * NL;
        const int k1 = k10 + l;
        if (k1 < a.L1)
            out[comp * cstride + (size_t)k3 * plane + k1] =
                cadd(res[k3 * NL2 + ln], cmulc(res[k3 * NL2 + NLT + ln], tw[k3]));
    }
}

// --------------------------------------------------------------- X inverse + epilogue
template <typename R, int NL>
__global__ void __launch_bounds__(1024) k_xinv(ConvArgs<R> a) {
    using C = cx<R>;
    constexpr int KS = NL + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + a.L1;
    C* scr = buf + (size_t)a.L1 * KS;
    __shared__ int any;
    __shared__ int64_t lbase[NL];
    __shared__ int lflag[NL];
    const int comp = blockIdx.y, j = blockIdx.z;
    const int nlines = a.n2 * a.n3;
    const int lin0 = blockIdx.x * NL;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    if (threadIdx.x < NL) {
        const int lin = lin0 + threadIdx.x;
        int f = 0;
        int64_t b = -1;
        if (lin < nlines) {
            f = a.line_flag[lin];
            const int i3 = udiv(lin, a.n2magic), i2 = lin - i3 * a.n2;
            if (f & 1) b = (int64_t)a.b1 * ((i2 - a.o2) + (int64_t)a.b2 * (i3 - a.o3));
        }
        lflag[threadIdx.x] = f;
        lbase[threadIdx.x] = b;
        if (f) atomicOr(&any, 1);
    }
    __syncthreads();
    if (!any) return;
    load_tw(tw, a.tw1, a.L1);
    const C* in = a.A + (((size_t)j * 3 + comp) * nlines + lin0) * a.L1;
    const int nvalid = min(NL, nlines - lin0) * a.L1;
    constexpr int U = 8;
    const int tot = NL * a.L1;
    for (int e0 = threadIdx.x; e0 < tot; e0 += U * blockDim.x) {
        C v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x;
            v[u] = czero<C>();
            if (e < nvalid && (lflag[udiv(e, a.L1magic)] & kLineLive)) v[u] = in[e];   // zero lines were not stored
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < tot) {
                const int l = udiv(e, a.L1magic), k = e - l * a.L1;
                buf[k * KS + l] = v[u];
            }
        }
    }
    __syncthreads();
    const C* res = fft_pp<true, NL, KS>(buf, scr, a.pl1, tw);
    const C* xb = a.X + (size_t)j * a.ldx + a.xoff + (size_t)comp * a.nb;
    C* yb = a.Y + (size_t)j * a.ldy + a.xoff + (size_t)comp * a.nb;
    const uint32_t b1magic = magic_div((uint32_t)a.b1);
    for (int e = threadIdx.x; e < NL * a.b1; e += blockDim.x) {
        const int l = udiv(e, b1magic), q1 = e - l * a.b1;
        if (!(lflag[l] & 1)) continue;
        const int64_t vb = lbase[l] + q1;
        const C x = xb[vb];
        C yv;
        if (a.mask[vb]) yv = csub(cmul(a.dinv[vb], x), res[(q1 + a.o1) * KS + l]);
        else yv = x;
        yb[vb] = yv;
    }
    if (a.nact > 0) {
        C* cco = a.cc + ((size_t)j * 3 + comp) * a.nact;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int l = warp; l < NL; l += blockDim.x >> 5) {
            const int lin = lin0 + l;
            if (!(lflag[l] & 2)) continue;
            for (int e = a.line_ptr[lin] + lane; e < a.line_ptr[lin + 1]; e += 32)
                cco[a.line_cidx[e]] = res[a.line_i1[e] * KS + l];
        }
    }
}

// --------------------------------------------------------------- launcher
// Each pass has a small set of (lines per CTA, threads per CTA) variants; the
// autotuner (conv_autotune) times them on the context's own buffers and keeps
// the fastest per pass.
struct Variant { int nl, threads; };
// (thread counts that match a stage's butterfly count, e.g. 16 per line for
// radix 16 on 256 points and 16 per half-line for radix 7 on 112 points, keep
// every thread busy in that stage)
static const Variant kXV[] = {{8, 128}, {8, 256}, {16, 256}, {16, 512}, {32, 512}, {32, 1024}};
static const Variant kZV[] = {{4, 256}, {4, 384}, {4, 512}, {8, 512}, {8, 768}, {8, 1024}, {16, 1024}};
constexpr int kNX = sizeof(kXV) / sizeof(kXV[0]);
constexpr int kNZ = sizeof(kZV) / sizeof(kZV[0]);
// Register-resident FP32 kernels (conv_reg.cuh) for the lengths they are built
// for, appended after the generic variants of each pass: x and y passes take NL
// lines per CTA (16 NL threads), the z pass NL = 4, 8, 16 lines (M = 112) or
// NL = 2, 4, 8 (M = 224) per CTA with 32 NL threads.
static const int kXR[] = {8, 16, 32};
constexpr int kNR = 3;
// z pass: k_zreg with NL from reg_zNL (variants 0-2), k_zreg_st with NL = 8 (3),
// NL = 16 (4, M = 112 only) and NL = 8 with the thread-pair middle phase (5,
// M = 224 only)
constexpr int kNRZ = 6;

template <typename R>
static ConvArgs<R> make_args(Ctx& c, const cx<R>* X, int64_t ldx, cx<R>* Y, int64_t ldy) {
    OpData<R>& d = data<R>(c);
    ConvArgs<R> a;
    a.n1 = c.ne[0]; a.n2 = c.ne[1]; a.n3 = c.ne[2];
    a.L1 = c.L[0]; a.L2 = c.L[1]; a.L3 = c.L[2];
    a.Lh1 = c.Lh[0]; a.Lh2 = c.Lh[1]; a.Lh3 = c.Lh[2];
    a.b1 = c.nb[0]; a.b2 = c.nb[1]; a.b3 = c.nb[2];
    a.o1 = c.off[0]; a.o2 = c.off[1]; a.o3 = c.off[2];
    a.L1magic = magic_div(a.L1);
    a.n2magic = magic_div(a.n2);
    a.nb = c.n_b; a.nact = c.nact;
    a.X = X; a.ldx = ldx; a.xoff = (int64_t)c.m_f + c.m_n;
    a.Y = Y; a.ldy = ldy;
    a.mask = c.mask; a.dinv = d.dinv;
    a.line_ptr = c.line_ptr; a.line_i1 = c.line_i1; a.line_cidx = c.line_cidx;
    a.line_flag = c.body_lines;
    a.gc = d.gc; a.cc = d.cc; a.A = d.bufA; a.B = d.bufB;
    a.spec = d.spec; a.tw1 = d.tw[0]; a.tw2 = d.tw[1]; a.tw3 = d.tw[2];
    const FFTPlan* pl = sizeof(R) == 4 ? c.plan16 : c.plan;
    a.pl1 = pl[0]; a.pl2 = pl[1]; a.pl3 = pl[2];
    a.pl3h = sizeof(R) == 4 ? c.plan3h16 : c.plan3h;
    a.zhalf = sizeof(R) == 4 && c.L[2] % 2 == 0 && a.pl3h.L == c.L[2] / 2 ? 1 : 0;
    return a;
}

template <typename R, int NL>
static void launch_x(const ConvArgs<R>& a, int p, int t, bool inv, cudaStream_t st) {
    const size_t sm = (size_t)a.L1 * (2 * NL + 3) * sizeof(cx<R>);
    dim3 g((a.n2 * a.n3 + NL - 1) / NL, 3, p);
    if (inv) k_xinv<R, NL><<<g, t, sm, st>>>(a);
    else k_xfwd<R, NL><<<g, t, sm, st>>>(a);
}
template <typename R, int NL>
static void launch_y(const ConvArgs<R>& a, int p, int t, bool inv, cudaStream_t st) {
    const size_t sm = (size_t)a.L2 * (2 * NL + 1) * sizeof(cx<R>) + (size_t)a.n2 * sizeof(int);
    dim3 g((a.L1 + NL - 1) / NL, a.n3, 3 * p);
    if (inv) k_ypass<R, NL, true><<<g, t, sm, st>>>(a);
    else k_ypass<R, NL, false><<<g, t, sm, st>>>(a);
}
template <typename R, int NL>
static void launch_z(const ConvArgs<R>& a, int p, int t, cudaStream_t st) {
    const size_t sm = (size_t)a.L3 * (6 * NL + 1) * sizeof(cx<R>);
    dim3 g((a.L1 + NL - 1) / NL, a.L2, p);
    if constexpr (sizeof(R) == 4) {   // FP32 only: the FP64 variant would spill
        if (a.zhalf) {
            k_zmul_h<R, NL><<<g, t, sm, st>>>(a);
            return;
        }
    }
    k_zmul<R, NL><<<g, t, sm, st>>>(a);
}

// ---- register variants (FP32): applicability, shared memory, launch
static bool reg_len_ok(int L) { return L == 256 || L == 512; }
static int reg_zR2(const ConvArgs<float>& a) {
    if (!a.zhalf) return 0;
    return a.L3 == 224 ? 7 : a.L3 == 448 ? 14 : 0;
}
static int reg_zNL(int R2, int rv) { return (R2 == 7 ? 4 : 2) << rv; }
static size_t reg_smem(const ConvArgs<float>& a, int pass, int rv) {
    const size_t cs = sizeof(float2);
    if (pass == 0 || pass == 4) {
        if (!reg_len_ok(a.L1)) return 0;
        const size_t L = a.L1, NL = kXR[rv], R1 = L / 16;
        return (L + NL * (L / 2 + 1) + NL * 16 * (R1 + 1)) * cs;
    }
    if (pass == 1 || pass == 3) {
        if (!reg_len_ok(a.L2)) return 0;
        return ((size_t)a.L2 + (size_t)kXR[rv] * a.L2) * cs + (size_t)a.n2 * sizeof(int);
    }
    const int R2 = reg_zR2(a);
    if (!R2) return 0;
    const size_t M = 16 * R2;
    if (rv >= 3) {   // staged kernel: twiddles, exchange, spectrum tile, staging lines
        const size_t NL = rv == 4 ? 16 : 8;
        if (a.L1 % NL != 0 || (rv == 4 && R2 != 7) || (rv == 5 && R2 != 14)) return 0;
        return (2 * M + 6 * M * NL + 6 * (size_t)a.Lh3 * NL + 3 * (size_t)a.n3 * NL) * cs;
    }
    const size_t NL = reg_zNL(R2, rv);
    return (2 * M + 6 * M * NL) * cs;
}

template <int R1, int NL>
static void launch_xreg(const ConvArgs<float>& a, int p, bool inv, cudaStream_t st) {
    const size_t sm = reg_smem(a, inv ? 4 : 0, NL == 8 ? 0 : NL == 16 ? 1 : 2);
    dim3 g((a.n2 * a.n3 + NL - 1) / NL, 3, p);
    if (inv) k_xinv_reg<R1, 16, NL><<<g, 16 * NL, sm, st>>>(a);
    else k_xfwd_reg<R1, 16, NL><<<g, 16 * NL, sm, st>>>(a);
}
template <int R1, int NL>
static void launch_yreg(const ConvArgs<float>& a, int p, bool inv, cudaStream_t st) {
    const size_t sm = ((size_t)a.L2 + (size_t)NL * a.L2) * sizeof(float2) + (size_t)a.n2 * sizeof(int);
    dim3 g((a.L1 + NL - 1) / NL, a.n3, 3 * p);
    if (inv) k_yreg<R1, 16, NL, true, false><<<g, 16 * NL, sm, st>>>(a);
    else k_yreg<R1, 16, NL, false, true><<<g, 16 * NL, sm, st>>>(a);
}
template <int R2, int NL>
static void launch_zreg(const ConvArgs<float>& a, int p, cudaStream_t st) {
    const size_t sm = (size_t)(2 * 16 * R2 + 6 * 16 * R2 * NL) * sizeof(float2);
    dim3 g((a.L1 + NL - 1) / NL, a.L2, p);
    k_zreg<R2, NL><<<g, 32 * NL, sm, st>>>(a);
}
template <int R2, int NL, bool SPLIT = false>
static void launch_zreg_st(const ConvArgs<float>& a, int p, cudaStream_t st) {
    const size_t sm = reg_smem(a, 2, SPLIT ? 5 : NL == 8 ? 3 : 4);
    dim3 g(a.L1 / NL, a.L2, 1);
    k_zreg_st<R2, NL, SPLIT><<<g, ZStaged<R2, NL, SPLIT>::NT, sm, st>>>(a, p);
}
template <int NL>
static void launch_xyreg(const ConvArgs<float>& a, int p, int pass, cudaStream_t st) {
    if (pass == 0 || pass == 4) {
        if (a.L1 == 256) launch_xreg<16, NL>(a, p, pass == 4, st);
        else launch_xreg<32, NL>(a, p, pass == 4, st);
    } else {
        if (a.L2 == 256) launch_yreg<16, NL>(a, p, pass == 3, st);
        else launch_yreg<32, NL>(a, p, pass == 3, st);
    }
}
static void run_reg_pass(const ConvArgs<float>& a, int p, int pass, int rv, cudaStream_t st) {
    if (pass == 2) {
        const int R2 = reg_zR2(a);
        if (rv == 3) {
            if (R2 == 7) launch_zreg_st<7, 8>(a, p, st);
            else launch_zreg_st<14, 8>(a, p, st);
            return;
        }
        if (rv == 4) {
            launch_zreg_st<7, 16>(a, p, st);
            return;
        }
        if (rv == 5) {
            launch_zreg_st<14, 8, true>(a, p, st);
            return;
        }
        if (R2 == 7) {
            if (rv == 0) launch_zreg<7, 4>(a, p, st);
            else if (rv == 1) launch_zreg<7, 8>(a, p, st);
            else launch_zreg<7, 16>(a, p, st);
        } else {
            if (rv == 0) launch_zreg<14, 2>(a, p, st);
            else if (rv == 1) launch_zreg<14, 4>(a, p, st);
            else launch_zreg<14, 8>(a, p, st);
        }
        return;
    }
    switch (kXR[rv]) {
        case 8: launch_xyreg<8>(a, p, pass, st); break;
        case 16: launch_xyreg<16>(a, p, pass, st); break;
        default: launch_xyreg<32>(a, p, pass, st); break;
    }
}

template <typename R>
static size_t smem_of(const ConvArgs<R>& a, int pass, int nl) {
    const size_t cs = sizeof(cx<R>);
    if (pass == 0 || pass == 4) return (size_t)a.L1 * (2 * nl + 3) * cs;
    if (pass == 1 || pass == 3) return (size_t)a.L2 * (2 * nl + 1) * cs + (size_t)a.n2 * sizeof(int);
    return (size_t)a.L3 * (6 * nl + 1) * cs;
}

// pass: 0 X-fwd, 1 Y-fwd, 2 Z, 3 Y-inv, 4 X-inv
template <typename R>
static void run_pass(const ConvArgs<R>& a, int p, int pass, int var, cudaStream_t st) {
    const int ng = pass == 2 ? kNZ : kNX;
    if (var >= ng) {
        if constexpr (sizeof(R) == 4) run_reg_pass(a, p, pass, var - ng, st);
        return;
    }
    if (pass == 2) {
        const Variant v = kZV[var];
        switch (v.nl) {
            case 4: launch_z<R, 4>(a, p, v.threads, st); break;
            case 8: launch_z<R, 8>(a, p, v.threads, st); break;
            default: launch_z<R, 16>(a, p, v.threads, st); break;
        }
        return;
    }
    const Variant v = kXV[var];
    const bool inv = pass > 2;
    if (pass == 0 || pass == 4) {
        switch (v.nl) {
            case 8: launch_x<R, 8>(a, p, v.threads, inv, st); break;
            case 16: launch_x<R, 16>(a, p, v.threads, inv, st); break;
            default: launch_x<R, 32>(a, p, v.threads, inv, st); break;
        }
    } else {
        switch (v.nl) {
            case 8: launch_y<R, 8>(a, p, v.threads, inv, st); break;
            case 16: launch_y<R, 16>(a, p, v.threads, inv, st); break;
            default: launch_y<R, 32>(a, p, v.threads, inv, st); break;
        }
    }
}

template <typename R>
void conv_apply(Ctx& c, int p, const cx<R>* X, int64_t ldx, cx<R>* Y, int64_t ldy,
                cudaStream_t st) {
    ConvArgs<R> a = make_args<R>(c, X, ldx, Y, ldy);
    OpData<R>& d = data<R>(c);
    const int ch = d.chunk;
    const int groups = (p + ch - 1) / ch;
    // algorithmic bytes of the launch groups: the three-pass schedule moves
    // 54 n_v complex values per RHS, plus the 6 spectrum octants once per group
    const double cs = sizeof(cx<R>);
    const double alg = 54.0 * (double)c.n_e * cs * p +
                       6.0 * groups * (double)c.Lh[0] * c.Lh[1] * c.Lh[2] * cs;
    ProfScope ps(c, sizeof(R) == 4 ? PG_FFTCONV : PG_FFTCONV64, st, alg);
    const int* tune = d.tune;
    for (int j0 = 0; j0 < p; j0 += ch) {
        const int pj = std::min(ch, p - j0);
        a.X = X + (size_t)j0 * ldx;
        a.Y = Y + (size_t)j0 * ldy;
        a.gc = d.gc + (size_t)j0 * 3 * c.nact;
        a.cc = d.cc + (size_t)j0 * 3 * c.nact;
        for (int pass = 0; pass < 5; ++pass) run_pass<R>(a, pj, pass, tune[pass], st);
        prof_count(c, 5);
    }
    VSIE_CUDA(cudaGetLastError());
}

// Time every variant of every pass (on the context's buffers; X = Y = a
// scratch vector) and keep the fastest.  Variants whose shared memory does not
// fit are skipped.  p = the context's max_rhs.
template <typename R>
void conv_autotune(Ctx& c) {
    OpData<R>& d = data<R>(c);
    int dev = 0, smax = 0;
    VSIE_CUDA(cudaGetDevice(&dev));
    VSIE_CUDA(cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int p = std::min(d.chunk, 4);
    cx<R>* xy = (cx<R>*)dalloc(c, (size_t)2 * c.N * p * sizeof(cx<R>));
    VSIE_CUDA(cudaMemset(xy, 0, (size_t)2 * c.N * p * sizeof(cx<R>)));
    const ConvArgs<R> a = make_args<R>(c, xy, c.N, xy + (size_t)c.N * p, c.N);
    cudaEvent_t e0, e1;
    VSIE_CUDA(cudaEventCreate(&e0));
    VSIE_CUDA(cudaEventCreate(&e1));
    std::string why = "no variant's shared memory fits";
    // VSIE_ZPASS_VARIANT=v restricts the FP32 z pass to variant v (tests and
    // tuning sweeps; a variant that does not apply leaves the pass without one)
    const char* zforce = sizeof(R) == 4 ? std::getenv("VSIE_ZPASS_VARIANT") : nullptr;
    const int zvar = zforce ? std::atoi(zforce) : -1;
    for (int pass = 0; pass < 5; ++pass) {
        const int ng = pass == 2 ? kNZ : kNX;
        const int nv = ng + (sizeof(R) == 4 ? (pass == 2 ? kNRZ : kNR) : 0);
        float best = 1e30f;
        int bi = -1;
        for (int v = 0; v < nv; ++v) {
            if (pass == 2 && zvar >= 0 && v != zvar) continue;
            if (v < ng) {
                const int nl = pass == 2 ? kZV[v].nl : kXV[v].nl;
                if (smem_of(a, pass, nl) > (size_t)smax) continue;
            } else {
                if constexpr (sizeof(R) == 4) {
                    const size_t sm = reg_smem(a, pass, v - ng);
                    if (sm == 0 || sm > (size_t)smax) continue;
                }
            }
            run_pass<R>(a, p, pass, v, 0);   // warm-up
            const cudaError_t le = cudaGetLastError();
            if (le != cudaSuccess) {
                why = std::string(cudaGetErrorString(le)) + " (variant " + std::to_string(v) + ")";
                continue;
            }
            VSIE_CUDA(cudaEventRecord(e0, 0));
            for (int it = 0; it < 3; ++it) run_pass<R>(a, p, pass, v, 0);
            VSIE_CUDA(cudaEventRecord(e1, 0));
            VSIE_CUDA(cudaEventSynchronize(e1));
            if (cudaGetLastError() != cudaSuccess) continue;
            float ms = 0;
            VSIE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            d.tune_ms[pass][v] = ms / 3;
            if (ms < best) { best = ms; bi = v; }
        }
        if (bi < 0) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            throw Error(VSIE_EUNSUPPORTED, "no FFT pass configuration fits this grid (pass " +
                                               std::to_string(pass) + ", precision " +
                                               std::to_string(sizeof(R) * 16) + " bits: " + why + ")");
        }
        d.tune[pass] = bi;
        if (std::getenv("VSIE_TRACE_TUNE")) {
            fprintf(stderr, "[vsie tune] FP%d pass %d L=(%d,%d,%d) p=%d chosen %d:", (int)sizeof(R) * 8, pass,
                    c.L[0], c.L[1], c.L[2], p, bi);
            for (int v = 0; v < nv; ++v) fprintf(stderr, " %.3f", d.tune_ms[pass][v]);
            fprintf(stderr, "\n");
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    auto& al = c.allocs;   // the scratch vectors are not kept with the context
    al.erase(std::remove(al.begin(), al.end(), (void*)xy), al.end());
    cudaFree(xy);
}

template <typename R>
void conv_set_attrs() {
    const int big = 220 * 1024;
#define VSIE_ATTR(k) VSIE_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, big))
    VSIE_ATTR((k_xfwd<R, 8>)); VSIE_ATTR((k_xfwd<R, 16>)); VSIE_ATTR((k_xfwd<R, 32>));
    VSIE_ATTR((k_xinv<R, 8>)); VSIE_ATTR((k_xinv<R, 16>)); VSIE_ATTR((k_xinv<R, 32>));
    VSIE_ATTR((k_ypass<R, 8, false>)); VSIE_ATTR((k_ypass<R, 16, false>)); VSIE_ATTR((k_ypass<R, 32, false>));
    VSIE_ATTR((k_ypass<R, 8, true>)); VSIE_ATTR((k_ypass<R, 16, true>)); VSIE_ATTR((k_ypass<R, 32, true>));
    VSIE_ATTR((k_zmul<R, 4>)); VSIE_ATTR((k_zmul<R, 8>)); VSIE_ATTR((k_zmul<R, 16>));
    VSIE_ATTR((k_zmul_h<R, 4>)); VSIE_ATTR((k_zmul_h<R, 8>)); VSIE_ATTR((k_zmul_h<R, 16>));
#define VSIE_CARVE(k) VSIE_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, \
                                                     (int)cudaSharedmemCarveoutMaxShared))
    if constexpr (sizeof(R) == 4) {
        // the register kernels fit several CTAs per SM only with the largest carveout
        VSIE_CARVE((k_zreg<7, 4>)); VSIE_CARVE((k_zreg<7, 8>)); VSIE_CARVE((k_zreg<7, 16>));
        VSIE_CARVE((k_zreg<14, 2>)); VSIE_CARVE((k_zreg<14, 4>)); VSIE_CARVE((k_zreg<14, 8>));
        VSIE_CARVE((k_yreg<16, 16, 16, false, true>)); VSIE_CARVE((k_yreg<16, 16, 16, true, false>));
        VSIE_CARVE((k_yreg<32, 16, 8, false, true>)); VSIE_CARVE((k_yreg<32, 16, 8, true, false>));
        VSIE_CARVE((k_xfwd_reg<16, 16, 8>)); VSIE_CARVE((k_xinv_reg<16, 16, 8>));
        VSIE_CARVE((k_xfwd_reg<32, 16, 8>)); VSIE_CARVE((k_xinv_reg<32, 16, 8>));
        VSIE_ATTR((k_xfwd_reg<16, 16, 8>)); VSIE_ATTR((k_xfwd_reg<16, 16, 16>)); VSIE_ATTR((k_xfwd_reg<16, 16, 32>));
        VSIE_ATTR((k_xfwd_reg<32, 16, 8>)); VSIE_ATTR((k_xfwd_reg<32, 16, 16>)); VSIE_ATTR((k_xfwd_reg<32, 16, 32>));
        VSIE_ATTR((k_xinv_reg<16, 16, 8>)); VSIE_ATTR((k_xinv_reg<16, 16, 16>)); VSIE_ATTR((k_xinv_reg<16, 16, 32>));
        VSIE_ATTR((k_xinv_reg<32, 16, 8>)); VSIE_ATTR((k_xinv_reg<32, 16, 16>)); VSIE_ATTR((k_xinv_reg<32, 16, 32>));
        VSIE_ATTR((k_yreg<16, 16, 8, false, true>)); VSIE_ATTR((k_yreg<16, 16, 16, false, true>));
        VSIE_ATTR((k_yreg<16, 16, 32, false, true>)); VSIE_ATTR((k_yreg<32, 16, 8, false, true>));
        VSIE_ATTR((k_yreg<32, 16, 16, false, true>)); VSIE_ATTR((k_yreg<32, 16, 32, false, true>));
        VSIE_ATTR((k_yreg<16, 16, 8, true, false>)); VSIE_ATTR((k_yreg<16, 16, 16, true, false>));
        VSIE_ATTR((k_yreg<16, 16, 32, true, false>)); VSIE_ATTR((k_yreg<32, 16, 8, true, false>));
        VSIE_ATTR((k_yreg<32, 16, 16, true, false>)); VSIE_ATTR((k_yreg<32, 16, 32, true, false>));
        VSIE_ATTR((k_zreg<7, 4>)); VSIE_ATTR((k_zreg<7, 8>)); VSIE_ATTR((k_zreg<7, 16>));
        VSIE_ATTR((k_zreg<14, 2>)); VSIE_ATTR((k_zreg<14, 4>)); VSIE_ATTR((k_zreg<14, 8>));
        VSIE_ATTR((k_zreg_st<7, 8, false>)); VSIE_ATTR((k_zreg_st<7, 16, false>));
        VSIE_ATTR((k_zreg_st<14, 8, false>)); VSIE_ATTR((k_zreg_st<14, 8, true>));
        VSIE_CARVE((k_zreg_st<7, 8, false>)); VSIE_CARVE((k_zreg_st<7, 16, false>));
        VSIE_CARVE((k_zreg_st<14, 8, false>)); VSIE_CARVE((k_zreg_st<14, 8, true>));
    }
#undef VSIE_ATTR
#undef VSIE_CARVE
}

template void conv_autotune<float>(Ctx&);
template void conv_autotune<double>(Ctx&);
// The five passes on body-only vectors (no near-coil contributions, body block
// at offset 0), with caller-provided work buffers A and B (used by the
// allocation-free entry point).
template <typename R>
void conv_apply_given_scratch(Ctx& c, int p, const cx<R>* Xb, int64_t ldx, cx<R>* Yb, int64_t ldy,
                              cx<R>* A, cx<R>* B, cudaStream_t st) {
    ConvArgs<R> a = make_args<R>(c, Xb, ldx, Yb, ldy);
    a.xoff = 0;
    a.nact = 0;
    a.A = A;
    a.B = B;
    const int* tune = data<R>(c).tune;
    for (int pass = 0; pass < 5; ++pass) run_pass<R>(a, p, pass, tune[pass], st);
    VSIE_CUDA(cudaGetLastError());
}
template void conv_apply_given_scratch<float>(Ctx&, int, const float2*, int64_t, float2*, int64_t,
                                              float2*, float2*, cudaStream_t);
template void conv_apply_given_scratch<double>(Ctx&, int, const double2*, int64_t, double2*,
                                               int64_t, double2*, double2*, cudaStream_t);

template void conv_apply<float>(Ctx&, int, const float2*, int64_t, float2*, int64_t, cudaStream_t);
template void conv_apply<double>(Ctx&, int, const double2*, int64_t, double2*, int64_t, cudaStream_t);
template void conv_set_attrs<float>();
template void conv_set_attrs<double>();

}  // namespace vsie
