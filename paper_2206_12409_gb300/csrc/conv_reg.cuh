// K1, FP32: register-resident passes of the FFT convolution for the transform
// lengths of the head grids (x, y: 256 = 16 x 16 and 512 = 32 x 16; z, half
// length M = L3 / 2: 112 = 16 x 7 and 224 = 16 x 14).  Included by conv.cu.
//
// A line of length L = R1 R2 is transformed in two register stages around one
// exchange through shared memory (decimation in time over n = t + R2 j):
//   stage A, thread t in [0, R2):  Y[t][k1] = w_L^(t k1) sum_j x[t + R2 j] w_R1^(j k1)
//   stage B, thread k1 in [0, R1): X[k1 + R1 k2] = sum_t Y[t][k1] w_R2^(t k2)
// Loads feed stage A straight from global memory and stage B stores straight to
// it, so each element crosses shared memory once per transform (the Stockham
// kernels of fft.cuh cross it once per stage plus once on each end).  Inputs
// known to be zero (the padded half of the x and y forward lines) are compile-
// time zeros, which removes their share of the first stage's arithmetic.
//
// The z pass runs the half-length scheme of k_zmul_h (even part x, odd part
// x w^n, two length-M transforms each way) with the spectrum multiply between
// the forward stage B and the inverse stage A on the same thread's registers:
//   forward A (radix 16) -> exchange -> forward B (radix R2) and multiply and
//   inverse A (radix R2) -> exchange -> inverse B (radix 16) and recombination
//   y[n] = y_even[n] + w^-n y_odd[n].
#pragma once

namespace vsie {

template <bool INV> __device__ __forceinline__ float2 twm(float2 a, float2 w) {
    return INV ? cmulc(a, w) : cmul(a, w);
}

// --------------------------------------------------------------- y pass
// CTA: NL consecutive k1 columns of one (i3, component, RHS) plane; threads
// R2 NL (stage A: one per (t, line); stage B loops over R1 NL butterflies).
// Shared memory: twiddles (L), exchange [t R1 + k1][line].
template <int R1, int R2, int NL, bool INV, bool HZ>
__global__ void __launch_bounds__(R2 * NL) k_yreg(ConvArgs<float> a) {
    using C = float2;
    constexpr int L = R1 * R2, NT = R2 * NL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* ex = tw + L;
    const int k10 = blockIdx.x * NL, i3 = blockIdx.y, ja = blockIdx.z;
    // rows i2 whose x line is zero: not read (forward), not written (inverse)
    int* rowf = reinterpret_cast<int*>(ex + (size_t)L * NL);
    for (int i = threadIdx.x; i < a.n2; i += NT) rowf[i] = a.line_flag[i + a.n2 * i3] & kLineLive;
    for (int i = threadIdx.x; i < L; i += NT) tw[i] = a.tw2[i];
    __syncthreads();
    const int nin = INV ? L : a.n2;
    const int nout = INV ? a.n2 : L;
    const size_t pl = (size_t)ja * a.n3 + i3;
    const C* in = INV ? a.B + pl * L * a.L1 : a.A + pl * a.n2 * a.L1;
    C* out = INV ? a.A + pl * a.n2 * a.L1 : a.B + pl * L * a.L1;
    {
        const int l = threadIdx.x % NL, t = threadIdx.x / NL;
        const int k1g = k10 + l;
        C v[R1];
#pragma unroll
        for (int j = 0; j < R1; ++j) {
            const int row = t + R2 * j;
            v[j] = make_float2(0.f, 0.f);
            if (!(HZ && j >= R1 / 2) && row < nin && k1g < a.L1 && (INV || rowf[row]))
                v[j] = in[(size_t)row * a.L1 + k1g];
        }
        __syncthreads();   // twiddles loaded
        dftR<INV>(v, int_<R1>());
#pragma unroll
        for (int k = 0; k < R1; ++k) ex[(t * R1 + k) * NL + l] = (k > 0 && t > 0) ? twm<INV>(v[k], tw[t * k]) : v[k];
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < R1 / R2; ++it) {
        const int w = threadIdx.x + it * NT;
        const int l = w % NL, k1 = w / NL;
        const int k1g = k10 + l;
        C v[R2];
#pragma unroll
        for (int t = 0; t < R2; ++t) v[t] = ex[(t * R1 + k1) * NL + l];
        dftR<INV>(v, int_<R2>());
        if (k1g < a.L1) {
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) {
                const int row = k1 + R1 * k2;
                if (row < nout && (!INV || rowf[row])) out[(size_t)row * a.L1 + k1g] = v[k2];
            }
        }
    }
}

// --------------------------------------------------------------- x forward
// CTA: NL lines (i2, i3) of one component and RHS; threads R2 NL.  The line is
// staged in shared memory first (body values under the mask, then the coil's
// projected values), because the coil contributions arrive as a sparse list.
// Shared memory: twiddles (L), staged lines [NL][L/2 + 1], exchange
// [NL][R2][R1 + 1] (padded: conflict-free in both stages).
template <int R1, int R2, int NL>
__global__ void __launch_bounds__(R2 * NL) k_xfwd_reg(ConvArgs<float> a) {
    using C = float2;
    constexpr int L = R1 * R2, LH = L / 2, NT = R2 * NL, XS = R2 * (R1 + 1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* sx = tw + L;
    C* ex = sx + NL * (LH + 1);
    __shared__ int64_t lbase[NL];
    __shared__ int llive[NL];
    const int comp = blockIdx.y, j = blockIdx.z;
    const int nlines = a.n2 * a.n3;
    const int lin0 = blockIdx.x * NL;
    int live = 0;
    if (threadIdx.x < NL) {
        const int lin = lin0 + threadIdx.x;
        int64_t b = -1;
        if (lin < nlines) {
            const int i3 = udiv(lin, a.n2magic), i2 = lin - i3 * a.n2;
            const int q2 = i2 - a.o2, q3 = i3 - a.o3;
            if (q2 >= 0 && q2 < a.b2 && q3 >= 0 && q3 < a.b3) b = (int64_t)a.b1 * (q2 + (int64_t)a.b2 * q3);
            live = a.line_flag[lin] & kLineLive;
        }
        lbase[threadIdx.x] = b;
        llive[threadIdx.x] = live;
    }
    for (int i = threadIdx.x; i < L; i += NT) tw[i] = a.tw1[i];
    if (!__syncthreads_or(live)) return;   // every line of this CTA is zero: nothing to store
    const C* xb = a.X + (size_t)j * a.ldx + a.xoff + (size_t)comp * a.nb;
    // the mask byte and the value are loaded independently (no load waits on
    // another); vacuum voxels are zeroed afterwards
#pragma unroll 4
    for (int e = threadIdx.x; e < NL * LH; e += NT) {
        const int l = e / LH, i1 = e - l * LH;
        const int q1 = i1 - a.o1;
        const int64_t lb = lbase[l];
        C v = make_float2(0.f, 0.f);
        if (lb >= 0 && q1 >= 0 && q1 < a.b1) {
            const C x = xb[lb + q1];
            v = a.mask[lb + q1] ? x : v;
        }
        sx[l * (LH + 1) + i1] = v;
    }
    __syncthreads();
    if (a.nact > 0) {
        const C* g = a.gc + ((size_t)j * 3 + comp) * a.nact;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int l = warp; l < NL; l += NT >> 5) {
            const int lin = lin0 + l;
            if (lin >= nlines) continue;
            for (int e = a.line_ptr[lin] + lane; e < a.line_ptr[lin + 1]; e += 32) {
                C& t = sx[l * (LH + 1) + a.line_i1[e]];
                t = cadd(t, g[a.line_cidx[e]]);
            }
        }
        __syncthreads();
    }
    {
        const int t = threadIdx.x % R2, l = threadIdx.x / R2;
        C v[R1];
#pragma unroll
        for (int jj = 0; jj < R1; ++jj) v[jj] = jj < R1 / 2 ? sx[l * (LH + 1) + t + R2 * jj] : make_float2(0.f, 0.f);
        dftR<false>(v, int_<R1>());
#pragma unroll
        for (int k = 0; k < R1; ++k) ex[l * XS + t * (R1 + 1) + k] = (k > 0 && t > 0) ? cmul(v[k], tw[t * k]) : v[k];
    }
    __syncthreads();
    C* out = a.A + (((size_t)j * 3 + comp) * nlines + lin0) * L;
#pragma unroll
    for (int it = 0; it < R1 / R2; ++it) {
        const int w = threadIdx.x + it * NT;
        const int k1 = w % R1, l = w / R1;
        C v[R2];
#pragma unroll
        for (int t = 0; t < R2; ++t) v[t] = ex[l * XS + t * (R1 + 1) + k1];
        dftR<false>(v, int_<R2>());
        if (lin0 + l < nlines && llive[l]) {
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) out[(size_t)l * L + k1 + R1 * k2] = v[k2];
        }
    }
}

// --------------------------------------------------------------- x inverse + epilogue
// Same CTA shape; stage A loads the spectrum line from global memory, stage B
// writes the first L/2 outputs to shared memory, from where the epilogue of
// k_xinv (diagonal, mask, vacuum identity, pFFT read-out) takes them.
template <int R1, int R2, int NL>
__global__ void __launch_bounds__(R2 * NL) k_xinv_reg(ConvArgs<float> a) {
    using C = float2;
    constexpr int L = R1 * R2, LH = L / 2, NT = R2 * NL, XS = R2 * (R1 + 1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* ex = tw + L;
    C* res = ex + NL * XS;
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
    for (int i = threadIdx.x; i < L; i += NT) tw[i] = a.tw1[i];
    const C* in = a.A + (((size_t)j * 3 + comp) * nlines + lin0) * L;
    {
        const int t = threadIdx.x % R2, l = threadIdx.x / R2;
        const bool ok = lin0 + l < nlines && (lflag[l] & kLineLive);   // zero lines were not stored
        C v[R1];
#pragma unroll
        for (int jj = 0; jj < R1; ++jj) v[jj] = ok ? in[(size_t)l * L + t + R2 * jj] : make_float2(0.f, 0.f);
        __syncthreads();   // twiddles loaded
        dftR<true>(v, int_<R1>());
#pragma unroll
        for (int k = 0; k < R1; ++k) ex[l * XS + t * (R1 + 1) + k] = (k > 0 && t > 0) ? cmulc(v[k], tw[t * k]) : v[k];
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < R1 / R2; ++it) {
        const int w = threadIdx.x + it * NT;
        const int k1 = w % R1, l = w / R1;
        C v[R2];
#pragma unroll
        for (int t = 0; t < R2; ++t) v[t] = ex[l * XS + t * (R1 + 1) + k1];
        dftR<true>(v, int_<R2>());
#pragma unroll
        for (int k2 = 0; k2 < R2 / 2; ++k2) res[l * (LH + 1) + k1 + R1 * k2] = v[k2];
    }
    __syncthreads();
    const C* xb = a.X + (size_t)j * a.ldx + a.xoff + (size_t)comp * a.nb;
    C* yb = a.Y + (size_t)j * a.ldy + a.xoff + (size_t)comp * a.nb;
    const uint32_t b1magic = magic_div((uint32_t)a.b1);
    for (int e = threadIdx.x; e < NL * a.b1; e += NT) {
        const int l = udiv(e, b1magic), q1 = e - l * a.b1;
        if (!(lflag[l] & 1)) continue;
        const int64_t vb = lbase[l] + q1;
        const C x = xb[vb];
        yb[vb] = a.mask[vb] ? csub(cmul(a.dinv[vb], x), res[l * (LH + 1) + q1 + a.o1]) : x;
    }
    if (a.nact > 0) {
        C* cco = a.cc + ((size_t)j * 3 + comp) * a.nact;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int l = warp; l < NL; l += NT >> 5) {
            const int lin = lin0 + l;
            if (!(lflag[l] & 2)) continue;
            for (int e = a.line_ptr[lin] + lane; e < a.line_ptr[lin + 1]; e += 32)
                cco[a.line_cidx[e]] = res[l * (LH + 1) + a.line_i1[e]];
        }
    }
}

// Exchange rows of 64 bytes (NL = 8 lines) fill half of the 32 banks.  Row m is
// stored at m ^ ((m >> 4) & 1) and spectrum-tile row r at r ^ ((r >> 1) & 1), so
// that the four row groups a warp touches at once (rows 16 apart in stage A,
// 14 apart in the middle phase's stores, 2 apart in the spectrum reads) fall two
// into each bank half.
__device__ __forceinline__ int zrow_sw(int m, int nl) { return nl == 8 ? m ^ ((m >> 4) & 1) : m; }
__device__ __forceinline__ int srow_sw(int r, int nl) { return nl == 8 ? r ^ ((r >> 1) & 1) : r; }

// --------------------------------------------------------------- z pass
// CTA: NL consecutive k1 columns at one k2, all three components, one RHS;
// 32 NL threads, one (even/odd half, k1, line) item each in the middle phase.
// Shared memory: twiddles (L3) and one exchange buffer
// [component][even/odd][m][line], m in [0, M), reused by both exchanges (the
// middle phase reads all of it before any thread overwrites it).
template <int R2, int NL>
__global__ void __launch_bounds__(32 * NL, 16 / NL) k_zreg(ConvArgs<float> a) {
    using C = float2;
    constexpr int M = 16 * R2, L3 = 2 * M, NT = 32 * NL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* ex = tw + L3;
    const int k10 = blockIdx.x * NL, j = blockIdx.z;
    // visit k2 and its mirror L2 - k2 back to back (they share spectrum octants)
    const int y = blockIdx.y;
    const int k2 = y == 0 ? 0 : ((y & 1) ? (y + 1) >> 1 : a.L2 - (y >> 1));
    for (int i = threadIdx.x; i < L3; i += NT) tw[i] = a.tw3[i];
    __syncthreads();
    const size_t plane = (size_t)a.L2 * a.L1;
    const size_t cstride = (size_t)a.n3 * plane;
    C* base = a.B + (size_t)j * 3 * cstride + (size_t)k2 * a.L1;
    // forward stage A on the even part x[n] and the odd part x[n] w^n (n < n3 <= M)
    for (int w = threadIdx.x; w < 3 * R2 * NL; w += NT) {
        const int l = w % NL, t = (w / NL) % R2, comp = w / (NL * R2);
        const int k1g = k10 + l;
        C e[16], o[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int n = t + R2 * q;
            C x = make_float2(0.f, 0.f);
            if (n < a.n3 && k1g < a.L1) x = base[comp * cstride + (size_t)n * plane + k1g];
            e[q] = x;
            o[q] = cmul(x, tw[n]);
        }
        dftR<false>(e, int_<16>());
        dftR<false>(o, int_<16>());
        C* de = ex + (size_t)(comp * 2) * M * NL + l;
        C* dodd = de + (size_t)M * NL;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            C we = e[k], wo = o[k];
            if (k > 0 && t > 0) {
                const C tt = tw[2 * t * k];    // w_M^(t k)
                we = cmul(we, tt);
                wo = cmul(wo, tt);
            }
            const int row = zrow_sw(t * 16 + k, NL);
            de[row * NL] = we;
            dodd[row * NL] = wo;
        }
    }
    __syncthreads();
    // forward stage B, spectrum multiply, inverse stage A: item (half, k1, line)
    {
        const int w = threadIdx.x;
        const int l = w % NL, k1 = (w / NL) % 16, half = w / (16 * NL);
        const int k1g = k10 + l;
        C v[3][R2];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const C* src = ex + (size_t)(c * 2 + half) * M * NL + l;
#pragma unroll
            for (int t = 0; t < R2; ++t) v[c][t] = src[zrow_sw(t * 16 + k1, NL) * NL];
        }
        __syncthreads();   // every item has read its inputs; the buffer is reused below
#pragma unroll
        for (int c = 0; c < 3; ++c) dftR<false>(v[c], int_<R2>());   // v[c][q]: frequency 2 (k1 + 16 q) + half
        if (k1g < a.L1) {
            const size_t oct = (size_t)a.Lh1 * a.Lh2 * a.Lh3;
            const int kk2 = k2 <= a.L2 / 2 ? k2 : a.L2 - k2;
            const float sg2 = k2 <= a.L2 / 2 ? 1.f : -1.f;
            const int kk1 = k1g <= a.L1 / 2 ? k1g : a.L1 - k1g;
            const float sg1 = k1g <= a.L1 / 2 ? 1.f : -1.f;
            const C* sp = a.spec + kk1 + (size_t)a.Lh1 * kk2;
            const size_t st3 = (size_t)a.Lh1 * a.Lh2;
#pragma unroll
            for (int q = 0; q < R2; ++q) {
                const int k3 = 2 * (k1 + 16 * q) + half;
                const int kk3 = k3 <= L3 / 2 ? k3 : L3 - k3;
                const float sg3 = k3 <= L3 / 2 ? 1.f : -1.f;
                const C* so = sp + st3 * kk3;
                const C txx = so[0], tyy = so[oct], tzz = so[2 * oct];
                const C txy = cscale(so[3 * oct], sg1 * sg2);
                const C txz = cscale(so[4 * oct], sg1 * sg3);
                const C tyz = cscale(so[5 * oct], sg2 * sg3);
                const C x = v[0][q], yv = v[1][q], z = v[2][q];
                C ox = cmul(txx, x), oy = cmul(txy, x), oz = cmul(txz, x);
                cfma(ox, txy, yv); cfma(ox, txz, z);
                cfma(oy, tyy, yv); cfma(oy, tyz, z);
                cfma(oz, tyz, yv); cfma(oz, tzz, z);
                v[0][q] = ox; v[1][q] = oy; v[2][q] = oz;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dftR<true>(v[c], int_<R2>());      // v[c][n1] = sum_q X[k1 + 16 q] w_R2^(-q n1)
            C* dst = ex + (size_t)(c * 2 + half) * M * NL + l;
#pragma unroll
            for (int n1 = 0; n1 < R2; ++n1)
                dst[zrow_sw(k1 * R2 + n1, NL) * NL] = (n1 > 0 && k1 > 0) ? cmulc(v[c][n1], tw[2 * n1 * k1]) : v[c][n1];
        }
    }
    __syncthreads();
    // inverse stage B (radix 16 over k1) and recombination y[n] = y_e[n] + w^-n y_o[n]
    for (int w = threadIdx.x; w < 3 * R2 * NL; w += NT) {
        const int l = w % NL, n1 = (w / NL) % R2, comp = w / (NL * R2);
        const int k1g = k10 + l;
        C e[16], o[16];
        const C* se = ex + (size_t)(comp * 2) * M * NL + l;
        const C* so = se + (size_t)M * NL;
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) {
            const int row = zrow_sw(k1 * R2 + n1, NL);
            e[k1] = se[row * NL];
            o[k1] = so[row * NL];
        }
        dftR<true>(e, int_<16>());
        dftR<true>(o, int_<16>());
        if (k1g < a.L1) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int n = n1 + R2 * q;
                if (n < a.n3) base[comp * cstride + (size_t)n * plane + k1g] = cadd(e[q], cmulc(o[q], tw[n]));
            }
        }
    }
}

// --------------------------------------------------------------- z pass, staged
// Same transform as k_zreg, reorganised so that the CTA's share of the spectrum
// and its input lines come from shared memory:
//   * CTA: NL consecutive k1 columns at one k2, all three components, and every
//     right-hand side of the launch group in turn (the spectrum tile is loaded
//     once per CTA, not once per right-hand side);
//   * the spectrum tile (6 components x (L3/2 + 1) k3 x NL columns) and the
//     input lines of right-hand side 0 arrive by cp.async at the start; while
//     right-hand side j is in its middle and final phases, the lines of j + 1
//     are fetched into the staging buffer, so the global-load latency of
//     stage A overlaps the arithmetic;
//   * NT = max(32 NL, 3 R2 NL rounded up to a warp) threads, so stage A and the
//     final phase take one round (k_zreg needs two at R2 = 14);
//   * exchange and spectrum rows use the bank swizzle of k_zreg (NL = 8).
// Shared memory: twiddles (L3), exchange 6 M NL, spectrum 6 (L3/2+1) NL,
// staging 3 n3 NL complex values.  Needs L1 % NL == 0 (16-byte cp.async).
template <int R2, int NL, bool SPLIT = false> struct ZStaged {
    static constexpr int M = 16 * R2;
    static constexpr int NT0 = (3 * R2 * NL + 31) / 32 * 32;
    static constexpr int NMID = (SPLIT ? 64 : 32) * NL;   // threads of the middle phase
    static constexpr int NT = NT0 > NMID ? NT0 : NMID;
    static constexpr int MINB = (R2 == 7 && NL == 8 && !SPLIT) ? 2 : 1;
};
__device__ __forceinline__ void cpa8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cpa16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int R2, int NL, bool SPLIT>
__global__ void __launch_bounds__(ZStaged<R2, NL, SPLIT>::NT, ZStaged<R2, NL, SPLIT>::MINB)
    k_zreg_st(ConvArgs<float> a, int p) {
    using C = float2;
    constexpr int M = ZStaged<R2, NL, SPLIT>::M, L3 = 2 * M, NT = ZStaged<R2, NL, SPLIT>::NT;
    static_assert(!SPLIT || (R2 % 2 == 0 && NT == 64 * NL), "split middle phase: even R2, one thread pair per item");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* ex = tw + L3;
    C* sp = ex + 6 * M * NL;
    C* pre = sp + (size_t)6 * a.Lh3 * NL;
    const int k10 = blockIdx.x * NL;
    const int y = blockIdx.y;
    const int k2 = y == 0 ? 0 : ((y & 1) ? (y + 1) >> 1 : a.L2 - (y >> 1));
    const int kk2 = k2 <= a.L2 / 2 ? k2 : a.L2 - k2;
    const float sg2 = k2 <= a.L2 / 2 ? 1.f : -1.f;
    const size_t plane = (size_t)a.L2 * a.L1;
    const size_t cstride = (size_t)a.n3 * plane;
    const size_t oct = (size_t)a.Lh1 * a.Lh2 * a.Lh3;
    const size_t st3 = (size_t)a.Lh1 * a.Lh2;
    for (int i = threadIdx.x; i < L3; i += NT) tw[i] = a.tw3[i];
    // spectrum tile: row r = c6 Lh3 + kk3, column l (each thread keeps one column;
    // NT is a multiple of NL, so the loops need no runtime division)
    static_assert(NT % NL == 0 && NT % (NL / 2) == 0, "thread count must tile the line columns");
    {
        const int l = threadIdx.x % NL, k1g = k10 + l;
        const int kk1 = k1g <= a.L1 / 2 ? k1g : a.L1 - k1g;
        const C* sb = a.spec + (size_t)kk2 * a.Lh1 + kk1;
        for (int c6 = 0; c6 < 6; ++c6)
            for (int kk3 = threadIdx.x / NL; kk3 < a.Lh3; kk3 += NT / NL)
                cpa8(sp + (size_t)srow_sw(c6 * a.Lh3 + kk3, NL) * NL + l, sb + c6 * oct + kk3 * st3);
    }
    auto prefetch = [&](int j) {
        const C* src = a.B + (size_t)j * 3 * cstride + (size_t)k2 * a.L1 + k10;
        const int part = threadIdx.x % (NL / 2);
        for (int comp = 0; comp < 3; ++comp)
            for (int n = threadIdx.x / (NL / 2); n < a.n3; n += NT / (NL / 2))
                cpa16(pre + (size_t)(comp * a.n3 + n) * NL + 2 * part, src + comp * cstride + (size_t)n * plane + 2 * part);
    };
    prefetch(0);
    cpa_commit();
    const int l1 = threadIdx.x % NL;
    const int k1g_mid = k10 + l1;
    const float sg1 = k1g_mid <= a.L1 / 2 ? 1.f : -1.f;
    for (int j = 0; j < p; ++j) {
        cpa_wait_all();
        __syncthreads();   // staged lines of j (and, at j = 0, spectrum and twiddles) are in
        // forward stage A: even part x[n], odd part x[n] w^n (n < n3 <= M)
        for (int w = threadIdx.x; w < 3 * R2 * NL; w += NT) {
            const int l = w % NL, t = (w / NL) % R2, comp = w / (NL * R2);
            C e[16], o[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int n = t + R2 * q;
                C x = make_float2(0.f, 0.f);
                if (n < a.n3) x = pre[(size_t)(comp * a.n3 + n) * NL + l];
                e[q] = x;
                o[q] = cmul(x, tw[n]);
            }
            dftR<false>(e, int_<16>());
            dftR<false>(o, int_<16>());
            C* de = ex + (size_t)(comp * 2) * M * NL + l;
            C* dodd = de + (size_t)M * NL;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                C we = e[k], wo = o[k];
                if (k > 0 && t > 0) {
                    const C tt = tw[2 * t * k];
                    we = cmul(we, tt);
                    wo = cmul(wo, tt);
                }
                const int row = zrow_sw(t * 16 + k, NL);
                de[row * NL] = we;
                dodd[row * NL] = wo;
            }
        }
        __syncthreads();   // exchange written; the staging buffer is free
        if (j + 1 < p) {
            prefetch(j + 1);
            cpa_commit();
        }
        if constexpr (!SPLIT) {
            // forward stage B, spectrum multiply, inverse stage A: item (half, k1, line)
            const bool act = threadIdx.x < 32 * NL;
            const int k1 = (threadIdx.x / NL) % 16, half = threadIdx.x / (16 * NL);
            C v[3][R2];
            if (act) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const C* src = ex + (size_t)(c * 2 + half) * M * NL + l1;
#pragma unroll
                    for (int t = 0; t < R2; ++t) v[c][t] = src[zrow_sw(t * 16 + k1, NL) * NL];
                }
            }
            __syncthreads();   // every item has read its inputs; the buffer is reused below
            if (act) {
#pragma unroll
                for (int c = 0; c < 3; ++c) dftR<false>(v[c], int_<R2>());
#pragma unroll
                for (int q = 0; q < R2; ++q) {
                    const int k3 = 2 * (k1 + 16 * q) + half;
                    const int kk3 = k3 <= L3 / 2 ? k3 : L3 - k3;
                    const float sg3 = k3 <= L3 / 2 ? 1.f : -1.f;
                    const C* so = sp + l1;
                    const C txx = so[(size_t)srow_sw(kk3, NL) * NL];
                    const C tyy = so[(size_t)srow_sw(a.Lh3 + kk3, NL) * NL];
                    const C tzz = so[(size_t)srow_sw(2 * a.Lh3 + kk3, NL) * NL];
                    const C txy = cscale(so[(size_t)srow_sw(3 * a.Lh3 + kk3, NL) * NL], sg1 * sg2);
                    const C txz = cscale(so[(size_t)srow_sw(4 * a.Lh3 + kk3, NL) * NL], sg1 * sg3);
                    const C tyz = cscale(so[(size_t)srow_sw(5 * a.Lh3 + kk3, NL) * NL], sg2 * sg3);
                    const C x = v[0][q], yv = v[1][q], z = v[2][q];
                    C ox = cmul(txx, x), oy = cmul(txy, x), oz = cmul(txz, x);
                    cfma(ox, txy, yv); cfma(ox, txz, z);
                    cfma(oy, tyy, yv); cfma(oy, tyz, z);
                    cfma(oz, tyz, yv); cfma(oz, tzz, z);
                    v[0][q] = ox; v[1][q] = oy; v[2][q] = oz;
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    dftR<true>(v[c], int_<R2>());
                    C* dst = ex + (size_t)(c * 2 + half) * M * NL + l1;
#pragma unroll
                    for (int n1 = 0; n1 < R2; ++n1)
                        dst[zrow_sw(k1 * R2 + n1, NL) * NL] = (n1 > 0 && k1 > 0) ? cmulc(v[c][n1], tw[2 * n1 * k1]) : v[c][n1];
                }
            }
        } else {
            // the same phase with every item on a pair of adjacent lanes: lane sub
            // takes the samples t = 2m + sub, so the radix-R2 transforms become two
            // radix-R2/2 halves joined by one shuffle exchange each way, and each lane
            // holds 3 x R2/2 values (half the registers, twice the threads)
            constexpr int RH = R2 / 2, WS = L3 / R2;   // tw[WS q] = exp(-2 pi i q / R2)
            const int it = threadIdx.x >> 1, sub = threadIdx.x & 1;
            const int lm = it % NL, k1 = (it / NL) % 16, half = it / (16 * NL);
            const float sg1m = k10 + lm <= a.L1 / 2 ? 1.f : -1.f;
            C v[3][RH];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const C* src = ex + (size_t)(c * 2 + half) * M * NL + lm;
#pragma unroll
                for (int m = 0; m < RH; ++m) v[c][m] = src[zrow_sw((2 * m + sub) * 16 + k1, NL) * NL];
            }
            __syncthreads();   // every item has read its inputs; the buffer is reused below
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dftR<false>(v[c], int_<RH>());   // sub 0: E[q], sub 1: O[q]
#pragma unroll
                for (int q = 0; q < RH; ++q) {
                    C pv;
                    pv.x = __shfl_xor_sync(0xffffffffu, v[c][q].x, 1);
                    pv.y = __shfl_xor_sync(0xffffffffu, v[c][q].y, 1);
                    const C e = sub ? pv : v[c][q];
                    C o = sub ? v[c][q] : pv;
                    if (q > 0) o = cmul(o, tw[WS * q]);
                    v[c][q] = sub ? csub(e, o) : cadd(e, o);   // X[q + RH sub]
                }
            }
#pragma unroll
            for (int q = 0; q < RH; ++q) {
                const int k3 = 2 * (k1 + 16 * (q + RH * sub)) + half;
                const int kk3 = k3 <= L3 / 2 ? k3 : L3 - k3;
                const float sg3 = k3 <= L3 / 2 ? 1.f : -1.f;
                const C* so = sp + lm;
                const C txx = so[(size_t)srow_sw(kk3, NL) * NL];
                const C tyy = so[(size_t)srow_sw(a.Lh3 + kk3, NL) * NL];
                const C tzz = so[(size_t)srow_sw(2 * a.Lh3 + kk3, NL) * NL];
                const C txy = cscale(so[(size_t)srow_sw(3 * a.Lh3 + kk3, NL) * NL], sg1m * sg2);
                const C txz = cscale(so[(size_t)srow_sw(4 * a.Lh3 + kk3, NL) * NL], sg1m * sg3);
                const C tyz = cscale(so[(size_t)srow_sw(5 * a.Lh3 + kk3, NL) * NL], sg2 * sg3);
                const C x = v[0][q], yv = v[1][q], z = v[2][q];
                C ox = cmul(txx, x), oy = cmul(txy, x), oz = cmul(txz, x);
                cfma(ox, txy, yv); cfma(ox, txz, z);
                cfma(oy, tyy, yv); cfma(oy, tyz, z);
                cfma(oz, tyz, yv); cfma(oz, tzz, z);
                v[0][q] = ox; v[1][q] = oy; v[2][q] = oz;
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                // inverse by decimation in frequency: even outputs from X[q] + X[q + RH],
                // odd outputs from (X[q] - X[q + RH]) exp(+2 pi i q / R2)
#pragma unroll
                for (int q = 0; q < RH; ++q) {
                    C pv;
                    pv.x = __shfl_xor_sync(0xffffffffu, v[c][q].x, 1);
                    pv.y = __shfl_xor_sync(0xffffffffu, v[c][q].y, 1);
                    if (sub == 0) {
                        v[c][q] = cadd(v[c][q], pv);
                    } else {
                        const C d = csub(pv, v[c][q]);
                        v[c][q] = q > 0 ? cmulc(d, tw[WS * q]) : d;
                    }
                }
                dftR<true>(v[c], int_<RH>());   // v[c][m]: output n1 = 2 m + sub
                C* dst = ex + (size_t)(c * 2 + half) * M * NL + lm;
#pragma unroll
                for (int m = 0; m < RH; ++m) {
                    const int n1 = 2 * m + sub;
                    dst[zrow_sw(k1 * R2 + n1, NL) * NL] = (n1 > 0 && k1 > 0) ? cmulc(v[c][m], tw[2 * n1 * k1]) : v[c][m];
                }
            }
        }
        __syncthreads();
        // inverse stage B (radix 16 over k1) and recombination y[n] = y_e[n] + w^-n y_o[n]
        C* base = a.B + (size_t)j * 3 * cstride + (size_t)k2 * a.L1;
        for (int w = threadIdx.x; w < 3 * R2 * NL; w += NT) {
            const int l = w % NL, n1 = (w / NL) % R2, comp = w / (NL * R2);
            C e[16], o[16];
            const C* se = ex + (size_t)(comp * 2) * M * NL + l;
            const C* so = se + (size_t)M * NL;
#pragma unroll
            for (int kq = 0; kq < 16; ++kq) {
                const int row = zrow_sw(kq * R2 + n1, NL);
                e[kq] = se[row * NL];
                o[kq] = so[row * NL];
            }
            dftR<true>(e, int_<16>());
            dftR<true>(o, int_<16>());
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int n = n1 + R2 * q;
                if (n < a.n3) base[comp * cstride + (size_t)n * plane + k10 + l] = cadd(e[q], cmulc(o[q], tw[n]));
            }
        }
        __syncthreads();   // the exchange buffer is free for the next right-hand side
    }
}

}  // namespace vsie
