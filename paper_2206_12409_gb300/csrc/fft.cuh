// Shared-memory Stockham FFT stages used by the convolution passes (K1) and by
// the spectra set-up.  A CTA transforms `nl` lines of length L held in shared
// memory; element (line, k) sits at buf[line * ls + k * ks].  Each stage of
// radix R reads every element once from `src` and writes it to `dst`
// (ping-pong), so one barrier per stage suffices.
//
// Stage t (radix R, Ns = product of the radices before it), butterfly j in
// [0, L/R): k = j mod Ns, inputs src[j + r L/R] twiddled by w^(r k) with
// w = exp(-+ 2 pi i / (Ns R)), radix-R DFT, outputs to dst[(j - k) R + k + r Ns].
// Twiddles come from a table tw[m] = exp(-2 pi i m / L) (conjugated for the
// inverse transform).  The inverse transform is unnormalised.
#pragma once
#include "vsie_internal.h"

namespace vsie {

// cos/sin(2 pi k / R) constants
#define C3S 0.86602540378443864676
#define C5C1 0.30901699437494742410
#define C5S1 0.95105651629515357212
#define C5C2 -0.80901699437494742410
#define C5S2 0.58778525229247312917
#define C7C1 0.62348980185873353053
#define C7S1 0.78183148246802980871
#define C7C2 -0.22252093395631440429
#define C7S2 0.97492791218182360702
#define C7C3 -0.90096886790241912624
#define C7S3 0.43388373911755812048
#define SQH 0.70710678118654752440

// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C rot90(C a) {
    C r;
    if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
    return r;
}

template <bool INV, typename C> __device__ __forceinline__ void dft2(C& a0, C& a1) {
    C t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
    C s02 = cadd(a0, a2), d02 = csub(a0, a2);
    C s13 = cadd(a1, a3), d13 = rot90<INV>(csub(a1, a3));
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = cadd(d02, d13);
    a3 = csub(d02, d13);
}

template <bool INV, typename C> __device__ __forceinline__ void dftR(C* v, int_<2>) { dft2<INV>(v[0], v[1]); }
template <bool INV, typename C> __device__ __forceinline__ void dftR(C* v, int_<4>) { dft4<INV>(v[0], v[1], v[2], v[3]); }

template <bool INV, typename C> __device__ __forceinline__ void dftR(C* v, int_<8>) {
    using R = decltype(v[0].x);
    C b[8];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        b[r] = cadd(v[r], v[r + 4]);
        b[r + 4] = csub(v[r], v[r + 4]);
    }
    // twiddles w8^r, r = 1, 2, 3 on the difference half
    const R q = (R)SQH;
    {
        C t = b[5];
        // w8 = (1 - i)/sqrt2 forward, (1 + i)/sqrt2 inverse
        if (INV) { b[5].x = q * (t.x - t.y); b[5].y = q * (t.x + t.y); }
        else { b[5].x = q * (t.x + t.y); b[5].y = q * (t.y - t.x); }
    }
    b[6] = rot90<INV>(b[6]);
    {
        C t = b[7];
        // w8^3 = (-1 - i)/sqrt2 forward, (-1 + i)/sqrt2 inverse
        if (INV) { b[7].x = -q * (t.x + t.y); b[7].y = q * (t.x - t.y); }
        else { b[7].x = q * (t.y - t.x); b[7].y = -q * (t.x + t.y); }
    }
    dft4<INV>(b[0], b[1], b[2], b[3]);
    dft4<INV>(b[4], b[5], b[6], b[7]);
    v[0] = b[0]; v[2] = b[1]; v[4] = b[2]; v[6] = b[3];
    v[1] = b[4]; v[3] = b[5]; v[5] = b[6]; v[7] = b[7];
}

template <bool INV, typename C> __device__ __forceinline__ void dftR(C* v, int_<3>) {
    using R = decltype(v[0].x);
    C t = cadd(v[1], v[2]);
    C d = csub(v[1], v[2]);
    C a0 = v[0];
    v[0] = cadd(a0, t);
    C m = a0;
    m.x -= (R)0.5 * t.x;
    m.y -= (R)0.5 * t.y;
    // (-+ i) s3 d
    C sd = rot90<INV>(d);
    sd.x *= (R)C3S;
    sd.y *= (R)C3S;
    v[1] = cadd(m, sd);
    v[2] = csub(m, sd);
}

// odd prime radix by symmetric pairs:
// A_q = a0 + sum_{r=1}^{(R-1)/2} [ (a_r + a_{R-r}) cos(2 pi r q / R) -+ i (a_r - a_{R-r}) sin(2 pi r q / R) ]
template <bool INV, int RR, typename C>
__device__ __forceinline__ void dft_odd(C* v, const double* cs, const double* sn) {
    using R = decltype(v[0].x);
    constexpr int H = (RR - 1) / 2;
    C sp[H], dm[H];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
        sp[r - 1] = cadd(v[r], v[RR - r]);
        dm[r - 1] = csub(v[r], v[RR - r]);
    }
    C a0 = v[0];
    C s0 = a0;
#pragma unroll
    for (int r = 0; r < H; ++r) s0 = cadd(s0, sp[r]);
    C out[RR];
    out[0] = s0;
#pragma unroll
    for (int q = 1; q <= H; ++q) {
        C re = a0, im = czero<C>();
#pragma unroll
        for (int r = 1; r <= H; ++r) {
            const int idx = (r * q) % RR;          // angle index 2 pi idx / R
            const int k = idx <= H ? idx : RR - idx;
            const R c = (R)cs[k - 1];
            const R s = (R)(idx <= H ? sn[k - 1] : -sn[k - 1]);
            re.x += c * sp[r - 1].x;
            re.y += c * sp[r - 1].y;
            im.x += s * dm[r - 1].x;
            im.y += s * dm[r - 1].y;
        }
        C ri = rot90<INV>(im);   // -i s d forward, +i s d inverse
        out[q] = cadd(re, ri);
        out[RR - q] = csub(re, ri);
    }
#pragma unroll
    for (int q = 0; q < RR; ++q) v[q] = out[q];
}

template <bool INV, typename C> __device__ __forceinline__ void dftR(C* v, int_<5>) {
    const double cs[2] = {C5C1, C5C2}, sn[2] = {C5S1, C5S2};
    dft_odd<INV, 5>(v, cs, sn);
}
template <bool INV, typename C> __device__ __forceinline__ void dftR(C* v, int_<7>) {
    const double cs[3] = {C7C1, C7C2, C7C3}, sn[3] = {C7S1, C7S2, C7S3};
    dft_odd<INV, 7>(v, cs, sn);
}

template <int RR, bool INV, typename C>
__device__ __forceinline__ void stockham_stage(const C* __restrict__ src, C* __restrict__ dst,
                                               int nl, int L, int ls, int ks, int Ns,
                                               const C* __restrict__ tw, bool line_fast) {
    const int nbf = L / RR;
    const int total = nl * nbf;
    const int twstep = L / (Ns * RR);
    for (int it = threadIdx.x; it < total; it += blockDim.x) {
        int line, j;
        if (line_fast) { line = it % nl; j = it / nl; }
        else { line = it / nbf; j = it - line * nbf; }
        const int k = j % Ns;
        const C* s = src + (size_t)line * ls;
        C v[RR];
#pragma unroll
        for (int r = 0; r < RR; ++r) v[r] = s[(size_t)(j + r * nbf) * ks];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < RR; ++r) {
                const C w = tw[r * k * twstep];
                v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
            }
        }
        dftR<INV>(v, int_<RR>());
        const int idx = (j - k) * RR + k;
        C* d = dst + (size_t)line * ls;
#pragma unroll
        for (int r = 0; r < RR; ++r) d[(size_t)(idx + r * Ns) * ks] = v[r];
    }
}

// Full transform of nl lines; returns the buffer that holds the result
// (either `a` or `b`).  Ends with __syncthreads().
template <bool INV, typename C>
__device__ C* fft_lines(C* a, C* b, int nl, int L, int ls, int ks, const FFTPlan& pl,
                        const C* tw, bool line_fast) {
    C* src = a;
    C* dst = b;
    int Ns = 1;
    for (int st = 0; st < pl.nst; ++st) {
        const int r = pl.rad[st];
        switch (r) {
            case 8: stockham_stage<8, INV>(src, dst, nl, L, ls, ks, Ns, tw, line_fast); break;
            case 4: stockham_stage<4, INV>(src, dst, nl, L, ls, ks, Ns, tw, line_fast); break;
            case 2: stockham_stage<2, INV>(src, dst, nl, L, ls, ks, Ns, tw, line_fast); break;
            case 3: stockham_stage<3, INV>(src, dst, nl, L, ls, ks, Ns, tw, line_fast); break;
            case 5: stockham_stage<5, INV>(src, dst, nl, L, ls, ks, Ns, tw, line_fast); break;
            default: stockham_stage<7, INV>(src, dst, nl, L, ls, ks, Ns, tw, line_fast); break;
        }
        __syncthreads();
        C* t = src; src = dst; dst = t;
        Ns *= r;
    }
    return src;
}

}  // namespace vsie
