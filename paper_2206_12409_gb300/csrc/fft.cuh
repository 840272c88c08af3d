// Shared-memory Stockham FFT used by the convolution passes (K1) and by the
// spectra set-up.  A CTA transforms NLT lines of length L held in shared
// memory, element (line, k) at buf[k * KS + line] (lines fastest, so that the
// threads of a warp touch consecutive addresses).  Each stage of radix R reads
// one buffer and writes the other (ping-pong), so a thread keeps only one
// butterfly's R values in registers.
//
// Stage (radix R, Ns = product of the radices before it), butterfly j in
// [0, L/R): k = j mod Ns, inputs at j + r L/R twiddled by w^(r k) with
// w = exp(-+ 2 pi i / (Ns R)), radix-R DFT, outputs to (j - k) R + k + r Ns.
// Twiddles come from tw[m] = exp(-2 pi i m / L) (conjugated for the inverse).
// The inverse transform is unnormalised.
#pragma once
#include "vsie_internal.h"

namespace vsie {

// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C rot90(C a) {
    C r;
    if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
    return r;
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
    C s02 = cadd(a0, a2), d02 = csub(a0, a2);
    C s13 = cadd(a1, a3), d13 = rot90<INV>(csub(a1, a3));
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = cadd(d02, d13);
    a3 = csub(d02, d13);
}

template <bool INV, typename C> __device__ __forceinline__ void dftR(C* v, int_<2>) {
    C t = v[0];
    v[0] = cadd(t, v[1]);
    v[1] = csub(t, v[1]);
}
template <bool INV, typename C> __device__ __forceinline__ void dftR(C* v, int_<4>) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
}

template <bool INV, typename C> __device__ __forceinline__ void dftR(C* v, int_<8>) {
    using R = decltype(v[0].x);
    C b[8];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        b[r] = cadd(v[r], v[r + 4]);
        b[r + 4] = csub(v[r], v[r + 4]);
    }
    constexpr R q = (R)0.70710678118654752440;
    {
        C t = b[5];   // times (1 -+ i)/sqrt2
        if (INV) { b[5].x = q * (t.x - t.y); b[5].y = q * (t.x + t.y); }
        else { b[5].x = q * (t.x + t.y); b[5].y = q * (t.y - t.x); }
    }
    b[6] = rot90<INV>(b[6]);
    {
        C t = b[7];   // times (-1 -+ i)/sqrt2
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
    constexpr R s3 = (R)0.86602540378443864676;
    C t = cadd(v[1], v[2]);
    C d = csub(v[1], v[2]);
    C a0 = v[0];
    v[0] = cadd(a0, t);
    C m = a0;
    m.x -= (R)0.5 * t.x;
    m.y -= (R)0.5 * t.y;
    C sd = rot90<INV>(d);
    sd.x *= s3;
    sd.y *= s3;
    v[1] = cadd(m, sd);
    v[2] = csub(m, sd);
}

// cos / sin (2 pi k / R), k = 1 .. (R-1)/2
template <typename R, int RR> struct OddConst;
template <typename R> struct OddConst<R, 5> {
    __device__ static constexpr R c(int k) { return k == 1 ? (R)0.30901699437494742410 : (R)-0.80901699437494742410; }
    __device__ static constexpr R s(int k) { return k == 1 ? (R)0.95105651629515357212 : (R)0.58778525229247312917; }
};
template <typename R> struct OddConst<R, 7> {
    __device__ static constexpr R c(int k) {
        return k == 1 ? (R)0.62348980185873353053 : k == 2 ? (R)-0.22252093395631440429 : (R)-0.90096886790241912624;
    }
    __device__ static constexpr R s(int k) {
        return k == 1 ? (R)0.78183148246802980871 : k == 2 ? (R)0.97492791218182360702 : (R)0.43388373911755812048;
    }
};

// odd prime radix by symmetric pairs:
// A_q = a0 + sum_{r=1}^{H} [ (a_r + a_{R-r}) cos(2 pi r q / R) -+ i (a_r - a_{R-r}) sin(2 pi r q / R) ]
template <bool INV, int RR, typename C>
__device__ __forceinline__ void dft_odd(C* v) {
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
    v[0] = s0;
#pragma unroll
    for (int q = 1; q <= H; ++q) {
        C re = a0, im = czero<C>();
#pragma unroll
        for (int r = 1; r <= H; ++r) {
            const int idx = (r * q) % RR;
            const int k = idx <= H ? idx : RR - idx;
            const R c = OddConst<R, RR>::c(k);
            const R s = idx <= H ? OddConst<R, RR>::s(k) : -OddConst<R, RR>::s(k);
            re.x += c * sp[r - 1].x;
            re.y += c * sp[r - 1].y;
            im.x += s * dm[r - 1].x;
            im.y += s * dm[r - 1].y;
        }
        C ri = rot90<INV>(im);
        // outputs q and R - q; write after all reads of v[1..] are done (sp/dm hold them)
        v[q] = cadd(re, ri);
        v[RR - q] = csub(re, ri);
    }
}
// a * exp(-+ i theta) with c = cos theta, s = sin theta (forward: minus)
template <bool INV, typename C, typename R>
__device__ __forceinline__ C twc(C a, R c, R s) {
    C r;
    if (INV) { r.x = a.x * c - a.y * s; r.y = a.y * c + a.x * s; }
    else { r.x = a.x * c + a.y * s; r.y = a.y * c - a.x * s; }
    return r;
}

// radix 16 as 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2,
// X[k1 + 4 k2] = sum_n2 w4^(n2 k2) w16^(n2 k1) sum_n1 w4^(n1 k1) x[4 n1 + n2]
template <bool INV, typename C> __device__ __forceinline__ void dftR(C* v, int_<16>) {
    using R = decltype(v[0].x);
    constexpr R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173;
    constexpr R q = (R)0.70710678118654752440;
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
    // y[n2][k1] at v[n2 + 4 k1]; twiddle by w16^(n2 k1)
    v[5] = twc<INV>(v[5], c1, s1);       // n2 1, k1 1: w^1
    v[9] = twc<INV>(v[9], q, q);         // n2 1, k1 2: w^2
    v[13] = twc<INV>(v[13], s1, c1);     // n2 1, k1 3: w^3
    v[6] = twc<INV>(v[6], q, q);         // n2 2, k1 1: w^2
    v[10] = rot90<INV>(v[10]);           // n2 2, k1 2: w^4
    v[14] = twc<INV>(v[14], -q, q);      // n2 2, k1 3: w^6
    v[7] = twc<INV>(v[7], s1, c1);       // n2 3, k1 1: w^3
    v[11] = twc<INV>(v[11], -q, q);      // n2 3, k1 2: w^6
    v[15] = twc<INV>(v[15], -c1, -s1);   // n2 3, k1 3: w^9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    // X[k1 + 4 k2] sits at v[4 k1 + k2]: transpose the 4 x 4 block
    C t[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[4 * k1 + k2];
}

template <bool INV, typename C> __device__ __forceinline__ void dftR(C* v, int_<5>) { dft_odd<INV, 5>(v); }
template <bool INV, typename C> __device__ __forceinline__ void dftR(C* v, int_<7>) { dft_odd<INV, 7>(v); }

// radix 2R from two radix-R transforms of the even and odd samples:
// X[k] = E[k] + w^k O[k], X[k + R] = E[k] - w^k O[k],  w = exp(-+ 2 pi i / (2R)),
// with c[k] = cos(pi k / R), s[k] = sin(pi k / R)
template <bool INV, int RH, typename C, typename R>
__device__ __forceinline__ void dft_even_odd(C* v, const R* c, const R* s) {
    C e[RH], o[RH];
#pragma unroll
    for (int r = 0; r < RH; ++r) {
        e[r] = v[2 * r];
        o[r] = v[2 * r + 1];
    }
    dftR<INV>(e, int_<RH>());
    dftR<INV>(o, int_<RH>());
#pragma unroll
    for (int k = 0; k < RH; ++k) {
        const C t = k == 0 ? o[0] : twc<INV>(o[k], c[k], s[k]);
        v[k] = cadd(e[k], t);
        v[k + RH] = csub(e[k], t);
    }
}

// radix 14 = 2 x 7
template <bool INV, typename C> __device__ __forceinline__ void dftR(C* v, int_<14>) {
    using R = decltype(v[0].x);
    const R c[7] = {(R)1.0, (R)0.90096886790241912624, (R)0.62348980185873353053, (R)0.22252093395631440429,
                    (R)-0.22252093395631440429, (R)-0.62348980185873353053, (R)-0.90096886790241912624};
    const R s[7] = {(R)0.0, (R)0.43388373911755812048, (R)0.78183148246802980871, (R)0.97492791218182360702,
                    (R)0.97492791218182360702, (R)0.78183148246802980871, (R)0.43388373911755812048};
    dft_even_odd<INV, 7>(v, c, s);
}

// radix 32 = 2 x 16
template <bool INV, typename C> __device__ __forceinline__ void dftR(C* v, int_<32>) {
    using R = decltype(v[0].x);
    const R c[16] = {(R)1.0, (R)0.98078528040323044913, (R)0.92387953251128675613, (R)0.83146961230254523708,
                     (R)0.70710678118654752440, (R)0.55557023301960222474, (R)0.38268343236508977173,
                     (R)0.19509032201612826785, (R)0.0, (R)-0.19509032201612826785, (R)-0.38268343236508977173,
                     (R)-0.55557023301960222474, (R)-0.70710678118654752440, (R)-0.83146961230254523708,
                     (R)-0.92387953251128675613, (R)-0.98078528040323044913};
    const R s[16] = {(R)0.0, (R)0.19509032201612826785, (R)0.38268343236508977173, (R)0.55557023301960222474,
                     (R)0.70710678118654752440, (R)0.83146961230254523708, (R)0.92387953251128675613,
                     (R)0.98078528040323044913, (R)1.0, (R)0.98078528040323044913, (R)0.92387953251128675613,
                     (R)0.83146961230254523708, (R)0.70710678118654752440, (R)0.55557023301960222474,
                     (R)0.38268343236508977173, (R)0.19509032201612826785};
    dft_even_odd<INV, 16>(v, c, s);
}

template <int RR, bool INV, int NLT, int KS, typename C>
__device__ __forceinline__ void stage_pp(const C* __restrict__ src, C* __restrict__ dst, int L,
                                         int Ns, uint32_t nsmagic, int twstep,
                                         const C* __restrict__ tw) {
    const int nbf = L / RR;
    const int total = NLT * nbf;
    for (int it = threadIdx.x; it < total; it += blockDim.x) {
        const int line = it % NLT, j = it / NLT;
        C v[RR];
#pragma unroll
        for (int r = 0; r < RR; ++r) v[r] = src[(j + r * nbf) * KS + line];
        const int k = nsmagic ? j - Ns * (int)__umulhi((uint32_t)j, nsmagic) : 0;
        if (k) {
            const int kt = k * twstep;
#pragma unroll
            for (int r = 1; r < RR; ++r) {
                const C w = tw[r * kt];
                v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
            }
        }
        dftR<INV>(v, int_<RR>());
        const int idx = (j - k) * RR + k;
#pragma unroll
        for (int r = 0; r < RR; ++r) dst[(idx + r * Ns) * KS + line] = v[r];
    }
}

// Full transform of the NLT lines held in `a` (element (line, k) at
// a[k * KS + line]); `b` is scratch of the same size.  Returns the buffer that
// holds the result.  Starts and ends synchronised.
template <bool INV, int NLT, int KS, typename C>
__device__ C* fft_pp(C* a, C* b, const FFTPlan& pl, const C* tw) {
    C* src = a;
    C* dst = b;
    for (int st = 0; st < pl.nst; ++st) {
        const int Ns = pl.ns[st];
        const uint32_t mg = pl.nsmagic[st];
        const int ts = pl.twstep[st];
        switch (pl.rad[st]) {
            case 16:
                // radix 16 is planned for FP32 only (FP64 plans stop at 8, keeping the
                // FP64 kernels' registers within their launch bounds)
                if constexpr (sizeof(C) == 8) stage_pp<16, INV, NLT, KS>(src, dst, pl.L, Ns, mg, ts, tw);
                break;
            case 8: stage_pp<8, INV, NLT, KS>(src, dst, pl.L, Ns, mg, ts, tw); break;
            case 4: stage_pp<4, INV, NLT, KS>(src, dst, pl.L, Ns, mg, ts, tw); break;
            case 2: stage_pp<2, INV, NLT, KS>(src, dst, pl.L, Ns, mg, ts, tw); break;
            case 3: stage_pp<3, INV, NLT, KS>(src, dst, pl.L, Ns, mg, ts, tw); break;
            case 5: stage_pp<5, INV, NLT, KS>(src, dst, pl.L, Ns, mg, ts, tw); break;
            default: stage_pp<7, INV, NLT, KS>(src, dst, pl.L, Ns, mg, ts, tw); break;
        }
        __syncthreads();
        C* t = src; src = dst; dst = t;
    }
    return src;
}

}  // namespace vsie
