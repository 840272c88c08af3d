// Set-up of the volume kernel spectra (Sec. II.B): the generating columns of
// the block-Toeplitz Z_bb, circulant-embedded at length L and transformed by
// the library's own FFT stages.
//
// Kernel, for integer voxel offsets d (units of h):
//   T(d) = h^3 (k0^2 I + grad grad) g (h d),  g = exp(-i k0 R) / (4 pi R),  d != 0
//   T(0) = [(2/3)(1 + i k0 a) exp(-i k0 a) - 1] I,  a = (3 / (4 pi))^(1/3) h
// (the field at the centre of the equal-volume sphere; the paper delegates the
// PWC discretisation of Z_bb to MARIE).  Closed form of the dyad:
//   (g / R^2) [ (k0^2 R^2 - 1 - i k0 R) delta_ab + (3 + 3 i k0 R - k0^2 R^2) Rh_a Rh_b ].
// Embedding: position k in [0, L) holds offset k (k < n), k - L (k > L - n), else 0.
// Stored: octant k_i in [0, L_i/2] of the 6 unique components (xx yy zz xy xz yz)
// of h^3 FFT(T) / (L1 L2 L3); the other octants follow from the parity of each
// component (diagonal: even in every axis; ab: odd in a and b).
#include "fft.cuh"
#include <cmath>

namespace vsie {

__global__ void k_generator(double2* __restrict__ t, int L1, int L2, int L3, int n1, int n2,
                            int n3, double h, double k0, double2 selfv) {
    const size_t tot = (size_t)L1 * L2 * L3;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot;
         e += (size_t)gridDim.x * blockDim.x) {
        const int k1 = e % L1;
        const int k2 = (e / L1) % L2;
        const int k3 = e / ((size_t)L1 * L2);
        int d[3];
        bool ok = true;
        const int k[3] = {k1, k2, k3}, n[3] = {n1, n2, n3}, L[3] = {L1, L2, L3};
        for (int i = 0; i < 3; ++i) {
            if (k[i] < n[i]) d[i] = k[i];
            else if (k[i] > L[i] - n[i]) d[i] = k[i] - L[i];
            else ok = false;
        }
        double2 v[6];
        for (int c = 0; c < 6; ++c) v[c] = make_double2(0.0, 0.0);
        if (ok) {
            if (d[0] == 0 && d[1] == 0 && d[2] == 0) {
                v[0] = v[1] = v[2] = selfv;
            } else {
                const double rx = h * d[0], ry = h * d[1], rz = h * d[2];
                const double R2 = rx * rx + ry * ry + rz * rz;
                const double R = sqrt(R2);
                double sn, cs;
                sincos(k0 * R, &sn, &cs);
                // g = (cos - i sin) / (4 pi R); scaled by h^3 / R^2
                const double pre = h * h * h / (4.0 * M_PI * R * R2);
                const double2 g = make_double2(pre * cs, -pre * sn);
                const double kR = k0 * R;
                const double2 A = cmul(g, make_double2(kR * kR - 1.0, -kR));
                const double2 B = cmul(g, make_double2(3.0 - kR * kR, 3.0 * kR));
                const double ux = rx / R, uy = ry / R, uz = rz / R;
                v[0] = cadd(A, cscale(B, ux * ux));
                v[1] = cadd(A, cscale(B, uy * uy));
                v[2] = cadd(A, cscale(B, uz * uz));
                v[3] = cscale(B, ux * uy);
                v[4] = cscale(B, ux * uz);
                v[5] = cscale(B, uy * uz);
            }
        }
        for (int c = 0; c < 6; ++c) t[c * tot + e] = v[c];
    }
}

// In-place FFT of a full L1 x L2 x L3 x ncomp array along one axis; a CTA
// transforms NL lines: consecutive lines along i1 (axis 0: lines are the
// (k2, k3, comp) rows, loaded transposed) or NL consecutive k1 (axes 1, 2).
template <int NL>
__global__ void __launch_bounds__(512) k_fft_axis(double2* __restrict__ t, int L1, int L2, int L3,
                                                  int ncomp, int axis, FFTPlan pl,
                                                  const double2* __restrict__ twg) {
    constexpr int KS = NL + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* tw = reinterpret_cast<double2*>(smem_raw);
    const int L = pl.L;
    double2* s0 = tw + L;
    double2* s1 = s0 + (size_t)KS * L;
    for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = twg[i];
    const size_t vol = (size_t)L1 * L2 * L3;
    if (axis == 0) {
        const size_t nlines = (size_t)L2 * L3 * ncomp;
        const size_t l0 = (size_t)blockIdx.x * NL;
        const size_t base = l0 * L1;
        const int nvalid = (int)min((size_t)NL, nlines - l0);
        for (int e = threadIdx.x; e < NL * L; e += blockDim.x) {
            const int l = e / L, k = e - l * L;
            s0[k * KS + l] = l < nvalid ? t[base + e] : make_double2(0, 0);
        }
        __syncthreads();
        const double2* r = fft_pp<false, NL, KS>(s0, s1, pl, tw);
        for (int e = threadIdx.x; e < nvalid * L; e += blockDim.x) {
            const int l = e / L, k = e - l * L;
            t[base + e] = r[k * KS + l];
        }
        return;
    }
    const int k10 = blockIdx.x * NL;
    const int other = blockIdx.y;
    size_t base, es;
    if (axis == 1) {
        const int k3 = other % L3, c = other / L3;
        base = (size_t)c * vol + (size_t)k3 * L1 * L2;
        es = L1;
    } else {
        const int k2 = other % L2, c = other / L2;
        base = (size_t)c * vol + (size_t)k2 * L1;
        es = (size_t)L1 * L2;
    }
    for (int e = threadIdx.x; e < NL * L; e += blockDim.x) {
        const int l = e % NL, k = e / NL;
        s0[k * KS + l] = (k10 + l) < L1 ? t[base + k * es + k10 + l] : make_double2(0, 0);
    }
    __syncthreads();
    const double2* r = fft_pp<false, NL, KS>(s0, s1, pl, tw);
    for (int e = threadIdx.x; e < NL * L; e += blockDim.x) {
        const int l = e % NL, k = e / NL;
        if (k10 + l < L1) t[base + k * es + k10 + l] = r[k * KS + l];
    }
}

template <typename R>
__global__ void k_octant(const double2* __restrict__ t, cx<R>* __restrict__ spec, int L1, int L2,
                         int L3, int Lh1, int Lh2, int Lh3, double scale) {
    const size_t oct = (size_t)Lh1 * Lh2 * Lh3;
    const size_t vol = (size_t)L1 * L2 * L3;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < 6 * oct;
         e += (size_t)gridDim.x * blockDim.x) {
        const int c = e / oct;
        const size_t o = e - c * oct;
        const int k1 = o % Lh1, k2 = (o / Lh1) % Lh2, k3 = o / ((size_t)Lh1 * Lh2);
        const double2 v = t[c * vol + k1 + (size_t)L1 * (k2 + (size_t)L2 * k3)];
        cx<R>* dummy = nullptr;
        spec[e] = to_c(cscale(v, scale), dummy);
    }
}

template <typename R>
void upload_twiddles(Ctx& c) {
    OpData<R>& d = data<R>(c);
    for (int ax = 0; ax < 3; ++ax) {
        const int L = c.L[ax];
        std::vector<cx<R>> tw(L);
        for (int m = 0; m < L; ++m) {
            const double ang = 2.0 * M_PI * (double)m / (double)L;
            tw[m].x = (R)std::cos(ang);
            tw[m].y = (R)(-std::sin(ang));
        }
        d.tw[ax] = (cx<R>*)dalloc(c, L * sizeof(cx<R>));
        VSIE_CUDA(cudaMemcpy(d.tw[ax], tw.data(), L * sizeof(cx<R>), cudaMemcpyHostToDevice));
    }
}

template <typename R>
void build_spectra(Ctx& c) {
    // double-precision generator and transform, shared by both precisions
    if (!c.f64.tw[0]) upload_twiddles<double>(c);
    OpData<R>& d = data<R>(c);
    if (!d.tw[0]) upload_twiddles<R>(c);
    const int L1 = c.L[0], L2 = c.L[1], L3 = c.L[2];
    const size_t vol = (size_t)L1 * L2 * L3;
    double2* t = nullptr;
    if (cudaMalloc(&t, 6 * vol * sizeof(double2)) != cudaSuccess)
        throw Error(VSIE_ENOMEM, "spectra set-up: cannot allocate the embedded generator");
    try {
        const double a = std::cbrt(3.0 / (4.0 * M_PI)) * c.h;
        const std::complex<double> e = std::exp(std::complex<double>(0.0, -c.k0 * a));
        const std::complex<double> sv =
            (2.0 / 3.0) * std::complex<double>(1.0, c.k0 * a) * e - 1.0;
        k_generator<<<2048, 256>>>(t, L1, L2, L3, c.ne[0], c.ne[1], c.ne[2], c.h, c.k0,
                                   make_double2(sv.real(), sv.imag()));
        VSIE_CUDA(cudaGetLastError());
        constexpr int NL = 8;
        VSIE_CUDA(cudaFuncSetAttribute(k_fft_axis<NL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024));
        for (int ax = 0; ax < 3; ++ax) {
            const int L = c.L[ax];
            const size_t sm = ((size_t)2 * (NL + 1) + 1) * L * sizeof(double2);
            if (ax == 0) {
                const size_t nlines = (size_t)L2 * L3 * 6;
                k_fft_axis<NL><<<(unsigned)((nlines + NL - 1) / NL), 256, sm>>>(
                    t, L1, L2, L3, 6, 0, c.plan[0], c.f64.tw[0]);
            } else {
                dim3 g((L1 + NL - 1) / NL, (ax == 1 ? L3 : L2) * 6);
                k_fft_axis<NL><<<g, 256, sm>>>(t, L1, L2, L3, 6, ax, c.plan[ax], c.f64.tw[ax]);
            }
            VSIE_CUDA(cudaGetLastError());
        }
        const size_t oct = (size_t)c.Lh[0] * c.Lh[1] * c.Lh[2];
        d.spec = (cx<R>*)dalloc(c, 6 * oct * sizeof(cx<R>));
        const double scale = c.h * c.h * c.h / (double)vol;
        k_octant<R><<<1024, 256>>>(t, d.spec, L1, L2, L3, c.Lh[0], c.Lh[1], c.Lh[2], scale);
        VSIE_CUDA(cudaGetLastError());
        VSIE_CUDA(cudaDeviceSynchronize());
    } catch (...) {
        cudaFree(t);
        throw;
    }
    cudaFree(t);
}

template void build_spectra<float>(Ctx&);
template void build_spectra<double>(Ctx&);
template void upload_twiddles<float>(Ctx&);
template void upload_twiddles<double>(Ctx&);

}  // namespace vsie
