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
// input once and its output once.
#include "fft.cuh"

namespace vsie {

template <typename R>
struct ConvArgs {
    int n1, n2, n3, L1, L2, L3, Lh1, Lh2, Lh3;
    int b1, b2, b3, o1, o2, o3;
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
};

template <typename C>
__device__ __forceinline__ void load_tw(C* s, const C* g, int L) {
    for (int i = threadIdx.x; i < L; i += blockDim.x) s[i] = g[i];
}

// --------------------------------------------------------------- X forward
template <typename R>
__global__ void __launch_bounds__(256) k_xfwd(ConvArgs<R> a, int NL) {
    using C = cx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* s0 = tw + a.L1;
    C* s1 = s0 + (size_t)NL * a.L1;
    const int comp = blockIdx.y, j = blockIdx.z;
    const int nlines = a.n2 * a.n3;
    const int lin0 = blockIdx.x * NL;
    load_tw(tw, a.tw1, a.L1);
    const C* xb = a.X + (size_t)j * a.ldx + a.xoff + (size_t)comp * a.nb;
    for (int e = threadIdx.x; e < NL * a.L1; e += blockDim.x) {
        const int l = e / a.L1, i1 = e - l * a.L1;
        const int lin = lin0 + l;
        C v = czero<C>();
        if (lin < nlines && i1 < a.n1) {
            const int i2 = lin % a.n2, i3 = lin / a.n2;
            const int q1 = i1 - a.o1, q2 = i2 - a.o2, q3 = i3 - a.o3;
            if (q1 >= 0 && q1 < a.b1 && q2 >= 0 && q2 < a.b2 && q3 >= 0 && q3 < a.b3) {
                const int64_t vb = q1 + (int64_t)a.b1 * (q2 + (int64_t)a.b2 * q3);
                if (a.mask[vb]) v = xb[vb];
            }
        }
        s0[e] = v;
    }
    __syncthreads();
    if (a.nact > 0) {
        const C* g = a.gc + ((size_t)j * 3 + comp) * a.nact;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int l = warp; l < NL; l += blockDim.x >> 5) {
            const int lin = lin0 + l;
            if (lin >= nlines) continue;
            for (int e = a.line_ptr[lin] + lane; e < a.line_ptr[lin + 1]; e += 32) {
                C& t = s0[(size_t)l * a.L1 + a.line_i1[e]];
                t = cadd(t, g[a.line_cidx[e]]);
            }
        }
        __syncthreads();
    }
    C* res = fft_lines<false>(s0, s1, NL, a.L1, a.L1, 1, a.pl1, tw, false);
    C* out = a.A + (((size_t)j * 3 + comp) * nlines + lin0) * a.L1;
    const int nvalid = min(NL, nlines - lin0) * a.L1;
    for (int e = threadIdx.x; e < nvalid; e += blockDim.x) out[e] = res[e];
}

// --------------------------------------------------------------- Y forward
template <typename R>
__global__ void __launch_bounds__(256) k_yfwd(ConvArgs<R> a, int NL) {
    using C = cx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* s0 = tw + a.L2;
    C* s1 = s0 + (size_t)NL * a.L2;
    const int k10 = blockIdx.x * NL, i3 = blockIdx.y, ja = blockIdx.z;
    load_tw(tw, a.tw2, a.L2);
    const C* in = a.A + ((size_t)ja * a.n3 + i3) * a.n2 * a.L1;
    for (int e = threadIdx.x; e < NL * a.L2; e += blockDim.x) {
        const int l = e % NL, i2 = e / NL;
        const int k1 = k10 + l;
        C v = czero<C>();
        if (i2 < a.n2 && k1 < a.L1) v = in[(size_t)i2 * a.L1 + k1];
        s0[e] = v;
    }
    __syncthreads();
    C* res = fft_lines<false>(s0, s1, NL, a.L2, 1, NL, a.pl2, tw, true);
    C* out = a.B + ((size_t)ja * a.n3 + i3) * a.L2 * a.L1;
    for (int e = threadIdx.x; e < NL * a.L2; e += blockDim.x) {
        const int l = e % NL, k2 = e / NL;
        const int k1 = k10 + l;
        if (k1 < a.L1) out[(size_t)k2 * a.L1 + k1] = res[e];
    }
}

// --------------------------------------------------------------- Z fused
template <typename R>
__global__ void __launch_bounds__(256) k_zmul(ConvArgs<R> a, int NL) {
    using C = cx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf[4];
    buf[0] = tw + a.L3;
    for (int q = 1; q < 4; ++q) buf[q] = buf[q - 1] + (size_t)NL * a.L3;
    const int k10 = blockIdx.x * NL, k2 = blockIdx.y, j = blockIdx.z;
    load_tw(tw, a.tw3, a.L3);
    const size_t plane = (size_t)a.L2 * a.L1;
    for (int comp = 0; comp < 3; ++comp) {
        const C* in = a.B + ((size_t)j * 3 + comp) * a.n3 * plane + (size_t)k2 * a.L1;
        C* s = buf[comp];
        for (int e = threadIdx.x; e < NL * a.L3; e += blockDim.x) {
            const int l = e % NL, i3 = e / NL;
            const int k1 = k10 + l;
            C v = czero<C>();
            if (i3 < a.n3 && k1 < a.L1) v = in[(size_t)i3 * plane + k1];
            s[e] = v;
        }
    }
    __syncthreads();
    // forward transforms; the scratch buffer rotates through the four slots
    int slot[3] = {0, 1, 2};
    int scratch = 3;
    for (int comp = 0; comp < 3; ++comp) {
        C* r = fft_lines<false>(buf[slot[comp]], buf[scratch], NL, a.L3, 1, NL, a.pl3, tw, true);
        if (r == buf[scratch]) { int t = slot[comp]; slot[comp] = scratch; scratch = t; }
    }
    // pointwise 3x3 multiply with the octant-stored symmetric spectra
    {
        const size_t oct = (size_t)a.Lh1 * a.Lh2 * a.Lh3;
        const int kk2 = k2 <= a.L2 / 2 ? k2 : a.L2 - k2;
        const R sg2 = k2 <= a.L2 / 2 ? (R)1 : (R)-1;
        C* sx = buf[slot[0]];
        C* sy = buf[slot[1]];
        C* sz = buf[slot[2]];
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
            const C x = sx[e], y = sy[e], z = sz[e];
            C ox = cmul(txx, x), oy = cmul(txy, x), oz = cmul(txz, x);
            cfma(ox, txy, y); cfma(ox, txz, z);
            cfma(oy, tyy, y); cfma(oy, tyz, z);
            cfma(oz, tyz, y); cfma(oz, tzz, z);
            sx[e] = ox; sy[e] = oy; sz[e] = oz;
        }
    }
    __syncthreads();
    for (int comp = 0; comp < 3; ++comp) {
        C* r = fft_lines<true>(buf[slot[comp]], buf[scratch], NL, a.L3, 1, NL, a.pl3, tw, true);
        if (r == buf[scratch]) { int t = slot[comp]; slot[comp] = scratch; scratch = t; }
    }
    for (int comp = 0; comp < 3; ++comp) {
        C* out = a.B + ((size_t)j * 3 + comp) * a.n3 * plane + (size_t)k2 * a.L1;
        const C* s = buf[slot[comp]];
        for (int e = threadIdx.x; e < NL * a.n3; e += blockDim.x) {
            const int l = e % NL, i3 = e / NL;
            const int k1 = k10 + l;
            if (k1 < a.L1) out[(size_t)i3 * plane + k1] = s[e];
        }
    }
}

// --------------------------------------------------------------- Y inverse
template <typename R>
__global__ void __launch_bounds__(256) k_yinv(ConvArgs<R> a, int NL) {
    using C = cx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* s0 = tw + a.L2;
    C* s1 = s0 + (size_t)NL * a.L2;
    const int k10 = blockIdx.x * NL, i3 = blockIdx.y, ja = blockIdx.z;
    load_tw(tw, a.tw2, a.L2);
    const C* in = a.B + ((size_t)ja * a.n3 + i3) * a.L2 * a.L1;
    for (int e = threadIdx.x; e < NL * a.L2; e += blockDim.x) {
        const int l = e % NL, k2 = e / NL;
        const int k1 = k10 + l;
        s0[e] = k1 < a.L1 ? in[(size_t)k2 * a.L1 + k1] : czero<C>();
    }
    __syncthreads();
    C* res = fft_lines<true>(s0, s1, NL, a.L2, 1, NL, a.pl2, tw, true);
    C* out = a.A + ((size_t)ja * a.n3 + i3) * a.n2 * a.L1;
    for (int e = threadIdx.x; e < NL * a.n2; e += blockDim.x) {
        const int l = e % NL, i2 = e / NL;
        const int k1 = k10 + l;
        if (k1 < a.L1) out[(size_t)i2 * a.L1 + k1] = res[e];
    }
}

// --------------------------------------------------------------- X inverse + epilogue
template <typename R>
__global__ void __launch_bounds__(256) k_xinv(ConvArgs<R> a, int NL) {
    using C = cx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* s0 = tw + a.L1;
    C* s1 = s0 + (size_t)NL * a.L1;
    __shared__ int any;
    const int comp = blockIdx.y, j = blockIdx.z;
    const int nlines = a.n2 * a.n3;
    const int lin0 = blockIdx.x * NL;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    if (threadIdx.x < NL && lin0 + (int)threadIdx.x < nlines && a.line_flag[lin0 + threadIdx.x])
        atomicOr(&any, 1);
    __syncthreads();
    if (!any) return;
    load_tw(tw, a.tw1, a.L1);
    const C* in = a.A + (((size_t)j * 3 + comp) * nlines + lin0) * a.L1;
    const int nvalid = min(NL, nlines - lin0) * a.L1;
    for (int e = threadIdx.x; e < NL * a.L1; e += blockDim.x) s0[e] = e < nvalid ? in[e] : czero<C>();
    __syncthreads();
    C* res = fft_lines<true>(s0, s1, NL, a.L1, a.L1, 1, a.pl1, tw, false);
    // body epilogue
    const C* xb = a.X + (size_t)j * a.ldx + a.xoff + (size_t)comp * a.nb;
    C* yb = a.Y + (size_t)j * a.ldy + a.xoff + (size_t)comp * a.nb;
    for (int e = threadIdx.x; e < NL * a.b1; e += blockDim.x) {
        const int l = e / a.b1, q1 = e - l * a.b1;
        const int lin = lin0 + l;
        if (lin >= nlines || !(a.line_flag[lin] & 1)) continue;
        const int i2 = lin % a.n2, i3 = lin / a.n2;
        const int q2 = i2 - a.o2, q3 = i3 - a.o3;
        const int64_t vb = q1 + (int64_t)a.b1 * (q2 + (int64_t)a.b2 * q3);
        const C x = xb[vb];
        C y;
        if (a.mask[vb]) y = csub(cmul(a.dinv[vb], x), res[(size_t)l * a.L1 + q1 + a.o1]);
        else y = x;
        yb[vb] = y;
    }
    if (a.nact > 0) {
        C* cco = a.cc + ((size_t)j * 3 + comp) * a.nact;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int l = warp; l < NL; l += blockDim.x >> 5) {
            const int lin = lin0 + l;
            if (lin >= nlines || !(a.line_flag[lin] & 2)) continue;
            for (int e = a.line_ptr[lin] + lane; e < a.line_ptr[lin + 1]; e += 32)
                cco[a.line_cidx[e]] = res[(size_t)l * a.L1 + a.line_i1[e]];
        }
    }
}

// --------------------------------------------------------------- launcher
static int pick_lines(int L, int nbufs, size_t csize, int maxl, size_t budget) {
    int nl = maxl;
    while (nl > 1 && (size_t)(nbufs * nl + 1) * L * csize > budget) nl >>= 1;
    return nl;
}

template <typename R>
static size_t smem_bytes(int L, int nl, int nbufs) {
    return ((size_t)nbufs * nl + 1) * L * sizeof(cx<R>);
}

template <typename R>
void conv_apply(Ctx& c, int p, const cx<R>* X, int64_t ldx, cx<R>* Y, int64_t ldy,
                cudaStream_t st) {
    OpData<R>& d = data<R>(c);
    ConvArgs<R> a;
    a.n1 = c.ne[0]; a.n2 = c.ne[1]; a.n3 = c.ne[2];
    a.L1 = c.L[0]; a.L2 = c.L[1]; a.L3 = c.L[2];
    a.Lh1 = c.Lh[0]; a.Lh2 = c.Lh[1]; a.Lh3 = c.Lh[2];
    a.b1 = c.nb[0]; a.b2 = c.nb[1]; a.b3 = c.nb[2];
    a.o1 = c.off[0]; a.o2 = c.off[1]; a.o3 = c.off[2];
    a.nb = c.n_b; a.nact = c.nact;
    a.X = X; a.ldx = ldx; a.xoff = (int64_t)c.m_f + c.m_n;
    a.Y = Y; a.ldy = ldy;
    a.mask = c.mask; a.dinv = d.dinv;
    a.line_ptr = c.line_ptr; a.line_i1 = c.line_i1; a.line_cidx = c.line_cidx;
    a.line_flag = c.body_lines;
    a.gc = d.gc; a.cc = d.cc; a.A = d.bufA; a.B = d.bufB;
    a.spec = d.spec; a.tw1 = d.tw[0]; a.tw2 = d.tw[1]; a.tw3 = d.tw[2];
    a.pl1 = c.plan[0]; a.pl2 = c.plan[1]; a.pl3 = c.plan[2];
    const size_t budget = 100 * 1024;
    const int cs = sizeof(cx<R>);
    const int maxl = sizeof(R) == 4 ? 16 : 8;
    // X forward
    {
        int nl = pick_lines(a.L1, 2, cs, maxl, budget);
        size_t sm = smem_bytes<R>(a.L1, nl, 2);
        dim3 g((a.n2 * a.n3 + nl - 1) / nl, 3, p);
        k_xfwd<R><<<g, 256, sm, st>>>(a, nl);
    }
    {
        int nl = pick_lines(a.L2, 2, cs, maxl, budget);
        size_t sm = smem_bytes<R>(a.L2, nl, 2);
        dim3 g((a.L1 + nl - 1) / nl, a.n3, 3 * p);
        k_yfwd<R><<<g, 256, sm, st>>>(a, nl);
    }
    {
        int nl = pick_lines(a.L3, 4, cs, maxl, budget + 16 * 1024);
        size_t sm = smem_bytes<R>(a.L3, nl, 4);
        dim3 g((a.L1 + nl - 1) / nl, a.L2, p);
        k_zmul<R><<<g, 256, sm, st>>>(a, nl);
    }
    {
        int nl = pick_lines(a.L2, 2, cs, maxl, budget);
        size_t sm = smem_bytes<R>(a.L2, nl, 2);
        dim3 g((a.L1 + nl - 1) / nl, a.n3, 3 * p);
        k_yinv<R><<<g, 256, sm, st>>>(a, nl);
    }
    {
        int nl = pick_lines(a.L1, 2, cs, maxl, budget);
        size_t sm = smem_bytes<R>(a.L1, nl, 2);
        dim3 g((a.n2 * a.n3 + nl - 1) / nl, 3, p);
        k_xinv<R><<<g, 256, sm, st>>>(a, nl);
    }
    VSIE_CUDA(cudaGetLastError());
}

template <typename R>
void conv_set_attrs() {
    const int big = 120 * 1024;
    VSIE_CUDA(cudaFuncSetAttribute(k_xfwd<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    VSIE_CUDA(cudaFuncSetAttribute(k_yfwd<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    VSIE_CUDA(cudaFuncSetAttribute(k_zmul<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    VSIE_CUDA(cudaFuncSetAttribute(k_yinv<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    VSIE_CUDA(cudaFuncSetAttribute(k_xinv<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
}

template void conv_apply<float>(Ctx&, int, const float2*, int64_t, float2*, int64_t, cudaStream_t);
template void conv_apply<double>(Ctx&, int, const double2*, int64_t, double2*, int64_t, cudaStream_t);
template void conv_set_attrs<float>();
template void conv_set_attrs<double>();

}  // namespace vsie
