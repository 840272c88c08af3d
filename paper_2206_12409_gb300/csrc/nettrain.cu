// The learned body preconditioner inside the solver, and its training on pairs
// that the context's own operator generates (not in the paper).
//
// Preconditioner (right, applied by flexible GMRES):
//   z_f = Z_ff^-1 v_f,  z_n = Z_nn^-1 v_n        (surface blocks, as the block
//                                                   preconditioner)
//   u   = D^-1 v_b,  s = RMS(u)                   (Jacobi-scaled body residual)
//   z_b = u + s * net([u / s; (eps_r - 1)/50; sigma])   on material voxels,
//   z_b = u                                           on vacuum voxels,
// so an all-zero network is the block preconditioner itself.
// Training pair: a smooth random body current e on the material voxels (white
// noise from a counter-based hash, box-blurred a seed-chosen number of times),
// r = Z_bb e by the FP32 operator; input from u = D^-1 r, target (e - u) / s.
#include "vsie_internal.h"

#include <algorithm>
#include <cmath>

namespace vsie {

struct Net;
Net* net_of(vsie_net* n);
void net_forward_input(Net& n, cudaStream_t st);
float* net_input(Net& n);
float* net_output(Net& n);
float* net_target(Net& n);
void net_ensure(Net& n, int d, int h, int w);
double net_train_on_target(Net& n, float lr, cudaStream_t st);

template <typename R>
void matvec_internal(Ctx& c, int p, const cx<R>* X, int64_t ldx, cx<R>* Y, int64_t ldy,
                     cudaStream_t st);

static int g1(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }
static int pad8(int n) { return (n + 7) / 8 * 8; }
constexpr int kRedBlocks = 152;

// splitmix64 finaliser of (seed, i): a counter-based generator
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// e[i] = complex standard normal (Box-Muller on two hashed uniforms), i < n
__global__ void k_noise(float2* e, int64_t n, uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t a = mix64(seed ^ mix64((uint64_t)i * 2 + 1)), b = mix64(seed ^ mix64((uint64_t)i * 2 + 2));
        const float u1 = ((a >> 40) + 0.5f) * (1.f / 16777216.f), u2 = (b >> 40) * (1.f / 16777216.f);
        const float rad = sqrtf(-2.f * logf(u1));
        float sn, cs;
        sincospif(2.f * u2, &sn, &cs);
        e[i] = make_float2(rad * cs, rad * sn);
    }
}

// 3 x 3 x 3 box average of each of the 3 components (clamped at the grid edge)
__global__ void k_blur(const float2* __restrict__ a, int n1, int n2, int n3, float2* __restrict__ b) {
    const int64_t nv = (int64_t)n1 * n2 * n3;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * nv; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i % nv, comp = i / nv;
        const int x = (int)(v % n1), y = (int)((v / n1) % n2), z = (int)(v / ((int64_t)n1 * n2));
        float2 s = make_float2(0.f, 0.f);
        int cnt = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int xx = x + dx, yy = y + dy, zz = z + dz;
                    if (xx < 0 || xx >= n1 || yy < 0 || yy >= n2 || zz < 0 || zz >= n3) continue;
                    const float2 t = a[comp * nv + xx + (int64_t)n1 * (yy + (int64_t)n2 * zz)];
                    s.x += t.x;
                    s.y += t.y;
                    ++cnt;
                }
        b[i] = make_float2(s.x / cnt, s.y / cnt);
    }
}

// partial sums of |d_v x[a v]|^2 over the body block of column c (blockIdx.y = c)
__global__ void __launch_bounds__(256) k_scaled_sumsq(const float2* __restrict__ X, int64_t ldx, int64_t off,
                                                      const float2* __restrict__ d, int64_t nb,
                                                      double* __restrict__ part) {
    const int c = blockIdx.y;
    const float2* x = X + (size_t)c * ldx + off;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * nb; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 u = cmul(x[i], d[i % nb]);
        s += (double)u.x * u.x + (double)u.y * u.y;
    }
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        part[(size_t)c * gridDim.x + blockIdx.x] = t;
    }
}

// scale[c] = sqrt(sum_b part[c][b] / (3 nb))   (one thread per column)
__global__ void k_scale_finish(const double* __restrict__ part, int nblk, int p, int64_t nb, float* __restrict__ scale) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)c * nblk + b];
    scale[c] = (float)std::sqrt(s / (3.0 * (double)nb));
}

// network input of column c: channels 2a, 2a+1 = re, im of u_a / s; 6, 7 = materials;
// zero on the padding of the (D, H, W) = (pad8 n3, pad8 n2, pad8 n1) grid
__global__ void k_pack(const float2* __restrict__ X, int64_t off, const float2* __restrict__ d,
                       const float* __restrict__ mat, const float* __restrict__ scale, int c, int n1, int n2,
                       int n3, int W, int H, int D, float* __restrict__ in) {
    const int64_t V = (int64_t)W * H * D, nb = (int64_t)n1 * n2 * n3;
    const float s = scale[c];
    const float is = s > 0.f ? 1.f / s : 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % W), y = (int)((i / W) % H), z = (int)(i / ((int64_t)W * H));
        float ch[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (x < n1 && y < n2 && z < n3) {
            const int64_t v = x + (int64_t)n1 * (y + (int64_t)n2 * z);
            for (int a = 0; a < 3; ++a) {
                const float2 u = cmul(X[off + a * nb + v], d[v]);
                ch[2 * a] = u.x * is;
                ch[2 * a + 1] = u.y * is;
            }
            ch[6] = mat[v];
            ch[7] = mat[nb + v];
        }
        for (int q = 0; q < 8; ++q) in[q * V + i] = ch[q];
    }
}

// z_b = u + s * (y_{2a} + i y_{2a+1}) on the material voxels of column c, z_b = u
// on vacuum voxels (their operator rows are the identity, so u is exact there;
// a correction of size s would swamp the material part)
__global__ void k_unpack(const float2* __restrict__ X, int64_t xoff, const float2* __restrict__ d,
                         const uint8_t* __restrict__ mask, const float* __restrict__ out,
                         const float* __restrict__ scale, int c, int n1, int n2, int n3, int W, int H,
                         float2* __restrict__ Y, int64_t yoff) {
    const int64_t nb = (int64_t)n1 * n2 * n3, V = (int64_t)W * H * (((n3 + 7) / 8) * 8);
    const float s = scale[c];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * nb; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i % nb;
        const int a = (int)(i / nb);
        const int x = (int)(v % n1), y = (int)((v / n1) % n2), z = (int)(v / ((int64_t)n1 * n2));
        const int64_t q = x + (int64_t)W * (y + (int64_t)H * z);
        const float2 u = cmul(X[xoff + i], d[v]);
        const float f = mask[v] ? s : 0.f;
        Y[yoff + i] = make_float2(u.x + f * out[(2 * a) * V + q], u.y + f * out[(2 * a + 1) * V + q]);
    }
}

// training target (6 x V): (e - u) / s on body voxels, zero on the padding
__global__ void k_target(const float2* __restrict__ e, const float2* __restrict__ r, const float2* __restrict__ d,
                         const float* __restrict__ scale, int n1, int n2, int n3, int W, int H, int D,
                         float* __restrict__ tg) {
    const int64_t V = (int64_t)W * H * D, nb = (int64_t)n1 * n2 * n3;
    const float s = scale[0];
    const float is = s > 0.f ? 1.f / s : 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % W), y = (int)((i / W) % H), z = (int)(i / ((int64_t)W * H));
        for (int a = 0; a < 3; ++a) {
            float re = 0.f, im = 0.f;
            if (x < n1 && y < n2 && z < n3) {
                const int64_t v = x + (int64_t)n1 * (y + (int64_t)n2 * z);
                const float2 u = cmul(r[a * nb + v], d[v]);
                const float2 ev = e[a * nb + v];
                re = (ev.x - u.x) * is;
                im = (ev.y - u.y) * is;
            }
            tg[(2 * a) * V + i] = re;
            tg[(2 * a + 1) * V + i] = im;
        }
    }
}

// e <- e * f on the material voxels, 0 elsewhere
__global__ void k_mask_scale(float2* e, const uint8_t* __restrict__ mask, int64_t nb, float f) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * nb; i += (int64_t)gridDim.x * blockDim.x) {
        const float m = mask[i % nb] ? f : 0.f;
        e[i] = make_float2(e[i].x * m, e[i].y * m);
    }
}

static void ensure_net_inputs(Ctx& c) {
    if (c.net_mat) return;
    std::vector<float> m(2 * (size_t)c.n_b);
    for (int64_t v = 0; v < c.n_b; ++v) {
        m[v] = (float)((c.eps_r[v] - 1.0) / 50.0);
        m[c.n_b + v] = (float)c.sigma[v];
    }
    c.net_mat = (float*)dalloc(c, m.size() * sizeof(float));
    VSIE_CUDA(cudaMemcpy(c.net_mat, m.data(), m.size() * sizeof(float), cudaMemcpyHostToDevice));
    c.net_part = (double*)dalloc(c, (size_t)kRedBlocks * std::max(c.max_rhs, 1) * sizeof(double));
    c.net_scale = (float*)dalloc(c, (size_t)std::max(c.max_rhs, 1) * sizeof(float));
}

void apply_learned_precond(Ctx& c, int p, const float2* X, int64_t ldx, float2* Y, int64_t ldy,
                           cudaStream_t st) {
    if (!c.net) throw Error(VSIE_EINVAL, "precond = 2 needs a network (vsie_net_attach)");
    build_block_precond(c);
    ensure_net_inputs(c);
    OpData<float>& d = data<float>(c);
    Net& net = *reinterpret_cast<Net*>(c.net);
    ProfScope ps(c, PG_PRECOND, st);
    const cx<float> one = mk<float2>(1, 0), zero = mk<float2>(0, 0);
    if (c.m_f > 0) apply_far_inverse32(c, p, X, ldx, Y, ldy, st);
    if (c.m_n > 0)
        cgemm<float>(c, OP_N, c.m_n, p, c.m_n, one, d.pc_Znni, c.m_n, 0, X + c.m_f, ldx, 0, zero,
                     Y + c.m_f, ldy, 0, 1, nullptr, nullptr, st);
    const int n1 = c.nb[0], n2 = c.nb[1], n3 = c.nb[2];
    const int W = pad8(n1), H = pad8(n2), D = pad8(n3);
    net_ensure(net, D, H, W);
    const int64_t off = (int64_t)c.m_f + c.m_n;
    k_scaled_sumsq<<<dim3(kRedBlocks, p), 256, 0, st>>>(X, ldx, off, d.pc_bdiag, c.n_b, c.net_part);
    k_scale_finish<<<1, 64, 0, st>>>(c.net_part, kRedBlocks, p, c.n_b, c.net_scale);
    prof_count(c, 2);
    const int64_t V = (int64_t)W * H * D;
    for (int j = 0; j < p; ++j) {
        k_pack<<<g1(V), 256, 0, st>>>(X + (size_t)j * ldx, off, d.pc_bdiag, c.net_mat, c.net_scale, j, n1, n2,
                                      n3, W, H, D, net_input(net));
        net_forward_input(net, st);
        k_unpack<<<g1(3 * c.n_b), 256, 0, st>>>(X + (size_t)j * ldx, off, d.pc_bdiag, c.mask, net_output(net),
                                                c.net_scale, j, n1, n2, n3, W, H, Y + (size_t)j * ldy, off);
        prof_count(c, 2 + 21);   // pack, unpack and the network's 21 launches
    }
    VSIE_CUDA(cudaGetLastError());
}

}  // namespace vsie

using namespace vsie;

extern "C" {

vsie_status vsie_precond_apply(vsie_ctx* ctx, int32_t p, const void* X, int64_t ldx, void* Y, int64_t ldy,
                               int32_t kind, vsie_stream stream) {
    if (!ctx) { set_global_err("null context"); return VSIE_EINVAL; }
    Ctx& c = *reinterpret_cast<Ctx*>(ctx);
    try {
        if (!X || !Y) throw Error(VSIE_EINVAL, "null X or Y");
        if (p < 1 || p > c.max_rhs) throw Error(VSIE_EINVAL, "p outside [1, max_rhs]");
        if (ldx < c.N || ldy < c.N) throw Error(VSIE_EINVAL, "leading dimension < N");
        if (!c.f32.ready) throw Error(VSIE_EUNSUPPORTED, "needs the C64 operator");
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        if (kind == 0) {
            build_block_precond(c);
            apply_block_precond<float>(c, p, (const float2*)X, ldx, (float2*)Y, ldy, st);
        } else if (kind == 2) {
            apply_learned_precond(c, p, (const float2*)X, ldx, (float2*)Y, ldy, st);
        } else {
            throw Error(VSIE_EINVAL, "kind must be 0 or 2");
        }
    } catch (const Error& e) {
        c.err = e.msg;
        return e.st;
    }
    return VSIE_OK;
}

vsie_status vsie_net_attach(vsie_ctx* ctx, vsie_net* net) {
    if (!ctx) { set_global_err("null context"); return VSIE_EINVAL; }
    reinterpret_cast<Ctx*>(ctx)->net = net;
    return VSIE_OK;
}

vsie_status vsie_net_train(vsie_ctx* ctx, vsie_net* net, int32_t steps, double lr, uint64_t seed,
                           float* losses_host, vsie_stream stream) {
    if (!ctx || !net) { set_global_err("null context or network"); return VSIE_EINVAL; }
    Ctx& c = *reinterpret_cast<Ctx*>(ctx);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    float2* e = nullptr;
    float2* X = nullptr;
    float2* Y = nullptr;
    try {
        if (steps < 0 || !(lr > 0)) throw Error(VSIE_EINVAL, "steps < 0 or lr <= 0");
        if (!c.f32.ready) throw Error(VSIE_EUNSUPPORTED, "training needs the C64 operator");
        build_block_precond(c);
        ensure_net_inputs(c);
        Net& nt = *net_of(net);
        const int n1 = c.nb[0], n2 = c.nb[1], n3 = c.nb[2];
        const int W = pad8(n1), H = pad8(n2), D = pad8(n3);
        net_ensure(nt, D, H, W);
        const int64_t nb = c.n_b, N = c.N, off = (int64_t)c.m_f + c.m_n;
        if (cudaMalloc(&e, 3 * nb * sizeof(float2)) != cudaSuccess ||
            cudaMalloc(&X, N * sizeof(float2)) != cudaSuccess ||
            cudaMalloc(&Y, N * sizeof(float2)) != cudaSuccess) {
            cudaGetLastError();
            throw Error(VSIE_ENOMEM, "training vectors");
        }
        OpData<float>& d = data<float>(c);
        std::vector<double> hp(kRedBlocks);
        for (int s = 0; s < steps; ++s) {
            const uint64_t sd = seed * 0x100000001B3ull + (uint64_t)s;
            // smooth random current on the material voxels (its scale cancels: input and
            // target are both divided by s)
            k_noise<<<g1(3 * nb), 256, 0, st>>>(e, 3 * nb, sd);
            const int nblur = (int)(sd % 4);
            for (int q = 0; q < nblur; ++q) {
                k_blur<<<g1(3 * nb), 256, 0, st>>>(e, n1, n2, n3, Y + off);
                VSIE_CUDA(cudaMemcpyAsync(e, Y + off, 3 * nb * sizeof(float2), cudaMemcpyDeviceToDevice, st));
            }
            k_mask_scale<<<g1(3 * nb), 256, 0, st>>>(e, c.mask, nb, 1.f);
            // r = Z e (surface parts of the input zero; body rows of the output)
            VSIE_CUDA(cudaMemsetAsync(X, 0, N * sizeof(float2), st));
            VSIE_CUDA(cudaMemcpyAsync(X + off, e, 3 * nb * sizeof(float2), cudaMemcpyDeviceToDevice, st));
            matvec_internal<float>(c, 1, X, N, Y, N, st);
            // input scale s = RMS(D^-1 r), input channels and the target
            k_scaled_sumsq<<<dim3(kRedBlocks, 1), 256, 0, st>>>(Y, N, off, d.pc_bdiag, nb, c.net_part);
            k_scale_finish<<<1, 64, 0, st>>>(c.net_part, kRedBlocks, 1, nb, c.net_scale);
            k_pack<<<g1((int64_t)W * H * D), 256, 0, st>>>(Y, off, d.pc_bdiag, c.net_mat, c.net_scale, 0, n1, n2,
                                                           n3, W, H, D, net_input(nt));
            k_target<<<g1((int64_t)W * H * D), 256, 0, st>>>(e, Y + off, d.pc_bdiag, c.net_scale, n1, n2, n3, W, H,
                                                             D, net_target(nt));
            VSIE_CUDA(cudaGetLastError());
            // learning rate decays linearly to a tenth over the run
            const double lr_s = lr * (1.0 - 0.9 * (double)s / (double)std::max(steps, 1));
            const double L = net_train_on_target(nt, (float)lr_s, st);
            if (losses_host) losses_host[s] = (float)L;
        }
        VSIE_CUDA(cudaStreamSynchronize(st));
    } catch (const Error& ex) {
        cudaFree(e); cudaFree(X); cudaFree(Y);
        c.err = ex.msg;
        return ex.st;
    }
    cudaFree(e); cudaFree(X); cudaFree(Y);
    return VSIE_OK;
}

}  // extern "C"
