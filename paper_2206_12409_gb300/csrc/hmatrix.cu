// Hierarchical (H-) matrix of the far-far conductor block Z_ff (Sec. II.B: the
// large conductor blocks are compressed by ACA; Eq. (hvsie_disc)).
//
//  * Cluster tree of the far RWG functions: recursive bisection of their
//    centres along the longest box axis at the median, down to `leaf` functions;
//    each cluster keeps the bounding box of its functions' supports.
//  * Block partition: a cluster pair (s, t) is admissible when
//    min(diam s, diam t) <= eta dist(s, t) (boxes of the supports); admissible
//    pairs become low-rank leaves U V^T, pairs of two leaf clusters dense leaves,
//    anything else is split (only the non-leaf side when one side is a leaf).
//  * Low-rank leaves: ACA with partial pivoting (Zhao et al. 2005) to the ACA
//    tolerance, one CTA per block, rows and columns read from the dense FP64
//    block assembled at set-up; a block whose ACA has not converged within its
//    rank cap is kept dense.
//  * Product y = Z_ff x, p right-hand sides, in three launches: gather x into
//    cluster order; t_b = V_b^T x(t_b) for every low-rank block; one CTA per
//    leaf row cluster sums its dense blocks and U_b t_b over every block that
//    covers it and scatters the rows back (no atomics, fixed order).
// FP64 data come from the ACA; the FP32 copies are the rounded FP64 factors.
#include "hmatrix.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <functional>
#include <numeric>

namespace vsie {

// ------------------------------------------------------------------ host: tree and blocks
namespace {
struct CNode {
    int b = 0, e = 0;
    double lo[3], hi[3];
    int c[2] = {-1, -1};
};

double diam(const CNode& n) {
    double s = 0;
    for (int d = 0; d < 3; ++d) s += (n.hi[d] - n.lo[d]) * (n.hi[d] - n.lo[d]);
    return std::sqrt(s);
}
double dist(const CNode& a, const CNode& b) {
    double s = 0;
    for (int d = 0; d < 3; ++d) {
        const double g = std::max({0.0, b.lo[d] - a.hi[d], a.lo[d] - b.hi[d]});
        s += g * g;
    }
    return std::sqrt(s);
}
}  // namespace

HmPlan hm_plan(int m, const double* centre, const double* slo, const double* shi, int leaf, double eta) {
    HmPlan P;
    P.m = m;
    P.perm.resize(m);
    std::iota(P.perm.begin(), P.perm.end(), 0);
    std::vector<CNode> nodes;
    std::function<int(int, int)> build = [&](int b, int e) -> int {
        CNode n;
        n.b = b;
        n.e = e;
        for (int d = 0; d < 3; ++d) { n.lo[d] = 1e300; n.hi[d] = -1e300; }
        double clo[3] = {1e300, 1e300, 1e300}, chi[3] = {-1e300, -1e300, -1e300};
        for (int i = b; i < e; ++i) {
            const int r = P.perm[i];
            for (int d = 0; d < 3; ++d) {
                n.lo[d] = std::min(n.lo[d], slo[3 * r + d]);
                n.hi[d] = std::max(n.hi[d], shi[3 * r + d]);
                clo[d] = std::min(clo[d], centre[3 * r + d]);
                chi[d] = std::max(chi[d], centre[3 * r + d]);
            }
        }
        const int id = (int)nodes.size();
        nodes.push_back(n);
        if (e - b > leaf) {
            int ax = 0;
            for (int d = 1; d < 3; ++d)
                if (chi[d] - clo[d] > chi[ax] - clo[ax]) ax = d;
            const int mid = b + (e - b) / 2;
            std::nth_element(P.perm.begin() + b, P.perm.begin() + mid, P.perm.begin() + e,
                             [&](int x, int y) {
                                 return centre[3 * x + ax] < centre[3 * y + ax] ||
                                        (centre[3 * x + ax] == centre[3 * y + ax] && x < y);
                             });
            const int c0 = build(b, mid);
            const int c1 = build(mid, e);
            nodes[id].c[0] = c0;
            nodes[id].c[1] = c1;
        }
        return id;
    };
    if (m > 0) build(0, m);
    // leaves in order partition [0, m)
    std::function<void(int)> leaves = [&](int id) {
        const CNode& n = nodes[id];
        if (n.c[0] < 0) {
            const int li = (int)P.rl_start.size();
            P.rl_start.push_back(n.b);
            (void)li;
            return;
        }
        leaves(n.c[0]);
        leaves(n.c[1]);
    };
    if (m > 0) leaves(0);
    P.rl_start.push_back(m);
    std::function<void(int, int)> part = [&](int s, int t) {
        const CNode& a = nodes[s];
        const CNode& b = nodes[t];
        const bool la = a.c[0] < 0, lb = b.c[0] < 0;
        const double d = dist(a, b);
        if (d > 0 && std::min(diam(a), diam(b)) <= eta * d) {
            P.blk.push_back({a.b, a.e - a.b, b.b, b.e - b.b, false});
        } else if (la && lb) {
            P.blk.push_back({a.b, a.e - a.b, b.b, b.e - b.b, true});
        } else if (la) {
            part(s, b.c[0]);
            part(s, b.c[1]);
        } else if (lb) {
            part(a.c[0], t);
            part(a.c[1], t);
        } else {
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) part(a.c[i], b.c[j]);
        }
    };
    if (m > 0) part(0, 0);
    return P;
}

// Row-leaf entry lists (which blocks cover each leaf row cluster, and where).
static void hm_entries(const HmPlan& P, std::vector<int>& ptr, std::vector<int>& eb, std::vector<int>& ero) {
    const int nrl = (int)P.rl_start.size() - 1;
    std::vector<std::vector<std::pair<int, int>>> lists(nrl);
    std::vector<int> leaf_at(P.m + 1, -1);
    for (int l = 0; l < nrl; ++l) leaf_at[P.rl_start[l]] = l;
    for (int b = 0; b < (int)P.blk.size(); ++b) {
        const auto& B = P.blk[b];
        int pos = B.r0;
        while (pos < B.r0 + B.nr) {
            const int l = leaf_at[pos];
            lists[l].push_back({b, pos - B.r0});
            pos = P.rl_start[l + 1];
        }
    }
    ptr.assign(1, 0);
    for (int l = 0; l < nrl; ++l) {
        for (auto& pr : lists[l]) {
            eb.push_back(pr.first);
            ero.push_back(pr.second);
        }
        ptr.push_back((int)eb.size());
    }
}

// ------------------------------------------------------------------ device: assembly
__global__ void k_hm_dense(const double2* __restrict__ Z, int64_t ldz, const int* __restrict__ perm,
                           const int4* __restrict__ blk, const int64_t* __restrict__ off, const int* __restrict__ ids,
                           double2* __restrict__ D64) {
    const int b = ids[blockIdx.x];
    const int4 B = blk[b];
    double2* D = D64 + off[b];
    const int64_t n = (int64_t)B.y * B.w;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
        const int i = (int)(e % B.y), j = (int)(e / B.y);
        D[e] = Z[(size_t)perm[B.x + i] + (size_t)ldz * perm[B.z + j]];
    }
}

__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// Block argmax of val (ties: smallest index) over the CTA; val < 0 = excluded.
__device__ void block_argmax(double val, int idx, double* sv, int* si, double& best, int& bi) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, val, o);
        const int oi = __shfl_down_sync(0xffffffffu, idx, o);
        if (ov > val || (ov == val && oi >= 0 && (idx < 0 || oi < idx))) { val = ov; idx = oi; }
    }
    if (lane == 0) { sv[w] = val; si[w] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = sv[0];
        int ii = si[0];
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
            if (sv[q] > v || (sv[q] == v && si[q] >= 0 && (ii < 0 || si[q] < ii))) { v = sv[q]; ii = si[q]; }
        sv[0] = v;
        si[0] = ii;
    }
    __syncthreads();
    best = sv[0];
    bi = si[0];
    __syncthreads();
}

__device__ double block_sum(double v, double* sv) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sv[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += sv[q];
        sv[0] = s;
    }
    __syncthreads();
    const double r = sv[0];
    __syncthreads();
    return r;
}

// ACA with partial pivoting of block ids[blockIdx.x] (rows perm[r0 + i], columns
// perm[c0 + j] of the dense Z); A ~= sum_l u_l v_l^T with u_l = U[:, l] (m rows,
// ld m) and v_l = V[:, l] (n rows, ld n).  rank[b] = k, or -1 when kcap terms did
// not reach the tolerance.  flags: m + n bytes of scratch per block.
constexpr int kAcaThreads = 256;
__global__ void __launch_bounds__(kAcaThreads)
k_hm_aca(const double2* __restrict__ Z, int64_t ldz, const int* __restrict__ perm, const int4* __restrict__ blk,
         const int* __restrict__ ids, const int64_t* __restrict__ uo, const int64_t* __restrict__ vo,
         const int64_t* __restrict__ fo, const int* __restrict__ kcap, double tol, double2* __restrict__ U,
         double2* __restrict__ V, unsigned char* __restrict__ flags, int* __restrict__ rank) {
    __shared__ double sv[32];
    __shared__ int si[32];
    __shared__ double2 sc[2];
    const int bi = blockIdx.x, b = ids[bi];
    const int4 B = blk[b];
    const int m = B.y, n = B.w, K = kcap[bi];
    double2* Ub = U + uo[bi];
    double2* Vb = V + vo[bi];
    unsigned char* ur = flags + fo[bi];
    unsigned char* uc = ur + m;
    for (int i = threadIdx.x; i < m + n; i += blockDim.x) ur[i] = 0;
    __syncthreads();
    int k = 0, i = 0, tries = 0;
    double normS2 = 0.0;
    bool conv = false;
    while (k < K && tries <= m) {
        if (threadIdx.x == 0) ur[i] = 1;
        const size_t zr = (size_t)perm[B.x + i];
        double best = -1.0;
        int jb = -1;
        {
            double bv = -1.0;
            int bj = -1;
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                double2 a = Z[zr + (size_t)ldz * perm[B.z + j]];
                for (int l = 0; l < k; ++l) a = csub(a, cmul(Ub[i + (size_t)m * l], Vb[j + (size_t)n * l]));
                Vb[j + (size_t)n * k] = a;
                const double v = uc[j] ? -1.0 : cabs2(a);
                if (v > bv) { bv = v; bj = j; }
            }
            block_argmax(bv, bj, sv, si, best, jb);
        }
        if (!(best > 0.0) || jb < 0) {
            // zero residual row: continue from the next unused row
            ++tries;
            double bv = -1.0;
            int bj = -1;
            for (int q = threadIdx.x; q < m; q += blockDim.x)
                if (!ur[q]) { bv = 1.0; bj = q; break; }
            double bb;
            int nx;
            block_argmax(bv, bj, sv, si, bb, nx);
            if (nx < 0) { conv = true; break; }
            i = nx;
            continue;
        }
        if (threadIdx.x == 0) {
            sc[0] = Vb[jb + (size_t)n * k];
            uc[jb] = 1;
        }
        __syncthreads();
        const double2 piv = sc[0];
        const double pn = cabs2(piv);
        const double2 ip = make_double2(piv.x / pn, -piv.y / pn);
        for (int j = threadIdx.x; j < n; j += blockDim.x) Vb[j + (size_t)n * k] = cmul(Vb[j + (size_t)n * k], ip);
        const size_t zc = (size_t)ldz * perm[B.z + jb];
        double bu = -1.0, nu2 = 0.0;
        int bq = -1;
        for (int q = threadIdx.x; q < m; q += blockDim.x) {
            double2 a = Z[zc + perm[B.x + q]];
            for (int l = 0; l < k; ++l) a = csub(a, cmul(Ub[q + (size_t)m * l], Vb[jb + (size_t)n * l]));
            Ub[q + (size_t)m * k] = a;
            nu2 += cabs2(a);
            const double v = ur[q] ? -1.0 : cabs2(a);
            if (v > bu) { bu = v; bq = q; }
        }
        __syncthreads();
        nu2 = block_sum(nu2, sv);
        double nv2 = 0.0;
        for (int j = threadIdx.x; j < n; j += blockDim.x) nv2 += cabs2(Vb[j + (size_t)n * k]);
        nv2 = block_sum(nv2, sv);
        // 2 Re sum_l (u_l^H u_k)(v_l^H v_k)
        double cross = 0.0;
        for (int l = 0; l < k; ++l) {
            double2 du = make_double2(0, 0), dv = make_double2(0, 0);
            for (int q = threadIdx.x; q < m; q += blockDim.x) du = cadd(du, cmulc(Ub[q + (size_t)m * k], Ub[q + (size_t)m * l]));
            for (int j = threadIdx.x; j < n; j += blockDim.x) dv = cadd(dv, cmulc(Vb[j + (size_t)n * k], Vb[j + (size_t)n * l]));
            const double dux = block_sum(du.x, sv), duy = block_sum(du.y, sv);
            const double dvx = block_sum(dv.x, sv), dvy = block_sum(dv.y, sv);
            cross += 2.0 * (dux * dvx - duy * dvy);
        }
        normS2 += nu2 * nv2 + cross;
        ++k;
        if (sqrt(nu2 * nv2) <= tol * sqrt(fmax(normS2, 0.0))) { conv = true; break; }
        double bb;
        int nx;
        block_argmax(bu, bq, sv, si, bb, nx);
        if (nx < 0) { conv = true; break; }
        i = nx;
    }
    if (threadIdx.x == 0) rank[bi] = (conv || k < K) ? k : -1;
}

__global__ void k_hm_narrow(const double2* __restrict__ a, float2* __restrict__ b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

// ------------------------------------------------------------------ device: product
template <typename R>
__global__ void k_hm_gather(int m, int p, const int* __restrict__ perm, const cx<R>* __restrict__ X, int64_t ldx,
                            cx<R>* __restrict__ xt) {
    const int64_t tot = (int64_t)m * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), c = (int)(e / m);
        xt[e] = X[(size_t)c * ldx + perm[i]];
    }
}

// t[(toff_b + l) NB + c] = sum_j V_b[j, l] xt[c0_b + j, c]  (one CTA per low-rank block,
// one warp per l)
template <typename R, int NB>
__global__ void __launch_bounds__(256) k_hm_vt(int m, int p, const int* __restrict__ lr, const int4* __restrict__ blk,
                                               const int* __restrict__ kb, const int64_t* __restrict__ voff,
                                               const int* __restrict__ toff, const cx<R>* __restrict__ V,
                                               const cx<R>* __restrict__ xt, cx<R>* __restrict__ t) {
    using C = cx<R>;
    const int b = lr[blockIdx.x];
    const int4 B = blk[b];
    const int n = B.w, k = kb[b];
    const C* Vb = V + voff[b];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int l = w; l < k; l += blockDim.x >> 5) {
        C acc[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) acc[c] = czero<C>();
        for (int j = lane; j < n; j += 32) {
            const C v = Vb[j + (size_t)n * l];
#pragma unroll
            for (int c = 0; c < NB; ++c)
                if (c < p) cfma(acc[c], v, xt[(size_t)c * m + B.z + j]);
        }
#pragma unroll
        for (int c = 0; c < NB; ++c) {
            if (c >= p) break;
            auto vx = acc[c].x, vy = acc[c].y;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                vx += __shfl_down_sync(0xffffffffu, vx, o);
                vy += __shfl_down_sync(0xffffffffu, vy, o);
            }
            if (lane == 0) t[(size_t)(toff[b] + l) * NB + c] = mk<C>(vx, vy);
        }
    }
}

// One CTA per leaf row cluster: rows [rs, re) in cluster order.  The CTA has ng
// groups of rt threads (rt = the largest leaf, a warp multiple); thread r of group g
// owns row r and the columns jj = g, g + ng, ... of every staged chunk, so ng loads
// of each row are in flight at once.  The ng partial sums are added in a fixed
// order at the end (group 0 takes those of groups 1, 2, ... in turn).
// Dynamic shared memory: max(kHmStage, rt) x NB complex values.
constexpr int kHmStage = 128;   // columns staged per step
template <typename R, int NB>
__global__ void __launch_bounds__(512) k_hm_rows(int m, int p, const int* __restrict__ perm,
                                                  const int* __restrict__ rl, const int* __restrict__ eptr,
                                                  const int* __restrict__ eblk, const int* __restrict__ eroff,
                                                  const int4* __restrict__ blk, const int* __restrict__ kb,
                                                  const int64_t* __restrict__ doff, const cx<R>* __restrict__ D,
                                                  const cx<R>* __restrict__ U, const int* __restrict__ toff,
                                                  const cx<R>* __restrict__ t, const cx<R>* __restrict__ xt,
                                                  cx<R>* __restrict__ Y, int64_t ldy, int rt) {
    using C = cx<R>;
    extern __shared__ __align__(16) unsigned char hm_smem[];
    C* sx = reinterpret_cast<C*>(hm_smem);
    const int L = blockIdx.x;
    const int rs = rl[L], nr = rl[L + 1] - rs;
    const int ng = blockDim.x / rt;
    const int grp = threadIdx.x / rt, r = threadIdx.x - grp * rt;
    C acc[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) acc[c] = czero<C>();
    for (int e = eptr[L]; e < eptr[L + 1]; ++e) {
        const int b = eblk[e], ro = eroff[e];
        const int4 B = blk[b];
        const int k = kb[b];
        const C* Ab = (k < 0 ? D : U) + doff[b];
        const int ncol = k < 0 ? B.w : k;
        for (int j0 = 0; j0 < ncol; j0 += kHmStage) {
            const int nj = min(kHmStage, ncol - j0);
            __syncthreads();
            for (int q = threadIdx.x; q < nj * NB; q += blockDim.x) {
                const int jj = q / NB, c = q - jj * NB;
                C v = czero<C>();
                if (c < p) v = k < 0 ? xt[(size_t)c * m + B.z + j0 + jj] : t[(size_t)(toff[b] + j0 + jj) * NB + c];
                sx[q] = v;
            }
            __syncthreads();
            if (r < nr) {
                const C* a = Ab + (size_t)(ro + r) + (size_t)B.y * j0;
                for (int jj = grp; jj < nj; jj += ng) {
                    const C av = a[(size_t)B.y * jj];
#pragma unroll
                    for (int c = 0; c < NB; ++c) cfma(acc[c], av, sx[jj * NB + c]);
                }
            }
        }
    }
    for (int g = 1; g < ng; ++g) {
        __syncthreads();
        if (grp == g && r < nr) {
#pragma unroll
            for (int c = 0; c < NB; ++c) sx[r * NB + c] = acc[c];
        }
        __syncthreads();
        if (grp == 0 && r < nr) {
#pragma unroll
            for (int c = 0; c < NB; ++c) acc[c] = cadd(acc[c], sx[r * NB + c]);
        }
    }
    if (grp == 0 && r < nr) {
        const int row = perm[rs + r];
#pragma unroll
        for (int c = 0; c < NB; ++c)
            if (c < p) Y[(size_t)c * ldy + row] = acc[c];
    }
}

// ------------------------------------------------------------------ build and apply
template <typename T>
static T* hm_up(Ctx& c, const std::vector<T>& v) {
    T* d = (T*)dalloc(c, std::max<size_t>(v.size(), 1) * sizeof(T));
    if (!v.empty()) VSIE_CUDA(cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return d;
}

void hm_build(Ctx& c, const HmPlan& P, const double2* dZ, int64_t ldz, double tol) {
    HmDev& H = c.hm;
    H.m = P.m;
    H.nrl = (int)P.rl_start.size() - 1;
    const int nb = (int)P.blk.size();
    H.nblk = nb;
    std::vector<int4> blk(nb);
    for (int b = 0; b < nb; ++b) blk[b] = make_int4(P.blk[b].r0, P.blk[b].nr, P.blk[b].c0, P.blk[b].nc);
    H.perm = hm_up(c, P.perm);
    H.rl = hm_up(c, P.rl_start);
    H.blk = hm_up(c, blk);
    // ---- low-rank blocks by ACA, in batches that bound the scratch
    constexpr int kCap = 96;
    std::vector<int> kb(nb, -1);   // -1: dense
    std::vector<int> lr_try;
    for (int b = 0; b < nb; ++b)
        if (!P.blk[b].dense) lr_try.push_back(b);
    std::vector<std::vector<double2>> hU(nb), hV(nb);   // compact factors of the low-rank blocks (host)
    {
        Ctx S;   // scratch allocations of the build
        S.device = c.device;
        try {
            size_t cap = 0;
            for (int b : lr_try) cap = std::max(cap, (size_t)(P.blk[b].nr + P.blk[b].nc) * std::min({kCap, P.blk[b].nr, P.blk[b].nc}));
            const size_t budget = std::max<size_t>(cap, (size_t)96 << 20);   // complex values per batch
            double2* Us = (double2*)dalloc(S, budget * sizeof(double2));   // U then V of each block
            unsigned char* fl = (unsigned char*)dalloc(S, (size_t)2 * P.m * std::max<size_t>(lr_try.size(), 1) + 16);
            size_t q0 = 0;
            while (q0 < lr_try.size()) {
                std::vector<int> ids, kc;
                std::vector<int64_t> uo, vo, fo;
                size_t used = 0, fused = 0;
                size_t q = q0;
                while (q < lr_try.size()) {
                    const auto& B = P.blk[lr_try[q]];
                    const int K = std::min({kCap, B.nr, B.nc});
                    const size_t need = (size_t)(B.nr + B.nc) * K;
                    if (used + need > budget && !ids.empty()) break;
                    ids.push_back(lr_try[q]);
                    kc.push_back(K);
                    uo.push_back((int64_t)used);
                    vo.push_back((int64_t)(used + (size_t)B.nr * K));
                    fo.push_back((int64_t)fused);
                    used += need;
                    fused += B.nr + B.nc;
                    ++q;
                }
                int* d_ids = hm_up(S, ids);
                int* d_kc = hm_up(S, kc);
                int64_t* d_uo = hm_up(S, uo);
                int64_t* d_fo = hm_up(S, fo);
                int* d_rank = (int*)dalloc(S, ids.size() * sizeof(int));
                k_hm_aca<<<(unsigned)ids.size(), kAcaThreads>>>(dZ, ldz, H.perm, H.blk, d_ids, d_uo,
                                                                hm_up(S, vo), d_fo, d_kc, tol, Us, Us, fl, d_rank);
                VSIE_CUDA(cudaGetLastError());
                std::vector<int> rk(ids.size());
                VSIE_CUDA(cudaMemcpy(rk.data(), d_rank, rk.size() * sizeof(int), cudaMemcpyDeviceToHost));
                for (size_t t = 0; t < ids.size(); ++t) {
                    const int b = ids[t];
                    if (rk[t] < 0) continue;   // stays dense
                    const auto& B = P.blk[b];
                    kb[b] = rk[t];
                    hU[b].resize((size_t)B.nr * rk[t]);
                    hV[b].resize((size_t)B.nc * rk[t]);
                    if (rk[t] > 0) {
                        VSIE_CUDA(cudaMemcpy(hU[b].data(), Us + uo[t], hU[b].size() * sizeof(double2), cudaMemcpyDeviceToHost));
                        VSIE_CUDA(cudaMemcpy(hV[b].data(), Us + vo[t], hV[b].size() * sizeof(double2), cudaMemcpyDeviceToHost));
                    }
                }
                for (void* ptr : S.allocs)
                    if (ptr != Us && ptr != fl) cudaFree(ptr);
                S.allocs = {Us, fl};
                q0 = q;
            }
        } catch (...) {
            for (void* ptr : S.allocs) cudaFree(ptr);
            throw;
        }
        for (void* ptr : S.allocs) cudaFree(ptr);
        S.allocs.clear();
    }
    // ---- layout: dense blocks in D, factors in U and V, t offsets of the low-rank blocks
    std::vector<int64_t> doff(nb, 0), voff(nb, 0);
    std::vector<int> toff(nb, 0), dense_ids, lr_ids;
    int64_t nD = 0, nU = 0, nV = 0;
    int nt = 0;
    for (int b = 0; b < nb; ++b) {
        const auto& B = P.blk[b];
        if (kb[b] < 0) {
            doff[b] = nD;
            nD += (int64_t)B.nr * B.nc;
            dense_ids.push_back(b);
        } else {
            doff[b] = nU;
            voff[b] = nV;
            toff[b] = nt;
            nU += (int64_t)B.nr * kb[b];
            nV += (int64_t)B.nc * kb[b];
            nt += kb[b];
            if (kb[b] > 0) lr_ids.push_back(b);
        }
    }
    std::vector<int64_t> dense_off;
    for (int b : dense_ids) dense_off.push_back(doff[b]);
    H.nlr = (int)lr_ids.size();
    H.nt = nt;
    H.kb = hm_up(c, kb);
    H.doff = hm_up(c, doff);
    H.voff = hm_up(c, voff);
    H.toff = hm_up(c, toff);
    H.lr = hm_up(c, lr_ids);
    std::vector<int> eptr, eb, ero;
    hm_entries(P, eptr, eb, ero);
    H.eptr = hm_up(c, eptr);
    H.eblk = hm_up(c, eb);
    H.eroff = hm_up(c, ero);
    H.nD = nD;
    H.nU = nU;
    H.nV = nV;
    // FP64 data
    H.D64 = (double2*)dalloc(c, std::max<int64_t>(nD, 1) * sizeof(double2));
    H.U64 = (double2*)dalloc(c, std::max<int64_t>(nU, 1) * sizeof(double2));
    H.V64 = (double2*)dalloc(c, std::max<int64_t>(nV, 1) * sizeof(double2));
    if (!dense_ids.empty()) {
        int* d_ids = hm_up(c, dense_ids);
        k_hm_dense<<<(unsigned)dense_ids.size(), 256>>>(dZ, ldz, H.perm, H.blk, H.doff, d_ids, H.D64);
        VSIE_CUDA(cudaGetLastError());
    }
    {
        std::vector<double2> u((size_t)nU), v((size_t)nV);
        for (int b = 0; b < nb; ++b) {
            if (kb[b] <= 0) continue;
            std::copy(hU[b].begin(), hU[b].end(), u.begin() + doff[b]);
            std::copy(hV[b].begin(), hV[b].end(), v.begin() + voff[b]);
        }
        if (nU) VSIE_CUDA(cudaMemcpy(H.U64, u.data(), u.size() * sizeof(double2), cudaMemcpyHostToDevice));
        if (nV) VSIE_CUDA(cudaMemcpy(H.V64, v.data(), v.size() * sizeof(double2), cudaMemcpyHostToDevice));
    }
    // FP32 copies
    H.D32 = (float2*)dalloc(c, std::max<int64_t>(nD, 1) * sizeof(float2));
    H.U32 = (float2*)dalloc(c, std::max<int64_t>(nU, 1) * sizeof(float2));
    H.V32 = (float2*)dalloc(c, std::max<int64_t>(nV, 1) * sizeof(float2));
    k_hm_narrow<<<2048, 256>>>(H.D64, H.D32, (size_t)nD);
    k_hm_narrow<<<2048, 256>>>(H.U64, H.U32, (size_t)nU);
    k_hm_narrow<<<2048, 256>>>(H.V64, H.V32, (size_t)nV);
    VSIE_CUDA(cudaGetLastError());
    // work buffers for 16 right-hand sides per pass
    H.xt64 = (double2*)dalloc(c, (size_t)P.m * 16 * sizeof(double2));
    H.t64 = (double2*)dalloc(c, (size_t)std::max(nt, 1) * 16 * sizeof(double2));
    H.xt32 = (float2*)H.xt64;   // FP32 and FP64 products never run at the same time
    H.t32 = (float2*)H.t64;
    H.ndense = (int)dense_ids.size();
    {   // one thread per row of the largest leaf row cluster (a warp multiple)
        int mr = 1;
        for (size_t l = 0; l + 1 < P.rl_start.size(); ++l) mr = std::max(mr, P.rl_start[l + 1] - P.rl_start[l]);
        H.rows_threads = std::min(256, (mr + 31) / 32 * 32);
    }
    VSIE_CUDA(cudaDeviceSynchronize());
    H.on = true;
    if (std::getenv("VSIE_TRACE")) {
        int kmax = 0, nfall = 0;
        for (int b = 0; b < nb; ++b) kmax = std::max(kmax, kb[b]);
        for (int b : lr_try) nfall += kb[b] < 0;
        fprintf(stderr, "[vsie H] m %d leaves %d blocks %d (dense %d, low rank %d, ACA fallbacks %d) max rank %d, "
                        "%.3f GB FP64 data (dense-block equivalent %.3f GB)\n",
                P.m, H.nrl, nb, H.ndense, H.nlr, nfall, kmax, (nD + nU + nV) * 16.0 / 1e9,
                (double)P.m * P.m * 16.0 / 1e9);
    }
}

template <typename R>
void hm_apply(Ctx& c, int p, const cx<R>* X, int64_t ldx, cx<R>* Y, int64_t ldy, cudaStream_t st) {
    HmDev& H = c.hm;
    const cx<R>* D = sizeof(R) == 8 ? (const cx<R>*)H.D64 : (const cx<R>*)H.D32;
    const cx<R>* U = sizeof(R) == 8 ? (const cx<R>*)H.U64 : (const cx<R>*)H.U32;
    const cx<R>* V = sizeof(R) == 8 ? (const cx<R>*)H.V64 : (const cx<R>*)H.V32;
    cx<R>* xt = sizeof(R) == 8 ? (cx<R>*)H.xt64 : (cx<R>*)H.xt32;
    cx<R>* t = sizeof(R) == 8 ? (cx<R>*)H.t64 : (cx<R>*)H.t32;
    for (int c0 = 0; c0 < p; c0 += 16) {
        const int pc = std::min(16, p - c0);
        const cx<R>* Xc = X + (size_t)c0 * ldx;
        cx<R>* Yc = Y + (size_t)c0 * ldy;
        const int64_t tot = (int64_t)H.m * pc;
        k_hm_gather<R><<<(int)std::min<int64_t>((tot + 255) / 256, 152 * 16), 256, 0, st>>>(H.m, pc, H.perm, Xc, ldx, xt);
        const int rt = H.rows_threads, ng = std::max(1, std::min(4, 512 / rt));
        if (pc <= 8) {
            const size_t sm = (size_t)std::max(kHmStage, rt) * 8 * sizeof(cx<R>);
            if (sm > 48 * 1024)
                VSIE_CUDA(cudaFuncSetAttribute(k_hm_rows<R, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            if (H.nlr) k_hm_vt<R, 8><<<H.nlr, 256, 0, st>>>(H.m, pc, H.lr, H.blk, H.kb, H.voff, H.toff, V, xt, t);
            k_hm_rows<R, 8><<<H.nrl, rt * ng, sm, st>>>(H.m, pc, H.perm, H.rl, H.eptr, H.eblk, H.eroff, H.blk, H.kb,
                                                        H.doff, D, U, H.toff, t, xt, Yc, ldy, rt);
        } else {
            const size_t sm = (size_t)std::max(kHmStage, rt) * 16 * sizeof(cx<R>);
            if (sm > 48 * 1024)
                VSIE_CUDA(cudaFuncSetAttribute(k_hm_rows<R, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            if (H.nlr) k_hm_vt<R, 16><<<H.nlr, 256, 0, st>>>(H.m, pc, H.lr, H.blk, H.kb, H.voff, H.toff, V, xt, t);
            k_hm_rows<R, 16><<<H.nrl, rt * ng, sm, st>>>(H.m, pc, H.perm, H.rl, H.eptr, H.eblk, H.eroff, H.blk, H.kb,
                                                         H.doff, D, U, H.toff, t, xt, Yc, ldy, rt);
        }
        prof_count(c, H.nlr ? 3 : 2);
    }
    VSIE_CUDA(cudaGetLastError());
}

template void hm_apply<float>(Ctx&, int, const float2*, int64_t, float2*, int64_t, cudaStream_t);
template void hm_apply<double>(Ctx&, int, const double2*, int64_t, double2*, int64_t, cudaStream_t);

}  // namespace vsie
