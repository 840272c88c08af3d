// Set-up assembly kernels (FP64): Galerkin EFIE entries between RWG functions
// (Eq. sie / Eq. disc_sie) and body-surface coupling entries (Eq. nvsie,
// Sec. IV.C quadrature), evaluated on the GPU.
//
// EFIE:  K_mn = <f_m, Gop f_n> = k0^2 \int\int f_m . f_n g - \int\int div f_m div' f_n g,
// written per triangle pair (T, T') through the moments (local coordinates
// about the centroids c, c')
//   A0 = \int\int g,  A1 = \int\int (r - c) g,  B1 = \int\int (r' - c') g,
//   C  = \int\int (r - c).(r' - c') g,
// so that with f = s l / (2A) (r - v):
//   contribution = s s' l l' / (4 A A') [ k0^2 (C - v'.A1 - v.B1 + v.v' A0) - 4 A0 ]
// (v, v' the free vertices relative to c, c').  Quadrature tier per pair, from
// the centroid distance d and the longer triangle diameter D:
//   near (shared vertex, or d < 2D): outer 7-point rule, inner 7-point rule on
//        g - 1/(4 pi R) plus analytic 1/R integrals, averaged with the same rule
//        with T and T' swapped (keeps K symmetric);
//   mid  (d < 6D): 6 x 6 points;   far: centroid x centroid.
// Analytic 1/R integrals over a flat triangle (Wilton et al. 1984, Graglia 1993):
//   I0 = sum_e t f - |d| sum_e [atan(t s+ / (R0^2 + |d| R+)) - atan(t s- / (R0^2 + |d| R-))],
//   I1 = (1/2) sum_e u (R0^2 f + s+ R+ - s- R-) - d n I0,
//   f = ln((R+ + s+) / (R- + s-)) (or the equal ratio (R- - s-)/(R+ - s+) when s+ + s- < 0).
//
// Coupling: K[(p, a), n] = \int_{V_p} [Gop f_n]_a dV with
//   Gop f (r) = k0^2 \int g f + \int (div' f) grad_r g,
// near: 2x2x2 Gauss points in the voxel x 6-point rule; far: centre x centroid.
#include "setup.h"

#include <cmath>

namespace vsie {

struct DQuad {
    int n;
    double b[7][3];
    double w[7];
};

// Published rules (weights sum to 1): Dunavant degree 4 (6 points), Radon
// degree 5 (7 points), centroid.
__constant__ DQuad c_rules[3];

static DQuad make_rule(int which) {
    DQuad q{};
    auto sym = [&](int& k, double a, double b, double w) {
        const double t[3][3] = {{a, b, b}, {b, a, b}, {b, b, a}};
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) q.b[k][j] = t[i][j];
            q.w[k++] = w;
        }
    };
    int k = 0;
    if (which == 0) {
        q.b[0][0] = q.b[0][1] = q.b[0][2] = 1.0 / 3.0;
        q.w[0] = 1.0;
        k = 1;
    } else if (which == 1) {
        sym(k, 0.108103018168070, 0.445948490915965, 0.223381589678011);
        sym(k, 0.816847572980459, 0.091576213509771, 0.109951743655322);
    } else {
        q.b[0][0] = q.b[0][1] = q.b[0][2] = 1.0 / 3.0;
        q.w[0] = 0.225;
        k = 1;
        sym(k, 0.059715871789770, 0.470142064105115, 0.132394152788506);
        sym(k, 0.797426985353087, 0.101286507323456, 0.125939180544827);
    }
    q.n = k;
    return q;
}

void upload_rules() {
    static bool done = false;
    if (done) return;
    DQuad r[3] = {make_rule(0), make_rule(1), make_rule(2)};
    VSIE_CUDA(cudaMemcpyToSymbol(c_rules, r, sizeof(r)));
    done = true;
}

struct V3 { double x, y, z; };
__device__ __forceinline__ V3 v3(const double* p) { return {p[0], p[1], p[2]}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double norm(V3 a) { return sqrt(dot(a, a)); }

struct CV3 { double2 x, y, z; };
__device__ __forceinline__ void cv_add(CV3& a, double2 s, V3 v) {
    a.x = cadd(a.x, cscale(s, v.x));
    a.y = cadd(a.y, cscale(s, v.y));
    a.z = cadd(a.z, cscale(s, v.z));
}
__device__ __forceinline__ double2 cv_dot(CV3 a, V3 v) {
    return cadd(cadd(cscale(a.x, v.x), cscale(a.y, v.y)), cscale(a.z, v.z));
}

// g(R) = exp(-i k R) / (4 pi R)
__device__ __forceinline__ double2 green(double R, double k0) {
    double s, c;
    sincos(k0 * R, &s, &c);
    const double f = 1.0 / (4.0 * M_PI * R);
    return make_double2(f * c, -f * s);
}
// g(R) - 1/(4 pi R) without cancellation; -i k / (4 pi) at R = 0
__device__ __forceinline__ double2 green_smooth(double R, double k0) {
    if (R == 0.0) return make_double2(0.0, -k0 / (4.0 * M_PI));
    double s, c;
    sincos(0.5 * k0 * R, &s, &c);
    const double f = 1.0 / (4.0 * M_PI * R);
    // exp(-i kR) - 1 = -2 sin^2(kR/2) - i sin(kR),  sin(kR) = 2 s c
    return make_double2(-2.0 * s * s * f, -2.0 * s * c * f);
}

__device__ void tri_point(const MeshDev& m, int t, int rule, int q, V3& p, double& w) {
    const int* v = m.tri + 3 * t;
    const V3 a = v3(m.xyz + 3 * v[0]), b = v3(m.xyz + 3 * v[1]), c = v3(m.xyz + 3 * v[2]);
    const DQuad& Q = c_rules[rule];
    p = Q.b[q][0] * a + Q.b[q][1] * b + Q.b[q][2] * c;
    w = Q.w[q] * m.area[t];
}

// analytic I0 = \int_T 1/R, I1 = \int_T (r' - r)/R for observation r
__device__ void potint(const MeshDev& m, int t, V3 r, double& I0, V3& I1) {
    const int* vi = m.tri + 3 * t;
    V3 P[3] = {v3(m.xyz + 3 * vi[0]), v3(m.xyz + 3 * vi[1]), v3(m.xyz + 3 * vi[2])};
    const V3 n = v3(m.normal + 3 * t);
    const double d = dot(r - P[0], n);
    const V3 rho = r - d * n;
    const double ad = fabs(d);
    double s0 = 0.0;
    V3 iv = {0, 0, 0};
    for (int k = 0; k < 3; ++k) {
        const V3 a = P[k], b = P[(k + 1) % 3];
        V3 l = b - a;
        l = (1.0 / norm(l)) * l;
        const V3 u = cross(l, n);
        const double sp = dot(b - rho, l), sm = dot(a - rho, l), tt = dot(a - rho, u);
        const double R0sq = tt * tt + d * d;
        const double Rp = norm(b - r), Rm = norm(a - r);
        double f;
        if (sp + sm >= 0.0) f = log(fmax(Rp + sp, 1e-300) / fmax(Rm + sm, 1e-300));
        else f = log(fmax(Rm - sm, 1e-300) / fmax(Rp - sp, 1e-300));
        s0 += tt * f - ad * (atan2(tt * sp, R0sq + ad * Rp) - atan2(tt * sm, R0sq + ad * Rm));
        iv = iv + (0.5 * (R0sq * f + sp * Rp - sm * Rm)) * u;
    }
    I0 = s0;
    I1 = iv - (d * s0) * n;
}

struct Mom { double2 A0; CV3 A1, B1; double2 C; };

__device__ __forceinline__ void mom_zero(Mom& M) {
    const double2 z = make_double2(0, 0);
    M.A0 = M.C = z;
    M.A1 = {z, z, z};
    M.B1 = {z, z, z};
}

__device__ void mom_regular(const MeshDev& ma, int ta, const MeshDev& mb, int tb, int rule,
                            double k0, Mom& M) {
    mom_zero(M);
    const V3 ca = v3(ma.centroid + 3 * ta), cb = v3(mb.centroid + 3 * tb);
    const int n = c_rules[rule].n;
    for (int i = 0; i < n; ++i) {
        V3 pa;
        double wa;
        tri_point(ma, ta, rule, i, pa, wa);
        const V3 la = pa - ca;
        for (int j = 0; j < n; ++j) {
            V3 pb;
            double wb;
            tri_point(mb, tb, rule, j, pb, wb);
            const V3 lb = pb - cb;
            const double2 G = cscale(green(norm(pa - pb), k0), wa * wb);
            M.A0 = cadd(M.A0, G);
            cv_add(M.A1, G, la);
            cv_add(M.B1, G, lb);
            M.C = cadd(M.C, cscale(G, dot(la, lb)));
        }
    }
}

// one direction: outer rule on ta, inner smooth rule + analytic on tb
__device__ void mom_singular_dir(const MeshDev& ma, int ta, const MeshDev& mb, int tb, double k0,
                                 Mom& M) {
    mom_zero(M);
    const V3 ca = v3(ma.centroid + 3 * ta), cb = v3(mb.centroid + 3 * tb);
    const int n = c_rules[2].n;
    for (int i = 0; i < n; ++i) {
        V3 pa;
        double wa;
        tri_point(ma, ta, 2, i, pa, wa);
        double2 J0 = make_double2(0, 0);
        CV3 J1 = {J0, J0, J0};
        for (int j = 0; j < n; ++j) {
            V3 pb;
            double wb;
            tri_point(mb, tb, 2, j, pb, wb);
            const double2 G = cscale(green_smooth(norm(pa - pb), k0), wb);
            J0 = cadd(J0, G);
            cv_add(J1, G, pb - cb);
        }
        double I0;
        V3 I1;
        potint(mb, tb, pa, I0, I1);
        const double q = 1.0 / (4.0 * M_PI);
        J0.x += q * I0;
        const V3 w1 = I1 + I0 * (pa - cb);
        J1.x.x += q * w1.x;
        J1.y.x += q * w1.y;
        J1.z.x += q * w1.z;
        const V3 la = pa - ca;
        M.A0 = cadd(M.A0, cscale(J0, wa));
        cv_add(M.A1, cscale(J0, wa), la);
        M.B1.x = cadd(M.B1.x, cscale(J1.x, wa));
        M.B1.y = cadd(M.B1.y, cscale(J1.y, wa));
        M.B1.z = cadd(M.B1.z, cscale(J1.z, wa));
        M.C = cadd(M.C, cscale(cv_dot(J1, la), wa));
    }
}

__device__ void tri_pair_moments(const MeshDev& ma, int ta, const MeshDev& mb, int tb, bool same,
                                 double k0, Mom& M) {
    const V3 ca = v3(ma.centroid + 3 * ta), cb = v3(mb.centroid + 3 * tb);
    const double d = norm(ca - cb);
    const double D = fmax(ma.diam[ta], mb.diam[tb]);
    int tier = d < 2.0 * D ? 0 : (d < 6.0 * D ? 1 : 2);
    if (same) {
        const int* va = ma.tri + 3 * ta;
        const int* vb = mb.tri + 3 * tb;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                if (va[i] == vb[j]) tier = 0;
    }
    if (tier == 2) {
        mom_regular(ma, ta, mb, tb, 0, k0, M);
    } else if (tier == 1) {
        mom_regular(ma, ta, mb, tb, 1, k0, M);
    } else {
        Mom f, b;
        mom_singular_dir(ma, ta, mb, tb, k0, f);
        mom_singular_dir(mb, tb, ma, ta, k0, b);
        M.A0 = cscale(cadd(f.A0, b.A0), 0.5);
        M.C = cscale(cadd(f.C, b.C), 0.5);
        M.A1.x = cscale(cadd(f.A1.x, b.B1.x), 0.5);
        M.A1.y = cscale(cadd(f.A1.y, b.B1.y), 0.5);
        M.A1.z = cscale(cadd(f.A1.z, b.B1.z), 0.5);
        M.B1.x = cscale(cadd(f.B1.x, b.A1.x), 0.5);
        M.B1.y = cscale(cadd(f.B1.y, b.A1.y), 0.5);
        M.B1.z = cscale(cadd(f.B1.z, b.A1.z), 0.5);
    }
}

// K[rows, cols] (or -K when negate) into out (column-major, ld = ldo); rows of
// RWG set a, columns of RWG set b.
__global__ void k_efie(MeshDev ma, MeshDev mb, bool same, int nr, const int* __restrict__ rows,
                       int nc, const int* __restrict__ cols, double k0, double sign,
                       double2* __restrict__ out, int64_t ldo) {
    const int64_t tot = (int64_t)nr * nc;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int ir = e % nr, ic = e / nr;
        const int m = rows ? rows[ir] : ir;
        const int n = cols ? cols[ic] : ic;
        double2 acc = make_double2(0, 0);
        for (int ha = 0; ha < 2; ++ha) {
            const int ta = ha == 0 ? ma.tplus[m] : ma.tminus[m];
            const int va = ha == 0 ? ma.vplus[m] : ma.vminus[m];
            const double sa = ha == 0 ? 1.0 : -1.0;
            const V3 vra = v3(ma.xyz + 3 * va) - v3(ma.centroid + 3 * ta);
            for (int hb = 0; hb < 2; ++hb) {
                const int tb = hb == 0 ? mb.tplus[n] : mb.tminus[n];
                const int vb = hb == 0 ? mb.vplus[n] : mb.vminus[n];
                const double sb = hb == 0 ? 1.0 : -1.0;
                const V3 vrb = v3(mb.xyz + 3 * vb) - v3(mb.centroid + 3 * tb);
                Mom M;
                tri_pair_moments(ma, ta, mb, tb, same, k0, M);
                const double2 vv = cadd(csub(csub(M.C, cv_dot(M.A1, vrb)), cv_dot(M.B1, vra)),
                                        cscale(M.A0, dot(vra, vrb)));
                const double pre = sa * sb * ma.len[m] * mb.len[n] / (4.0 * ma.area[ta] * mb.area[tb]);
                const double2 t = csub(cscale(vv, k0 * k0), cscale(M.A0, 4.0));
                acc = cadd(acc, cscale(t, pre));
            }
        }
        out[(size_t)ir + (size_t)ic * ldo] = cscale(acc, sign);
    }
}

// Gop f_n at point r (one RWG, rule for its triangles)
__device__ void gop_rwg(const MeshDev& m, int n, V3 r, int rule, double k0, double2 E[3]) {
    E[0] = E[1] = E[2] = make_double2(0, 0);
    for (int h = 0; h < 2; ++h) {
        const int t = h == 0 ? m.tplus[n] : m.tminus[n];
        const int v = h == 0 ? m.vplus[n] : m.vminus[n];
        const double s = h == 0 ? 1.0 : -1.0;
        const V3 pv = v3(m.xyz + 3 * v);
        const double l = m.len[n], A = m.area[t];
        const int nq = c_rules[rule].n;
        for (int q = 0; q < nq; ++q) {
            V3 p;
            double w;
            tri_point(m, t, rule, q, p, w);
            const V3 Rv = r - p;
            const double R = norm(Rv);
            const double2 g = cscale(green(R, k0), w);
            // k0^2 s l/(2A) g (p - v)
            const double c1 = k0 * k0 * s * l / (2.0 * A);
            const V3 f = p - pv;
            // (s l / A) g * (-(1 + i k R) / R^2) Rv
            const double c2 = s * l / A / (R * R);
            const double2 gk = cmul(g, make_double2(-1.0, -k0 * R));   // -(1 + i kR) g
            E[0] = cadd(E[0], cadd(cscale(g, c1 * f.x), cscale(gk, c2 * Rv.x)));
            E[1] = cadd(E[1], cadd(cscale(g, c1 * f.y), cscale(gk, c2 * Rv.y)));
            E[2] = cadd(E[2], cadd(cscale(g, c1 * f.z), cscale(gk, c2 * Rv.z)));
        }
    }
}

// Coupling block: out[a][iv + ldo * ic] (component-major planes, plane stride
// pstride) = sign * K[(vox[iv], a), cols[ic]]; with only >= 0 just that
// component is written, at out[iv + ldo * ic].
__global__ void k_coupling(MeshDev m, GridDev g, int nvx, const int64_t* __restrict__ vox, int nc,
                           const int* __restrict__ cols, double k0, bool near, double sign,
                           double2* __restrict__ out, int64_t ldo, int64_t pstride, int only) {
    const int64_t tot = (int64_t)nvx * nc;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int iv = e % nvx, ic = e / nvx;
        const int64_t v = vox ? vox[iv] : iv;
        const int n = cols ? cols[ic] : ic;
        const int i1 = v % g.n[0];
        const int i2 = (v / g.n[0]) % g.n[1];
        const int i3 = v / ((int64_t)g.n[0] * g.n[1]);
        const V3 c = {g.origin[0] + g.h * i1, g.origin[1] + g.h * i2, g.origin[2] + g.h * i3};
        double2 acc[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
        if (near) {
            const double o = 0.5 * g.h / sqrt(3.0);
            for (int q = 0; q < 8; ++q) {
                const V3 p = {c.x + ((q & 1) ? o : -o), c.y + ((q & 2) ? o : -o),
                              c.z + ((q & 4) ? o : -o)};
                double2 E[3];
                gop_rwg(m, n, p, 1, k0, E);
                for (int a = 0; a < 3; ++a) acc[a] = cadd(acc[a], cscale(E[a], 0.125));
            }
        } else {
            gop_rwg(m, n, c, 0, k0, acc);
        }
        const double h3 = g.h * g.h * g.h * sign;
        if (only >= 0) {
            out[(size_t)iv + (size_t)ic * ldo] = cscale(acc[only], h3);
        } else {
            for (int a = 0; a < 3; ++a)
                out[(size_t)a * pstride + (size_t)iv + (size_t)ic * ldo] = cscale(acc[a], h3);
        }
    }
}

// Field Gop f_n at points ctr[ic] + pts[ip] (pFFT fit): out[3 np ic + a np + ip]
__global__ void k_field_points(MeshDev m, int np, const double* __restrict__ pts, int nc,
                               const int* __restrict__ cols, const double* __restrict__ ctr,
                               double k0, double2* __restrict__ out) {
    const int64_t tot = (int64_t)np * nc;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int ip = e % np, ic = e / np;
        const int n = cols ? cols[ic] : ic;
        const V3 r = {ctr[3 * ic] + pts[3 * ip], ctr[3 * ic + 1] + pts[3 * ip + 1],
                      ctr[3 * ic + 2] + pts[3 * ip + 2]};
        double2 E[3];
        gop_rwg(m, n, r, 1, k0, E);
        for (int a = 0; a < 3; ++a) out[(size_t)3 * np * ic + (size_t)a * np + ip] = E[a];
    }
}

// Tested incident plane wave (Sec. II.A; the conductor rows of Eq. (hvsie)):
// out[m] = scale \int f_m . e0 exp(-i k0 khat . r) dS over both triangles of RWG
// m, by the 6-point rule.  geo holds, per RWG and per half (T+, then T-), the
// three vertices, the free vertex and s l / 2 (13 doubles), so that
// \int_T f . E dS = (s l / 2) sum_q w_q (r_q - v) . E(r_q) (rule weights sum to 1).
__global__ void k_pw_surface(int m, const double* __restrict__ geo, V3 khat, V3 e0, double k0,
                             double2 scale, double2* __restrict__ out) {
    const DQuad& Q = c_rules[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int hf = 0; hf < 2; ++hf) {
            const double* g = geo + (size_t)26 * i + 13 * hf;
            const V3 a = v3(g), b = v3(g + 3), c = v3(g + 6), v = v3(g + 9);
            const double sl2 = g[12];
            for (int q = 0; q < Q.n; ++q) {
                const V3 r = Q.b[q][0] * a + Q.b[q][1] * b + Q.b[q][2] * c;
                double sn, cs;
                sincos(k0 * dot(khat, r), &sn, &cs);
                const double f = Q.w[q] * sl2 * dot(r - v, e0);
                acc.x += f * cs;    // exp(-i phi) = cos phi - i sin phi
                acc.y -= f * sn;
            }
        }
        out[i] = cmul(scale, acc);
    }
}

void planewave_surface(int m, const double* geo, const double khat[3], const double e0[3], double k0,
                       double2 scale, double2* out, cudaStream_t st) {
    upload_rules();
    if (m <= 0) return;
    const V3 kh = {khat[0], khat[1], khat[2]}, e = {e0[0], e0[1], e0[2]};
    k_pw_surface<<<(m + 127) / 128, 128, 0, st>>>(m, geo, kh, e, k0, scale, out);
    VSIE_CUDA(cudaGetLastError());
}

// Grid part of the near block, summed directly over stencil pairs (the pFFT
// reading of Sec. III with Z_nn dense): for near RWG m, n with stencils S_m, S_n
// (voxel s^3 blocks at base_m, base_n of the extended grid) and weights W,
//   Z[m + ld n] += h^3 sum_{a, q in S_m} sum_{b, q' in S_n}
//                  W[m][a s^3 + q] T_ab(q - q') W[n][b s^3 + q'],
// with T the voxel kernel of the body operator (T(d) = h^3 (k0^2 + grad grad) g
// at d h, the equal-volume-sphere self term at d = 0).  This equals h^3 P^T K P
// through the aperiodic grid convolution exactly (the embedding adds no
// periodic images), at a cost of m_n^2 (2 s - 1)^3 kernel values.  One CTA per
// row m (its weights in shared memory), threads over n.
__device__ void voxel_kernel6(int dx, int dy, int dz, double h, double k0, double2 selfv, double2 T[6]) {
    if (dx == 0 && dy == 0 && dz == 0) {
        T[0] = T[1] = T[2] = selfv;
        T[3] = T[4] = T[5] = make_double2(0.0, 0.0);
        return;
    }
    const double rx = h * dx, ry = h * dy, rz = h * dz;
    const double R2 = rx * rx + ry * ry + rz * rz;
    const double R = sqrt(R2);
    double sn, cs;
    sincos(k0 * R, &sn, &cs);
    const double pre = h * h * h / (4.0 * M_PI * R * R2);
    const double2 g = make_double2(pre * cs, -pre * sn);
    const double kR = k0 * R;
    const double2 A = cmul(g, make_double2(kR * kR - 1.0, -kR));
    const double2 B = cmul(g, make_double2(3.0 - kR * kR, 3.0 * kR));
    const double ux = rx / R, uy = ry / R, uz = rz / R;
    T[0] = cadd(A, cscale(B, ux * ux));
    T[1] = cadd(A, cscale(B, uy * uy));
    T[2] = cadd(A, cscale(B, uz * uz));
    T[3] = cscale(B, ux * uy);
    T[4] = cscale(B, ux * uz);
    T[5] = cscale(B, uy * uz);
}

__global__ void k_ptkp(int mn, int s, const double2* __restrict__ W, const int* __restrict__ base, double h,
                       double k0, double2 selfv, double2* __restrict__ Z, int64_t ldz) {
    extern __shared__ __align__(16) unsigned char ptkp_smem[];
    double2* wm = reinterpret_cast<double2*>(ptkp_smem);
    const int s3 = s * s * s, m = blockIdx.x;
    for (int i = threadIdx.x; i < 3 * s3; i += blockDim.x) wm[i] = W[(size_t)m * 3 * s3 + i];
    const int bm0 = base[3 * m], bm1 = base[3 * m + 1], bm2 = base[3 * m + 2];
    __syncthreads();
    const double h3 = h * h * h;
    for (int n = threadIdx.x; n < mn; n += blockDim.x) {
        const double2* wn = W + (size_t)n * 3 * s3;
        const int d0 = bm0 - base[3 * n], d1 = bm1 - base[3 * n + 1], d2 = bm2 - base[3 * n + 2];
        double2 acc = make_double2(0.0, 0.0);
        for (int ez = 1 - s; ez < s; ++ez)
            for (int ey = 1 - s; ey < s; ++ey)
                for (int ex = 1 - s; ex < s; ++ex) {
                    // q - q' = (ex, ey, ez) within the stencils
                    double2 T[6];
                    voxel_kernel6(d0 + ex, d1 + ey, d2 + ez, h, k0, selfv, T);
                    double2 C[3][3];
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) C[a][b] = make_double2(0.0, 0.0);
                    for (int qz = max(0, ez); qz < min(s, s + ez); ++qz)
                        for (int qy = max(0, ey); qy < min(s, s + ey); ++qy)
                            for (int qx = max(0, ex); qx < min(s, s + ex); ++qx) {
                                const int q = qx + s * (qy + s * qz);
                                const int qq = (qx - ex) + s * ((qy - ey) + s * (qz - ez));
                                for (int a = 0; a < 3; ++a) {
                                    const double2 wa = wm[a * s3 + q];
                                    for (int b = 0; b < 3; ++b) cfma(C[a][b], wa, wn[b * s3 + qq]);
                                }
                            }
                    // sum_ab T_ab C_ab with T symmetric: xx yy zz xy xz yz
                    cfma(acc, T[0], C[0][0]);
                    cfma(acc, T[1], C[1][1]);
                    cfma(acc, T[2], C[2][2]);
                    cfma(acc, T[3], cadd(C[0][1], C[1][0]));
                    cfma(acc, T[4], cadd(C[0][2], C[2][0]));
                    cfma(acc, T[5], cadd(C[1][2], C[2][1]));
                }
        double2* z = Z + (size_t)m + (size_t)n * ldz;
        *z = cadd(*z, cscale(acc, h3));
    }
}

void ptkp_add(int mn, int s, const double2* W, const int* base, double h, double k0, double2 selfv, double2* Z,
              int64_t ldz) {
    if (mn <= 0) return;
    const size_t sm = (size_t)3 * s * s * s * sizeof(double2);
    if (sm > 48 * 1024) VSIE_CUDA(cudaFuncSetAttribute(k_ptkp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_ptkp<<<mn, 128, sm>>>(mn, s, W, base, h, k0, selfv, Z, ldz);
    VSIE_CUDA(cudaGetLastError());
}

static int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 127) / 128, 152 * 64); }

void efie_block(const MeshDev& ma, const MeshDev& mb, bool same, int nr, const int* rows, int nc,
                const int* cols, double k0, double sign, double2* out, int64_t ldo) {
    upload_rules();
    if ((int64_t)nr * nc == 0) return;
    k_efie<<<grid_for((int64_t)nr * nc), 128>>>(ma, mb, same, nr, rows, nc, cols, k0, sign, out, ldo);
    VSIE_CUDA(cudaGetLastError());
}

void coupling_block(const MeshDev& m, const GridDev& g, int nvx, const int64_t* vox, int nc,
                    const int* cols, double k0, bool near, double sign, double2* out, int64_t ldo,
                    int64_t pstride, int only) {
    upload_rules();
    if ((int64_t)nvx * nc == 0) return;
    k_coupling<<<grid_for((int64_t)nvx * nc), 128>>>(m, g, nvx, vox, nc, cols, k0, near, sign, out,
                                                      ldo, pstride, only);
    VSIE_CUDA(cudaGetLastError());
}

void field_points(const MeshDev& m, int np, const double* pts, int nc, const int* cols,
                  const double* ctr, double k0, double2* out) {
    upload_rules();
    if ((int64_t)np * nc == 0) return;
    k_field_points<<<grid_for((int64_t)np * nc), 128>>>(m, np, pts, nc, cols, ctr, k0, out);
    VSIE_CUDA(cudaGetLastError());
}

}  // namespace vsie
