// vsie_rhs_planewave: the right-hand side of Eq. (hvsie) for an incident plane
// wave E_inc(r) = e0 exp(-i k0 khat . r) (Sec. II.A, time convention
// exp(+i omega t)).  With Z = D - K and E-field testing, the scattered field of
// the currents is Gop J / (i omega eps0), so
//   conductor row m:        i omega eps0 \int f_m . E_inc dS   (6-point rule per
//                           triangle, k_pw_surface in assemble.cu);
//   body row (voxel p, a):  i omega eps0 h^3 E_inc,a(r_p) on material voxels,
//                           0 on vacuum voxels (identity rows).
#include "setup.h"

#include <cmath>

namespace vsie {

__global__ void k_pw_body(int64_t nb, int n1, int n2, double h, double ox, double oy, double oz,
                          double kx, double ky, double kz, double ex, double ey, double ez, double k0,
                          double2 scale, const uint8_t* __restrict__ mask, double2* __restrict__ out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nb;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (!mask[v]) {
            out[v] = out[nb + v] = out[2 * nb + v] = make_double2(0.0, 0.0);
            continue;
        }
        const int i1 = (int)(v % n1);
        const int i2 = (int)((v / n1) % n2);
        const int64_t i3 = v / ((int64_t)n1 * n2);
        const double x = ox + h * i1, y = oy + h * i2, z = oz + h * (double)i3;
        double sn, cs;
        sincos(k0 * (kx * x + ky * y + kz * z), &sn, &cs);
        const double2 ph = cmul(scale, make_double2(cs, -sn));
        out[v] = cscale(ph, ex);
        out[nb + v] = cscale(ph, ey);
        out[2 * nb + v] = cscale(ph, ez);
    }
}

}  // namespace vsie

using namespace vsie;

extern "C" vsie_status vsie_rhs_planewave(vsie_ctx* ctx, const double k_hat[3], const double e0[3], void* B,
                                          vsie_stream stream) {
    if (!ctx) { set_global_err("null context"); return VSIE_EINVAL; }
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    try {
        if (!k_hat || !e0 || !B) throw Error(VSIE_EINVAL, "null k_hat, e0 or B");
        double kn = 0, en = 0, ke = 0;
        for (int d = 0; d < 3; ++d) {
            if (!std::isfinite(k_hat[d]) || !std::isfinite(e0[d])) throw Error(VSIE_EINVAL, "non-finite k_hat or e0");
            kn += k_hat[d] * k_hat[d];
            en += e0[d] * e0[d];
            ke += k_hat[d] * e0[d];
        }
        if (!(kn > 0)) throw Error(VSIE_EINVAL, "k_hat must be non-zero");
        kn = std::sqrt(kn);
        if (std::fabs(ke) / kn > 1e-9 * std::sqrt(en)) throw Error(VSIE_EINVAL, "e0 must be orthogonal to k_hat");
        const int m = c->m_f + c->m_n;
        if (m > 0 && !c->rwg_geo)
            throw Error(VSIE_EUNSUPPORTED, "context has no conductor geometry (created from parts or loaded)");
        const double kh[3] = {k_hat[0] / kn, k_hat[1] / kn, k_hat[2] / kn};
        const double2 scale = make_double2(0.0, c->omega * kEps0);   // i omega eps0
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        double2* out = (double2*)B;
        planewave_surface(m, c->rwg_geo, kh, e0, c->k0, scale, out, st);
        const double h3 = c->h * c->h * c->h;
        const int blocks = (int)std::min<int64_t>((c->n_b + 255) / 256, 152 * 16);
        k_pw_body<<<blocks, 256, 0, st>>>(c->n_b, c->nb[0], c->nb[1], c->h, c->origin[0], c->origin[1],
                                          c->origin[2], kh[0], kh[1], kh[2], e0[0], e0[1], e0[2], c->k0,
                                          cscale(scale, h3), c->mask, out + m);
        VSIE_CUDA(cudaGetLastError());
    } catch (const Error& e) {
        c->err = e.msg;
        return e.st;
    }
    return VSIE_OK;
}
