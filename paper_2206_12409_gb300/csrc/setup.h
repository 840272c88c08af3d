// Internal declarations of the geometry set-up (vsie_setup): RWG meshes on the
// device and the assembly kernels of assemble.cu.
#pragma once
#include "vsie_internal.h"

namespace vsie {

// Device view of a triangle mesh and its RWG functions (all arrays device).
struct MeshDev {
    const double* xyz = nullptr;       // nverts x 3
    const int* tri = nullptr;          // ntris x 3
    const double* area = nullptr;      // ntris
    const double* centroid = nullptr;  // ntris x 3
    const double* normal = nullptr;    // ntris x 3 (from the vertex order)
    const double* diam = nullptr;      // ntris, longest edge
    const int* tplus = nullptr;        // m
    const int* tminus = nullptr;
    const int* vplus = nullptr;        // free vertices
    const int* vminus = nullptr;
    const double* len = nullptr;       // m, edge lengths
    int ntris = 0, m = 0;
};

struct GridDev {
    int n[3];
    double h;
    double origin[3];
};

// Host RWG construction (same conventions as documented in vsie.h):
// interior edges sorted by (min vertex, max vertex); T+ = adjacent triangle
// with the smaller index; ports map vertex pairs to edge indices.
struct MeshHost {
    std::vector<double> xyz;
    std::vector<int> tri;
    std::vector<double> area, centroid, normal, diam, len;
    std::vector<int> tplus, tminus, vplus, vminus;
    std::vector<int> ports;   // edge index per port
    int m = 0, ntris = 0;
};

MeshHost build_rwg(const vsie_mesh& mesh);
MeshDev upload_mesh(Ctx& c, const MeshHost& h);

void efie_block(const MeshDev& ma, const MeshDev& mb, bool same, int nr, const int* rows, int nc,
                const int* cols, double k0, double sign, double2* out, int64_t ldo);
void coupling_block(const MeshDev& m, const GridDev& g, int nvx, const int64_t* vox, int nc,
                    const int* cols, double k0, bool near, double sign, double2* out, int64_t ldo,
                    int64_t pstride, int only = -1);
void field_points(const MeshDev& m, int np, const double* pts, int nc, const int* cols,
                  const double* ctr, double k0, double2* out);
// out[m] = scale \int f_m . e0 exp(-i k0 khat . r) dS for m RWG functions
// described by geo (26 doubles each: see k_pw_surface)
// Z[m + ldz n] += h^3 (P^T T P)[m, n] for the mn near RWG (direct stencil-pair sum)
void ptkp_add(int mn, int s, const double2* W, const int* base, double h, double k0, double2 selfv, double2* Z,
              int64_t ldz);
void planewave_surface(int m, const double* geo, const double khat[3], const double e0[3], double k0,
                       double2 scale, double2* out, cudaStream_t st);

}  // namespace vsie
