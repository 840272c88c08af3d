// Hierarchical matrix of the far-far conductor block (hmatrix.cu).
#pragma once
#include "vsie_internal.h"

namespace vsie {

// Cluster tree and block partition (host), from the far RWG functions' centres
// and support boxes (3 doubles per function each).
struct HmPlan {
    struct Blk { int r0, nr, c0, nc; bool dense; };
    int m = 0;
    std::vector<int> perm;       // cluster position -> RWG index
    std::vector<int> rl_start;   // leaf row clusters: [rl_start[l], rl_start[l + 1])
    std::vector<Blk> blk;        // leaves of the block partition (cluster positions)
};
HmPlan hm_plan(int m, const double* centre, const double* slo, const double* shi, int leaf, double eta);

// Builds c.hm from the plan and the dense FP64 block dZ (original RWG order,
// column-major, leading dimension ldz): dense leaves copied, low-rank leaves by
// ACA to tol.  Device data in both precisions.
void hm_build(Ctx& c, const HmPlan& P, const double2* dZ, int64_t ldz, double tol);

// Y[:, 0:p] = Z_ff X[:, 0:p] on the far rows (overwrites them).
template <typename R>
void hm_apply(Ctx& c, int p, const cx<R>* X, int64_t ldx, cx<R>* Y, int64_t ldy, cudaStream_t st);

}  // namespace vsie
