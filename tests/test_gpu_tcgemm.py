"""The preconditioner's far-block inverse applied on the tensor cores (tcgen05,
TMA, split TF32; include/vsie.h dense_gemm = 0) against the SIMT row-panel
product of the same inverse (dense_gemm = 1), through vsie_precond_apply: the
two FP32 products agree to FP32 accuracy for 1 to 20 right-hand sides (the
kernel works in 16-column passes), for an even m_f (1536) and an odd one (35:
the row pitch is padded for TMA)."""
import numpy as np
import pytest

from paper_2206_12409_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _odd_far_problem():
    g, er, sg = I.sphere_phantom((6, 6, 6), 10e-3, 25e-3, 50.0, 0.6)
    shield = I.open_cylinder(0.1, 0.2, n_theta=7, n_z=2)     # 7 x 5 = 35 interior edges
    return I.Problem("odd far block", g, er, sg, 298e6, None, shield, None, (0, 0, 0), 3, 1e-6, 1e-6, 1)


def _apply(ctx, x, V, torch):
    N, p = x.shape
    X = torch.from_numpy(np.ascontiguousarray(x.T)).to(torch.complex64).cuda()
    Y = torch.full_like(X, float("nan"))
    V.vsie_precond_apply(ctx, p, X.data_ptr(), N, Y.data_ptr(), N, 0)
    torch.cuda.synchronize()
    return Y.cpu().numpy().T.astype(np.complex128)


@pytest.mark.parametrize("which", ["sphere_loop_shield", "odd"])
def test_tensor_core_far_inverse_matches_simt(which, sphere_loop_shield):
    import torch
    from paper_2206_12409_gb300 import vsie as V
    prob = sphere_loop_shield if which == "sphere_loop_shield" else _odd_far_problem()
    tc = V.setup_problem(prob, max_rhs=20, dense_gemm=0)
    simt = V.setup_problem(prob, max_rhs=20, dense_gemm=1)
    try:
        N, mf, mn, nb = V.vsie_sizes(tc)
        assert (mf % 2 == 1) == (which == "odd")
        for p in (1, 3, 16, 20):
            x = I.random_vectors(N, p, seed=70 + p)
            y_tc = _apply(tc, x, V, torch)
            y_si = _apply(simt, x, V, torch)
            assert np.isfinite(y_tc).all()
            e = np.linalg.norm(y_tc[:mf] - y_si[:mf]) / np.linalg.norm(y_si[:mf])
            print(f"[tensor-core far inverse] {which} m_f={mf} p={p} rel_diff={e:.2e}")
            assert e <= 2e-5
            assert np.array_equal(y_tc[mf:], y_si[mf:])          # other blocks untouched
    finally:
        V.vsie_destroy(tc)
        V.vsie_destroy(simt)
