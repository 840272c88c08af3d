"""vsie_save / vsie_load: a context set up on the GPU, written to a file and read
back, gives the same operator (FP64 and FP32 matvecs) and the same port
right-hand sides; corrupt or missing files are rejected."""
import numpy as np
import pytest

from paper_2206_12409_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_save_load_round_trip(tmp_path):
    import torch
    from paper_2206_12409_gb300 import vsie as V
    prob = I.problem_sphere_loop_shield()
    ctx = V.setup_problem(prob, max_rhs=2)
    path = tmp_path / "op.vsie"
    try:
        V.vsie_save(ctx, path)
        ctx2 = V.vsie_load(path)
    except Exception:
        V.vsie_destroy(ctx)
        raise
    try:
        N = V.vsie_sizes(ctx)[0]
        assert V.vsie_sizes(ctx2) == V.vsie_sizes(ctx)
        x = I.random_vectors(N, 2).T.copy()
        X = torch.from_numpy(x).cuda()
        Y1, Y2 = torch.empty_like(X), torch.empty_like(X)
        V.vsie_matvec(ctx, 2, X.data_ptr(), N, Y1.data_ptr(), N, V.VSIE_C128)
        V.vsie_matvec(ctx2, 2, X.data_ptr(), N, Y2.data_ptr(), N, V.VSIE_C128)
        torch.cuda.synchronize()
        assert torch.linalg.norm(Y1 - Y2) <= 1e-13 * torch.linalg.norm(Y1)
        X32 = X.to(torch.complex64)
        Z1, Z2 = torch.empty_like(X32), torch.empty_like(X32)
        V.vsie_matvec(ctx, 2, X32.data_ptr(), N, Z1.data_ptr(), N, V.VSIE_C64)
        V.vsie_matvec(ctx2, 2, X32.data_ptr(), N, Z2.data_ptr(), N, V.VSIE_C64)
        torch.cuda.synchronize()
        assert torch.linalg.norm(Z1 - Z2) <= 1e-6 * torch.linalg.norm(Z1)
        B1 = torch.zeros((1, N), dtype=torch.complex128, device="cuda")
        B2 = torch.zeros_like(B1)
        V.vsie_rhs_ports(ctx, [0], 1.0, B1.data_ptr(), N)
        V.vsie_rhs_ports(ctx2, [0], 1.0, B2.data_ptr(), N)
        torch.cuda.synchronize()
        assert torch.equal(B1, B2) and torch.count_nonzero(B1) == 1
    finally:
        V.vsie_destroy(ctx)
        V.vsie_destroy(ctx2)
