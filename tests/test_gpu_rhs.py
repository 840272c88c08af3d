"""GPU plane-wave right-hand side (vsie_rhs_planewave) against the oracle's
(oracle/rhs.py), on the sphere + loop + shield workload set up from geometry:
conductor rows (shield and coil RWG) and body rows, each to 1e-12."""
import numpy as np
import pytest

from oracle import rhs
from paper_2206_12409_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k_hat,e0", [((0, 0, 1), (1, 0, 0)), ((0.6, 0.0, 0.8), (0.8, 0.0, -0.6)),
                                      ((1, 1, 1), (1, -1, 0))])
def test_planewave_rhs_vs_oracle(sphere_loop_shield, k_hat, e0):
    import torch
    from paper_2206_12409_gb300 import vsie as V
    prob = sphere_loop_shield
    ctx = V.setup_problem(prob, max_rhs=1)
    try:
        N, mf, mn, nb = V.vsie_sizes(ctx)
        B = torch.full((N,), float("nan"), dtype=torch.complex128, device="cuda")
        V.vsie_rhs_planewave(ctx, k_hat, e0, B.data_ptr())
        torch.cuda.synchronize()
        b = B.cpu().numpy()
    finally:
        V.vsie_destroy(ctx)
    bo = rhs.planewave(prob, k_hat, e0)
    assert bo.shape == b.shape
    for name, sl in (("far", slice(0, mf)), ("near", slice(mf, mf + mn)), ("body", slice(mf + mn, None))):
        err = np.linalg.norm(b[sl] - bo[sl]) / np.linalg.norm(bo[sl])
        print(f"[planewave rhs] {name} rows rel_err={err:.2e}")
        assert err <= 1e-12, (name, err)


def test_planewave_rejects_bad_input(sphere_loop_shield):
    import torch
    from paper_2206_12409_gb300 import vsie as V
    ctx = V.setup_problem(sphere_loop_shield, max_rhs=1)
    try:
        N = V.vsie_sizes(ctx)[0]
        B = torch.zeros((N,), dtype=torch.complex128, device="cuda")
        for kh, e in (((0, 0, 0), (1, 0, 0)), ((0, 0, 1), (0, 0, 1))):
            with pytest.raises(V.VsieError) as ex:
                V.vsie_rhs_planewave(ctx, kh, e, B.data_ptr())
            assert ex.value.status == V.VSIE_EINVAL
    finally:
        V.vsie_destroy(ctx)
