import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libvsie")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def sphere_loop_shield():
    from paper_2206_12409_gb300 import inputs as I
    return I.problem_sphere_loop_shield()


@pytest.fixture(scope="session")
def hybrid_parts(sphere_loop_shield):
    from oracle import hybrid
    return hybrid.build_parts(sphere_loop_shield)


@pytest.fixture(scope="session")
def dense_reference(sphere_loop_shield):
    from oracle import hybrid
    return hybrid.dense_operator(sphere_loop_shield)


def oracle_parts_to_abi(P):
    """Marshal the oracle's operator parts into a vsie_parts struct (test
    infrastructure: the oracle is the source of these inputs, never the
    reverse)."""
    import numpy as np
    from paper_2206_12409_gb300 import vsie as V
    pre = P.pre.tocsr()
    pre.sort_indices()
    return V.make_parts(
        m_f=P.m_f, m_n=P.m_n, stencil=P.s, W=P.W, base=P.base,
        pre_rowptr=pre.indptr.astype(np.int64), pre_col=pre.indices.astype(np.int32),
        pre_val=pre.data.astype(np.complex128), Znn=P.Znn, U=P.U, V=P.V, Zff=P.Zff, tt=P.tt)


def gpu_matvec(ctx, x, precision, ld=None):
    """Run vsie_matvec on a host complex array x (N, p) and return (N, p)."""
    import numpy as np
    import torch
    from paper_2206_12409_gb300 import vsie as V
    N, p = x.shape
    ld = N if ld is None else ld
    dt = torch.complex128 if precision == V.VSIE_C128 else torch.complex64
    X = torch.zeros((p, ld), dtype=dt)
    X[:, :N] = torch.from_numpy(np.ascontiguousarray(x.T))
    X = X.cuda()
    Y = torch.full((p, ld), float("nan"), dtype=dt, device="cuda")
    V.vsie_matvec(ctx, p, X.data_ptr(), ld, Y.data_ptr(), ld, precision)
    torch.cuda.synchronize()
    y = Y.cpu().numpy().T[:N]
    return y.astype(np.complex128)
