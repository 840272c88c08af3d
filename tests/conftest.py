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


def input_blocks(P):
    """Unknowns of the three input blocks of Eq. (hvsie): far and near surface
    currents, body currents."""
    mf, mn = P.m_f, P.m_n
    return {"far": slice(0, mf), "near": slice(mf, mf + mn), "body": slice(mf + mn, None)}


def output_blocks(P):
    """Rows of the three output blocks: far and near surface rows, and the body
    rows of material voxels (rows of vacuum voxels return their input)."""
    import numpy as np
    mf, mn = P.m_f, P.m_n
    rows = {k: np.zeros(P.N, bool) for k in ("far", "near", "body")}
    rows["far"][:mf] = True
    rows["near"][mf:mf + mn] = True
    rows["body"][mf + mn:] = np.tile(P.chi != 0, 3)
    return rows


def block_parity(ctx, P, precision, tol, p=1, seed=8, label=""):
    """Each block of Eq. (hvsie_disc) on its own: for every input block alone
    (the others zero) the relative L2 error of every non-empty output block of
    the GPU matvec against oracle.hybrid.matvec on the same parts.  A small
    output block therefore cannot hide behind a large one.  Prints the table,
    asserts every entry <= tol and returns it."""
    import numpy as np
    from paper_2206_12409_gb300 import inputs as I
    from oracle import hybrid
    x0 = I.random_vectors(P.N, p, seed=seed)
    errs = {}
    for iname, sl in input_blocks(P).items():
        x = np.zeros_like(x0)
        x[sl] = x0[sl]
        yo = hybrid.matvec(P, x)
        y = gpu_matvec(ctx, x, precision)
        assert np.isfinite(y).all(), (label, iname)
        for oname, rows in output_blocks(P).items():
            den = np.linalg.norm(yo[rows])
            if den == 0:
                continue
            errs[f"{iname}->{oname}"] = float(np.linalg.norm((y - yo)[rows]) / den)
    print(f"[block parity] {label} precision={precision} p={p} tol={tol:g} " +
          " ".join(f"{k}={v:.2e}" for k, v in errs.items()))
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, (label, precision, bad)
    return errs
