"""GPU parity of the hybrid-VSIE matvec (Eq. hvsie_disc) on a mid-size workload
that reaches the kernel paths of the head-size workload, block by block.

problem_coil_array_mid: 1824 far RWG (the last 256-row panel of the FP32 far
block is partial), 1024 near RWG (the tall-skinny kernels for the near block and
the U factor), TT ranks above 100 (r2 n3 >= 1024: the tall-skinny and
inner-product kernels of the middle TT cores, split-K on the transposed chain),
precorrection pairs in both directions, FFT lengths 54 x 54 x 48 (radices 2 and
3, half-length Z pass) and p = 8 right-hand sides, the bench's batch width.
The operator parts come from the oracle (oracle.hybrid.build_parts); the GPU
applies them through vsie_create + vsie_matvec."""
import numpy as np
import pytest

from paper_2206_12409_gb300 import inputs as I
from oracle import hybrid
from tests.conftest import block_parity, gpu_matvec, oracle_parts_to_abi

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 2e-5}


@pytest.fixture(scope="module")
def mid_ctx():
    from paper_2206_12409_gb300 import vsie as V
    prob = I.problem_coil_array_mid()
    P = hybrid.build_parts(prob)
    parts, keep = oracle_parts_to_abi(P)
    g = prob.grid
    ctx = V.vsie_create(V.make_grid(g.n, g.h, g.origin), prob.eps_r, prob.sigma, prob.freq_hz,
                        V.make_options(ext_n=prob.ext_n, ext_offset=prob.ext_offset, max_rhs=8),
                        parts)
    yield ctx, P
    V.vsie_destroy(ctx)


def test_mid_workload_reaches_head_paths(mid_ctx):
    """The shapes that select the head workload's kernels are present."""
    _, P = mid_ctx
    assert P.m_f % 256 != 0 and P.m_n >= 1024
    r = [(c[1].shape[2], c[2].shape[2]) for c in P.tt]
    assert all(r2 * P.body.n[2] >= 1024 and r3 > 100 for r2, r3 in r), r
    assert P.pre.nnz > 0


@pytest.mark.parametrize("prec", [0, 1])
def test_mid_blocks(mid_ctx, prec):
    ctx, P = mid_ctx
    block_parity(ctx, P, prec, TOL[prec], p=8, seed=21, label="coil array mid")


@pytest.mark.parametrize("prec", [0, 1])
def test_mid_whole_matvec(mid_ctx, prec):
    ctx, P = mid_ctx
    x = I.random_vectors(P.N, 8, seed=22)
    yo = hybrid.matvec(P, x)
    y = gpu_matvec(ctx, x, prec)
    M3 = np.tile(P.chi != 0, 3)
    rows = np.concatenate([np.ones(P.m_f + P.m_n, bool), M3])
    err = np.linalg.norm((y - yo)[rows]) / np.linalg.norm(yo[rows])
    print(f"[mid whole] precision={prec} rel_err={err:.3e}")
    assert err <= TOL[prec]
