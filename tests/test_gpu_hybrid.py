"""GPU parity of the full hybrid-VSIE matvec (Eq. hvsie_disc) with the oracle's
operator parts passed through vsie_create: FP64 <= 1e-10, FP32 <= 2e-5."""
import numpy as np
import pytest

from paper_2206_12409_gb300 import inputs as I
from oracle import hybrid
from tests.conftest import block_parity, gpu_matvec, oracle_parts_to_abi

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 2e-5}


@pytest.fixture(scope="module")
def ctx_and_parts(sphere_loop_shield, hybrid_parts):
    from paper_2206_12409_gb300 import vsie as V
    prob = sphere_loop_shield
    P = hybrid_parts
    parts, keep = oracle_parts_to_abi(P)
    g = prob.grid
    ctx = V.vsie_create(V.make_grid(g.n, g.h, g.origin), prob.eps_r, prob.sigma, prob.freq_hz,
                        V.make_options(ext_n=prob.ext_n, ext_offset=prob.ext_offset, max_rhs=8),
                        parts)
    yield ctx, P
    V.vsie_destroy(ctx)


def _err(y, yo, P):
    M3 = np.tile(P.chi != 0, 3)
    rows = np.concatenate([np.ones(P.m_f + P.m_n, bool), M3])
    return np.linalg.norm((y - yo)[rows]) / np.linalg.norm(yo[rows])


@pytest.mark.parametrize("p", [1, 3])
def test_hybrid_matvec_parity(ctx_and_parts, p):
    from paper_2206_12409_gb300 import vsie as V
    ctx, P = ctx_and_parts
    assert V.vsie_sizes(ctx) == (P.N, P.m_f, P.m_n, P.body.nv)
    x = I.random_vectors(P.N, p, seed=7)
    yo = hybrid.matvec(P, x)
    for prec in (V.VSIE_C128, V.VSIE_C64):
        y = gpu_matvec(ctx, x, prec)
        assert _err(y, yo, P) <= TOL[prec], (prec, _err(y, yo, P))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", [1, 8])
def test_hybrid_blocks_separately(ctx_and_parts, prec, p):
    """Each input block alone (far, near, body) against every output block, so
    that no block hides behind a larger one: the FP32 body rows (about 1e-5 of
    the whole output norm) are held to 2e-5 on their own."""
    ctx, P = ctx_and_parts
    block_parity(ctx, P, prec, TOL[prec], p=p, seed=8 + p, label="sphere+loop+shield")
