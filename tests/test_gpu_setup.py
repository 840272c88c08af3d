"""GPU set-up from geometry (vsie_setup) against the oracle's definitions, on
the sphere + loop + closed-shield workload: deterministic parts to ~1e-9,
compressed parts to their tolerances, and the whole operator against the
oracle's hybrid and dense operators."""
import numpy as np
import pytest

from paper_2206_12409_gb300 import inputs as I
from oracle import hybrid, coupling, rwg, tt as ott, physics
from tests.conftest import block_parity, gpu_matvec, output_blocks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup_ctx(sphere_loop_shield):
    from paper_2206_12409_gb300 import vsie as V
    ctx = V.setup_problem(sphere_loop_shield, max_rhs=8)
    parts = V.parts_to_numpy(ctx, sphere_loop_shield.grid.n)
    yield ctx, parts
    V.vsie_destroy(ctx)


def test_sizes(setup_ctx, hybrid_parts):
    from paper_2206_12409_gb300 import vsie as V
    ctx, parts = setup_ctx
    assert V.vsie_sizes(ctx) == (hybrid_parts.N, hybrid_parts.m_f, hybrid_parts.m_n,
                                 hybrid_parts.body.nv)


def test_projection_and_stencils(setup_ctx, hybrid_parts):
    _, parts = setup_ctx
    P = hybrid_parts
    assert np.array_equal(parts["base"], P.base)
    assert np.linalg.norm(parts["W"] - P.W) <= 1e-8 * np.linalg.norm(P.W)


def test_precorrection(setup_ctx, hybrid_parts):
    _, parts = setup_ctx
    pre = hybrid_parts.pre.tocsr()
    pre.sort_indices()
    assert np.array_equal(parts["pre_rowptr"], pre.indptr)
    assert np.array_equal(parts["pre_col"], pre.indices)
    assert np.linalg.norm(parts["pre_val"] - pre.data) <= 1e-8 * np.linalg.norm(pre.data)


def test_near_block(setup_ctx, hybrid_parts):
    _, parts = setup_ctx
    Z = hybrid_parts.Znn
    assert np.linalg.norm(parts["Znn"] - Z) <= 1e-9 * np.linalg.norm(Z)


def test_far_blocks(setup_ctx, hybrid_parts, dense_reference):
    _, parts = setup_ctx
    P = hybrid_parts
    assert np.linalg.norm(parts["Zff"] - P.Zff) <= 1e-10 * np.linalg.norm(P.Zff)
    Zfn = P.U @ P.V.conj().T     # oracle ACA is exact (full rank) at this size
    Zg = parts["U"] @ parts["V"].conj().T
    assert np.linalg.norm(Zg - Zfn) <= 1e-5 * np.linalg.norm(Zfn)


def test_tt_against_exact_far_coupling(setup_ctx, sphere_loop_shield):
    """TT reconstruction vs the exact (1 x 1-point) far coupling on every entry,
    within the TT tolerance."""
    _, parts = setup_ctx
    prob = sphere_loop_shield
    _, k0 = physics.omega_k0(prob.freq_hz)
    rs = rwg.build(prob.shield)
    K = coupling.K_block(prob.grid, np.arange(prob.grid.nv), rs, np.arange(rs.m), k0, near=False)
    for a in range(3):
        T = -K[a].reshape(tuple(prob.grid.n) + (rs.m,), order="F")
        R = ott.tt_full(parts["tt"][a])
        assert np.linalg.norm(R - T) <= prob.tt_tol * np.linalg.norm(T)


def test_matvec_vs_oracle_hybrid_and_dense(setup_ctx, sphere_loop_shield, hybrid_parts,
                                           dense_reference):
    from paper_2206_12409_gb300 import vsie as V
    ctx, _ = setup_ctx
    P = hybrid_parts
    x = I.random_vectors(P.N, 2, seed=5)
    M3 = np.tile(P.chi != 0, 3)
    x[P.m_f + P.m_n:][~M3] = 0
    y = gpu_matvec(ctx, x, V.VSIE_C128)
    yh = hybrid.matvec(P, x)
    assert np.linalg.norm(y - yh) <= 2e-6 * np.linalg.norm(yh)
    # per output block against the oracle's own parts: the set-up's parts are
    # independent approximations (ACA, TT cross) at tolerance 1e-6 and a pFFT
    # fit equal to the oracle's to ~1e-8, so every block agrees to ~1e-6
    for name, rows in output_blocks(P).items():
        e = np.linalg.norm((y - yh)[rows]) / np.linalg.norm(yh[rows])
        print(f"[setup vs oracle parts] {name} rows: {e:.2e}")
        assert e <= 1e-5, (name, e)
    Z, idx = dense_reference
    yd = hybrid.dense_matvec(sphere_loop_shield, Z, idx, x)
    assert np.linalg.norm(y - yd) <= 2e-3 * np.linalg.norm(yd)


@pytest.mark.parametrize("p", [5, 20])
def test_multi_rhs_matvec_equals_single_rhs(sphere_loop_shield, p):
    """A p-column matvec (p above the 16-column width of the tall-skinny and
    panel kernels takes their chunked and generic paths) equals p one-column
    matvecs, in FP64 and FP32."""
    import torch
    from paper_2206_12409_gb300 import vsie as V
    ctx = V.setup_problem(sphere_loop_shield, max_rhs=p)
    try:
        N = V.vsie_sizes(ctx)[0]
        x = I.random_vectors(N, p).T.copy()
        for prec, dt, tol in ((V.VSIE_C128, torch.complex128, 1e-13), (V.VSIE_C64, torch.complex64, 1e-5)):
            X = torch.from_numpy(x).to(dt).cuda()
            Y = torch.empty_like(X)
            V.vsie_matvec(ctx, p, X.data_ptr(), N, Y.data_ptr(), N, prec)
            Y1 = torch.empty_like(X)
            for j in range(p):
                V.vsie_matvec(ctx, 1, X[j].data_ptr(), N, Y1[j].data_ptr(), N, prec)
            torch.cuda.synchronize()
            assert (torch.linalg.norm(Y - Y1) / torch.linalg.norm(Y1)).item() < tol
    finally:
        V.vsie_destroy(ctx)


def _oracle_parts_with(P, g):
    """The oracle's Parts with the operator parts the GPU set-up produced (its
    projection, precorrection, near block, ACA factors, far block and TT cores);
    spectra and materials stay the oracle's own."""
    import dataclasses
    import scipy.sparse as sp
    nb = P.body.nv
    if g.get("pre_nnz", 0):
        pre = sp.csr_matrix((g["pre_val"], g["pre_col"], g["pre_rowptr"]), shape=(3 * nb, g["m_n"]))
    else:
        pre = sp.csr_matrix((3 * nb, g["m_n"]), dtype=np.complex128)
    return dataclasses.replace(P, W=g["W"], base=g["base"], pre=pre, Znn=g["Znn"], U=g["U"],
                               V=g["V"], Zff=g["Zff"], tt=g["tt"])


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 2e-5)])
def test_matvec_blocks_with_setup_parts(setup_ctx, hybrid_parts, prec, tol):
    """The matvec of a vsie_setup context, block by block, against the oracle's
    matvec applied to the parts that set-up computed (the parts themselves are
    checked against the oracle's in the tests above)."""
    ctx, parts = setup_ctx
    Pg = _oracle_parts_with(hybrid_parts, parts)
    block_parity(ctx, Pg, prec, tol, p=2, seed=31, label="vsie_setup parts")
