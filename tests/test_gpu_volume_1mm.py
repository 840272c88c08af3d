"""GPU body operator at the 1 mm head size (192 x 192 x 224 voxels in the
256 x 256 x 224 extended grid, FFT lengths 512 x 512 x 448: the register
kernels for 512-point lines and the 224-point half-length z pass), checked on
sampled output rows against the oracle's direct sum (oracle.volume.rows_matvec:
the definition of Z_bb x, no FFT), and over every row by the property that the
FP32 and FP64 operators agree."""
import numpy as np
import pytest

from oracle import physics, volume
from paper_2206_12409_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("zv", [None, 9, 10, 12])
def test_volume_1mm_sampled_rows_and_precisions(zv, monkeypatch):
    """zv: the z-pass variant forced through VSIE_ZPASS_VARIANT (None: tuned);
    9 is k_zreg with 8 lines per CTA, 10 the staged k_zreg_st, 12 the staged kernel
    with its middle phase on thread pairs."""
    import torch
    if zv is not None:
        monkeypatch.setenv("VSIE_ZPASS_VARIANT", str(zv))
    from paper_2206_12409_gb300 import vsie as V
    g, er, sg = I.layered_head_phantom((192, 192, 224), 1e-3)
    f = 298e6
    ctx = V.vsie_create(V.make_grid(g.n, g.h, g.origin), er, sg, f,
                        V.make_options(ext_n=(256, 256, 224), ext_offset=(32, 32, 0), max_rhs=2))
    try:
        N = V.vsie_sizes(ctx)[0]
        assert N == 3 * g.nv
        x = I.random_vectors(N, 2, seed=77)
        ys = {}
        for prec, dt in ((V.VSIE_C128, torch.complex128), (V.VSIE_C64, torch.complex64)):
            X = torch.from_numpy(np.ascontiguousarray(x.T)).to(dt).cuda()
            Y = torch.full_like(X, float("nan"))
            V.vsie_matvec(ctx, 2, X.data_ptr(), N, Y.data_ptr(), N, prec)
            torch.cuda.synchronize()
            ys[prec] = Y.cpu().numpy().T.astype(np.complex128)
            del X, Y
    finally:
        V.vsie_destroy(ctx)
    chi = physics.chi(er, sg, f)
    _, k0 = physics.omega_k0(f)
    mat = np.nonzero(chi != 0)[0]
    rng = np.random.default_rng(3)
    rows = [a * g.nv + int(v) for a, v in zip((0, 1, 2, 0, 1, 2, 0, 1), rng.choice(mat, 8, replace=False))]
    rows += [int(np.nonzero(chi == 0)[0][0]), 2 * g.nv + int(mat[-1])]
    yo = volume.rows_matvec(g, chi, k0, x, rows)
    for prec, tol in ((V.VSIE_C128, 1e-10), (V.VSIE_C64, 2e-5)):
        e = np.linalg.norm(ys[prec][rows] - yo) / np.linalg.norm(yo)
        print(f"[1 mm sampled rows] precision={prec} rel_err={e:.2e}")
        assert e <= tol
    M3 = np.tile(chi != 0, 3)
    d = np.linalg.norm((ys[V.VSIE_C64] - ys[V.VSIE_C128])[M3]) / np.linalg.norm(ys[V.VSIE_C128][M3])
    print(f"[1 mm all rows] FP32 vs FP64 rel_diff={d:.2e}")
    assert d <= 2e-5
