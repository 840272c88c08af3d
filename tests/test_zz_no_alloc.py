"""The allocation-free body operator (vsie_volume_matvec_static) against the
ordinary matvec.

Callers that cannot allocate device memory while the operator runs (fixed
memory pools, real-time loops, runtimes that own all device memory) use that entry
point; its FFT work space is a fixed 32 MiB device array inside the library.
This file is collected last so that a failure here comes after every other
test has run."""
import numpy as np
import pytest

from paper_2206_12409_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_static_matches_matvec_twice():
    import torch
    from paper_2206_12409_gb300 import vsie as V
    g, er, sg = I.sphere_phantom((12, 12, 12), 5e-3, 25e-3, 50.0, 0.6)
    ctx = V.vsie_create(V.make_grid(g.n, g.h, g.origin), er, sg, 298e6, V.make_options(max_rhs=2))
    try:
        N = V.vsie_sizes(ctx)[0]
        assert N == 3 * g.nv            # volume-only context: unknowns are the body block
        for prec, dt, tol in ((V.VSIE_C128, torch.complex128, 1e-10),
                              (V.VSIE_C64, torch.complex64, 2e-5)):
            for call in range(2):       # two calls in a row share the static work space
                x = I.random_vectors(N, 2, seed=40 + call)
                X = torch.from_numpy(np.ascontiguousarray(x.T)).to(dt).cuda()
                Y0 = torch.empty_like(X)
                Y1 = torch.full_like(X, float("nan"))
                V.vsie_matvec(ctx, 2, X.data_ptr(), N, Y0.data_ptr(), N, prec)
                V.vsie_volume_matvec_static(ctx, 2, X.data_ptr(), N, Y1.data_ptr(), N, prec)
                torch.cuda.synchronize()
                y0 = Y0.cpu().numpy().astype(np.complex128)
                y1 = Y1.cpu().numpy().astype(np.complex128)
                assert np.linalg.norm(y1 - y0) <= tol * np.linalg.norm(y0)
    finally:
        V.vsie_destroy(ctx)


def test_static_rejects_oversize_request():
    from paper_2206_12409_gb300 import vsie as V
    g, er, sg = I.sphere_phantom((96, 96, 112), 2e-3, 0.08, 50.0, 0.6)
    ctx = V.vsie_create(V.make_grid(g.n, g.h, g.origin), er, sg, 298e6,
                        V.make_options(max_rhs=1, precisions=2))
    try:
        import torch
        N = V.vsie_sizes(ctx)[0]
        X = torch.zeros((1, N), dtype=torch.complex64, device="cuda")
        with pytest.raises(V.VsieError) as e:
            V.vsie_volume_matvec_static(ctx, 1, X.data_ptr(), N, X.data_ptr(), N, V.VSIE_C64)
        assert e.value.status == V.VSIE_EINVAL
    finally:
        V.vsie_destroy(ctx)


def test_static_on_coil_context_after_unrelated_call():
    """On a context with a near coil (extended grid, coil-active lines) the
    allocation-free call equals the body rows of vsie_matvec given zero surface
    inputs.  A call with more right-hand sides and other data runs first, so
    the shared work space holds unrelated values when the checked call starts."""
    import torch
    from paper_2206_12409_gb300 import vsie as V
    prob = I.problem_sphere_loop_shield()
    ctx = V.setup_problem(prob, max_rhs=4)
    try:
        N, mf, mn, nb = V.vsie_sizes(ctx)
        off = mf + mn
        for prec, dt, tol in ((V.VSIE_C128, torch.complex128, 1e-10),
                              (V.VSIE_C64, torch.complex64, 2e-5)):
            junk = torch.from_numpy(np.ascontiguousarray(I.random_vectors(3 * nb, 4, seed=90).T)).to(dt).cuda()
            junk_out = torch.empty_like(junk)
            V.vsie_volume_matvec_static(ctx, 4, junk.data_ptr(), 3 * nb, junk_out.data_ptr(), 3 * nb, prec)
            x = np.zeros((N, 2), np.complex128)
            x[off:] = I.random_vectors(3 * nb, 2, seed=91)
            X = torch.from_numpy(np.ascontiguousarray(x.T)).to(dt).cuda()
            Y0 = torch.empty_like(X)
            V.vsie_matvec(ctx, 2, X.data_ptr(), N, Y0.data_ptr(), N, prec)
            Xb = X[:, off:].contiguous()
            Yb = torch.full_like(Xb, float("nan"))
            V.vsie_volume_matvec_static(ctx, 2, Xb.data_ptr(), 3 * nb, Yb.data_ptr(), 3 * nb, prec)
            torch.cuda.synchronize()
            y0 = Y0[:, off:].cpu().numpy().astype(np.complex128)
            y1 = Yb.cpu().numpy().astype(np.complex128)
            assert np.isfinite(y1).all()
            assert np.linalg.norm(y1 - y0) <= tol * np.linalg.norm(y0), (prec, np.linalg.norm(y1 - y0) / np.linalg.norm(y0))
    finally:
        V.vsie_destroy(ctx)
