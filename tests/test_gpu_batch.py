"""vsie_solve_batch (uneven batch of independent problems): concurrent solves on
per-thread streams give the same solutions as one-by-one solves, and bad
batches are rejected."""
import numpy as np
import pytest

from oracle import mie
from paper_2206_12409_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _problems():
    out = []
    # spheres of different sizes and materials (uneven batch)
    for N, eps, sig in ((8, 50.0, 0.6), (12, 10.0, 0.3), (16, 2.0, 0.0), (10, 80.0, 2.2)):
        h = 50e-3 / N
        g, er, sg = I.sphere_phantom(n=(N + 2,) * 3, h=h, radius=25e-3, eps_r=eps, sigma=sig)
        out.append(I.Problem("sphere", g, er, sg, 298e6))
    return out


def test_batch_matches_single_solves():
    import torch
    from paper_2206_12409_gb300 import vsie as V
    probs = _problems()
    ctxs = [V.setup_problem(pr, max_rhs=1) for pr in probs]
    try:
        Ns = [V.vsie_sizes(c)[0] for c in ctxs]
        Bs = []
        for pr, c, N in zip(probs, ctxs, Ns):
            b = np.zeros(N, np.complex128)
            nb = 3 * pr.grid.nv
            b[N - nb:] = mie.body_rhs(pr.grid, pr.eps_r, pr.sigma, pr.freq_hz)
            Bs.append(torch.from_numpy(b).cuda()[None, :])
        o = V.vsie_solve_opts()
        o.mode, o.restart, o.maxit, o.inner_tol = 1, 50, 3000, 1e-3
        X1 = [torch.zeros_like(B) for B in Bs]
        for c, B, X, N in zip(ctxs, Bs, X1, Ns):
            st, _ = V.vsie_solve(c, 1, B.data_ptr(), N, X.data_ptr(), N, 1e-6, o)
            assert st == V.VSIE_OK
        X2 = [torch.zeros_like(B) for B in Bs]
        st, sts, infos = V.vsie_solve_batch(ctxs, [1] * len(ctxs), [B.data_ptr() for B in Bs], Ns,
                                            [X.data_ptr() for X in X2], Ns, 1e-6, o, nthreads=4)
        torch.cuda.synchronize()
        assert st == V.VSIE_OK and all(s == V.VSIE_OK for s in sts)
        for a, b, inf in zip(X1, X2, infos):
            assert torch.linalg.norm(a - b) <= 1e-12 * torch.linalg.norm(a)
            assert inf.relres[0] <= 1e-6
        # a context twice is rejected
        st, _, _ = V.vsie_solve_batch([ctxs[0], ctxs[0]], [1, 1], [Bs[0].data_ptr()] * 2, [Ns[0]] * 2,
                                      [X2[0].data_ptr()] * 2, [Ns[0]] * 2, 1e-6, o)
        assert st == V.VSIE_EINVAL
    finally:
        for c in ctxs:
            V.vsie_destroy(c)
