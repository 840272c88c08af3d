"""GPU learned preconditioner (csrc/net.cu, csrc/nettrain.cu) against the FP64
oracle network (oracle/unet.py): forward pass, every parameter gradient and
the input gradient, one training step (loss and Adam update); then training on
operator-generated pairs and its use inside flexible GMRES."""
import numpy as np
import pytest

from oracle import unet

pytestmark = pytest.mark.gpu


def _bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _params(seed):
    """Oracle He-normal weights rounded to BF16 (the kernels' weight precision),
    small random biases rounded to FP32."""
    rng = np.random.default_rng(seed + 100)
    P = unet.init_params(seed)
    for k in P:
        P[k] = _bf16(P[k]) if k.endswith(".w") else np.float32(0.05 * rng.standard_normal(P[k].shape)).astype(np.float64)
    return P


def _pack(P):
    return np.concatenate([np.concatenate([P[n + ".w"].ravel(), P[n + ".b"]]) for n, *_ in unet.LAYERS])


def _unpack(v):
    out, off = {}, 0
    for n, ci, co, k in unet.LAYERS:
        nw = co * ci * k ** 3
        out[n + ".w"] = v[off:off + nw].reshape(co, ci, k, k, k)
        out[n + ".b"] = v[off + nw:off + nw + co]
        off += nw + co
    return out


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


@pytest.fixture(scope="module")
def net_case():
    import torch
    from paper_2206_12409_gb300 import vsie as V
    P = _params(7)
    rng = np.random.default_rng(8)
    D, H, W = 16, 8, 24                       # ragged: three different multiples of 8
    x = rng.standard_normal((8, D, H, W)).astype(np.float32)
    net = V.vsie_net_create(1)
    assert V.vsie_net_num_params(net) == _pack(P).size
    V.vsie_net_set_params(net, _pack(P))
    yield V, torch, net, P, x, (D, H, W)
    V.vsie_net_destroy(net)


def test_forward_matches_oracle(net_case):
    V, torch, net, P, x, (D, H, W) = net_case
    X = torch.from_numpy(x).cuda()
    Y = torch.empty((6, D, H, W), dtype=torch.float32, device="cuda")
    V.vsie_net_forward(net, D, H, W, X.data_ptr(), Y.data_ptr())
    torch.cuda.synchronize()
    yo, _ = unet.forward(P, x.astype(np.float64))
    assert _rel(Y.cpu().numpy(), yo) < 1e-4


def test_backward_matches_oracle(net_case):
    V, torch, net, P, x, (D, H, W) = net_case
    rng = np.random.default_rng(9)
    dy = rng.standard_normal((6, D, H, W)).astype(np.float32)
    X = torch.from_numpy(x).cuda()
    DY = torch.from_numpy(dy).cuda()
    DX = torch.empty((8, D, H, W), dtype=torch.float32, device="cuda")
    g = _unpack(V.vsie_net_backward(net, D, H, W, X.data_ptr(), DY.data_ptr(), DX.data_ptr()))
    _, tape = unet.forward(P, x.astype(np.float64))
    G, gx = unet.backward(P, tape, dy.astype(np.float64))
    for k in G:
        assert _rel(g[k], G[k]) < 1e-3, k
    assert _rel(DX.cpu().numpy(), gx) < 1e-3


def test_training_step_matches_oracle():
    import torch
    from paper_2206_12409_gb300 import vsie as V
    P = _params(11)
    rng = np.random.default_rng(12)
    D, H, W = 8, 16, 8
    x = rng.standard_normal((8, D, H, W)).astype(np.float32)
    t = rng.standard_normal((6, D, H, W)).astype(np.float32)
    net = V.vsie_net_create(2)
    try:
        V.vsie_net_set_params(net, _pack(P))
        lr = 1e-3
        X = torch.from_numpy(x).cuda()
        T = torch.from_numpy(t).cuda()
        loss = V.vsie_net_step(net, D, H, W, X.data_ptr(), T.data_ptr(), lr)
        new = _unpack(V.vsie_net_get_params(net).astype(np.float64))
    finally:
        V.vsie_net_destroy(net)
    Lo, G = unet.loss_and_grad(P, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - Lo) < 1e-5 * Lo
    Q = {k: v.copy() for k, v in P.items()}
    unet.adam_step(Q, G, {k: 0 * v for k, v in P.items()}, {k: 0 * v for k, v in P.items()}, 1, lr=lr)
    for k in P:
        big = np.abs(G[k]) > 1e-3 * np.abs(G[k]).max()     # away from the sign decision at g = 0
        d = np.abs(new[k] - Q[k])
        assert d[big].max(initial=0) < 1e-6 + 1e-3 * lr, k
        assert d.max() <= 2 * lr + 1e-6, k


def _head(seed):
    from paper_2206_12409_gb300 import inputs as I
    g, er, sg = I.layered_head_phantom(n=(32, 32, 40), h=6.5e-3, seed=seed)
    return I.Problem("head_small", g, er, sg, 298e6)


def _solve(V, torch, ctx, prob, precond, mode=1):
    from oracle import mie
    N = V.vsie_sizes(ctx)[0]
    b = mie.body_rhs(prob.grid, prob.eps_r, prob.sigma, prob.freq_hz)
    B = torch.from_numpy(b.copy()).cuda()[None, :]
    X = torch.zeros_like(B)
    o = V.vsie_solve_opts()
    o.mode, o.restart, o.maxit, o.precond, o.inner_tol = mode, 50, 3000, precond, 1e-3
    st, info = V.vsie_solve(ctx, 1, B.data_ptr(), N, X.data_ptr(), N, 1e-6, o)
    return st, info.iters[0], info.relres[0]


def test_trained_network_reduces_iterations_on_held_out_phantom():
    """Train on phantom A (pairs from A's own operator), then solve the plane-wave
    problem of a different phantom B: flexible GMRES with the network needs fewer
    iterations than with the block preconditioner alone, and both reach a true
    FP64 relative residual of 1e-6."""
    import torch
    from paper_2206_12409_gb300 import vsie as V
    pa, pb = _head(1), _head(2)
    ca = V.setup_problem(pa, max_rhs=1)
    cb = V.setup_problem(pb, max_rhs=1)
    net = V.vsie_net_create(3)
    try:
        st0, it0, rr0 = _solve(V, torch, cb, pb, 0)
        L = V.vsie_net_train(ca, net, 6000, lr=1e-3, seed=5)
        assert np.mean(L[-50:]) < 0.6 * np.mean(L[:50])
        V.vsie_net_attach(cb, net)
        st1, it1, rr1 = _solve(V, torch, cb, pb, 2)
        st2, it2, rr2 = _solve(V, torch, cb, pb, 2, mode=0)
    finally:
        V.vsie_destroy(ca)
        V.vsie_destroy(cb)
        V.vsie_net_destroy(net)
    assert st0 == st1 == st2 == V.VSIE_OK
    assert max(rr0, rr1, rr2) <= 1e-6
    assert it1 < 0.85 * it0 and it2 < 0.85 * it0, (it0, it1, it2)


def test_zero_network_equals_block_preconditioner():
    import torch
    from paper_2206_12409_gb300 import vsie as V
    from paper_2206_12409_gb300 import inputs as I
    g, er, sg = I.layered_head_phantom(n=(16, 16, 24), h=1.3e-2, seed=4)
    ctx = V.setup_problem(I.Problem("h", g, er, sg, 298e6), max_rhs=2)
    net = V.vsie_net_create(1)
    try:
        V.vsie_net_set_params(net, np.zeros(V.vsie_net_num_params(net), np.float32))
        V.vsie_net_attach(ctx, net)
        N = V.vsie_sizes(ctx)[0]
        rng = np.random.default_rng(0)
        x = (rng.standard_normal((2, N)) + 1j * rng.standard_normal((2, N))).astype(np.complex64)
        X = torch.from_numpy(x).cuda()
        Y0, Y2 = torch.zeros_like(X), torch.zeros_like(X)
        V.vsie_precond_apply(ctx, 2, X.data_ptr(), N, Y0.data_ptr(), N, 0)
        V.vsie_precond_apply(ctx, 2, X.data_ptr(), N, Y2.data_ptr(), N, 2)
        torch.cuda.synchronize()
        assert torch.equal(Y0, Y2)
    finally:
        V.vsie_destroy(ctx)
        V.vsie_net_destroy(net)


def test_learned_preconditioner_application_matches_oracle():
    """vsie_precond_apply (kind 2) against the oracle's restatement of the
    preconditioner (Jacobi scaling, RMS normalisation, network, masked
    correction) on a small head phantom, with the same parameters."""
    import torch
    from paper_2206_12409_gb300 import vsie as V
    from paper_2206_12409_gb300 import inputs as I
    g, er, sg = I.layered_head_phantom(n=(16, 16, 20), h=1.3e-2, seed=6)
    prob = I.Problem("h", g, er, sg, 298e6)
    ctx = V.setup_problem(prob, max_rhs=2)
    P = _params(21)
    net = V.vsie_net_create(1)
    try:
        V.vsie_net_set_params(net, _pack(P))
        V.vsie_net_attach(ctx, net)
        N = V.vsie_sizes(ctx)[0]
        assert N == 3 * g.nv
        rng = np.random.default_rng(22)
        x = (rng.standard_normal((2, N)) + 1j * rng.standard_normal((2, N))).astype(np.complex64)
        X = torch.from_numpy(x).cuda()
        Y = torch.zeros_like(X)
        V.vsie_precond_apply(ctx, 2, X.data_ptr(), N, Y.data_ptr(), N, 2)
        torch.cuda.synchronize()
        y = Y.cpu().numpy()
        for c in range(2):
            zo = unet.apply_preconditioner(P, g, er, sg, prob.freq_hz, x[c].astype(np.complex128))
            assert _rel(y[c], zo) < 1e-4
    finally:
        V.vsie_destroy(ctx)
        V.vsie_net_destroy(net)
