"""Port network and lumped loads through the C ABI (vsie_rhs_ports, vsie_solve,
vsie_set_loads, vsie_port_network) against oracle.ports on the two-loop problem
(two strip loops, a lossy sphere and a small shield).  The device and the oracle
assemble and compress the operator independently (pFFT projection, TT and ACA at
1e-6).  The operator's condition number is ~1e7 here, and entry-wise relative
noise of 1e-6 on the oracle's operator moves Y by 2.4e-4 of its largest entry, so
Y is compared at 5e-4.  Z and S follow from Y by the same closed forms on both
sides (1e-10); a series load moves Z_00 by exactly Z_L (to the solve accuracy)."""
import numpy as np
import pytest

from paper_2206_12409_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def two():
    from paper_2206_12409_gb300 import vsie as V
    from oracle import hybrid, physics, ports
    p = I.problem_two_loops()
    ctx = V.setup_problem(p, max_rhs=2)
    rows, lens = ports.port_rows(p)
    w, _ = physics.omega_k0(p.freq_hz)
    Zh, _ = ports.hybrid_dense(hybrid.build_parts(p))
    ref = ports.solve_network(Zh, rows, lens, w)
    yield V, ctx, p, ref
    V.vsie_destroy(ctx)


def _network(V, ctx, z0=50.0):
    import torch
    N = V.vsie_sizes(ctx)[0]
    B = torch.zeros((2, N), dtype=torch.complex128, device="cuda")
    V.vsie_rhs_ports(ctx, [0, 1], 1.0, B.data_ptr(), N)
    X = torch.zeros_like(B)
    o = V.vsie_solve_opts()
    o.mode, o.restart, o.maxit = 0, 200, 4000
    st, info = V.vsie_solve(ctx, 2, B.data_ptr(), N, X.data_ptr(), N, 1e-12, o)
    assert st == V.VSIE_OK, (st, info.relres[0], info.relres[1])
    return V.vsie_port_network(ctx, [0, 1], X.data_ptr(), N, z0)


def test_network_against_oracle(two):
    from oracle import ports
    V, ctx, p, (Yo, Zo, So) = two
    Y, Z, S = _network(V, ctx)
    e = np.abs(Y - Yo).max() / np.abs(Yo).max()
    print(f"[port network] |Y - Y_oracle| / |Y| = {e:.2e}; Z00 = {Z[0, 0]:.4f} ohm")
    assert e <= 5e-4
    assert np.abs(Y - Y.T).max() <= 1e-9 * np.abs(Y).max()
    _, Zc, Sc = ports.network(Y, 50.0)
    assert np.abs(Z - Zc).max() <= 1e-10 * np.abs(Zc).max()
    assert np.abs(S - Sc).max() <= 1e-10
    _, _, S75 = _network(V, ctx, 75.0)
    assert np.abs(S75 - ports.network(Y, 75.0)[2]).max() <= 1e-9


def test_series_load_and_reset(two):
    V, ctx, p, _ = two
    _, Z0, _ = _network(V, ctx)
    zl = 3.0 - 20j
    V.vsie_set_loads(ctx, [0], [zl])
    try:
        _, Z1, _ = _network(V, ctx)
    finally:
        V.vsie_set_loads(ctx, [], [])
    D = Z1 - Z0
    print(f"[port load] Z00 shift {D[0, 0]:.6f} for Z_L = {zl}")
    assert abs(D[0, 0] - zl) <= 1e-5 * np.abs(Z0).max()
    D[0, 0] = 0
    assert np.abs(D).max() <= 1e-5 * np.abs(Z0).max()
    _, Z2, _ = _network(V, ctx)
    assert np.abs(Z2 - Z0).max() <= 1e-6 * np.abs(Z0).max()


def test_load_and_network_argument_errors(two):
    import torch
    V, ctx, p, _ = two
    for ports_, z in (([2], [1.0]), ([-1], [1.0]), ([0, 0], [1.0, 2.0]), ([0], [np.nan])):
        with pytest.raises(V.VsieError) as e:
            V.vsie_set_loads(ctx, ports_, z)
        assert e.value.status == V.VSIE_EINVAL
    N = V.vsie_sizes(ctx)[0]
    X = torch.zeros((2, N), dtype=torch.complex128, device="cuda")
    with pytest.raises(V.VsieError) as e:
        V.vsie_port_network(ctx, [0, 1], X.data_ptr(), N, 50.0)
    assert e.value.status == V.VSIE_EBREAKDOWN


def test_drive_rhs_and_cp_mode(two):
    """vsie_rhs_drive with the two-loop circularly polarised voltages equals the
    oracle's superposition of single-port delta-gap columns (rwg.rhs_ports), and
    the solved port currents equal Y v (linearity of the solve)."""
    import torch
    from oracle import physics, ports, rwg
    V, ctx, p, _ = two
    N = V.vsie_sizes(ctx)[0]
    v = V.cp_mode_voltages(2) * (0.7 + 0.2j)
    B = torch.zeros((1, N), dtype=torch.complex128, device="cuda")
    V.vsie_rhs_drive(ctx, [0, 1], v, B.data_ptr())
    b = B.cpu().numpy()[0]
    w, _ = physics.omega_k0(p.freq_hz)
    rows, lens = ports.port_rows(p)
    rc = rwg.build(p.coil)
    cols = rwg.rhs_ports(rc, w, physics.EPS0)
    ref = np.zeros(N, complex)
    ref[rows] = cols[rc.ports, np.arange(2)] * v
    assert np.abs(b - ref).max() <= 1e-15 * np.abs(ref).max()
    assert np.count_nonzero(b) == 2
    X = torch.zeros_like(B)
    o = V.vsie_solve_opts()
    o.mode, o.restart, o.maxit = 0, 200, 4000
    st, _ = V.vsie_solve(ctx, 1, B.data_ptr(), N, X.data_ptr(), N, 1e-12, o)
    assert st == V.VSIE_OK
    x = X.cpu().numpy()[0]
    Y = _network(V, ctx)[0]
    I = x[rows] * lens
    assert np.abs(I - Y @ v).max() <= 1e-6 * np.abs(I).max()
    for bad in (([0, 0], v), ([0, 5], v), ([0, 1], [np.inf, 1.0])):
        with pytest.raises(V.VsieError) as e:
            V.vsie_rhs_drive(ctx, bad[0], bad[1], B.data_ptr())
        assert e.value.status == V.VSIE_EINVAL
