"""Pins of oracle.ports (lumped loads and port network, Sec. IV.B and V): textbook
two-port closed forms for the Y -> Z -> S step; the loop inductance and radiation
resistance of a strip loop through the network path; and, on the two-loop
problem with a lossy body and the uncompressed dense operator, reciprocity,
the mirror symmetry of the geometry, passivity and the exact shift of Z_ii by a
series load."""
import numpy as np
import pytest

from paper_2206_12409_gb300 import inputs as I
from oracle import efie, hybrid, physics, ports, rwg


def test_matched_t_attenuator():
    """A T attenuator with voltage ratio K matched to z0 has S11 = S22 = 0 and
    S21 = S12 = 1/K; its arms are z0 (K-1)/(K+1) and its leg 2 z0 K/(K^2-1)."""
    z0, K = 50.0, 3.0
    za = z0 * (K - 1) / (K + 1)
    zc = 2 * z0 * K / (K * K - 1)
    Z = np.array([[za + zc, zc], [zc, za + zc]], complex)
    Y, Z2, S = ports.network(np.linalg.inv(Z), z0)
    assert np.abs(Z2 - Z).max() < 1e-12 * np.abs(Z).max()
    assert abs(S[0, 0]) < 1e-14 and abs(S[1, 1]) < 1e-14
    assert abs(S[1, 0] - 1 / K) < 1e-14 and abs(S[0, 1] - 1 / K) < 1e-14


def test_one_port_limits():
    """S of a one-port: matched load 0, short -1, open (tiny Y) +1, and the
    reflection coefficient (Z - z0)/(Z + z0) for a reactive load."""
    z0 = 50.0
    assert abs(ports.network([[1 / z0]], z0)[2][0, 0]) < 1e-15
    assert abs(ports.network([[1e12]], z0)[2][0, 0] + 1) < 1e-9
    assert abs(ports.network([[1e-12]], z0)[2][0, 0] - 1) < 1e-9
    zl = 20 + 35j
    assert abs(ports.network([[1 / zl]], z0)[2][0, 0] - (zl - z0) / (zl + z0)) < 1e-14


def test_loop_impedance_through_the_network():
    """The 40 mm strip loop at 10 MHz: Z_in from solve_network on the EFIE
    operator has X = omega mu0 R (ln(8R/a) - 2), a = w/4, within 5% and
    R = 20 pi^2 (C/lambda)^4 within 3%."""
    f = 10e6
    r = rwg.build(I.loop_strip(40e-3, 2e-3, 128))
    w, k0 = physics.omega_k0(f)
    Z = -efie.K_dense(r, r, k0, True)
    _, Zp, _ = ports.solve_network(Z, r.ports, r.length[r.ports], w)
    L = physics.MU0 * 0.04 * (np.log(8 * 0.04 / 0.5e-3) - 2)
    assert abs(Zp[0, 0].imag / (w * L) - 1) < 0.05
    Rrad = 20 * np.pi ** 2 * (2 * np.pi * 0.04 * f / physics.C0) ** 4
    assert abs(Zp[0, 0].real / Rrad - 1) < 0.03


@pytest.fixture(scope="module")
def two_loops():
    p = I.problem_two_loops()
    Z, _ = hybrid.dense_operator(p)
    rows, lens = ports.port_rows(p)
    w, _ = physics.omega_k0(p.freq_hz)
    return p, Z, rows, lens, w


def test_port_rows(two_loops):
    p, Z, rows, lens, w = two_loops
    mf = rwg.build(p.shield).m
    rc = rwg.build(p.coil)
    assert rows.tolist() == [mf + e for e in rc.ports] and rows.size == 2
    assert np.allclose(lens, rc.length[rc.ports])


def test_reciprocity_symmetry_passivity(two_loops):
    """Y = Y^T; the loops are images of each other under a half turn about z that
    maps body, shield and grid onto themselves, so Y00 = Y11; the body and the
    radiation take power, so Re Z is positive definite and I - S^H S positive
    semidefinite."""
    p, Z, rows, lens, w = two_loops
    Y, Zp, S = ports.solve_network(Z, rows, lens, w)
    assert np.abs(Y - Y.T).max() <= 1e-12 * np.abs(Y).max()
    assert abs(Y[0, 0] - Y[1, 1]) <= 1e-9 * abs(Y[0, 0])
    assert np.linalg.eigvalsh((Zp + Zp.conj().T) / 2).min() > 0
    assert np.linalg.eigvalsh(np.eye(2) - S.conj().T @ S).min() > 0


@pytest.mark.parametrize("zl", [3.0 - 20j, 0.5 + 100j, -1j / (2 * np.pi * 298e6 * 5e-12)])
def test_series_load_shifts_z_by_exactly_zl(two_loops, zl):
    """A series element at port 0 adds Z_L to Z_00 and leaves the rest of the
    port impedance matrix unchanged (the load is in series with the source)."""
    p, Z, rows, lens, w = two_loops
    _, Z0, _ = ports.solve_network(Z, rows, lens, w)
    _, Z1, _ = ports.solve_network(Z, rows, lens, w, loads={0: zl})
    D = Z1 - Z0
    assert abs(D[0, 0] - zl) <= 1e-9 * max(abs(zl), np.abs(Z0).max())
    D[0, 0] = 0
    assert np.abs(D).max() <= 1e-9 * np.abs(Z0).max()


def test_compressed_network_close_to_dense(two_loops):
    """The network of the compressed operator (TT, ACA, pFFT with the 3^3
    stencil) is within 1e-3 of the dense operator's."""
    p, Z, rows, lens, w = two_loops
    Yd = ports.solve_network(Z, rows, lens, w)[0]
    Zh, sel = ports.hybrid_dense(hybrid.build_parts(p))
    assert (sel[:rows.max() + 1] == np.arange(rows.max() + 1)).all()
    Yh = ports.solve_network(Zh, rows, lens, w)[0]
    assert np.abs(Yh - Yd).max() <= 1e-3 * np.abs(Yd).max()
