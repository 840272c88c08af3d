"""Pins of oracle.tucker (Tucker/HOSVD compression of the body block's Green
generators, Sec. II.A): exact at full rank, within the HOSVD error bound when
truncated, multilinear rank (1, 1, 1) for a separable tensor, the parity
re-embedding of the exact octants equal to the direct evaluation at every
offset, and the body matvec with the compressed generators within a small
multiple of the tolerance of the uncompressed product."""
import numpy as np
import pytest

from oracle import physics, tucker, volume
from paper_2206_12409_gb300 import inputs as I


def _rand(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


def test_full_rank_reconstruction_is_exact():
    T = _rand((5, 6, 7), 1)
    core, U = tucker.hosvd(T, 0.0)
    assert core.shape == (5, 6, 7)
    assert np.abs(tucker.reconstruct(core, U) - T).max() <= 1e-12 * np.abs(T).max()


@pytest.mark.parametrize("tol", [1e-1, 1e-2, 1e-3])
def test_truncation_error_bound(tol):
    # a tensor with decaying multilinear spectrum
    r = np.random.default_rng(2)
    A, B, C = (np.linalg.qr(_rand((12, 12), s))[0] for s in (3, 4, 5))
    S = _rand((12, 12, 12), 6) * np.exp(-0.6 * np.add.outer(np.add.outer(np.arange(12), np.arange(12)), np.arange(12)))
    T = np.einsum("ia,jb,kc,abc->ijk", A, B, C, S)
    core, U = tucker.hosvd(T, tol)
    err = np.linalg.norm(tucker.reconstruct(core, U) - T) / np.linalg.norm(T)
    assert err <= tol
    assert max(core.shape) < 12            # something was truncated


def test_separable_tensor_has_rank_one():
    a, b, c = _rand(7, 7), _rand(8, 8), _rand(9, 9)
    T = np.einsum("i,j,k->ijk", a, b, c)
    core, U = tucker.hosvd(T, 1e-12)
    assert core.shape == (1, 1, 1)
    assert np.abs(tucker.reconstruct(core, U) - T).max() <= 1e-12 * np.abs(T).max()


@pytest.mark.parametrize("n,L", [((5, 4, 6), None), ((5, 4, 6), (12, 9, 14))])
def test_parity_embedding_matches_direct_evaluation(n, L):
    _, k0 = physics.omega_k0(298e6)
    h = 5e-3
    G = tucker.generator_octants(n, h, k0)
    E = tucker.embed_octants(G, n, L)
    D = volume.embedded_kernel(n, h, k0, L)
    assert np.abs(E - D).max() <= 1e-12 * np.abs(D).max()


def test_compressed_generators_in_the_body_matvec():
    """24^3 sphere at 5 mm, 298 MHz: at tol 1e-6 the matvec differs from the
    uncompressed one by less than 1e-5 and every component compresses."""
    g, er, sg = I.sphere_phantom((24, 24, 24), 5e-3, 55e-3, 50.0, 0.6)
    _, k0 = physics.omega_k0(298e6)
    chi = physics.chi(er, sg, 298e6)
    x = I.random_vectors(3 * g.nv, 1, seed=9)
    y0 = volume.fft_matvec(g, chi, k0, x)
    spec, ranks = tucker.compressed_spectra(g.n, g.h, k0, 1e-6)
    y1 = volume.fft_matvec(g, chi, k0, x, spec=spec)
    M3 = np.tile(chi != 0, 3)
    e = np.linalg.norm((y1 - y0)[M3]) / np.linalg.norm(y0[M3])
    assert e <= 1e-5, e
    assert all(max(r) < 24 for r in ranks), ranks
