"""Port network of the conductors: lumped loads and the Y, Z, S matrices of the
ports (Sec. IV.B and V: the coil ports with their tuning and matching elements).

Test infrastructure only (see oracle/__init__.py).

Every port is driven in turn by a 1 V delta gap (right-hand side
i omega eps0 V l_m on its edge, rwg.rhs_ports) with the other ports shorted.  The
current through the edge of port i for the excitation of port j is
I_ij = j_i l_i, so Y = I / (1 V), Z = Y^-1 and S = (Z - z0 I)(Z + z0 I)^-1.
A lumped impedance Z_L in series with a port edge m drops -Z_L I_m across the gap,
which moves to the left-hand side as i omega eps0 Z_L l_m^2 on the diagonal entry
(m, m) of the operator.

Pinned by (tests/test_oracle_ports.py): reciprocity Y = Y^T (the operator is
complex-symmetric); a series load Z_L at port i adds exactly Z_L to Z_ii and
nothing else; passivity with a lossy body (I - S^H S positive semidefinite); and,
through the single-loop input impedance 1 / (j l), the low-frequency loop
inductance pin of tests/test_oracle_surface.py.
"""
from __future__ import annotations

import numpy as np

from . import hybrid, physics, rwg


def load_diagonal(omega, length, z_load):
    """Diagonal addition of a series load Z_L on an edge of length l."""
    return 1j * omega * physics.EPS0 * np.asarray(z_load, complex) * np.asarray(length, float) ** 2


def network(I, z0=50.0):
    """(Y, Z, S) from the port currents I (nports x nports) of 1 V drives."""
    Y = np.asarray(I, complex)
    Z = np.linalg.inv(Y)
    E = np.eye(Y.shape[0])
    S = (Z - z0 * E) @ np.linalg.inv(Z + z0 * E)
    return Y, Z, S


def port_rows(prob):
    """Unknown indices and edge lengths of the ports, [shield ports; coil ports]."""
    rows, lens = [], []
    mf = 0
    if prob.shield is not None:
        rf = rwg.build(prob.shield)
        rows += list(rf.ports)
        lens += list(rf.length[rf.ports])
        mf = rf.m
    if prob.coil is not None:
        rc = rwg.build(prob.coil)
        rows += [mf + e for e in rc.ports]
        lens += list(rc.length[rc.ports])
    return np.asarray(rows, int), np.asarray(lens, float)


def solve_network(Z, rows, lens, omega, z0=50.0, loads=None):
    """Port network of the dense operator Z over the unknowns that the port rows
    index.  loads: {port index: Z_L}."""
    Z = np.array(Z, complex)
    for q, zl in (loads or {}).items():
        Z[rows[q], rows[q]] += load_diagonal(omega, lens[q], zl)
    n = rows.size
    B = np.zeros((Z.shape[0], n), complex)
    for j in range(n):
        B[rows[j], j] = 1j * omega * physics.EPS0 * 1.0 * lens[j]
    X = np.linalg.solve(Z, B)
    I = X[rows, :] * lens[:, None]
    return network(I, z0)


def hybrid_dense(P):
    """The compressed hybrid operator of Eq. (hvsie_disc) (oracle.hybrid.matvec on
    the parts P) as a dense matrix, column by column (small problems), restricted
    to the active unknowns [j_f; j_n; j_b on material voxels].  Returns (Z, sel),
    sel the indices of those unknowns in the full vector."""
    nb = P.chi.size
    mat = np.nonzero(P.chi != 0)[0]
    sel = np.concatenate([np.arange(P.m_f + P.m_n)]
                         + [P.m_f + P.m_n + a * nb + mat for a in range(3)])
    Z = np.zeros((sel.size, sel.size), complex)
    for c0 in range(0, sel.size, 64):
        c1 = min(c0 + 64, sel.size)
        E = np.zeros((P.N, c1 - c0), complex)
        E[sel[c0:c1], np.arange(c1 - c0)] = 1.0
        Z[:, c0:c1] = hybrid.matvec(P, E)[sel]
    return Z, sel
