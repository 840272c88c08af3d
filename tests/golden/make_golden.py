"""Writes tests/golden/oracle_values.json from the FP64 oracle only.

These stored values freeze the oracle's arithmetic: tests/test_golden.py
recomputes them and fails on any change, so that a change to the oracle is
deliberate (the file is regenerated by running this script, and the change is
justified by the passage of the paper or the reading it follows).  Inputs are
fixed numbers and the seeded generators of paper_2206_12409_gb300.inputs.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import mie, physics, volume  # noqa: E402
from paper_2206_12409_gb300 import inputs as I  # noqa: E402


def c2l(z):
    z = np.asarray(z, np.complex128).ravel()
    return [[float(v.real), float(v.imag)] for v in z]


def values():
    f = 298e6
    _, k0 = physics.omega_k0(f)
    out = {"freq_hz": f}
    out["self_term"] = {str(h): c2l(physics.self_term(k0, h)) for h in (2e-3, 5e-3, 1e-2)}
    offs = [(1, 0, 0), (1, 1, 0), (2, 1, 1), (0, 3, -2)]
    out["voxel_kernel_h5mm"] = {str(o): c2l(physics.voxel_kernel(np.array(o), 5e-3, k0)) for o in offs}
    pts = np.array([[0.0, 0.0, 0.0], [5e-3, -3e-3, 8e-3], [-1.2e-2, 4e-3, -6e-3]])
    out["mie_interior_eps50_sig0.6_a25mm"] = c2l(mie.interior_field(pts, 25e-3, 50.0, 0.6, f))
    g, er, sg = I.sphere_phantom(n=(5, 5, 5), h=1e-2, radius=20e-3, eps_r=50.0, sigma=0.6)
    chi = physics.chi(er, sg, f)
    x = I.random_vectors(3 * g.nv, 1).ravel()
    y = volume.dense_matvec(g, chi, k0, x).ravel()
    out["dense_body_matvec_5cube_every7th"] = c2l(y[::7])
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_values.json"), "w") as fh:
        json.dump(values(), fh, indent=1)
    print("wrote", os.path.join(HERE, "oracle_values.json"))
