"""FP64 CPU oracle for the hybrid-VSIE method (arXiv 2206.12409).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library never
calls it, and it shares no code with the CUDA library: every formula here is
written out again from the paper (and, where the paper is silent, from the
physics it cites), in plain NumPy/SciPy, slow and obviously correct.

Modules
-------
physics   constants, susceptibility, dyadic Green's function, self term (Sec. II.A)
volume    dense and FFT (Toeplitz) body operator Z_bb (Sec. II.B)
rwg       RWG basis and triangle quadrature (Sec. II.B, Eq. disc_sie)
potint    analytic 1/R potential integrals over a triangle (singularity extraction)
efie      Galerkin coil/shield matrix Z_cc (Eq. sie, Eq. disc_sie)
coupling  body-surface coupling Z_cb, near (8 x 6 points) and far (1 x 1) (Sec. IV.C)
pfft      precorrected-FFT projection, interpolation and precorrection (Sec. II.C, III)
aca       adaptive cross approximation with partial pivoting (Eq. for U V^*)
tt        TT-SVD, TT reconstruction and the TT matvecs of Eq. (mvp) and Eq. (tmvp)
hybrid    operator parts and the hybrid-VSIE matvec of Eq. (hvsie_disc)
gmres     GMRES(m) and flexible GMRES (Sec. III.A)
mie       Mie series for the field inside a homogeneous sphere (solver-level pin)
rhs       plane-wave right-hand side of the hybrid system (Sec. II.A)
ports     lumped loads and the Y, Z, S matrices of the ports (Sec. IV.B, V)
tucker    Tucker (HOSVD) compression of the body block's Green generators (Sec. II.A)

Parity status of each function is stated in its docstring; functions without an
independent pin say "parity unpinned".
"""
