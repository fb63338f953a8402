"""CPU FP64 oracle for the Bernstein-Bezier DG acoustic solver (Chan & Warburton,
"GPU-accelerated Bernstein-Bezier discontinuous Galerkin methods for wave problems").

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, independent restatement of
what the paper's method computes.  It shares no code, tables or constants with the CUDA
library.  Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
import it; the product path never does.

Modules
  operators  exact (rational) reference-element operators: Bernstein basis, derivative
             matrices (Lemma 1), mass / face-mass matrices, degree elevation, L0, l_j and
             the face lift L^f = M^{-1} M^f (Section 3.1).
  mesh       connectivity, trace matching and affine geometry (Section 3).
  dg         the semi-discrete right-hand side (Section 2 weak form, eq. (discrete_var)),
             the energy, low-storage RK4, point sources and receivers.
  nodal      Warp & Blend nodes and the nodal (Lagrange) operators (Section 3.1).
  adjoint    the discrete adjoint of the fully discrete scheme and the wavespeed gradient.

Parity unpinned: see the header of ``oracle.nodal`` (Warp & Blend node values are pinned
only through the paper's printed condition numbers).
"""
