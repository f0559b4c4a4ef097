"""CPU oracle for the XRL hot path -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, FP64 NumPy restatement of what the method
computes, written from the paper (Sec. II, eqs. 1-12, Algorithm 1).  Only the
test suite, the smoke check and the CPU-baseline leg of the benchmark may
import it; the CUDA library never does, and the two share no code.  The only
thing both sides consume is the seeded mesh generator package `meshgen`.

Modules and what pins them (tests under tests/test_oracle_*.py):

* quadrature  -- Gauss-Legendre based triangle rules.  Pinned by exact
  integration of monomials (closed-form moments of the reference triangle).
* panels      -- panel geometry, analytic potential of a uniform triangle,
  closed-form self integral, the near/far rule table and the dense matrix
  P (Sec. II-A eq. 6, Sec. II-C).  Pinned by brute-force adaptive quadrature,
  the Reynolds-transport edge identity for the self term, the point-charge
  limit, scaling P(s*geom) = P/s, symmetry and positive definiteness.
  Rectangular panels of hybrid meshes (panels.Panels, P as the area-weighted
  sum over the two triangles of each rectangle) are pinned by the closed-form
  self and edge-adjacent integrals of coplanar rectangles and by a reduced
  2-D quadrature of aligned rectangle pairs (tests/test_oracle_rect.py).
* esi         -- the double-plane surface impedance (eq. 3).  Pinned by its
  DC and high-frequency limits and by the skin depths the paper prints.
* circuit     -- PEEC branches, centroid-midpoint matrices A_t (Algorithm 1,
  eq. 4-5), fundamental-cycle loop matrix M (Sec. II-B), loop impedance
  (eq. 7-8), direct solve and port R, L.  Pinned by the uniform-current
  identity of the CM transform, M B^T = 0, the cycle-space dimension, DC
  resistance rho*L/A of a bar, reciprocity, positive definiteness of R and L,
  the Neumann mutual inductance of two parallel thin bars, and agreement with
  an independent nodal (MNA) formulation on small meshes.
* precond     -- the diagonal-of-P preconditioner Q (eq. 10) built densely.
  Pinned by Q equalling the loop operator with P replaced by diag(P), and
  by positive definiteness of its real and imaginary parts.  The diagonal-of-L
  comparison preconditioner of Sec. II-D and Table IV (circuit.precond_matrix_L:
  the loop-space Z_s kept whole plus the branch diagonal of the inductance) is
  pinned by the loop operator with its potential part switched off plus a
  per-branch sum written out from the edge midpoints and panel centroids,
  complex symmetry, positive definiteness and the sparsity of eq. 10.

Parity unpinned: none of the functions above is without a pin; the paper
prints no worked numeric example of A, P, Q or Z, so the pins are closed
forms, invariants and brute force as listed.
"""
