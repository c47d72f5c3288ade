"""Plain, slow FP64 CPU oracle for the GenEO-preconditioned laminate solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link anything in this package: only the tests, the smoke check and the
benchmark's CPU-baseline leg use it.  It shares no code with the CUDA
library; the only module both sides read is the seeded input description in
``paper_1707_04228_gb300/inputs.py``, which holds none of the method's
arithmetic.

Modules
  fem    -- Q2 hexahedron, Gauss rule, orthotropic/isotropic stiffness and its
            rotation, mesh geometry, element stiffness, assembly, loads,
            Dirichlet lifting, direct solve, stress recovery (Sections 2.1-2.3).
  geneo  -- overlapping decomposition, partition of unity, local Dirichlet and
            Neumann matrices, GenEO eigenproblems, coarse space, additive
            two-level Schwarz, PCG (Section 2.3).
  adjoint -- adjoint gradient of the resin stress p-norm with respect to the
            misalignment angles, by direct solves (Section 3).
  serendipity -- the 20-node serendipity hexahedron of the paper's own code
            (Section 2.1) on the same laminates; no GPU counterpart yet.

Every function cites the passage it follows.  Where the paper is silent the
docstring says which reading is taken.  Parity unpinned: none of the paper's
printed stress figures (Fig. stresses, Table per) are used, since they need a
different geometry, element and boundary conditions.
"""
