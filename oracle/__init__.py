"""CPU oracle for the space-time Galerkin FEM of the linear Schroedinger equation.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) imports, calls, links or executes anything under this folder.
Only the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg
use it.  It shares no code with the CUDA path: the only shared module is
`synth` (seeded input data, no method arithmetic).

Everything is plain FP64 (complex128) NumPy/SciPy, written from the paper's
definitions, slow and obviously correct:

  quadrature   Gauss-Legendre (Newton on Legendre polynomials) and a collapsed
               (Duffy) triangle rule.                 -- used for eq. (matrix_x),
                                                         eq. (matrix_t), the load
  fe_time      M_t, B_t, m_t from their integral definitions, eq. (matrix_t),
               P1 and P2 Lagrange elements, t0 DOF removed (Section 3).
  fe_space     structured triangulation, M_x, A_x from eq. (matrix_x), P1.
  fe_mesh      M_x, A_x of eq. (matrix_x) on any triangle (d = 2) or tetrahedron
               (d = 3) mesh, Lagrange P1 and P2, Dirichlet DOFs removed.
  assemble     explicit space-time prism assembly of K = iB_t (x) M_x + M_t (x) A_x
               (eq. LGS) straight from the sesquilinear form a(u,v) of eq.
               (VF_inhomogen) on each prism; load vector and lifting of
               eq. (VF_FEM).
  solve        SuperLU / dense solve of the explicit K; space-eigenbasis solve
               (independent cross-check); Bartels-Stewart (Schur) and fast
               diagonalisation (eig) Kronecker solvers of Section 3; FP64
               Kronecker residual; adjoint.
  timedec      step 1 of the Kronecker solver: (iB_t)^{-1} M_t = X_t S_t X_t^{-1},
               kappa_2(X_t) (Section 3, Table 2).
  norms        space-time L2(Q) and H1(Q)-seminorm errors (Section 4).
  cpu_fdm      independent CPU FP64 FDM over a process pool (the timed CPU
               baseline; mirrors the paper's per-core sparse direct solves).

Pins (tests/test_oracle_*.py) tie every function to something other than itself:
closed-form element matrices, identities, exact quadrature of polynomials,
dense brute force, two independent solvers, the paper's kappa_2(X_t) columns
(Tables 2-3) and its errors / convergence orders (Tables 1-3).
"""
