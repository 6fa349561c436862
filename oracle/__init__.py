"""Plain, slow CPU oracle for the high-order FEM fast direct Poisson solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA path and never imports it.

What it computes, and from which passage of Zlotnik & Zlotnik (arXiv:1609.07758):

* ``element``  -- exact local stiffness/mass matrices A, C of the equispaced
  Lagrange element on [-1, 1] and their 3x3 block form (Sect. 2, par. 1, Eq. matrAC).
* ``hp``       -- Python ``decimal`` helpers (pi, cos, sqrt) used where FP64 is
  not accurate enough (the paper itself used quadruple precision, Sect. 2 par. 5).
* ``spectrum`` -- the 1D spectrum of A v = lambda C v from Theorem 1: element
  eigenpairs of (A~, C~) (Lemma 1), the roots of the theta-equation (Eq. theta),
  the vectors p_k^(l) (Lemma 2) and the C-norms (Theorem 2, part 2).
* ``assemble`` -- the global 1D matrices (Eq. eig_glob) and the N-D operator
  (Eq. bvp glob 2), dense, in exact or FP64 arithmetic.
* ``solve``    -- algorithm (a) written as plain dense mode products with the
  eigenvector matrices (Eq. decomp v 2), and a brute-force exact Kronecker solve.
* ``load``     -- the FEM average f^h by (n+1)-point Gauss quadrature (Sect. 2 par. 5).

Parity status of each function is stated in its docstring; every function is
pinned by ``tests/test_oracle_*.py`` (marked ``not gpu``).
"""
