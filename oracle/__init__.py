"""CPU FP64 oracle for the Zolotarev-filter interior eigensolver (Li & Yang, arXiv:1701.08935).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` use it.  It shares no code with
``paper_1701_08935_gb300`` (no kernels, helpers, tables or constant generators);
the only shared module is the seeded input generator
``synth`` (a top-level module outside the package), which holds no arithmetic of the method.

Every function is a plain, slow, readable restatement of the paper's
definitions in float64 / complex128, written with numpy (library primitives
such as ``numpy.linalg.eigh`` or ``scipy.sparse.linalg.splu`` serve as single
steps where the paper's definition is a standard matrix operation).

Modules
-------
elliptic  Jacobi elliptic functions and complete elliptic integrals (AGM).
filter    Zolotarev functions (Thm 1), composition (Thm 2, eq. S), Moebius map
          (eq. req), R_ab (eq. R2), partial fractions (Prop 1, Cor 1, Prop 2).
ordering  nested-dissection ordering, assembly tree and front structures.
factor    no-pivot LU of the permuted shifted matrix (dense, small N).
apply     filtered block R_ab(B^-1 A) X: exact partial fractions and the hybrid
          Algorithm 2 (inner direct solves + shift-invariant GMRES).
eigs      Algorithm 1 (subspace iteration + Rayleigh-Ritz), residual metrics,
          Sylvester inertia counts, dense brute force.
"""
