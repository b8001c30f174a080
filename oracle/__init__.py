"""FP64 CPU oracle for the RWG-discretised EFIE and the refinement-free
Calderon multiplicative preconditioner (RF-CMP) of Adrian, Andriulli, Eibert
(arXiv 1803.08333).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product path (``paper_1803_08333_gb300``) never imports it,
and it never imports the product path: the two share no code.  Both take their
inputs from ``synth`` (seeded meshes and plane waves).

Plain, slow, obviously correct: numpy/scipy in float64/complex128, loops or
vectorised numpy over triangle pairs, dense linear algebra from numpy where a
library routine is a step (LU, Cholesky, eigenvalues).  Each function cites the
passage of the paper it follows.

Modules
  topology   edges, c+/c-, free vertices, Sigma, Lambda, genus  (Sec. 2, Eq. RWGdef, Eq. qHofj)
  quadrature 7-point triangle rule and per-cell geometry
  potentials analytic integrals of 1/R and (r'-p)/R over a triangle
  efie       T_A, V, T_Phi = Sigma V Sigma^T, T, excitation e  (Sec. 2)
  gram       G_ll, G_pp, G_ff, P1 stiffness matrix Delta        (Sec. 2)
  rfcmp      projectors, P_o, P_m, alpha/beta/gamma, A, b        (Sec. 3, Sec. 4)
  krylov     CG, CGS, dense LU solve                              (Sec. 3.4, Sec. 4)
  farfield   scattered far field and bistatic RCS
  mie        Mie series of a PEC sphere (textbook closed form)

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` (closed forms, identities, brute force, Mie series).
"""
