"""FP64 CPU oracle for the reduced-basis iteration (RBI) and RB-preconditioned CG.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or run
this package; only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline /
reference legs of `bench.py` use it.  It shares no code with the CUDA library:
the two read the same seeded inputs from `workloads` and nothing else.

Plain, slow and written to be checked by eye against the paper:
  problem.py   the affine parametrized operator A(mu) = sum_q theta_q(mu) A_q and
               load f(mu) = sum_r phi_r(mu) f_r (eq. 1, eq. 12), finite differences
  smoothers.py the smoother S(A, b, y) of eq. 8 (red-black / lexicographic
               Gauss-Seidel, Jacobi)
  direct.py    truth solves x(mu) = A(mu)^{-1} f(mu) (sparse direct, CG)
  rb.py        reduced system (eqs. 2, 2b, 12b, 12c), RBI (Alg. 2), RBCG (Alg. 3)
  greedy.py    greedy sampling with modified Gram-Schmidt (Alg. 1) and the
               adaptive greedy whose snapshots are RBCG solves (Alg. 4)

Parity pins (tests/test_oracle_*.py) tie every function to something outside
itself: a dense matrix built by a different route, closed-form Laplacian
eigen-solutions, textbook Gauss-Seidel / CG from library routines, and the
lemmas of Section 3.2.
"""
