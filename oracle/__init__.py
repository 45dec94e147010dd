"""Plain FP64 CPU oracle for the low-rank parameter-dependent FSI method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` use it.  It shares no code, header,
table or constant generator with the CUDA library under
``paper_2008_10275_gb300/``; the only common input is the seeded generator
module ``paper_2008_10275_gb300.inputs`` which holds no arithmetic of the
method.

Contents (each function cites the passage of the paper it follows):

* ``fsi``       -- mesh, DOF layout, Dirichlet data b_D and the Q2/Q2/Q1 finite
                   element residual R(x; mu, nu) and Jacobian J(x; mu, nu) of the
                   stationary FSI weak form (Sec. 2, Eq. (fsi_problem_weak1)),
                   both assembled directly and as the affine pieces
                   R0, Rmu, Rnu / J0, Jmu', Jnu' (Sec. 3, Eq. (pardep_matrix1));
                   the four-parameter forms of Sec. 4.4 (``*4``).
* ``params``    -- little-endian ordering, clustering into K subsets, upper
                   median index, diagonal matrices (Sec. 3.3, Def. 1, Eq.
                   (clustering1), Ex. 1-2; Sec. 3.4 Def. "Diagonal Matrices").
* ``newton``    -- per-parameter Newton iteration with a sparse direct solve
                   (Sec. 3.2, Eq. (newton_step_indiv1); four parameters,
                   Sec. 4.4).
* ``lowrank``   -- the subset matrix equation F(S_k) = B_k (Sec. 3.4, Eq.
                   (rhs_matrix1), Eq. (newton_matrix1)), its brute-force
                   column-by-column solution (Eq. (newtonstep_vectornot1)), the
                   mean-based preconditioner (Sec. 4.2) and the truncated,
                   preconditioned Chebyshev iteration and GMRES on dense
                   matrices.
* ``algorithm1``-- Algorithm 1 and the relative residual of Sec. 5.1.2.

Every floating-point computation is FP64.  Parity pins live in
``tests/test_oracle_*.py``.
"""
