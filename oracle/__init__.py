"""CPU FP64 oracle for the multilevel local-and-parallel P1 eigensolver.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The product path (the CUDA library and its Python binding) never
imports, calls or links anything here, and this package imports nothing from
the product.

It restates, plainly and slowly, what the paper (Li, Han, Xie, You, "Local and
parallel finite element algorithm based on multilevel discretization for
eigenvalue problem") computes:

* ``mesh``      - coarse triangulation T_H, regular (red) refinement T_{h_k}
                  (Section 4.2), nodal interpolation between nested P1 spaces;
* ``fem``       - P1 stiffness a(u,v) = (kappa grad u, grad v) and mass
                  b(u,v) = (u,v) (Sections 2.2 and 3), element by element;
* ``partition`` - D_j, Omega_j, G_j and G_{m+1} (Section 4, before Algorithm 4.1);
* ``multilevel``- Algorithm 4.2 (level-1 eigenproblem, then Correction steps),
                  Algorithm 4.1 (auxiliary local problems, gluing with the
                  G_{m+1} problem, Rayleigh-Ritz on V_{0H} + span{u~});
* ``multiple``  - the same for the q smallest eigenpairs (the subspace form: one
                  correction per eigenpair, one Rayleigh-Ritz on
                  V_{0H} + span{u~_1 .. u~_q}; Section 4's multiple-eigenvalue remark,
                  Table 1);
* ``tensor``    - Example 2's full-tensor coefficient and weighted mass (Section 6);
* ``p2``        - quadratic elements for Example 1 (Section 6);
* ``cube3d``    - the d = 3 case on box domains with Kuhn tetrahedra (Sections 2.1 and
                  4.2), run through the same ``multilevel`` / ``multiple`` steps.

Everything is float64, with sparse direct solves (``scipy.sparse.linalg.splu``)
and dense generalized symmetric eigensolves (``scipy.linalg.eigh``).

Parity status: every function here is pinned by a ``-m "not gpu"`` test against
a closed form, a brute-force computation, an exact identity or a special case
(see ``tests/test_oracle_*.py``). The absolute numbers of Table 1 are NOT
reproducible (the paper does not state its mesh, H, delta or subdomains), so
those values are "parity unpinned"; only their convergence orders are pinned.
"""
