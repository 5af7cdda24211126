"""FP64 CPU oracle for the matrix-oriented FEM (MO-FEM) / MO-PCG method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library, its
C ABI or the Python binding) may import, call, link or execute anything in this
package.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` use it.

It is a plain, slow, obviously-correct restatement of Frittelli & Sgura,
"Matrix-oriented FEM formulation for stationary and time-dependent PDEs on
x-normal domains" (arXiv 2109.01173), written in numpy/scipy in float64:

* :mod:`oracle.fem1d`      -- 1D Lagrange P_k bases, quadrature and the weighted
                              1D FEM matrices (Sec. 3.1-3.3).
* :mod:`oracle.operator`   -- the Kronecker / multiterm-Sylvester operator and
                              right-hand side on a two-profile x-normal domain
                              (Sec. 3.2, Eq. kronecker_mass_distorted; Sec. 5,
                              Eq. laplace_cap-shaped-domain_sylvester).
* :mod:`oracle.assembly2d` -- independent vector-form 2D assembly on the
                              physical (curvilinear) mesh plus a direct solve
                              (Sec. 5, Eq. laplace_xnormal_FEM); used only to pin
                              the Kronecker decomposition.
* :mod:`oracle.pcg`        -- MO-PCG (Sec. 5, Eqs. laplace_xnormal_pcg /
                              laplace_xnormal_pcg_iteration, standard PCG
                              reading), vector PCG, and the preconditioners:
                              reduced-approach two-term Sylvester solve (Sec. 4,
                              Eq. reduced_formula_for_u), the paper's single-term
                              product preconditioner (Sec. 5, Eq.
                              vector_preconditioner) and AUA (Eq. precSquare).
* :mod:`oracle.closed_form` -- closed-form P1 Dirichlet reduced solve on the
                              square (Sec. 4.1).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, brute-force 2D assembly or manufactured
solutions; none is "parity unpinned".
"""
