"""FP64 CPU oracle for the BRAS mass-inverse approximation (test infrastructure only).

This package is the slow, plain reference that the CUDA path is checked against.  Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` may import it; the product path never does.  It shares no code with the
CUDA library: the only common input is the seeded generator
``paper_2607_12138_b300.meshgen``, which holds none of the method's arithmetic.

Modules
-------
``polynomials``  dense monomial polynomials and exact simplex integrals.
``elements``     reference Lagrange / Nedelec / Raviart-Thomas / BDM elements by monomial
                 spans dualised against the documented dof functionals (tetrahedra and
                 triangles; first kinds N1curl / RT and second kinds N2curl / BDM, the
                 second kinds' face and interior moments taken against the first kinds'
                 own nodal bases); the Bernstein basis (space "h1b") by multinomial
                 expansion.
``assembly``     Piola metrics (Sec. 2.4, Eq. piola_mass_pullbacks), element matrices,
                 assembled M (Eq. M_PMbrP), multiplicity D, explicit BRAS
                 (Eq. mhatinvbras_def), Jacobi diag(M).
``solvers``      textbook PCG with the paper's stopping rule (Sec. 3), damped fixed point,
                 Chebyshev semi-iteration, power iteration, CG-Lanczos, dense spectral tools
                 (Eq. spectral-kappa).
``schur``        mixed Poisson divergence matrix and Schur complements -S = B M^{-1} B^T,
                 -S~ = B M_bras^{-1} B^T (Sec. 4, Sec. 5.1) for RT_k or BDM_k / DG_{k-1}.
``gradient``     adjoint gradient of the density-weighted mass solve.
``sampled``      one-dof-at-a-time BRAS / mass outputs for meshes too large to assemble.

Parity status: every function here is pinned by a ``-m "not gpu"`` test against a
closed form, a theorem of the paper, a value printed in the paper, or brute force.
The Lagrange elements of order 3-4, the N1curl / RT elements of order 2-4 and the
N2curl / BDM elements of order 3-4 use this project's documented node / moment convention,
which differs from the paper's (GLL nodes, Firedrake moments): their kappa values are
unpinned against the paper's tables, while the theorems (SPD, lambda_min >= 1,
one-element exactness, Lemma bras_exact_inverse_correction, Theorem
bras_lambda_max_projector), conformity and polynomial reproduction pin them.  The Bernstein
basis is canonical and is pinned to Table 1 at every order; N2curl / BDM of orders 1-2 are
pinned to Tables 2-3.
"""
