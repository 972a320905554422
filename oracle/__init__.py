"""FP64 CPU oracle for the shifted Laplace rational-filter eigensolver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import, call or
link this code: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path; both sides only share the seeded input generators
of ``workloads/``.

Modules, each citing the passage of the paper it follows:

* ``poles``     -- rational filter Phi (Eq. for Phi(lambda), Eq. of the SLRF
                   filter, Section 3.1), quadrature-rule pole sets on a circle
                   (Section 3.2), SLRF least-squares design (Section 3.1),
                   separation factor (Definition 3.1).
* ``filter``    -- the filter operator U = sum_j 2 Re(w_j (A - sigma_j B)^{-1} B V)
                   with sparse direct LU per pole (Section 3, conjugate-pair
                   reduction; Algorithm 1, steps solve / accumulate), and the
                   residual-corrected form of the same operator.
* ``rr``        -- Rayleigh-Ritz and residual norms (Algorithm 1, projection,
                   small eigenproblem and stopping rule).
* ``subspace``  -- Algorithm 1 end to end with exact solves.
* ``inertia``   -- eigenvalue counts in (0, gamma] by Sylvester's law of
                   inertia; closed-form 1D/2D spectra.

Parity status: the SLRF optimiser (Section 3.1) is "parity unpinned": the paper
does not state the optimiser, grid, starting points or a pole-distinctness
constraint, so the design is checked by properties only (real on the real axis,
conjugate symmetry, scaling in gamma, growth of the separation factor with N).
The Gauss-Chebyshev rule is pinned only by its ordering properties because the
paper gives no formula for it.  Everything else is pinned to closed forms,
brute force or library routines in ``tests/test_oracle_pins.py``.
"""
