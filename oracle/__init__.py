"""FP64 CPU oracle for the GMRF probabilistic PDE solver (arXiv 2503.08343).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code with the CUDA path; both take their
inputs from ``paper_2503_08343_gb300.workloads``, which holds no method
arithmetic.

The oracle computes the plain definitions, slowly and in float64:

* ``fem``     P1 element assembly on structured grids, the lumped-mass SPDE
              precision Q = K^T M^-1 K (Sec. 2.2, eq. sparse-prec-matrix),
              the implicit-Euler space-time prior (Sec. 2.4, App. A) and the
              Dirichlet constraint of App. B, all as an explicit sparse root B
              with Q = B^T B.
* ``observe`` observation matrices: point data (regression rows,
              Sec. 3.1), collocation rows of linear advection-diffusion and of
              Burgers' equation (Sec. 3.1, Sec. 3.3).
* ``linalg``  banded Cholesky (Sec. 3.2, "sparse Cholesky decomposition") and
              Takahashi selected inversion for exact marginal variances.
* ``rng``     Philox4x32-10 (Salmon et al., SC'11) and Box-Muller normals,
              written from the published definitions.
* ``infer``   affine conditioning (Sec. 3.1, eq. posterior-mean), perturbation
              samples through a left square root (Sec. 3.2), the
              Rao-Blackwellised variance estimator (Siden et al. 2018),
              Gauss-Newton with backtracking line search (Sec. 3.3) and the
              Gaussian log marginal likelihood with its gradient.

Pins (tests marked ``not gpu``) tie each function to something other than
itself: closed forms, brute force on tiny inputs, textbook special cases
(dense GP conditioning, Kalman smoothing) and invariants.  Functions without
such a pin say "parity unpinned" in their docstring.
"""
