"""Plain FP64 CPU oracle for the IPM hot path (Kusch, Wolters, Frank, arXiv:1912.09238).

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference arm may import it. The product path (the CUDA
library under ``paper_1912_09238_gb300/``) never imports, links or calls anything here,
and nothing here imports the product. The two share no code.

What it computes, module by module (each function cites the passage it follows):

* ``basis``    -- total-degree multi-indices (Sec. 2, Eq. numberBasisFcts), orthonormal
                  Legendre gPC basis (Sec. 2, Eq. SGClosure), tensor Gauss-Legendre
                  quadrature <.>_Q (Sec. 3.1).
* ``entropy``  -- entropies s, their gradients, the ansatz u_s = (grad s)^-1 (Sec. 3.1),
                  the Jacobian grad u_s and the Legendre transform s_* (Sec. 2, Eq. dualProblem;
                  App. B for Euler, with the sign correction of the alpha exponent).
* ``physics``  -- Burgers (App. A) and Euler (Sec. 7.1) fluxes, wave speeds, the
                  Lax-Friedrichs numerical flux (App. A, Eq. numFluxAnalytic, per-node form).
* ``dual``     -- the discrete dual cost L (Eq. L), its gradient and Hessian (Sec. 3.1),
                  the Newton map d (Eq. dualIterationFunction) with an Armijo line search,
                  and the stopping criterion (Eq. tauCrit).
* ``scheme1d`` -- the kinetic-flux moment update c (Eq. momentIterationFunction /
                  Eq. momentUpQuadrature), Algorithm 1 (IPM) and Algorithm 2 (One-Shot IPM)
                  for 1-D problems, the steady residual (Eq. residualSteady).
* ``scheme2d`` -- the same on structured 2-D quadrilateral meshes (Sec. 7 Euler system).
* ``adaptive`` -- the smoothness indicator (Eq. errorIndicator) and Algorithm 3.
* ``collocation`` -- Stochastic Collocation (Sec. 2, Sec. 7): the deterministic scheme with the
                  same flux run once per quadrature node, each node on its own time steps.

Everything is float64 numpy. Vectorisation over cells (and over quadrature nodes) is the
only liberty taken: every cell still runs its own iteration with its own stopping test;
no blocking, fusion or reordering beyond the paper's definitions.

Parity status of each function is stated in its module docstring ("pinned by" lists
the tests in ``tests/test_oracle_*.py`` that fix it against the paper or mathematics).
"""
