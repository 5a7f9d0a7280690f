"""Plain FP64 CPU oracle for the D2Q9 stream-and-collide method of Coreixas, Wissocq,
Chopard & Latt, "Impact of collision models on the physical properties and the stability
of lattice Boltzmann methods" (arXiv:2002.05265).

THIS PACKAGE IS TEST INFRASTRUCTURE. Only the test suite, the smoke check of the package
entry module and the CPU-baseline leg of the benchmark may import it. The product path
(the CUDA library and its Python binding) never imports, links or calls anything here,
and nothing here imports the product path.

Design rules followed throughout:
  * every function cites the section / equation of the paper it restates;
  * the arithmetic is the paper's definition written out literally in FP64 (numpy),
    vectorised over lattice nodes only, with no blocking, fusion or reordering;
  * every function works unchanged on complex128 arrays, so that exact derivatives can be
    taken by the complex-step method (used for the collision Jacobian of Appendix A);
  * the state is the pre-collision population field f[i, y, x] (9 x ny x nx), streamed by
    an explicit periodic push, which is deliberately a different organisation from the
    GPU kernels (pull, fused, deviation variables).

Modules
  d2q9         lattice constants (Sec. 2)
  moments      raw / Hermite / central / central-Hermite / cumulant transforms (App. B)
  equilibrium  extended and second-order equilibria (Eq. extendedFeq)
  collision    BGK, RM, HM, CM, CHM, K, PR, RR collision models (App. B)
  lbm          macroscopic fields, periodic streaming, time stepping (Eq. StreamCollide)
  lsa          collision Jacobian and the discrete eigenproblem (App. A)
  adjoint      reference gradients of a final-state loss (complex step through a run)

Parity status: K (cumulant) is pinned internally and against the paper's simulation
statements (Sec. 5b; tests/test_oracle_k_readings.py); its agreement with the paper's
linear-stability statements (Secs. 4b, 4c) is "parity unpinned": no reading of the cumulant
rebuild reproduces those and the simulations together.
"""

from . import d2q9, moments, equilibrium, collision, lbm, lsa, adjoint  # noqa: F401
