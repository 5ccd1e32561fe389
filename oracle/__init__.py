"""CPU oracle for y = sgn(gamma5 D_w(mu)) x by the nested Krylov method.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, double-precision
restatement of the paper's definitions (Bloch & Heybrock, "A nested Krylov
subspace method for the overlap operator", Lattice 2009). Only the test suite,
the smoke check and the CPU-baseline leg of the benchmark may import it. The
CUDA library never calls it, and it never calls the CUDA library; the two share
only the seeded input generators in ``ovinputs``.

Modules
  dirac   -- gamma matrices, the Wilson-Dirac operator with chemical potential,
             A = gamma5 D_w(mu) and its adjoint (Sec. 1, Eq. (Dov)).
  krylov  -- outer Lanczos / two-sided Lanczos, the preconditioned inner
             Krylov level, Roberts-Higham, recombination, stopping rule
             (Sec. 2, Eqs. (approximation), (Roberts); Sec. 3, Eqs. (nested),
             (precond)).
  exact   -- the spectral definition (Eq. (specdef)) for dense matrices, the
             Roberts-Higham iteration on a full dense matrix, and the
             closed-form free-field sign function through the FFT.
  deflation -- the critical eigenpairs of a dense matrix and the deflated sign
             function f(A)x = R f(Lambda) L^dag x + f(A)(I - R L^dag)x (Sec. 2).
  mlp     -- the sizing network: forward, gradient, Adam (not in the paper).

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, exact identities or brute force; none is "parity unpinned".
"""
from . import dirac, krylov, exact, deflation  # noqa: F401
