"""Deflation of the critical eigenvalues (oracle; test infrastructure).

Sec. 2 (the deflation paragraph): with m eigenvalues lambda_i of A near the
discontinuity of sgn, their right eigenvectors r_i and left eigenvectors l_i
(L_m^dag R_m = 1),

    f(A) x = R_m f(Lambda_m) (L_m^dag x) + f(A) (I - R_m L_m^dag) x,

where the first term is exact and the second is the Krylov approximation of
Eq. (approximation) applied to the deflated source (nested, Sec. 3).

Readings where the paper is silent (listed in the design notes):
  * which eigenvalues are critical: the m of smallest magnitude |lambda| (at mu = 0,
    A is Hermitian and these are exactly the ones nearest the imaginary axis);
  * sgn(lambda) = sgn(Re lambda) (Eq. (specdef) with the sign of the real part);
  * left eigenvectors are eigenvectors of A^dag for conj(lambda_i), scaled so that
    l_i^dag r_i = 1 (then L^dag R = 1 for distinct eigenvalues).
"""
import numpy as np

from . import krylov


def critical_eigenpairs(A, m, hermitian):
    """(lam, R, L) of the m eigenvalues of smallest magnitude of the dense matrix A, by
    full diagonalisation (small sizes only). hermitian: eigh, L = R (orthonormal)."""
    if hermitian:
        w, U = np.linalg.eigh(A)
        idx = np.argsort(np.abs(w))[:m]
        R = U[:, idx]
        return w[idx].astype(complex), R, R.copy()
    w, Rf = np.linalg.eig(A)
    idx = np.argsort(np.abs(w))[:m]
    # left eigenvectors: rows of R_full^{-1} (Y^dag A = Lambda Y^dag with Y^dag = R^{-1})
    Linv = np.linalg.inv(Rf)
    R = Rf[:, idx]
    L = np.conj(Linv[idx, :]).T  # l_i^dag = row i of R^{-1}, so l_i^dag r_j = delta_ij
    return w[idx], R, L


def deflate_source(x, R, L):
    """(c, x') with c = L^dag x and x' = (I - R L^dag) x."""
    c = np.conj(L.T) @ x
    return c, x - R @ c


def deflated_sign_apply(apply_A, apply_AH, x, hermitian, lam, R, L, **kw):
    """y ~ sgn(A) x = R sgn(Lambda) L^dag x + sgn(A) (I - R L^dag) x, the second term by
    krylov.sign_apply (same keywords). Returns (y, info) of the Krylov part."""
    c, xp = deflate_source(x, R, L)
    y2, info = krylov.sign_apply(apply_A, apply_AH, xp, hermitian, **kw)
    s = np.where(np.real(lam) >= 0, 1.0, -1.0)
    return R @ (s * c) + y2, info
