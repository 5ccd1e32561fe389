"""Exact sign functions (oracle; test infrastructure).

* sign_spectral: Eq. (specdef), f(A) = U diag(f(lambda_i)) U^{-1}, with
  sgn(z) = sgn(Re z) for complex eigenvalues (Sec. 1). Dense, small lattices.
* roberts_higham_dense: Eq. (Roberts) on the full n x n matrix, an independent
  route to sgn(A) on small lattices.
* free-field closed form: for U = 1, plane waves e^{i p.x} diagonalise D_w(mu):
    D(p) = m_w + sum_nu (1 - cos pt_nu) + i sum_nu gamma_nu sin pt_nu,
  with pt_nu = p_nu for x, y, z and pt_t = p_t - i mu, momenta p_i = 2 pi n_i / L_i
  and p_t = (2 n_t + 1) pi / L_t (antiperiodic). sgn(gamma5 D(p)) is a 4 x 4
  eigenproblem per momentum; the field is moved to momentum space by the FFT.
"""
import numpy as np

from .dirac import GAMMA, GAMMA5


def sign_of_eigs(lam, hermitian):
    return np.sign(lam.real) if not hermitian else np.sign(lam)


def sign_spectral(A, hermitian):
    """sgn(A) = U diag(sgn Re lambda) U^{-1} (Eq. (specdef))."""
    if hermitian:
        lam, U = np.linalg.eigh(A)
        return (U * np.sign(lam)[None, :]) @ np.conj(U.T), lam
    lam, U = np.linalg.eig(A)
    return (U * np.sign(lam.real)[None, :]) @ np.linalg.inv(U), lam


def sign_spectral_apply(A, x, hermitian):
    """sgn(A) x without forming sgn(A): U (sgn(Lambda) (U^{-1} x))."""
    if hermitian:
        lam, U = np.linalg.eigh(A)
        return U @ (np.sign(lam) * (np.conj(U.T) @ x)), lam
    lam, U = np.linalg.eig(A)
    return U @ (np.sign(lam.real) * np.linalg.solve(U, x)), lam


def roberts_higham_dense(A, rh_tol=1e-12, maxit=200):
    S = np.array(A, dtype=np.complex128)
    for it in range(1, maxit + 1):
        Sn = 0.5 * (S + np.linalg.inv(S))
        d = np.linalg.norm(Sn - S)
        S = Sn
        if d <= rh_tol * np.linalg.norm(S):
            return S, it
    raise RuntimeError("Roberts-Higham did not converge")


def free_momenta(dims, antiperiodic=True):
    """Momentum grids (pt, pz, py, px) matching numpy's FFT index order."""
    lx, ly, lz, lt = (int(d) for d in dims)
    px = 2 * np.pi * np.arange(lx) / lx
    py = 2 * np.pi * np.arange(ly) / ly
    pz = 2 * np.pi * np.arange(lz) / lz
    pt = 2 * np.pi * np.arange(lt) / lt + (np.pi / lt if antiperiodic else 0.0)
    return np.meshgrid(pt, pz, py, px, indexing="ij")


def free_dirac_momentum(dims, m_w, mu, antiperiodic=True):
    """D(p) as an array (Lt, Lz, Ly, Lx, 4, 4)."""
    pt, pz, py, px = free_momenta(dims, antiperiodic)
    ptil = [px, py, pz, pt - 1j * mu]
    D = np.zeros(pt.shape + (4, 4), dtype=np.complex128)
    mass = m_w + sum(1.0 - np.cos(p) for p in ptil)
    D += mass[..., None, None] * np.eye(4)
    for nu in range(4):
        D += 1j * np.sin(ptil[nu])[..., None, None] * GAMMA[nu]
    return D


def free_sign_apply(x, dims, m_w, mu, antiperiodic=True):
    """sgn(gamma5 D_w(mu)) x for the free field U = 1 (closed form + FFT)."""
    lx, ly, lz, lt = (int(d) for d in dims)
    psi = np.asarray(x).reshape(lt, lz, ly, lx, 4, 3)
    t = np.arange(lt).reshape(lt, 1, 1, 1, 1, 1)
    twist = np.exp(1j * np.pi * t / lt) if antiperiodic else np.ones_like(t, dtype=complex)
    phi = psi / twist  # periodic in t
    phat = np.fft.fftn(phi, axes=(0, 1, 2, 3))
    A = np.einsum("st,...tu->...su", GAMMA5, free_dirac_momentum(dims, m_w, mu, antiperiodic))
    lam, U = np.linalg.eig(A)
    S = np.einsum("...ij,...j,...jk->...ik", U, np.sign(lam.real), np.linalg.inv(U))
    yhat = np.einsum("...st,...tc->...sc", S, phat)
    y = np.fft.ifftn(yhat, axes=(0, 1, 2, 3)) * twist
    return y.reshape(np.shape(x))


def plane_wave(dims, n_mom, chi, antiperiodic=True):
    """e^{i p.x} chi (chi: 4 x 3 spin-colour), momentum integers n_mom = (nx, ny, nz, nt)."""
    lx, ly, lz, lt = (int(d) for d in dims)
    nx, ny, nz, nt = n_mom
    p = [2 * np.pi * nx / lx, 2 * np.pi * ny / ly, 2 * np.pi * nz / lz,
         (2 * np.pi * nt + (np.pi if antiperiodic else 0.0)) / lt]
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return (ph[..., None, None] * np.asarray(chi)[None, None, None, None]).reshape(-1), p
