"""Pins of the oracle's deflation (Sec. 2, the deflation paragraph): the critical
eigenpairs satisfy the eigen-equations and L^dag R = 1, the deflated source has no
component along them, the deflated result equals the spectral definition (Eq. (specdef)),
and deflation lowers the Krylov dimension needed."""
import numpy as np
import pytest

import ovinputs as oi
from conftest import rel
from oracle import deflation, dirac, exact, krylov


def ops(U, dims, m_w, mu):
    return (lambda v: dirac.A_apply(U, v, dims, m_w, mu), lambda v: dirac.AH_apply(U, v, dims, m_w, mu))


@pytest.fixture(scope="module")
def nonherm():
    dims, mu = (2, 2, 2, 4), 0.3
    U = oi.gauge_field(dims, "haar", 0)
    A = dirac.dense_A(U, dims, -1.5, mu)
    return dict(dims=dims, mu=mu, U=U, A=A, x=oi.gaussian_source(dims, 1))


def test_critical_eigenpairs_hermitian(haar44):
    A = haar44[0.0]["A"]
    lam, R, L = deflation.critical_eigenpairs(A, 12, True)
    assert np.linalg.norm(A @ R - R * lam[None, :]) < 1e-11 * np.linalg.norm(A)
    assert np.allclose(np.conj(L.T) @ R, np.eye(12), atol=1e-12)
    # the 12 of smallest magnitude: no other eigenvalue is smaller
    assert np.abs(lam).max() <= np.sort(np.abs(haar44[0.0]["lam"]))[12] + 1e-14


def test_critical_eigenpairs_nonhermitian(nonherm):
    A = nonherm["A"]
    lam, R, L = deflation.critical_eigenpairs(A, 10, False)
    assert np.linalg.norm(A @ R - R * lam[None, :]) < 1e-11 * np.linalg.norm(A)
    assert np.linalg.norm(np.conj(A.T) @ L - L * np.conj(lam)[None, :]) < 1e-10 * np.linalg.norm(A)
    assert np.allclose(np.conj(L.T) @ R, np.eye(10), atol=1e-11)
    assert np.abs(lam).max() <= np.sort(np.abs(np.linalg.eigvals(A)))[10] + 1e-12


def test_deflated_source_has_no_critical_component(nonherm):
    lam, R, L = deflation.critical_eigenpairs(nonherm["A"], 10, False)
    c, xp = deflation.deflate_source(nonherm["x"], R, L)
    assert np.abs(np.conj(L.T) @ xp).max() < 1e-12 * np.linalg.norm(nonherm["x"])
    assert rel(xp + R @ c, nonherm["x"]) < 1e-15


def test_deflated_sign_equals_spectral_definition_hermitian(haar44):
    d = haar44
    lam, R, L = deflation.critical_eigenpairs(d[0.0]["A"], 16, True)
    fA, fAH = ops(d["U"], d["dims"], d["m_w"], 0.0)
    y, info = deflation.deflated_sign_apply(fA, fAH, d["x"], True, lam, R, L, k_max=400, l=64, tol=1e-10)
    assert info["status"] == krylov.OK
    assert rel(y, d[0.0]["S"] @ d["x"]) < 2e-10


def test_deflated_sign_equals_spectral_definition_nonhermitian(nonherm):
    lam, R, L = deflation.critical_eigenpairs(nonherm["A"], 10, False)
    fA, fAH = ops(nonherm["U"], nonherm["dims"], -1.5, nonherm["mu"])
    y, info = deflation.deflated_sign_apply(fA, fAH, nonherm["x"], False, lam, R, L, k_max=384, l=100, tol=1e-10)
    yex, _ = exact.sign_spectral_apply(nonherm["A"], nonherm["x"], False)
    assert info["status"] == krylov.OK
    assert rel(y, yex) < 1e-9


def test_deflation_lowers_the_krylov_dimension(haar44):
    """Removing the 16 eigenvalues of smallest magnitude widens the gap around zero (on
    these Haar links from |lambda| >= 0.264 to >= 0.354, a factor 1.34), so the stopping
    rule stops at a smaller k for the same tolerance (the Krylov dimension needed grows
    about as the inverse of the gap: 390 -> 310 measured)."""
    d = haar44
    fA, fAH = ops(d["U"], d["dims"], d["m_w"], 0.0)
    lam, R, L = deflation.critical_eigenpairs(d[0.0]["A"], 16, True)
    _, i0 = krylov.sign_apply(fA, fAH, d["x"], True, 400, 64, 1e-10)
    _, i1 = deflation.deflated_sign_apply(fA, fAH, d["x"], True, lam, R, L, k_max=400, l=64, tol=1e-10)
    assert i1["status"] == krylov.OK and i1["k"] < 0.85 * i0["k"], (i0["k"], i1["k"])


def test_no_deflation_is_the_plain_method(nonherm):
    fA, fAH = ops(nonherm["U"], nonherm["dims"], -1.5, nonherm["mu"])
    n = nonherm["x"].size
    empty = np.zeros((n, 0), dtype=complex)
    y0, _ = krylov.sign_apply(fA, fAH, nonherm["x"], False, 200, 60, 0, k_fixed=200)
    y1, _ = deflation.deflated_sign_apply(fA, fAH, nonherm["x"], False, np.zeros(0, complex), empty, empty,
                                          k_max=200, l=60, tol=0, k_fixed=200)
    assert np.array_equal(y0, y1)
