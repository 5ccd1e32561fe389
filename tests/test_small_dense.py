"""The host routines of the eigensolver's Rayleigh-Ritz step (csrc/ov_small.cpp) against
their definitions: A V = V diag(w) with unit columns (general and Hermitian matrices,
including repeated eigenvalues), R^dag R = A with Rinv R = 1, A A^-1 = 1, and A = Q R with Q
unitary and R upper triangular. The file is
compiled alone with the host compiler for this test (no GPU needed)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHIM = r'''
#include <cuda_runtime.h>
namespace ov {
bool small_eig(int n, const double2* A, double2* w, double2* V);
bool small_eigh(int n, const double2* A, double* w, double2* V);
bool small_chol_inv(int n, const double2* A, double2* Rinv);
bool small_inv(int n, const double2* A, double2* X);
bool small_qr_q(int n, const double2* A, double2* Q);
}
extern "C" int t_eig(int n, const double2* A, double2* w, double2* V) { return ov::small_eig(n, A, w, V); }
extern "C" int t_eigh(int n, const double2* A, double* w, double2* V) { return ov::small_eigh(n, A, w, V); }
extern "C" int t_chol(int n, const double2* A, double2* R) { return ov::small_chol_inv(n, A, R); }
extern "C" int t_inv(int n, const double2* A, double2* X) { return ov::small_inv(n, A, X); }
extern "C" int t_qr(int n, const double2* A, double2* Q) { return ov::small_qr_q(n, A, Q); }
'''


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("small")
    shim = d / "shim.cpp"
    shim.write_text(SHIM)
    so = d / "libsmall.so"
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    src = os.path.join(ROOT, "paper_0910_2918_gb300", "csrc", "ov_small.cpp")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I" + cuda_inc, str(shim), src, "-o", str(so)],
                   check=True)
    return ctypes.CDLL(str(so))


def c128p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def rand_c(rng, n):
    return rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))


@pytest.mark.parametrize("n", [1, 2, 7, 24, 48])
def test_general_eig(lib, n):
    rng = np.random.default_rng(n)
    A = np.ascontiguousarray(rand_c(rng, n))
    w = np.zeros(n, complex)
    V = np.zeros((n, n), complex)
    assert lib.t_eig(n, c128p(A), c128p(w), c128p(V)) == 1
    assert np.linalg.norm(A @ V - V * w[None, :]) < 1e-11 * np.linalg.norm(A)
    assert np.allclose(np.linalg.norm(V, axis=0), 1.0)
    assert np.allclose(np.sort_complex(w), np.sort_complex(np.linalg.eigvals(A)), atol=1e-10 * np.abs(w).max())


def test_general_eig_of_a_projection_with_clustered_spectrum(lib):
    """Ritz matrices of the eigensolver: nearly normal, eigenvalues close together."""
    rng = np.random.default_rng(3)
    n = 32
    X = np.eye(n) + 0.1 * rand_c(rng, n)
    ev = 0.3 + 0.01 * rng.standard_normal(n) + 0.001j * rng.standard_normal(n)
    A = np.ascontiguousarray(X @ np.diag(ev) @ np.linalg.inv(X))
    w = np.zeros(n, complex)
    V = np.zeros((n, n), complex)
    assert lib.t_eig(n, c128p(A), c128p(w), c128p(V)) == 1
    assert np.linalg.norm(A @ V - V * w[None, :]) < 1e-10 * np.linalg.norm(A)


@pytest.mark.parametrize("n", [1, 5, 32])
def test_hermitian_eig(lib, n):
    rng = np.random.default_rng(10 + n)
    B = rand_c(rng, n)
    A = np.ascontiguousarray(B + B.conj().T)
    A[0, 0] = A[0, 0].real
    if n > 4:  # a repeated eigenvalue
        Q, _ = np.linalg.qr(rand_c(rng, n))
        ev = np.linspace(-1, 1, n)
        ev[2] = ev[3]
        A = np.ascontiguousarray(Q @ np.diag(ev) @ Q.conj().T)
    w = np.zeros(n)
    V = np.zeros((n, n), complex)
    assert lib.t_eigh(n, c128p(A), w.ctypes.data_as(ctypes.c_void_p), c128p(V)) == 1
    assert np.all(np.diff(w) >= -1e-12)
    assert np.linalg.norm(A @ V - V * w[None, :]) < 1e-11 * max(1.0, np.linalg.norm(A))
    assert np.allclose(V.conj().T @ V, np.eye(n), atol=1e-12)


def test_cholesky_inverse_and_inverse(lib):
    rng = np.random.default_rng(5)
    n = 20
    B = rand_c(rng, n)
    A = np.ascontiguousarray(B.conj().T @ B + n * np.eye(n))
    Ri = np.zeros((n, n), complex)
    assert lib.t_chol(n, c128p(A), c128p(Ri)) == 1
    R = np.linalg.inv(Ri)
    assert np.allclose(np.triu(R), R, atol=1e-12)
    assert np.linalg.norm(R.conj().T @ R - A) < 1e-12 * np.linalg.norm(A)
    X = np.zeros((n, n), complex)
    C = np.ascontiguousarray(rand_c(rng, n))
    assert lib.t_inv(n, c128p(C), c128p(X)) == 1
    assert np.allclose(C @ X, np.eye(n), atol=1e-11)
    # not positive definite: refused
    A2 = np.ascontiguousarray(-A)
    assert lib.t_chol(n, c128p(A2), c128p(Ri)) == 0


@pytest.mark.parametrize("n", [1, 5, 40, 64])
def test_qr_unitary_factor(lib, n):
    rng = np.random.default_rng(100 + n)
    A = np.ascontiguousarray(rand_c(rng, n))
    Q = np.zeros((n, n), complex)
    assert lib.t_qr(n, c128p(A), c128p(Q)) == 1
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(n)) < 1e-13 * n
    R = Q.conj().T @ A
    assert np.linalg.norm(np.tril(R, -1)) < 1e-12 * np.linalg.norm(A)  # leading spans kept


def test_qr_dependent_columns(lib):
    # columns 1 and 3 repeat column 0: Q stays unitary and column 0's direction leads
    rng = np.random.default_rng(7)
    n = 6
    A = rand_c(rng, n)
    A[:, 1] = A[:, 0]
    A[:, 3] = 2j * A[:, 0]
    A = np.ascontiguousarray(A)
    Q = np.zeros((n, n), complex)
    assert lib.t_qr(n, c128p(A), c128p(Q)) == 1
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(n)) < 1e-12
    q0 = A[:, 0] / np.linalg.norm(A[:, 0])
    assert abs(abs(np.vdot(Q[:, 0], q0)) - 1.0) < 1e-12
    R = Q.conj().T @ A
    assert np.linalg.norm(np.tril(R, -1)) < 1e-11 * np.linalg.norm(A)
