"""The overlap operator inside an iterative solver (Sec. 1: D_ov is what solvers need).
ov_solve runs CG on the normal equations of D(m) = (1 - m/2) D_ov + m, each D and D^dag
application a nested sign apply; its solution is compared with the dense solve of the
same operator built from the exact sign function (the spectral definition, Sec. 2)."""
import numpy as np
import pytest

import ovinputs as oi
from gpu_util import rel
from oracle import dirac, exact

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ov():
    import paper_0910_2918_gb300 as ov

    return ov


def gamma5(n):
    return np.where((np.arange(n) % 12) < 6, 1.0, -1.0)


def dense_massive_overlap(S, mass):
    n = S.shape[0]
    D_ov = np.eye(n) + gamma5(n)[:, None] * S
    return (1.0 - 0.5 * mass) * D_ov + mass * np.eye(n)


def test_solve_hermitian_vs_dense(ov, haar44):
    d = haar44
    mass = 0.2
    D = dense_massive_overlap(d[0.0]["S"], mass)
    b = np.stack([oi.gaussian_source(d["dims"], 7), oi.gaussian_source(d["dims"], 8)])
    x = np.zeros_like(b)
    with ov.Overlap(d["dims"], d["U"], d["m_w"], 0.0, "fp64", opts=ov.make_opts(check_interval=10)) as op:
        rc, its, res = op.solve(b, x, mass=mass, tol=1e-9, maxit=200, sign_tol=1e-11, k_max=600, l=120)
    assert rc == 0 and np.all(res <= 1e-9) and np.all(its > 0)
    for r in range(2):
        xr = np.linalg.solve(D, b[r])
        assert np.linalg.norm(D @ x[r] - b[r]) / np.linalg.norm(b[r]) < 5e-9
        assert rel(x[r], xr) < 1e-7


def test_solve_non_hermitian_vs_dense(ov):
    """mu = 0.3: D^dag needs the sign function of A^dag = gamma5 D_w(-mu)."""
    dims, mu, m_w, mass = (2, 2, 2, 4), 0.3, -1.5, 0.3
    U = oi.gauge_field(dims, "haar", 0)
    S, _ = exact.sign_spectral(dirac.dense_A(U, dims, m_w, mu), False)
    D = dense_massive_overlap(S, mass)
    b = oi.gaussian_source(dims, 3).reshape(1, -1)
    x = np.zeros_like(b)
    with ov.Overlap(dims, U, m_w, mu, "fp64", opts=ov.make_opts(check_interval=10)) as op:
        rc, its, res = op.solve(b, x, mass=mass, tol=1e-9, maxit=300, sign_tol=1e-11, k_max=384, l=120)
    assert rc == 0 and res[0] <= 1e-9
    assert np.linalg.norm(D @ x[0] - b[0]) / np.linalg.norm(b[0]) < 5e-9
    assert rel(x[0], np.linalg.solve(D, b[0])) < 1e-7


def test_solve_zero_rhs_and_device_buffers(ov):
    import torch

    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "near_unit", 1, eps=0.3)
    b = np.stack([np.zeros(12 * 256, dtype=np.complex128), oi.gaussian_source(dims, 2)])
    xh = np.zeros_like(b)
    with ov.Overlap(dims, U, -1.5, 0.2, "fp64", opts=ov.make_opts(check_interval=10)) as op:
        rc, its, res = op.solve(b, xh, mass=0.5, tol=1e-8)
        bd = torch.from_numpy(b).cuda()
        xd = torch.zeros_like(bd)
        rc2, its2, res2 = op.solve(bd, xd, mass=0.5, tol=1e-8)
    assert rc == 0 and rc2 == 0
    assert its[0] == 0 and np.all(xh[0] == 0) and res[0] == 0.0
    assert np.array_equal(xd.cpu().numpy(), xh)
