"""Deflation of the critical eigenvalues (Sec. 2, the deflation paragraph) on the GPU:
the device eigensolver against full diagonalisation, the deflated apply against the
oracle's deflated_sign_apply with the same eigenpairs, and the exact answer."""
import numpy as np
import pytest

import ovinputs as oi
from gpu_util import oracle_ops, rel
from oracle import deflation, dirac, exact, krylov

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ov():
    import paper_0910_2918_gb300 as ov

    return ov


def test_eigensolver_hermitian_vs_diagonalisation(ov, haar44):
    d = haar44
    m = 12
    with ov.Overlap(d["dims"], d["U"], d["m_w"], 0.0, "fp64") as op:
        rc, lam, res = op.deflate(m, tol=1e-11, maxit=300)
        lam_g, R, L = op.deflation(m)
    assert rc == 0 and np.all(res <= 1e-11)
    exact_lam = d[0.0]["lam"][np.argsort(np.abs(d[0.0]["lam"]))[:m]]
    assert np.allclose(np.sort(lam.real), np.sort(exact_lam), rtol=0, atol=1e-10)
    assert np.abs(lam.imag).max() == 0.0
    A = d[0.0]["A"]
    Rt = R.T  # columns are eigenvectors
    assert np.linalg.norm(A @ Rt - Rt * lam[None, :]) < 1e-10 * np.linalg.norm(Rt)
    assert np.allclose(R.conj() @ R.T, np.eye(m), atol=1e-12) and np.array_equal(R, L)


def test_eigensolver_nonhermitian_vs_diagonalisation(ov):
    dims, mu, m = (2, 2, 2, 4), 0.3, 10
    U = oi.gauge_field(dims, "haar", 0)
    A = dirac.dense_A(U, dims, -1.5, mu)
    with ov.Overlap(dims, U, -1.5, mu, "fp64") as op:
        rc, lam, res = op.deflate(m, tol=1e-11, maxit=300)
        lam_g, R, L = op.deflation(m)
    assert rc == 0 and np.all(res <= 1e-11)
    ev = np.linalg.eigvals(A)
    ev = ev[np.argsort(np.abs(ev))[:m]]
    for z in lam:  # every computed eigenvalue is one of the m smallest
        assert np.abs(ev - z).min() < 1e-9
    Rt, Lt = R.T, L.T
    assert np.linalg.norm(A @ Rt - Rt * lam[None, :]) < 1e-10 * np.linalg.norm(Rt)
    assert np.linalg.norm(A.conj().T @ Lt - Lt * lam.conj()[None, :]) < 1e-9 * np.linalg.norm(Lt)
    assert np.allclose(Lt.conj().T @ Rt, np.eye(m), atol=1e-10)


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_deflated_apply_vs_oracle_fixed_k(ov, prec, mu):
    """The deflated apply at fixed (k, l) equals the oracle's deflated_sign_apply run with
    the eigenpairs the GPU computed (Sec. 2: exact part plus the Krylov part on the
    deflated source)."""
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "haar", 0)
    x = oi.gaussian_source(dims, 1)
    k, l, m = 120, 110, 8
    y = np.zeros((1, x.size), dtype=np.complex128)
    with ov.Overlap(dims, U, -1.5, mu, prec, opts=ov.make_opts(k_fixed=k)) as op:
        rc, lam, res = op.deflate(m, tol=1e-10, maxit=300)
        lam_g, R, L = op.deflation(m)
        rc, info = op.sign_apply(x.reshape(1, -1).copy(), y, 0.0, k, l)
    fA, fAH = oracle_ops(U, dims, -1.5, mu)
    yo, io = deflation.deflated_sign_apply(fA, fAH, x, mu == 0.0, lam_g, R.T, L.T, k_max=k, l=l, tol=0, k_fixed=k)
    assert rel(y[0], yo) < 1e-10, rel(y[0], yo)


def test_deflated_apply_exact_and_faster(ov, haar44):
    """With the stopping rule: the deflated apply reaches the spectral definition's answer
    with a smaller Krylov dimension than the plain one (the 16 eigenvalues of smallest
    magnitude removed from the Krylov part), also through ov_apply (D_ov = 1 + gamma5 sgn)."""
    d = haar44
    x = d["x"].reshape(1, -1).copy()
    yex = d[0.0]["S"] @ d["x"]
    with ov.Overlap(d["dims"], d["U"], d["m_w"], 0.0, "fp64", opts=ov.make_opts(check_interval=10)) as op:
        y0 = np.zeros_like(x)
        rc0, i0 = op.sign_apply(x, y0, 1e-10, 600, 64)
        op.deflate(16, tol=1e-11, maxit=300)
        y1 = np.zeros_like(x)
        rc1, i1 = op.sign_apply(x, y1, 1e-10, 600, 64)
        yd = np.zeros_like(x)
        op.apply(x, yd, 1e-10, 600, 64)
    assert rc0 == 0 and rc1 == 0
    assert rel(y1[0], yex) < 2e-10 and rel(y0[0], yex) < 2e-10
    assert i1[0]["k"] < 0.85 * i0[0]["k"], (i0[0]["k"], i1[0]["k"])
    g5 = np.where((np.arange(x.size) % 12) < 6, 1.0, -1.0)
    assert rel(yd[0], x[0] + g5 * yex) < 2e-10


def test_deflated_solver_adjoint(ov):
    """ov_solve at mu != 0 with deflation: D^dag needs sgn(A^dag), deflated with the roles
    of the left and right eigenvectors swapped; the solution equals the dense solve."""
    dims, mu, mass = (2, 2, 2, 4), 0.3, 0.3
    U = oi.gauge_field(dims, "haar", 0)
    S, _ = exact.sign_spectral(dirac.dense_A(U, dims, -1.5, mu), False)
    n = S.shape[0]
    g5 = np.where((np.arange(n) % 12) < 6, 1.0, -1.0)
    D = (1 - mass / 2) * (np.eye(n) + g5[:, None] * S) + mass * np.eye(n)
    b = oi.gaussian_source(dims, 3).reshape(1, -1)
    x = np.zeros_like(b)
    with ov.Overlap(dims, U, -1.5, mu, "fp64", opts=ov.make_opts(check_interval=10)) as op:
        op.deflate(8, tol=1e-11, maxit=300)
        rc, its, res = op.solve(b, x, mass=mass, tol=1e-9, maxit=300, sign_tol=1e-11, k_max=384, l=120)
    assert rc == 0
    assert rel(x[0], np.linalg.solve(D, b[0])) < 1e-7


def test_batch_deflation_per_lattice(ov):
    """A batch handle deflates every lattice in the same launches (one eigensolver job per
    lattice and side): each lattice's eigenvalues are those of full diagonalisation, and the
    deflated batch apply equals the deflated single-lattice applies."""
    probs = [((4, 4, 4, 4), "haar", 0, -1.5, 0.0), ((2, 2, 2, 4), "haar", 0, -1.5, 0.3),
             ((2, 4, 2, 4), "haar", 5, -1.4, 0.2)]
    m, k = 8, 60
    Us = [oi.gauge_field(d, kind, seed) for d, kind, seed, _, _ in probs]
    xs = [oi.gaussian_source(d, 11 + i).reshape(1, -1).copy() for i, (d, _, _, _, _) in enumerate(probs)]
    hb = ov.ov_batch_create([p[0] for p in probs], Us, [p[3] for p in probs], [p[4] for p in probs], "fp64",
                            opts=ov.make_opts(k_fixed=k))
    try:
        rc, lam, res, used = ov.ov_deflate(hb, m, tol=1e-11, maxit=300, nlat=len(probs))
        ys = [np.zeros_like(x) for x in xs]
        ov.ov_batch_sign_apply(hb, xs, ys, 0.0, k, 50)
    finally:
        ov.ov_destroy(hb)
    assert rc == 0 and list(used) == [m] * len(probs)
    for i, (d, kind, seed, m_w, mu) in enumerate(probs):
        ev = np.linalg.eigvals(dirac.dense_A(Us[i], d, m_w, mu))
        ev = ev[np.argsort(np.abs(ev))[:m]]
        for z in lam[i]:
            assert np.abs(ev - z).min() < 1e-9
        y1 = np.zeros_like(xs[i])
        with ov.Overlap(d, Us[i], m_w, mu, "fp64", opts=ov.make_opts(k_fixed=k)) as op:
            op.deflate(m, tol=1e-11, maxit=300)
            op.sign_apply(xs[i], y1, 0.0, k, 50)
        assert rel(ys[i][0], y1[0]) < 1e-10, (i, rel(ys[i][0], y1[0]))


def test_deflated_handle_runs_strict_steps(ov):
    """With deflation attached a double-float handle ignores opts.relax: its float hopping
    error would put back components along the removed eigenvectors. The deflated apply with
    relax set is bitwise the one without, and counts no relaxed step."""
    dims, mu, k = (4, 4, 4, 4), 0.3, 160
    U = oi.gauge_field(dims, "haar", 0)
    x = oi.gaussian_source(dims, 2).reshape(1, -1).copy()
    out = []
    for relax in (0.0, 0.5):
        y = np.zeros_like(x)
        # one block size for both handles: the autotuner may pick different ones, and the
        # block partial sums of the reductions follow the block size
        with ov.Overlap(dims, U, -1.5, mu, "df64", opts=ov.make_opts(k_fixed=k, relax=relax, block_size=128)) as op:
            op.deflate(8, tol=1e-10, maxit=300)
            op.reset_stats()
            op.sign_apply(x, y, 0.0, k, 100)
            out.append((y, op.stats()["relaxed_steps"]))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == 0 and out[1][1] == 0


def test_deflated_apply_several_right_hand_sides(ov):
    """Several right-hand sides of one lattice in one deflated apply: each equals the
    deflated apply of that source alone (the projections c = L^dag x are per column) and
    the oracle's deflated_sign_apply with the same eigenpairs at fixed k."""
    dims, mu, k, l, m = (4, 4, 4, 4), 0.3, 120, 110, 8
    U = oi.gauge_field(dims, "haar", 0)
    X = np.stack([oi.gaussian_source(dims, 20 + i) for i in range(3)])
    Y = np.zeros_like(X)
    with ov.Overlap(dims, U, -1.5, mu, "fp64", opts=ov.make_opts(k_fixed=k)) as op:
        rc, lam, res = op.deflate(m, tol=1e-11, maxit=300)
        lam_g, R, L = op.deflation(m)
        rc, info = op.sign_apply(X.copy(), Y, 0.0, k, l)
        singles = []
        for i in range(3):
            y1 = np.zeros((1, X.shape[1]), dtype=np.complex128)
            op.sign_apply(X[i:i + 1].copy(), y1, 0.0, k, l)
            singles.append(y1[0])
    fA, fAH = oracle_ops(U, dims, -1.5, mu)
    for i in range(3):
        assert rel(Y[i], singles[i]) < 1e-12
        yo, _ = deflation.deflated_sign_apply(fA, fAH, X[i], False, lam_g, R.T, L.T, k_max=k, l=l, tol=0, k_fixed=k)
        assert rel(Y[i], yo) < 1e-10, (i, rel(Y[i], yo))
