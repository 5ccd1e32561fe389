"""Pins of the oracle's nested Krylov sign function (Secs. 1-3).

Each test fixes the oracle against something other than itself: the spectral
definition (Eq. (specdef)) on dense 4^4 matrices, the free-field closed form,
exact identities of the method (W^dag V = 1, H_k = W^dag A V, Eq. (precond),
the l x l corner property of naive nesting), or invariants of sgn.
"""
import numpy as np
import pytest

import ovinputs as oi
from oracle import dirac, exact, krylov
from conftest import rel

try:
    from threadpoolctl import threadpool_limits
except ImportError:  # pragma: no cover
    threadpool_limits = None


@pytest.fixture(autouse=True)
def _one_blas_thread(request):
    """Small dense ops run far faster on one BLAS thread; large dense
    factorisations (marked 'dense') keep all threads."""
    if threadpool_limits is None or request.node.get_closest_marker("dense"):
        yield
        return
    with threadpool_limits(limits=1, user_api="blas"):
        yield


def ops(U, dims, m_w, mu):
    return (lambda v: dirac.A_apply(U, v, dims, m_w, mu),
            lambda v: dirac.AH_apply(U, v, dims, m_w, mu))


# ---- P1: spectral definition on dense 4^4 (Eq. (specdef)) -----------------

def test_p1_hermitian_lanczos_vs_eigh(haar44):
    d = haar44
    fA, fAH = ops(d["U"], d["dims"], d["m_w"], 0.0)
    y, info = krylov.sign_apply(fA, fAH, d["x"], True, 400, 64, 1e-10)
    yref = d[0.0]["S"] @ d["x"]
    assert info["status"] == krylov.OK
    assert info["k"] <= 400
    assert rel(y, yref) < 2e-10
    # the a-posteriori estimate is of the size of the true error
    assert rel(y, yref) < 20 * max(info["err_est"], 1e-12)


def test_p1_two_sided_vs_eig_not_converged():
    """mu != 0, sgn(z) = sgn(Re z): a small k_max stops short of 1e-10, and the
    a-posteriori estimate must then track the true error."""
    dims = (4, 4, 2, 4)
    U = oi.gauge_field(dims, "haar", 0)
    x = oi.gaussian_source(dims, 1)
    A = dirac.dense_A(U, dims, -1.5, 0.3)
    yref, lam = exact.sign_spectral_apply(A, x, False)
    fA, fAH = ops(U, dims, -1.5, 0.3)
    y, info = krylov.sign_apply(fA, fAH, x, False, 200, 100, 1e-10)
    err = rel(y, yref)
    assert info["status"] == krylov.NOT_CONVERGED
    assert 1e-9 < err < 1e-3
    assert info["err_est"] / 30 < err < 30 * info["err_est"]


def test_p1_two_sided_small_lattice_converges():
    dims = (2, 2, 2, 4)
    U = oi.gauge_field(dims, "haar", 0)
    x = oi.gaussian_source(dims, 1)
    A = dirac.dense_A(U, dims, -1.5, 0.3)
    yref, lam = exact.sign_spectral_apply(A, x, False)
    assert np.abs(lam.real).min() > 0.1  # unique answer: no eigenvalue on the imaginary axis
    fA, fAH = ops(U, dims, -1.5, 0.3)
    y, info = krylov.sign_apply(fA, fAH, x, False, 400, 100, 1e-10)
    assert info["status"] == krylov.OK
    assert rel(y, yref) < 1e-9


# ---- P2: Roberts-Higham on the full matrix vs eigendecomposition ------------

@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_p2_dense_roberts_higham(mu):
    dims = (2, 2, 2, 4)
    U = oi.gauge_field(dims, "haar", 5)
    A = dirac.dense_A(U, dims, -1.5, mu)
    S_rh, its = exact.roberts_higham_dense(A)
    S_ev, _ = exact.sign_spectral(A, mu == 0.0)
    assert np.linalg.norm(S_rh - S_ev) / np.linalg.norm(S_ev) < 1e-12
    assert its < 30


# ---- P3: free field closed form at any volume ------------------------------

@pytest.mark.parametrize("dims,mu,l", [((8, 8, 8, 8), 0.0, 80), ((4, 4, 4, 8), 0.5, 120), ((6, 4, 4, 6), 0.2, 100)])
def test_p3_free_field(dims, mu, l):
    U = oi.gauge_field(dims, "unit", 0)
    x = oi.gaussian_source(dims, 1)
    yref = exact.free_sign_apply(x, dims, -1.5, mu)
    fA, fAH = ops(U, dims, -1.5, mu)
    y, info = krylov.sign_apply(fA, fAH, x, mu == 0.0, 400, l, 1e-10)
    assert info["status"] == krylov.OK
    assert rel(y, yref) < 2e-9


def test_p3_inner_estimate_flags_small_l():
    """With l too small at mu != 0 the outer estimate alone would pass; the
    inner estimate must flag the result (this is why the stopping rule has it)."""
    dims = (4, 4, 4, 8)
    U = oi.gauge_field(dims, "unit", 0)
    x = oi.gaussian_source(dims, 1)
    yref = exact.free_sign_apply(x, dims, -1.5, 0.5)
    fA, fAH = ops(U, dims, -1.5, 0.5)
    y, info = krylov.sign_apply(fA, fAH, x, False, 400, 50, 1e-10)
    assert rel(y, yref) > 1e-8
    assert info["status"] == krylov.NOT_CONVERGED
    assert info["err_est"] > 1e-8


# ---- P4: gauge covariance (exact at fixed k) --------------------------------

@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_p4_gauge_covariance(mu):
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "near_unit", 2, eps=0.4)
    om = oi.gauge_rotation(dims, 3)
    x = oi.gaussian_source(dims, 4)
    Up = dirac.gauge_rotate_links(U, om, dims)
    xp = dirac.gauge_rotate_spinor(x, om, dims)
    y, i1 = krylov.sign_apply(*ops(U, dims, -1.5, mu), x, mu == 0.0, 400, 40, 0, k_fixed=60)
    yp, i2 = krylov.sign_apply(*ops(Up, dims, -1.5, mu), xp, mu == 0.0, 400, 40, 0, k_fixed=60)
    assert rel(yp, dirac.gauge_rotate_spinor(y, om, dims)) < 1e-11
    assert np.allclose(i1["alpha"], i2["alpha"], atol=1e-12)


def test_p4_pure_gauge_free_field():
    """Pure-gauge links Omega(x) Omega(x+nu)^dag: y = Omega y_free(Omega^dag x)."""
    dims = (4, 4, 4, 8)
    om = oi.gauge_rotation(dims, 6)
    U = dirac.gauge_rotate_links(oi.gauge_field(dims, "unit", 0), om, dims)
    x = oi.gaussian_source(dims, 7)
    x0 = dirac.gauge_rotate_spinor(x, np.conj(np.swapaxes(om, -1, -2)), dims)
    yref = dirac.gauge_rotate_spinor(exact.free_sign_apply(x0, dims, -1.5, 0.0), om, dims)
    y, info = krylov.sign_apply(*ops(U, dims, -1.5, 0.0), x, True, 400, 60, 1e-10)
    assert rel(y, yref) < 2e-9


# ---- P5, P6: two-sided Lanczos identities -----------------------------------

def test_p5_two_sided_reduces_to_lanczos_at_mu0():
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "haar", 0)
    x = oi.gaussian_source(dims, 1)
    fA, fAH = ops(U, dims, -1.5, 0.0)
    o1 = krylov.Outer(fA, fAH, x, True)
    o2 = krylov.Outer(fA, fAH, x, False)
    for _ in range(30):
        o1.step()
        o2.step()
    assert np.allclose(np.real(o2.alpha), o1.alpha, atol=1e-12)
    assert np.abs(np.imag(o2.alpha)).max() < 1e-12
    assert np.allclose(np.abs(o2.gamma), o1.beta, atol=1e-12)
    assert np.allclose(o2.gamma, o2.beta, atol=1e-12)
    assert np.linalg.norm(o2.w - o2.v) < 1e-10


def test_p6_biorthogonality_and_ritz_matrix():
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "near_unit", 0, eps=0.4)
    x = oi.gaussian_source(dims, 1)
    fA, fAH = ops(U, dims, -1.5, 0.3)
    o = krylov.Outer(fA, fAH, x, False)
    W = [o.w]
    for _ in range(20):
        o.step()
        W.append(o.w)
    V = np.stack(o.V, axis=1)
    Wm = np.stack(W[:20], axis=1)
    assert np.abs(np.conj(Wm.T) @ V - np.eye(20)).max() < 1e-10
    AV = np.stack([fA(V[:, j]) for j in range(20)], axis=1)
    assert np.abs(np.conj(Wm.T) @ AV - o.H()).max() < 1e-10


# ---- P7: Roberts-Higham vs eigendecomposition -------------------------------

def test_p7_roberts_higham_small():
    rng = np.random.default_rng(0)
    # symmetric indefinite with eigenvalues away from 0
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    lam = np.concatenate([rng.uniform(0.3, 5, 25), -rng.uniform(0.3, 5, 15)])
    T = (Q * lam) @ Q.T
    S, its, ok = krylov.roberts_higham(T)
    assert ok
    assert np.abs(S - (Q * np.sign(lam)) @ Q.T).max() < 1e-12
    # complex, non-normal, eigenvalues off the imaginary axis
    X = rng.standard_normal((30, 30)) + 1j * rng.standard_normal((30, 30))
    ev = np.concatenate([rng.uniform(0.3, 3, 18), -rng.uniform(0.3, 3, 12)]) + 1j * rng.uniform(-2, 2, 30)
    T = X @ np.diag(ev) @ np.linalg.inv(X)
    S, its, ok = krylov.roberts_higham(T)
    Sref = X @ np.diag(np.sign(ev.real)) @ np.linalg.inv(X)
    assert ok
    assert np.linalg.norm(S - Sref) / np.linalg.norm(Sref) < 1e-10


def test_p7_roberts_higham_reports_failure():
    T = np.diag([1.0, -1.0, 1e-300])  # singular in double: not converged or inf
    with np.errstate(all="ignore"):
        try:
            S, its, ok = krylov.roberts_higham(T, maxit=5)
        except np.linalg.LinAlgError:
            ok = False
    assert not ok or not np.all(np.isfinite(S))


# ---- P8, P9: the inner level ------------------------------------------------

@pytest.mark.parametrize("hermitian,mu", [(True, 0.0), (False, 0.3)])
def test_p8_nested_with_l_equal_k_is_nonnested(hermitian, mu):
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "near_unit", 1, eps=0.4)
    x = oi.gaussian_source(dims, 2)
    o = krylov.Outer(*ops(U, dims, -1.5, mu), x, hermitian)
    for _ in range(40):
        o.step()
    H = o.H()
    c_n, _, ok, leff = krylov.nested_sign_e1(H, 40, hermitian)
    c_0, _, ok0 = krylov.nonnested_sign_e1(H)
    S, _ = exact.sign_spectral(H, hermitian)
    assert leff == 40
    assert np.linalg.norm(c_n - c_0) < 1e-9
    assert np.linalg.norm(c_0 - S[:, 0]) < 1e-11


def test_p8_preconditioning_identity_and_gap():
    """sgn(H) = sgn(H + H^{-1}) (Eq. (precond)); for Hermitian H the spectrum of
    H + H^{-1} has no point in (-2, 2) (Sec. 3, Fig. 2)."""
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "haar", 0)
    x = oi.gaussian_source(dims, 1)
    o = krylov.Outer(*ops(U, dims, -1.5, 0.0), x, True)
    for _ in range(80):
        o.step()
    H = o.H()
    M = H + np.linalg.inv(H)
    S1, l1 = exact.sign_spectral(H, True)
    S2, l2 = exact.sign_spectral(M, True)
    assert np.abs(S1 - S2).max() < 1e-10
    assert np.abs(l2).min() >= 2.0 - 1e-10
    # condition-number improvement (reported by the paper as about 10x)
    assert (np.abs(l1).max() / np.abs(l1).min()) > 2 * (np.abs(l2).max() / np.abs(l2).min())


def test_p9_naive_nesting_sees_only_the_corner():
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "haar", 0)
    x = oi.gaussian_source(dims, 1)
    o = krylov.Outer(*ops(U, dims, -1.5, 0.0), x, True)
    for _ in range(60):
        o.step()
    H = o.H()
    l = 15
    c, Q = krylov.naive_nested_sign_e1(H, l, True)
    # the inner basis is [e_1 .. e_l] up to signs
    assert np.abs(np.abs(Q[:l, :]) - np.eye(l)).max() < 1e-12
    assert np.abs(Q[l:, :]).max() < 1e-12
    S, _ = exact.sign_spectral(H[:l, :l], True)
    ref = np.zeros(60)
    ref[:l] = S[:, 0]
    assert np.abs(c - ref).max() < 1e-10


# ---- P10: invariants of sgn at any size -------------------------------------

def test_p10_invariants_hermitian():
    dims = (6, 6, 6, 6)
    U = oi.gauge_field(dims, "near_unit", 4, eps=0.3)
    fA, fAH = ops(U, dims, -1.6, 0.0)
    x = oi.gaussian_source(dims, 5)
    u = oi.gaussian_source(dims, 6)
    kw = dict(hermitian=True, k_max=600, l=80, tol=1e-10)
    Sx, _ = krylov.sign_apply(fA, fAH, x, **kw)
    Su, _ = krylov.sign_apply(fA, fAH, u, **kw)
    SSx, _ = krylov.sign_apply(fA, fAH, Sx, **kw)
    assert rel(SSx, x) < 1e-8
    assert abs(np.linalg.norm(Sx) - np.linalg.norm(x)) < 1e-8
    assert abs(np.vdot(u, Sx) - np.vdot(Su, x)) < 1e-8
    SAx, _ = krylov.sign_apply(fA, fAH, fA(x), **kw)
    assert rel(SAx, fA(Sx)) < 1e-8


def test_p10_adjoint_relation_nonhermitian():
    """<u, S(mu) x> = <S(-mu) u, x>: A(mu)^dag = A(-mu), so sgn(A(mu))^dag = sgn(A(-mu))."""
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "near_unit", 4, eps=0.3)
    x = oi.gaussian_source(dims, 5)
    u = oi.gaussian_source(dims, 6)
    kw = dict(hermitian=False, k_max=600, l=110, tol=1e-10)
    Sx, i1 = krylov.sign_apply(*ops(U, dims, -1.5, 0.3), x, **kw)
    Sm_u, i2 = krylov.sign_apply(*ops(U, dims, -1.5, -0.3), u, **kw)
    assert i1["status"] == krylov.OK and i2["status"] == krylov.OK
    assert abs(np.vdot(u, Sx) - np.vdot(Sm_u, x)) < 1e-9
    # and the Hermitian form of the identity fails at mu != 0
    Su, _ = krylov.sign_apply(*ops(U, dims, -1.5, 0.3), u, **kw)
    assert abs(np.vdot(u, Sx) - np.vdot(Su, x)) > 1e-4


# ---- P11: scale invariance (kappa normalisation) ----------------------------

def test_p11_kappa_normalisation():
    """The Krylov space and sgn are invariant under A -> 2 kappa A, so the
    non-nested result and the nested one with l = k do not depend on the
    normalisation, while alpha scales by 2 kappa. (The nested result with
    l < k does depend on it: H + H^{-1} is not scale invariant.)"""
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "haar", 0)
    x = oi.gaussian_source(dims, 1)
    m_w = -1.5
    two_kappa = 2.0 / (2 * m_w + 8)
    fA, fAH = ops(U, dims, m_w, 0.0)
    sA, sAH = (lambda v: two_kappa * fA(v)), (lambda v: two_kappa * fAH(v))
    y1, i1 = krylov.sign_apply(fA, fAH, x, True, 400, 40, 0, k_fixed=80, nested=False)
    y2, i2 = krylov.sign_apply(sA, sAH, x, True, 400, 40, 0, k_fixed=80, nested=False)
    assert rel(y2, y1) < 1e-11
    assert np.allclose(i2["alpha"], two_kappa * i1["alpha"], atol=1e-12)
    y3, _ = krylov.sign_apply(sA, sAH, x, True, 400, 80, 0, k_fixed=80)
    assert rel(y3, y1) < 1e-9
    y4, _ = krylov.sign_apply(sA, sAH, x, True, 400, 20, 0, k_fixed=80)
    y5, _ = krylov.sign_apply(fA, fAH, x, True, 400, 20, 0, k_fixed=80)
    assert rel(y4, y5) > 1e-8


# ---- P12: Ginsparg-Wilson relation at mu = 0 --------------------------------

@pytest.mark.dense
def test_p12_ginsparg_wilson_dense(haar44):
    S = haar44[0.0]["S"]
    A = haar44[0.0]["A"]
    n = S.shape[0]
    g5 = np.kron(np.eye(n // 12), np.kron(dirac.GAMMA5, np.eye(3)))
    D = np.eye(n) + g5 @ S
    gw = g5 @ D + D @ g5 - D @ g5 @ D
    assert np.linalg.norm(gw) <= 1e-10 * np.linalg.norm(D)
    assert np.linalg.norm(S @ S - np.eye(n)) < 1e-10 * np.sqrt(n)
    assert np.linalg.norm(S @ A - A @ S) < 1e-10 * np.linalg.norm(A)
    assert np.linalg.norm(S - np.conj(S.T)) < 1e-12 * np.sqrt(n)


def test_p12_ginsparg_wilson_vector():
    """gamma5 D x + D gamma5 x = D gamma5 D x with D = 1 + gamma5 S, three applies."""
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "near_unit", 3, eps=0.3)
    fA, fAH = ops(U, dims, -1.5, 0.0)
    x = oi.gaussian_source(dims, 9)
    g5 = lambda v: dirac.gamma5_apply(v, dims)
    kw = dict(hermitian=True, k_max=600, l=80, tol=1e-11)
    D = lambda v: v + g5(krylov.sign_apply(fA, fAH, v, **kw)[0])
    lhs = g5(D(x)) + D(g5(x))
    rhs = D(g5(D(x)))
    assert rel(lhs, rhs) < 1e-8


# ---- recombination and edge cases -------------------------------------------

@pytest.mark.parametrize("hermitian,mu", [(True, 0.0), (False, 0.3)])
def test_two_pass_equals_stored(hermitian, mu):
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "near_unit", 1, eps=0.4)
    x = oi.gaussian_source(dims, 2)
    y1, i1 = krylov.sign_apply(*ops(U, dims, -1.5, mu), x, hermitian, 400, 60, 1e-10, two_pass=False)
    y2, i2 = krylov.sign_apply(*ops(U, dims, -1.5, mu), x, hermitian, 400, 60, 1e-10, two_pass=True)
    assert i1["k"] == i2["k"]
    assert rel(y2, y1) < 1e-13


def test_eigenvector_source_lucky_breakdown():
    """x an eigenvector of A: the Krylov space is one-dimensional and the
    answer sgn(lambda) x is exact after one step."""
    dims = (2, 2, 2, 2)
    U = oi.gauge_field(dims, "haar", 0)
    A = dirac.dense_A(U, dims, -1.5, 0.0)
    lam, Uv = np.linalg.eigh(A)
    x = Uv[:, 3]
    y, info = krylov.sign_apply(*ops(U, dims, -1.5, 0.0), x, True, 50, 10, 1e-10)
    assert info["k"] == 1
    assert info["status"] == krylov.OK
    assert rel(y, np.sign(lam[3]) * x) < 1e-12


def test_k_max_not_converged():
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "haar", 0)
    x = oi.gaussian_source(dims, 1)
    y, info = krylov.sign_apply(*ops(U, dims, -1.5, 0.0), x, True, 30, 20, 1e-10)
    assert info["status"] == krylov.NOT_CONVERGED
    assert info["k"] == 30
    assert info["err_est"] > 1e-10
