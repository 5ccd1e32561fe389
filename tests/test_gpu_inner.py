"""Inner level parity: tridiagonal GEPP, inner Lanczos / two-sided Lanczos on
H + H^{-1}, Roberts-Higham (Sec. 3, Eqs. (nested), (precond); Eq. (Roberts))."""
import numpy as np
import pytest

import ovinputs as oi
from gpu_util import oracle_ops
from oracle import krylov

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ov():
    import paper_0910_2918_gb300 as ov

    return ov


@pytest.fixture(scope="module", params=["df64", "df64_plain", "fp64"])
def handle(ov, request):
    """Both arithmetics of the inner level's serial parts (float pairs, the default, and FP64),
    the float-pair form with determinant-scaled (default) and plain Roberts-Higham steps."""
    dims = (2, 2, 2, 2)
    arith = ov.binding.OV_INNER_FP64 if request.param == "fp64" else ov.binding.OV_INNER_DF64
    h = ov.ov_create(dims, oi.gauge_field(dims, "unit", 0), -1.5, 0.0,
                     opts=ov.make_opts(inner_arith=arith, rh_scaling=0 if request.param == "df64_plain" else 1))
    yield h
    ov.ov_destroy(h)


def ritz(mu, k, seed=0, dims=(4, 4, 4, 4), kind="haar"):
    U = oi.gauge_field(dims, kind, seed, eps=0.4)
    x = oi.gaussian_source(dims, seed + 1)
    o = krylov.Outer(*oracle_ops(U, dims, -1.5, mu), x, mu == 0.0)
    for _ in range(k):
        o.step()
    return o


def pack(outers, ld):
    A = np.zeros((len(outers), ld), complex)
    B = np.zeros_like(A)
    G = np.zeros_like(A)
    ks = []
    for i, o in enumerate(outers):
        k = o.k
        ks.append(k)
        A[i, :k] = o.alpha
        B[i, 1:k] = o.beta[1:k]
        G[i, 1:k] = o.gamma[1:k]
    return ks, A, B, G


@pytest.mark.parametrize("mu,l", [(0.0, 80), (0.3, 110), (0.3, 120), (0.0, 120)])
def test_inner_sign_vs_oracle(ov, handle, mu, l):
    """Parity at an inner dimension where the inner level has converged."""
    outers = [ritz(mu, k, seed=s) for k, s in ((150, 0), (97, 2), (64, 4))]
    ks, A, B, G = pack(outers, 160)
    rc, c, est, its = ov.ov_inner_sign(handle, ks, A, B, G, mu == 0.0, l)
    assert rc == 0
    for i, o in enumerate(outers):
        H = o.H()
        cref, _, ok, leff = krylov.nested_sign_e1(H, l, mu == 0.0)
        k = ks[i]
        est_ref = krylov.inner_estimate(H, leff, mu == 0.0, cref, leff < min(l, k))
        assert est_ref < 1e-11
        assert np.linalg.norm(c[i, :k] - cref) / np.linalg.norm(cref) < 1e-10
        assert np.all(c[i, k:] == 0)
        assert est[i] < 1e-10


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_inner_sign_unconverged_is_valid(ov, handle, mu):
    """Below convergence the nested vector is not unique: the inner Lanczos basis
    loses orthogonality early, so roundoff (a 1e-15 change of H^{-1} u) moves c by a
    fraction of the approximation error. What is unique is sgn(H) e_1; both sides
    must be within their estimate of it, and the estimates must agree in size."""
    outers = [ritz(mu, k, seed=s) for k, s in ((150, 0), (97, 2), (64, 4))]
    ks, A, B, G = pack(outers, 160)
    rc, c, est, its = ov.ov_inner_sign(handle, ks, A, B, G, mu == 0.0, 30)
    for i, o in enumerate(outers):
        H = o.H()
        k = ks[i]
        S, _, _ = krylov.roberts_higham(H)
        exact = S[:, 0]
        cref, _, ok, leff = krylov.nested_sign_e1(H, 30, mu == 0.0)
        est_ref = krylov.inner_estimate(H, leff, mu == 0.0, cref, False)
        assert np.linalg.norm(c[i, :k] - exact) <= 3 * est[i]
        assert np.linalg.norm(cref - exact) <= 3 * est_ref
        assert 0.1 < est[i] / est_ref < 10


def test_inner_sign_exact_when_l_equals_k(ov, handle):
    o = ritz(0.3, 30, seed=6)
    ks, A, B, G = pack([o], 40)
    rc, c, est, its = ov.ov_inner_sign(handle, ks, A, B, G, False, 30)
    S, _, _ = krylov.roberts_higham(o.H())
    assert np.linalg.norm(c[0, :30] - S[:, 0]) < 1e-10
    assert est[0] == 0.0


def test_roberts_higham_dense(ov, handle):
    rng = np.random.default_rng(1)
    mats = []
    for m in (120, 57, 8):
        X = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
        ev = np.concatenate([rng.uniform(0.3, 3, m // 2), -rng.uniform(0.3, 3, m - m // 2)]) + 1j * rng.uniform(-1, 1, m)
        mats.append((X @ np.diag(ev) @ np.linalg.inv(X), X, ev))
    for T, X, ev in mats:
        rc, S, its = ov.ov_rh_sign(handle, T[None])
        assert rc == 0
        Sref, it_ref, ok = krylov.roberts_higham(T)
        assert np.linalg.norm(S[0] - Sref) / np.linalg.norm(Sref) < 1e-10
        assert abs(int(its[0]) - it_ref) <= 1


def test_roberts_higham_singular_reports(ov, handle):
    T = np.zeros((1, 6, 6), complex)
    T[0, :3, :3] = np.eye(3)
    rc, S, its = ov.ov_rh_sign(handle, T)
    assert rc == ov.binding.OV_ERR_RH_NOCONV


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_inner_arithmetics_agree(ov, mu):
    """The float-pair and FP64 inner levels give the same converged c (1e-12) and the
    same inner estimate in size."""
    outers = [ritz(mu, k, seed=s) for k, s in ((200, 8), (120, 9))]
    ks, A, B, G = pack(outers, 200)
    dims = (2, 2, 2, 2)
    out = {}
    for arith in (ov.binding.OV_INNER_DF64, ov.binding.OV_INNER_FP64):
        h = ov.ov_create(dims, oi.gauge_field(dims, "unit", 0), -1.5, 0.0, opts=ov.make_opts(inner_arith=arith))
        out[arith] = ov.ov_inner_sign(h, ks, A, B, G, mu == 0.0, 110)
        ov.ov_destroy(h)
    (rd, cd, ed, _), (rf, cf, ef, _) = out[ov.binding.OV_INNER_DF64], out[ov.binding.OV_INNER_FP64]
    assert rd == 0 and rf == 0
    for i, k in enumerate(ks):
        assert np.linalg.norm(cd[i, :k] - cf[i, :k]) / np.linalg.norm(cf[i, :k]) < 1e-12
        assert ed[i] < 1e-10 and ef[i] < 1e-10


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_scaled_roberts_higham_same_sign_fewer_steps(ov, mu):
    """Determinant-scaled Roberts-Higham steps in the inner level reach the same sgn(T_l) e_1
    (1e-12) as the plain iteration of Eq. (Roberts), in fewer inversions."""
    outers = [ritz(mu, k, seed=s) for k, s in ((200, 8), (120, 9), (64, 3))]
    ks, A, B, G = pack(outers, 200)
    dims = (2, 2, 2, 2)
    out = {}
    for sc in (0, 1):
        h = ov.ov_create(dims, oi.gauge_field(dims, "unit", 0), -1.5, 0.0, opts=ov.make_opts(rh_scaling=sc))
        out[sc] = ov.ov_inner_sign(h, ks, A, B, G, mu == 0.0, 110)
        ov.ov_destroy(h)
    (r0, c0, e0, i0), (r1, c1, e1, i1) = out[0], out[1]
    assert r0 == 0 and r1 == 0
    for i, k in enumerate(ks):
        assert np.linalg.norm(c1[i, :k] - c0[i, :k]) / np.linalg.norm(c0[i, :k]) < 1e-12
        assert e1[i] < 1e-10
    assert np.sum(i1) < np.sum(i0), (i0, i1)
