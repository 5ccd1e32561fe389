"""Pins of the oracle's Wilson-Dirac operator (Sec. 1, Eq. (Dov)).

The operator formula is not printed in the paper; these tests fix it against
the free-field closed form (plane waves), the Clifford algebra, gamma5
Hermiticity and gauge covariance, and against a brute-force site loop.
"""
import itertools

import numpy as np
import pytest

import ovinputs as oi
from oracle import dirac, exact
from conftest import rel


def test_gamma_algebra():
    G = dirac.GAMMA
    for a, b in itertools.product(range(4), range(4)):
        assert np.allclose(G[a] @ G[b] + G[b] @ G[a], 2.0 * (a == b) * np.eye(4))
    for a in range(4):
        assert np.allclose(G[a], np.conj(G[a].T))
    # chiral basis: gamma5 = gamma1 gamma2 gamma3 gamma4 = diag(1, 1, -1, -1)
    assert np.allclose(dirac.GAMMA5, np.diag([1, 1, -1, -1]))


@pytest.mark.parametrize("mu", [0.0, 0.3, -0.2])
@pytest.mark.parametrize("n_mom", [(0, 0, 0, 0), (1, 2, 3, 1), (3, 0, 1, 2), (2, 2, 2, 3)])
def test_plane_wave_closed_form(mu, n_mom):
    """A e^{ip.x} chi = e^{ip.x} gamma5 D(p) chi with D(p) = m + sum(1 - cos pt)
    + i sum gamma sin pt, pt_t = p_t - i mu: fixes the projector sign, the
    direction of e^{+mu}, the 1/2 normalisation and the antiperiodic t boundary."""
    dims = (4, 4, 6, 4)
    U = oi.gauge_field(dims, "unit", 0)
    chi = oi.complex_gaussian(np.random.default_rng(7), (4, 3))
    x, _ = exact.plane_wave(dims, n_mom, chi)
    Ax = dirac.A_apply(U, x, dims, -1.5, mu)
    D = exact.free_dirac_momentum(dims, -1.5, mu)
    nx, ny, nz, nt = n_mom
    Ap = dirac.GAMMA5 @ D[nt, nz, ny, nx]
    ref = np.einsum("st,vtc->vsc", Ap, x.reshape(-1, 4, 3)).reshape(-1)
    assert rel(Ax, ref) < 1e-13


def _brute_wilson(U, psi, dims, m_w, mu):
    """Site-by-site loop over neighbours with explicit index arithmetic."""
    lx, ly, lz, lt = dims
    V = lx * ly * lz * lt
    U = U.reshape(V, 4, 3, 3)
    psi = psi.reshape(V, 4, 3)
    out = np.zeros_like(psi)
    G = dirac.GAMMA

    def coords(s):
        return [s % lx, (s // lx) % ly, (s // (lx * ly)) % lz, s // (lx * ly * lz)]

    def site(c):
        return c[0] + lx * (c[1] + ly * (c[2] + lz * c[3]))

    L = [lx, ly, lz, lt]
    for s in range(V):
        c = coords(s)
        acc = np.zeros((4, 3), dtype=complex)
        for nu in range(4):
            cf = list(c)
            cf[nu] += 1
            sign_f = 1.0
            if cf[nu] == L[nu]:
                cf[nu] = 0
                if nu == 3:
                    sign_f = -1.0
            cb = list(c)
            cb[nu] -= 1
            sign_b = 1.0
            if cb[nu] < 0:
                cb[nu] = L[nu] - 1
                if nu == 3:
                    sign_b = -1.0
            sf, sb = site(cf), site(cb)
            ef = np.exp(mu) if nu == 3 else 1.0
            eb = np.exp(-mu) if nu == 3 else 1.0
            for a in range(3):
                for spin in range(4):
                    for t in range(4):
                        pf = (1.0 if spin == t else 0.0) - G[nu][spin, t]
                        pb = (1.0 if spin == t else 0.0) + G[nu][spin, t]
                        for b in range(3):
                            acc[spin, a] += ef * sign_f * pf * U[s, nu, a, b] * psi[sf, t, b]
                            acc[spin, a] += eb * sign_b * pb * np.conj(U[sb, nu, b, a]) * psi[sb, t, b]
        out[s] = (m_w + 4.0) * psi[s] - 0.5 * acc
    return out.reshape(-1)


def test_brute_force_site_loop():
    dims = (2, 3, 2, 4)
    U = oi.gauge_field(dims, "haar", 11)
    psi = oi.gaussian_source(dims, 12)
    for mu in (0.0, 0.25):
        assert rel(dirac.wilson_apply(U, psi, dims, -1.3, mu), _brute_wilson(U, psi, dims, -1.3, mu)) < 1e-13


def test_gamma5_hermiticity():
    """A is Hermitian at mu = 0; <u, A v> = <A^dag u, v> with A^dag = gamma5 D_w(-mu)."""
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "haar", 3)
    u = oi.gaussian_source(dims, 4)
    v = oi.gaussian_source(dims, 5)
    lhs = np.vdot(u, dirac.A_apply(U, v, dims, -1.5, 0.0))
    rhs = np.vdot(dirac.A_apply(U, u, dims, -1.5, 0.0), v)
    assert abs(lhs - rhs) < 1e-12
    lhs = np.vdot(u, dirac.A_apply(U, v, dims, -1.5, 0.4))
    rhs = np.vdot(dirac.AH_apply(U, u, dims, -1.5, 0.4), v)
    assert abs(lhs - rhs) < 1e-12
    # and it is not Hermitian at mu != 0
    rhs_wrong = np.vdot(dirac.A_apply(U, u, dims, -1.5, 0.4), v)
    assert abs(lhs - rhs_wrong) > 1e-3


def test_gauge_covariance_operator():
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "near_unit", 8, eps=0.4)
    om = oi.gauge_rotation(dims, 9)
    x = oi.gaussian_source(dims, 10)
    Up = dirac.gauge_rotate_links(U, om, dims)
    xp = dirac.gauge_rotate_spinor(x, om, dims)
    for mu in (0.0, 0.3):
        lhs = dirac.A_apply(Up, xp, dims, -1.5, mu)
        rhs = dirac.gauge_rotate_spinor(dirac.A_apply(U, x, dims, -1.5, mu), om, dims)
        assert rel(lhs, rhs) < 1e-13


def test_inputs_are_su3():
    dims = (2, 2, 2, 2)
    for kind in ("haar", "near_unit"):
        U = oi.gauge_field(dims, kind, 1, eps=0.3).reshape(-1, 3, 3)
        assert np.allclose(U @ np.conj(np.swapaxes(U, -1, -2)), np.eye(3), atol=1e-13)
        assert np.allclose(np.linalg.det(U), 1.0, atol=1e-13)
