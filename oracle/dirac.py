"""Wilson-Dirac operator with chemical potential (oracle; test infrastructure).

Sec. 1, Eq. (Dov): D_ov(mu) = 1 + gamma5 sgn(gamma5 D_w(mu)), with -2 < m_w < 0
and mu entering the time links as prescribed by Hasenfratz and Karsch. The paper
does not print D_w; this module uses the standard form

  (D_w psi)(x) = (m_w + 4) psi(x)
      - 1/2 sum_nu [ (1 - gamma_nu) e^{+mu delta_{nu,t}} U_nu(x) psi(x + nu)
                   + (1 + gamma_nu) e^{-mu delta_{nu,t}} U_nu(x - nu)^dag psi(x - nu) ],

periodic in x, y, z and antiperiodic in t (a hop that wraps in t picks up -1),
with the DeGrand-Rossi (chiral) gamma basis, gamma5 = gamma1 gamma2 gamma3 gamma4.
A = gamma5 D_w(mu) is Hermitian at mu = 0 (Sec. 1); its adjoint is
A^dag = gamma5 D_w(-mu), because gamma5 D_w(mu) gamma5 = D_w(-mu)^dag.

Field layout: psi has shape (..., Lt, Lz, Ly, Lx, 4, 3), i.e. a flat vector of
length 12 V with index 12*site + 3*spin + colour reshapes to it directly.
Links have shape (V, 4, 3, 3) = (Lt, Lz, Ly, Lx, 4, 3, 3) after reshape.
"""
import numpy as np

I4 = np.eye(4, dtype=np.complex128)

# DeGrand-Rossi basis; index 0..3 = x, y, z, t.
GAMMA = np.array([
    [[0, 0, 0, 1j], [0, 0, 1j, 0], [0, -1j, 0, 0], [-1j, 0, 0, 0]],
    [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],
    [[0, 0, 1j, 0], [0, 0, 0, -1j], [-1j, 0, 0, 0], [0, 1j, 0, 0]],
    [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],
], dtype=np.complex128)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]

# lattice axis of direction nu in a field of shape (..., Lt, Lz, Ly, Lx, 4, 3)
_FIELD_AXIS = {0: -3, 1: -4, 2: -5, 3: -6}
# lattice axis of direction nu in links of shape (Lt, Lz, Ly, Lx, 4, 3, 3)
_LINK_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}


def _lattice_shape(dims):
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def as_field(vec, dims):
    """Flat spinor(s) (..., 12V) -> (..., Lt, Lz, Ly, Lx, 4, 3)."""
    vec = np.asarray(vec)
    return vec.reshape(vec.shape[:-1] + _lattice_shape(dims) + (4, 3))


def as_links(u, dims):
    return np.asarray(u).reshape(_lattice_shape(dims) + (4, 3, 3))


def _shift(psi, nu, step, antiperiodic):
    """psi(x + step*nu) (step = +1 forward, -1 backward), with the t-boundary sign."""
    ax = _FIELD_AXIS[nu]
    out = np.roll(psi, -step, axis=ax)
    if nu == 3 and antiperiodic:
        lt = psi.shape[ax]
        idx = [slice(None)] * psi.ndim
        # forward: the site t = Lt-1 received psi(t = 0) across the boundary;
        # backward: the site t = 0 received psi(t = Lt-1).
        idx[ax] = lt - 1 if step == 1 else 0
        out[tuple(idx)] *= -1.0
    return out


def wilson_apply(u, psi_vec, dims, m_w, mu, antiperiodic=True):
    """D_w(mu) psi for flat spinor(s) psi_vec of shape (..., 12V)."""
    links = as_links(u, dims)
    psi = as_field(psi_vec, dims)
    out = (m_w + 4.0) * psi
    hop = np.zeros_like(psi)
    for nu in range(4):
        unu = links[..., nu, :, :]
        fac_f = np.exp(mu) if nu == 3 else 1.0
        fac_b = np.exp(-mu) if nu == 3 else 1.0
        # forward hop: (1 - gamma_nu) e^{mu} U_nu(x) psi(x + nu)
        psi_f = _shift(psi, nu, +1, antiperiodic)
        chi = np.einsum("...ab,...sb->...sa", unu, psi_f)
        hop += fac_f * np.einsum("st,...tc->...sc", I4 - GAMMA[nu], chi)
        # backward hop: (1 + gamma_nu) e^{-mu} U_nu(x - nu)^dag psi(x - nu)
        ub = np.roll(unu, 1, axis=_LINK_AXIS[nu])
        psi_b = _shift(psi, nu, -1, antiperiodic)
        chi = np.einsum("...ba,...sb->...sa", np.conj(ub), psi_b)
        hop += fac_b * np.einsum("st,...tc->...sc", I4 + GAMMA[nu], chi)
    out = out - 0.5 * hop
    return out.reshape(np.shape(psi_vec))


def gamma5_apply(psi_vec, dims):
    psi = as_field(psi_vec, dims)
    return np.einsum("st,...tc->...sc", GAMMA5, psi).reshape(np.shape(psi_vec))


def A_apply(u, psi_vec, dims, m_w, mu, antiperiodic=True):
    """A psi = gamma5 D_w(mu) psi."""
    return gamma5_apply(wilson_apply(u, psi_vec, dims, m_w, mu, antiperiodic), dims)


def AH_apply(u, psi_vec, dims, m_w, mu, antiperiodic=True):
    """A^dag psi = gamma5 D_w(-mu) psi."""
    return gamma5_apply(wilson_apply(u, psi_vec, dims, m_w, -mu, antiperiodic), dims)


def dense_A(u, dims, m_w, mu, antiperiodic=True, chunk=512):
    """The n x n matrix of A (columns A e_i), for small lattices only."""
    n = 12 * int(np.prod(dims))
    out = np.empty((n, n), dtype=np.complex128)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        e = np.zeros((c1 - c0, n), dtype=np.complex128)
        e[np.arange(c1 - c0), np.arange(c0, c1)] = 1.0
        out[:, c0:c1] = A_apply(u, e, dims, m_w, mu, antiperiodic).T
    return out


def gauge_rotate_links(u, omega, dims):
    """U'_nu(x) = Omega(x) U_nu(x) Omega(x + nu)^dag (gauge transformation)."""
    links = as_links(u, dims)
    om = np.asarray(omega).reshape(_lattice_shape(dims) + (3, 3))
    out = np.empty_like(links)
    for nu in range(4):
        om_f = np.roll(om, -1, axis=_LINK_AXIS[nu])
        out[..., nu, :, :] = om @ links[..., nu, :, :] @ np.conj(np.swapaxes(om_f, -1, -2))
    return out.reshape(np.shape(u))


def gauge_rotate_spinor(psi_vec, omega, dims):
    """psi'(x) = Omega(x) psi(x) (acts on colour)."""
    psi = as_field(psi_vec, dims)
    om = np.asarray(omega).reshape(_lattice_shape(dims) + (3, 3))
    return np.einsum("...ab,...sb->...sa", om, psi).reshape(np.shape(psi_vec))
