"""Random draws for synthetic lattice workloads (no Dirac-operator arithmetic)."""
import numpy as np


def lattice_volume(dims):
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def complex_gaussian(rng, shape):
    """(N(0,1) + i N(0,1)) / sqrt(2), so E|z|^2 = 1."""
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) / np.sqrt(2.0)


def haar_su3(rng, count):
    """`count` Haar-random SU(3) matrices, shape (count, 3, 3).

    QR of a complex Gaussian matrix with the phases of R's diagonal moved into
    Q gives a Haar-distributed U(3) element (Mezzadri, Notices AMS 54 (2007)
    592); dividing by the principal cube root of its determinant puts it in
    SU(3).
    """
    z = complex_gaussian(rng, (count, 3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    ph = d / np.abs(d)
    q = q * ph[:, None, :]
    det = np.linalg.det(q)
    q = q / (det ** (1.0 / 3.0))[:, None, None]
    return q


def near_unit_su3(rng, count, eps):
    """`count` matrices exp(i*eps*H), H Hermitian traceless from a complex Gaussian.

    H = (G + G^dag)/2 - tr(.)/3; the exponential is taken through eigh, which is
    exact for Hermitian H.
    """
    g = complex_gaussian(rng, (count, 3, 3))
    h = 0.5 * (g + np.conj(np.swapaxes(g, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)[None]
    w, v = np.linalg.eigh(h)
    ph = np.exp(1j * eps * w)
    return np.einsum("nij,nj,nkj->nik", v, ph, np.conj(v))


def gauge_field(dims, kind, seed, eps=0.3):
    """Gauge links U[V][4][3][3] (complex128).

    kind: 'haar' (Haar-random SU(3)), 'near_unit' (exp(i*eps*H)) or 'unit'
    (free field U = 1).
    """
    V = lattice_volume(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "haar":
        u = haar_su3(rng, V * 4)
    elif kind == "near_unit":
        u = near_unit_su3(rng, V * 4, eps)
    elif kind == "unit":
        u = np.broadcast_to(np.eye(3, dtype=np.complex128), (V * 4, 3, 3)).copy()
    else:
        raise ValueError(kind)
    return np.ascontiguousarray(u.reshape(V, 4, 3, 3))


def round_links_fp32(u):
    """Links rounded once to complex64 and widened back to complex128.

    Single-precision runs use exactly these values, so the operator of a
    single-precision run is the same operator the double-precision oracle sees.
    """
    return u.astype(np.complex64).astype(np.complex128)


def gaussian_source(dims, seed, normalize=True):
    V = lattice_volume(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    x = complex_gaussian(rng, 12 * V)
    if normalize:
        x = x / np.linalg.norm(x)
    return x


def point_source(dims, site, spin, colour):
    V = lattice_volume(dims)
    x = np.zeros(12 * V, dtype=np.complex128)
    x[12 * site + 3 * spin + colour] = 1.0
    return x


def point_sources_12(dims, site=0):
    """The 12 spin-colour point sources at one site, shape (12, n)."""
    return np.stack([point_source(dims, site, s, c) for s in range(4) for c in range(3)])


def gauge_rotation(dims, seed):
    """Haar SU(3) matrix per site, shape (V, 3, 3) (a random gauge transformation)."""
    V = lattice_volume(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    return haar_su3(rng, V)


def problem_batch_48(seed_base=0):
    """48 independent problems of uneven size: 12 each of 4^4, 6^4, 6^3x12, 8^4.

    Problem i: Haar links if i is even, else near-unit links with eps_i drawn
    from U[0.2, 0.5]; mu_i from U[0, 0.5]; m_w = -1.5; one Gaussian source.
    Returns a list of dicts with keys dims, kind, eps, mu, m_w, gauge_seed,
    source_seed.
    """
    shapes = [(4, 4, 4, 4), (6, 6, 6, 6), (6, 6, 6, 12), (8, 8, 8, 8)]
    rng = np.random.Generator(np.random.PCG64(seed_base + 4848))
    probs = []
    for i in range(48):
        dims = shapes[i // 12]
        mu = float(rng.uniform(0.0, 0.5))
        eps = float(rng.uniform(0.2, 0.5))
        kind = "haar" if i % 2 == 0 else "near_unit"
        probs.append(dict(dims=dims, kind=kind, eps=eps if kind == "near_unit" else 0.0,
                          mu=mu, m_w=-1.5, gauge_seed=seed_base + i,
                          source_seed=seed_base + i + 1))
    return probs


def training_problems(count=2000, seed_base=1000):
    """Small problems for learning (k, l): 6^4, 6^3x8, 8^3x6, 8^4, mu ~ U[0,0.5],
    eps ~ U[0.2,0.5], m_w ~ U[-1.8,-1.3], seeds seed_base + i; the source is a Gaussian
    (even i) or a spin-colour point source at site 0 (odd i)."""
    shapes = [(6, 6, 6, 6), (6, 6, 6, 8), (8, 8, 8, 6), (8, 8, 8, 8)]
    out = []
    for i in range(count):
        rng = np.random.Generator(np.random.PCG64(seed_base + i))
        dims = shapes[int(rng.integers(0, 4))]
        mu = float(rng.uniform(0.0, 0.5))
        eps = float(rng.uniform(0.2, 0.5))
        m_w = float(rng.uniform(-1.8, -1.3))
        sc = int(rng.integers(0, 12))
        out.append(dict(dims=dims, kind="near_unit", eps=eps, mu=mu, m_w=m_w,
                        gauge_seed=seed_base + i, source_seed=seed_base + i + 100000,
                        source="gaussian" if i % 2 == 0 else "point", spin=sc // 3, colour=sc % 3))
    return out


def training_problems_rough(count=400, seed_base=20000):
    """Problems for learning (k, l) that include rough fields and the shapes of the
    48-lattice batch: 4^4, 6^4, 6^3x8, 6^3x12, 8^3x6, 8^4; Haar links (half of them) or
    near-unit links with eps ~ U[0.2, 0.5]; mu ~ U[0, 0.5], m_w ~ U[-1.8, -1.3]; seeds
    seed_base + i (disjoint from the batch's and from training_problems'); a Gaussian
    source (even i) or a spin-colour point source at site 0 (odd i)."""
    shapes = [(4, 4, 4, 4), (6, 6, 6, 6), (6, 6, 6, 8), (6, 6, 6, 12), (8, 8, 8, 6), (8, 8, 8, 8)]
    out = []
    for i in range(count):
        rng = np.random.Generator(np.random.PCG64(seed_base + i))
        dims = shapes[int(rng.integers(0, len(shapes)))]
        kind = "haar" if rng.uniform() < 0.5 else "near_unit"
        mu = float(rng.uniform(0.0, 0.5))
        eps = float(rng.uniform(0.2, 0.5))
        m_w = float(rng.uniform(-1.8, -1.3))
        sc = int(rng.integers(0, 12))
        out.append(dict(dims=dims, kind=kind, eps=eps if kind == "near_unit" else 0.0, mu=mu, m_w=m_w,
                        gauge_seed=seed_base + i, source_seed=seed_base + i + 100000,
                        source="gaussian" if i % 2 == 0 else "point", spin=sc // 3, colour=sc % 3))
    return out


def training_problems_large(count=120, seed_base=40000):
    """Larger problems for learning (k, l): 10^4, 12^4, 12^3x16, 16^4, near-unit links with
    eps ~ U[0.2, 0.5], mu ~ U[0, 0.5], m_w ~ U[-1.8, -1.3]; seeds seed_base + i (disjoint
    from every evaluation workload's); a Gaussian source (even i) or a spin-colour point
    source at site 0 (odd i)."""
    shapes = [(10, 10, 10, 10), (12, 12, 12, 12), (12, 12, 12, 16), (16, 16, 16, 16)]
    out = []
    for i in range(count):
        rng = np.random.Generator(np.random.PCG64(seed_base + i))
        dims = shapes[int(rng.integers(0, len(shapes)))]
        mu = float(rng.uniform(0.0, 0.5))
        eps = float(rng.uniform(0.2, 0.5))
        m_w = float(rng.uniform(-1.8, -1.3))
        sc = int(rng.integers(0, 12))
        out.append(dict(dims=dims, kind="near_unit", eps=eps, mu=mu, m_w=m_w,
                        gauge_seed=seed_base + i, source_seed=seed_base + i + 100000,
                        source="gaussian" if i % 2 == 0 else "point", spin=sc // 3, colour=sc % 3))
    return out


def problem_source(p):
    """The source of a problem dict from training_problems / problem_batch_48."""
    if p.get("source", "gaussian") == "point":
        return point_source(p["dims"], 0, p["spin"], p["colour"])
    return gaussian_source(p["dims"], p["source_seed"])
