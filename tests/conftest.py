import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libov")
    config.addinivalue_line("markers", "slow: long CPU test")
    config.addinivalue_line("markers", "dense: large dense linear algebra (all BLAS threads)")


@pytest.fixture(scope="session")
def haar44():
    """4^4 Haar links (seed 0), m_w = -1.5, Gaussian source (seed 1), the dense
    A at mu = 0 with its exact sign function (eigh)."""
    import ovinputs as oi
    from oracle import dirac, exact

    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "haar", 0)
    x = oi.gaussian_source(dims, 1)
    out = dict(dims=dims, U=U, x=x, m_w=-1.5)
    A = dirac.dense_A(U, dims, -1.5, 0.0)
    S, lam = exact.sign_spectral(A, True)
    out[0.0] = dict(A=A, S=S, lam=lam)
    return out


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))
