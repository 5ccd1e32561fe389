"""Stencil parity: A x = gamma5 D_w(mu) x and A^dag x on the GPU vs the oracle (Sec. 1)."""
import numpy as np
import pytest

import ovinputs as oi
from gpu_util import links_for, rel
from oracle import dirac

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-14, "df64": 5e-14, "fp32": 2e-6}


@pytest.fixture(scope="module")
def ov():
    import paper_0910_2918_gb300 as ov

    return ov


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("dims,mu", [((4, 4, 4, 4), 0.0), ((4, 6, 2, 8), 0.3), ((3, 5, 4, 6), -0.2),
                                     ((8, 8, 8, 8), 0.2)])
def test_stencil_vs_oracle(ov, prec, dims, mu):
    U = oi.gauge_field(dims, "haar", 3)
    Ul = links_for(prec, U)
    x = np.stack([oi.gaussian_source(dims, s) for s in (4, 5, 6)])
    y = np.zeros_like(x)
    with ov.Overlap(dims, U, -1.5, mu, prec) as op:
        for dag in (False, True):
            op.wilson_apply(x, y, dagger=dag)
            f = dirac.AH_apply if dag else dirac.A_apply
            for r in range(3):
                assert rel(y[r], f(Ul, x[r], dims, -1.5, mu)) < TOL[prec]


def test_stencil_periodic_time_and_device_buffers(ov):
    import torch

    dims = (4, 4, 4, 6)
    U = oi.gauge_field(dims, "near_unit", 1, eps=0.4)
    x = oi.gaussian_source(dims, 2).reshape(1, -1)
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros_like(xd)
    with ov.Overlap(dims, torch.from_numpy(U).cuda(), -1.2, 0.1, "fp64", t_antiperiodic=False) as op:
        op.wilson_apply(xd, yd)
    ref = dirac.A_apply(U, x[0], dims, -1.2, 0.1, antiperiodic=False)
    assert rel(yd.cpu().numpy()[0], ref) < 1e-14


def test_stencil_full_size_bench_lattice(ov):
    """16^4, 12 point sources, the bench's launch shape (double-float)."""
    dims = (16, 16, 16, 16)
    U = oi.gauge_field(dims, "near_unit", 0, eps=0.3)
    x = oi.point_sources_12(dims)
    x[:, :] += 1e-3 * oi.gaussian_source(dims, 9)[None, :]
    y = np.zeros_like(x)
    with ov.Overlap(dims, U, -1.6, 0.2, "df64") as op:
        op.wilson_apply(x, y)
    for r in (0, 5, 11):
        assert rel(y[r], dirac.A_apply(U, x[r], dims, -1.6, 0.2)) < 5e-14
