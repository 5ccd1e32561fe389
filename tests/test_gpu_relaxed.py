"""Relaxed double-float steps (opts.relax): the late outer steps run their hopping sum in
float arithmetic while vectors, recurrence, dot products and coefficients stay
double-float. Not part of the paper's method (inexact Krylov relaxation of the matvec
accuracy), so it is judged against converged answers: the free-field closed form and
strict double-float runs that the parity tests tie to the oracle."""
import numpy as np
import pytest

import ovinputs as oi
from gpu_util import rel
from oracle import exact

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ov():
    import paper_0910_2918_gb300 as ov

    return ov


def run(ov, dims, U, m_w, mu, x, tol, k_max, l, prec="df64", **opts):
    xs = np.ascontiguousarray(np.atleast_2d(x))
    y = np.zeros_like(xs)
    with ov.Overlap(dims, U, m_w, mu, prec, opts=ov.make_opts(**opts)) as op:
        rc, info = op.sign_apply(xs, y, tol, k_max, l)
        st = op.stats()
    return rc, y, info, st


def test_relaxed_free_field_closed_form(ov):
    dims = (4, 4, 4, 8)
    U = oi.gauge_field(dims, "unit", 0)
    x = oi.gaussian_source(dims, 1)
    yex = exact.free_sign_apply(x, dims, -1.5, 0.5)
    rc, ys, infos, sts = run(ov, dims, U, -1.5, 0.5, x, 1e-10, 400, 120, check_interval=25, block_size=128)
    assert infos[0]["status"] == 0 and rel(ys[0], yex) < 2e-9
    # k_ref = the strict run's k (first_check), float hopping from half of it
    k = infos[0]["k"]
    rc, y, info, st = run(ov, dims, U, -1.5, 0.5, x, 1e-10, 400, 120, check_interval=25, first_check=k, relax=0.5)
    assert info[0]["status"] == 0
    assert 0 < st["relaxed_steps"] < st["outer_steps"]
    assert rel(y[0], yex) < 1e-8
    # no reference step: relaxation stays off (same block size: bitwise the strict run)
    rc, y0, info0, st0 = run(ov, dims, U, -1.5, 0.5, x, 1e-10, 400, 120, check_interval=25, relax=0.5,
                             block_size=128)
    assert st0["relaxed_steps"] == 0 and np.array_equal(y0, ys)


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_relaxed_matches_strict_converged(ov, mu):
    """8^4 near-unit links: the relaxed run stopped at 1e-10 is within 1e-8 of the strict
    double-float run (Lanczos at mu = 0, two-sided at mu != 0)."""
    dims = (8, 8, 8, 8)
    U = oi.gauge_field(dims, "near_unit", 0, eps=0.4)
    x = oi.gaussian_source(dims, 1)
    rc, ys, infos, sts = run(ov, dims, U, -1.5, mu, x, 1e-10, 800, 100, check_interval=25, first_check=100)
    k = infos[0]["k"]
    rc, yr, infor, str_ = run(ov, dims, U, -1.5, mu, x, 1e-10, 800, 100, check_interval=25, first_check=k,
                              relax=0.5)
    assert infos[0]["status"] == 0 and infor[0]["status"] == 0
    assert sts["relaxed_steps"] == 0 and str_["relaxed_steps"] > 0
    assert rel(yr[0], ys[0]) < 1e-8


def test_relaxed_two_pass_and_stored_agree_at_convergence(ov):
    """Both recombination modes switch to float hopping at the same step; at a converged k
    both are within 1e-8 of the strict run. (Float hopping on the high words turns
    roundoff-level differences of the vectors into ~1e-7 differences of late matvecs, so
    the two modes agree to the relaxation error, not to roundoff.)"""
    dims = (4, 4, 4, 8)
    U = oi.gauge_field(dims, "near_unit", 3, eps=0.4)
    x = oi.gaussian_source(dims, 4)
    rc, ys, infos, sts = run(ov, dims, U, -1.5, 0.3, x, 1e-10, 600, 100, check_interval=25, block_size=128)
    k = infos[0]["k"]
    out = []
    for recomb in (0, 1):
        rc, y, info, st = run(ov, dims, U, -1.5, 0.3, x, 1e-10, 600, 100, check_interval=25, first_check=k,
                              relax=0.5, recombination=recomb, block_size=128)
        assert info[0]["status"] == 0 and st["relaxed_steps"] > 0
        assert rel(y[0], ys[0]) < 1e-8
        out.append(y[0])
    assert rel(out[1], out[0]) < 1e-8


def test_relax_only_affects_double_float_handles(ov):
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "near_unit", 1, eps=0.4)
    x = oi.gaussian_source(dims, 2)
    for prec in ("fp64", "fp32"):
        rc, y, info, st = run(ov, dims, U, -1.5, 0.2, x, 1e-6, 200, 40, prec=prec, relax=0.5)
        assert st["relaxed_steps"] == 0
    with pytest.raises(ov.OvError):
        run(ov, dims, U, -1.5, 0.2, x, 1e-6, 200, 40, relax=1.5)
