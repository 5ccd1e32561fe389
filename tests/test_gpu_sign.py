"""End-to-end parity of y = sgn(gamma5 D_w(mu)) x (Secs. 2-3) through the C-ABI.

FP64 and double-float runs must match the oracle to 1e-10 at identical (k, l); the
FP32 run within its stated bound. The oracle sees the operator the GPU run sees
(float runs use links rounded once to float). Parity at fixed (k, l) is asserted
with l large enough for the inner level to converge: below that the nested vector
depends on roundoff (see test_gpu_inner.test_inner_sign_unconverged_is_valid)."""
import numpy as np
import pytest

import ovinputs as oi
from gpu_util import links_for, oracle_sign, rel
from oracle import dirac, exact, krylov

pytestmark = pytest.mark.gpu

PARITY = {"fp64": 1e-10, "df64": 1e-10}


@pytest.fixture(scope="module")
def ov():
    import paper_0910_2918_gb300 as ov

    return ov


def gpu_sign(ov, dims, U, m_w, mu, x, prec="fp64", tol=1e-10, k_max=400, l=60, apply=False, **opts):
    xs = np.ascontiguousarray(np.atleast_2d(x))
    y = np.zeros_like(xs)
    with ov.Overlap(dims, U, m_w, mu, prec, opts=ov.make_opts(**opts)) as op:
        rc, info = (op.apply if apply else op.sign_apply)(xs, y, tol, k_max, l)
    return rc, y, info


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("mu,l", [(0.0, 80), (0.3, 110)])
@pytest.mark.parametrize("recomb", [0, 1])
def test_fixed_k_parity(ov, prec, mu, l, recomb):
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "haar", 0)
    x = oi.gaussian_source(dims, 1)
    k = 150
    rc, y, info = gpu_sign(ov, dims, U, -1.5, mu, x, prec, k_max=k, l=l, k_fixed=k, recombination=recomb)
    yo, io = oracle_sign(links_for(prec, U), dims, -1.5, mu, x, k_max=k, l=l, tol=0, k_fixed=k)
    assert info[0]["k"] == k and info[0]["l"] == io["l"]
    assert rel(y[0], yo) < PARITY[prec]


def test_c1_hermitian_stopping_rule_vs_oracle_and_exact(ov, haar44):
    """4^4 Haar, mu = 0, FP64, k <= 400, l = 64, tol 1e-10 (checked vs diagonalisation)."""
    d = haar44
    rc, y, info = gpu_sign(ov, d["dims"], d["U"], -1.5, 0.0, d["x"], "fp64", 1e-10, 400, 64)
    yo, io = oracle_sign(d["U"], d["dims"], -1.5, 0.0, d["x"], k_max=400, l=64, tol=1e-10)
    assert rc == 0 and info[0]["status"] == 0
    assert info[0]["k"] == io["k"]
    assert rel(y[0], yo) < 1e-10
    assert rel(y[0], d[0.0]["S"] @ d["x"]) < 2e-10
    assert info[0]["err_est"] == pytest.approx(io["err_est"], rel=1e-3)


def test_two_sided_stopping_rule_small_lattice(ov):
    """The stop is a threshold decision on an estimate that carries roundoff, so the
    two sides may stop one check apart when the estimate sits at tol; the answers are
    then compared with the exact one instead of with each other."""
    dims = (2, 2, 2, 4)
    U = oi.gauge_field(dims, "haar", 0)
    x = oi.gaussian_source(dims, 1)
    rc, y, info = gpu_sign(ov, dims, U, -1.5, 0.3, x, "fp64", 1e-10, 400, 100)
    yo, io = oracle_sign(U, dims, -1.5, 0.3, x, k_max=400, l=100, tol=1e-10)
    yex, _ = exact.sign_spectral_apply(dirac.dense_A(U, dims, -1.5, 0.3), x, False)
    assert info[0]["status"] == 0 and abs(info[0]["k"] - io["k"]) <= 10
    if info[0]["k"] == io["k"]:
        assert rel(y[0], yo) < 1e-10
    assert rel(y[0], yex) < 1e-9 and rel(yo, yex) < 1e-9


def test_c2_two_sided_8444_fixed_k(ov):
    """8^4 near-unit (eps 0.4), mu = 0.3, m_w = -1.5, FP64, two-sided Lanczos."""
    dims = (8, 8, 8, 8)
    U = oi.gauge_field(dims, "near_unit", 0, eps=0.4)
    x = oi.gaussian_source(dims, 1)
    k, l = 120, 100
    rc, y, info = gpu_sign(ov, dims, U, -1.5, 0.3, x, "fp64", k_max=k, l=l, k_fixed=k)
    yo, io = oracle_sign(U, dims, -1.5, 0.3, x, k_max=k, l=l, tol=0, k_fixed=k)
    assert rel(y[0], yo) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_c2_two_sided_stopping_rule_8444(ov, prec):
    """The 8^4 workload whole: near-unit links exp(i 0.4 H), mu = 0.3, m_w = -1.5, one
    Gaussian source, tol 1e-10, k <= 800, l = 100, a check every 10 steps, against the
    oracle's own stopping run (it stops at k = 310). The stop is a threshold decision on
    an estimate carrying roundoff, so the two may stop one check apart (the estimate at
    k = 300 sits at 1e-10 while the answer there is 3.8e-10 from the one at k = 310);
    the GPU answer is then compared with the oracle run to the GPU's own k. The two-sided
    process at k = 310 amplifies differences of arithmetic: a 1e-15 relative change of x
    moves the oracle's own k = 310 answer by 1e-11, so the double-float run (2^-48 a
    rounding against FP64's 2^-53) agrees with the FP64 oracle to a few 1e-10 there (the
    inner level at this k is not sensitive: a 1e-14 change of H_k moves c by 1e-13)."""
    dims = (8, 8, 8, 8)
    U = oi.gauge_field(dims, "near_unit", 0, eps=0.4)
    x = oi.gaussian_source(dims, 1)
    rc, y, info = gpu_sign(ov, dims, U, -1.5, 0.3, x, prec, 1e-10, 800, 100, check_interval=10)
    yo, io = oracle_sign(U, dims, -1.5, 0.3, x, k_max=800, l=100, tol=1e-10, check_interval=10)
    assert rc == 0 and info[0]["status"] == 0 and io["status"] == 0
    assert abs(info[0]["k"] - io["k"]) <= 10
    if info[0]["k"] != io["k"]:
        yo, io = oracle_sign(U, dims, -1.5, 0.3, x, k_max=800, l=100, tol=0, k_fixed=info[0]["k"])
    bar = 1e-10 if prec == "fp64" else 3e-10
    assert rel(y[0], yo) < bar, (info[0]["k"], io["k"], rel(y[0], yo))


def test_free_field_closed_form(ov):
    dims = (4, 4, 4, 8)
    U = oi.gauge_field(dims, "unit", 0)
    x = oi.gaussian_source(dims, 1)
    yex = exact.free_sign_apply(x, dims, -1.5, 0.5)
    for prec in ("fp64", "df64"):
        rc, y, info = gpu_sign(ov, dims, U, -1.5, 0.5, x, prec, 1e-10, 400, 120)
        assert info[0]["status"] == 0
        assert rel(y[0], yex) < 2e-9


def test_mixed_precision_bound(ov):
    """FP32 vectors and links, double coefficients: error vs the FP64 oracle <= 1e-6."""
    dims = (8, 8, 8, 8)
    U = oi.gauge_field(dims, "near_unit", 0, eps=0.3)
    x = oi.point_source(dims, 0, 1, 2)
    rc, y, info = gpu_sign(ov, dims, U, -1.6, 0.2, x, "fp32", 1e-7, 600, 100)
    assert info[0]["status"] == 0
    yo, io = oracle_sign(oi.round_links_fp32(U), dims, -1.6, 0.2, x, k_max=600, l=100, tol=1e-9,
                         check_interval=20)
    assert rel(y[0], yo) < 1e-6


def test_batch_equals_single_and_apply(ov):
    """Same block size on both sides: the batched right-hand sides reproduce single runs
    bitwise (reductions are per right-hand side)."""
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "near_unit", 2, eps=0.4)
    X = oi.point_sources_12(dims, site=5)
    rc, Y, infos = gpu_sign(ov, dims, U, -1.5, 0.2, X, "df64", 1e-10, 400, 100, block_size=128)
    assert rc == 0 and len(infos) == 12
    for r in (0, 7, 11):
        rc1, y1, i1 = gpu_sign(ov, dims, U, -1.5, 0.2, X[r], "df64", 1e-10, 400, 100, block_size=128)
        assert i1[0]["k"] == infos[r]["k"]
        assert np.array_equal(Y[r], y1[0])
    rc, D, _ = gpu_sign(ov, dims, U, -1.5, 0.2, X[:3], "df64", 1e-10, 400, 100, apply=True, block_size=128)
    g5 = lambda v: dirac.gamma5_apply(v, dims)
    for r in range(3):
        assert rel(D[r], X[r] + g5(Y[r])) < 1e-13


def test_device_buffers_match_host_buffers(ov):
    import torch

    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "haar", 0)
    x = oi.gaussian_source(dims, 1).reshape(1, -1)
    rc, yh, _ = gpu_sign(ov, dims, U, -1.5, 0.0, x, "fp64", 1e-10, 400, 64)
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros_like(xd)
    with ov.Overlap(dims, U, -1.5, 0.0, "fp64") as op:
        op.sign_apply(xd, yd, 1e-10, 400, 64)
    assert np.array_equal(yd.cpu().numpy(), yh)


def test_bitwise_reproducible(ov):
    """Fixed-order reductions: the same block size gives bitwise equal results, and a
    handle reuses its autotuned block size, so repeated calls on it are bitwise equal."""
    dims = (6, 4, 4, 6)
    U = oi.gauge_field(dims, "near_unit", 3, eps=0.4)
    x = oi.gaussian_source(dims, 4)
    r1 = gpu_sign(ov, dims, U, -1.5, 0.25, x, "df64", 1e-9, 400, 80, block_size=128)
    r2 = gpu_sign(ov, dims, U, -1.5, 0.25, x, "df64", 1e-9, 400, 80, block_size=128)
    assert np.array_equal(r1[1], r2[1])
    xs = x.reshape(1, -1).copy()
    with ov.Overlap(dims, U, -1.5, 0.25, "df64") as op:
        ya, yb = np.zeros_like(xs), np.zeros_like(xs)
        op.sign_apply(xs, ya, 1e-9, 400, 80)
        op.sign_apply(xs, yb, 1e-9, 400, 80)
    assert np.array_equal(ya, yb)


# ---- edge cases -------------------------------------------------------------

def test_zero_source(ov):
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "haar", 0)
    x = np.zeros((2, 12 * 256), complex)
    x[1] = oi.gaussian_source(dims, 1)
    rc, y, info = gpu_sign(ov, dims, U, -1.5, 0.0, x, "fp64", 1e-8, 400, 60)
    assert np.all(y[0] == 0)
    assert np.all(np.isfinite(y[1])) and np.linalg.norm(y[1]) > 0.5


def test_eigenvector_source_is_exact_after_one_step(ov):
    dims = (2, 2, 2, 2)
    U = oi.gauge_field(dims, "haar", 0)
    A = dirac.dense_A(U, dims, -1.5, 0.0)
    lam, V = np.linalg.eigh(A)
    x = V[:, 5]
    rc, y, info = gpu_sign(ov, dims, U, -1.5, 0.0, x, "fp64", 1e-10, 50, 10)
    assert info[0]["k"] == 1 and info[0]["status"] == 0
    assert rel(y[0], np.sign(lam[5]) * x) < 1e-12


def test_ragged_volume_and_tiny_k(ov):
    dims = (3, 5, 2, 7)  # V = 210, not a multiple of the block size
    U = oi.gauge_field(dims, "near_unit", 1, eps=0.3)
    x = oi.gaussian_source(dims, 2)
    rc, y, info = gpu_sign(ov, dims, U, -1.5, 0.1, x, "fp64", 1e-10, 7, 20)  # k_max < check interval
    yo, io = oracle_sign(U, dims, -1.5, 0.1, x, k_max=7, l=20, tol=1e-10)
    assert info[0]["k"] == 7 == io["k"] and rc == 1
    assert rel(y[0], yo) < 1e-10


def test_argument_errors(ov):
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "unit", 0)
    x = oi.gaussian_source(dims, 1).reshape(1, -1)
    y = np.zeros_like(x)
    with ov.Overlap(dims, U, -1.5, 0.0) as op:
        with pytest.raises(ov.OvError) as e:
            op.sign_apply(x, y, 1e-8, 100, 121)
        assert e.value.code == -7
        with pytest.raises(ov.OvError) as e:
            op.sign_apply(x, y, 1e-8, 2000, 60)
        assert e.value.code == -7
        with pytest.raises(ov.OvError):
            op.sign_apply(x, y, 1e-8, 100, 0)


def test_not_converged_warning_with_small_l(ov):
    """The inner estimate flags an inner dimension that is too small (status 1)."""
    dims = (4, 4, 4, 8)
    U = oi.gauge_field(dims, "unit", 0)
    x = oi.gaussian_source(dims, 1)
    rc, y, info = gpu_sign(ov, dims, U, -1.5, 0.5, x, "fp64", 1e-10, 400, 50)
    yo, io = oracle_sign(U, dims, -1.5, 0.5, x, k_max=400, l=50, tol=1e-10)
    assert rc == 1 and info[0]["status"] == 1 == io["status"]
    assert info[0]["k"] == io["k"]
    assert rel(y[0], yo) < 1e-10


def test_adaptive_schedule_fewer_checks_same_answer(ov):
    """The adaptive check schedule (next check where the outer estimate's log-linear
    decay reaches tol) stops at k >= the fixed schedule's k with fewer checks."""
    dims = (6, 6, 6, 6)
    U = oi.gauge_field(dims, "near_unit", 0, eps=0.3)
    x = oi.gaussian_source(dims, 1)
    res = {}
    for sched in (0, 1):
        xs = x.reshape(1, -1).copy()
        y = np.zeros_like(xs)
        with ov.Overlap(dims, U, -1.6, 0.2, "fp64", opts=ov.make_opts(check_schedule=sched, check_interval=10)) as op:
            rc, info = op.sign_apply(xs, y, 1e-9, 600, 90)
            res[sched] = (y[0], info[0], op.stats())
    (y0, i0, s0), (y1, i1, s1) = res[0], res[1]
    assert i0["status"] == 0 and i1["status"] == 0
    assert s1["checks"] < s0["checks"]
    assert i1["k"] >= i0["k"]
    assert rel(y1, y0) < 5e-9


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_overlapped_checks_equal_serial_order(ov, mu):
    """Checks overlapped with speculative outer steps give the serial result bitwise: same
    stop, same estimates, same vector (the speculative steps only add coefficients and basis
    vectors beyond the check's k)."""
    dims = (8, 8, 8, 8)
    U = oi.gauge_field(dims, "near_unit", 0, eps=0.4)
    X = oi.point_sources_12(dims, site=9)[:4]
    out = []
    for ovl in (0, 1):
        rc, y, info = gpu_sign(ov, dims, U, -1.5, mu, X, "df64", 1e-10, 800, 100, check_interval=25,
                               first_check=100, block_size=128, overlap_checks=ovl)
        out.append((y, info))
    (y0, i0), (y1, i1) = out
    assert [i["k"] for i in i0] == [i["k"] for i in i1]
    assert [i["err_est"] for i in i0] == [i["err_est"] for i in i1]
    assert [i["status"] for i in i1] == [0] * 4
    assert np.array_equal(y0, y1)


def test_final_check_runs_when_speculative_steps_reach_k_max(ov):
    """A check 5 steps before k_max lets speculative steps (run while the check is
    evaluated) reach k_max; the step at k_max must still be checked and the result
    recombined there: k = k_max, status OV_NOT_CONVERGED at an unreachable tol, and y
    equal to the oracle at the same fixed k (it once came back empty with k = 0)."""
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "near_unit", 2, eps=0.4)
    x = oi.gaussian_source(dims, 3)
    k_max, l = 80, 80  # l_eff = k: the inner level is exact, parity holds at any k
    for mu in (0.0, 0.3):
        rc, y, info = gpu_sign(ov, dims, U, -1.5, mu, x, "fp64", 1e-14, k_max, l, check_interval=25,
                               first_check=k_max - 5, overlap_checks=1)
        assert info[0]["k"] == k_max and rc == 1 and info[0]["status"] == 1
        yo, io = oracle_sign(U, dims, -1.5, mu, x, k_max=k_max, l=l, tol=0, k_fixed=k_max)
        assert rel(y[0], yo) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_serious_breakdown_returns_the_error(ov, prec):
    """A serious breakdown of two-sided Lanczos (|w~^dag v~| <= breakdown_tol ||v~|| ||w~||),
    forced from the host with a huge threshold: the call returns OV_ERR_BREAKDOWN at the
    first check (no hang, the handle stays usable), as the oracle reports it at step 1."""
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "near_unit", 2, eps=0.4)
    x = oi.gaussian_source(dims, 3)
    with ov.Overlap(dims, U, -1.5, 0.3, prec, opts=ov.make_opts(breakdown_tol=1e6)) as op:
        y = np.zeros((1, x.size), dtype=np.complex128)
        with pytest.raises(ov.OvError) as e:
            op.sign_apply(x.reshape(1, -1).copy(), y, 1e-10, 200, 60)
        assert e.value.code == ov.binding.OV_ERR_BREAKDOWN
        # the same handle still works with the default threshold
        op.set_opts(breakdown_tol=1e-14, k_fixed=40)
        rc, info = op.sign_apply(x.reshape(1, -1).copy(), y, 1e-10, 40, 40)
        assert rc == 0 and info[0]["k"] == 40
    fA, fAH = (lambda v: dirac.A_apply(U, v, dims, -1.5, 0.3)), (lambda v: dirac.AH_apply(U, v, dims, -1.5, 0.3))
    out = krylov.Outer(fA, fAH, x, False, breakdown_tol=1e6)
    out.step()
    assert out.status == krylov.ERR_BREAKDOWN


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_auto_recombination_falls_back_to_the_double_pass(ov, monkeypatch, mu):
    """OV_RECOMB_AUTO stores the basis while device memory lasts; when a basis allocation
    fails mid-run (here: a cap of one 64-step chunk, injected through OV_BASIS_CAP_BYTES)
    the run continues in the double pass and the answer equals the stored one."""
    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "near_unit", 4, eps=0.4)
    x = oi.gaussian_source(dims, 5).reshape(1, -1)
    k = 150
    pool = 12 * 256 * 16  # one FP64 vector of the 4^4 lattice, bytes
    ys, stats = {}, {}
    for mode, cap in (("stored", None), ("auto_capped", 64 * pool + 1)):
        if cap is None:
            monkeypatch.delenv("OV_BASIS_CAP_BYTES", raising=False)
        else:
            monkeypatch.setenv("OV_BASIS_CAP_BYTES", str(cap))
        recomb = 0 if mode == "stored" else 2
        y = np.zeros_like(x)
        with ov.Overlap(dims, U, -1.5, mu, "fp64", opts=ov.make_opts(k_fixed=k, recombination=recomb)) as op:
            rc, info = op.sign_apply(x, y, 0.0, k, 100)
            stats[mode] = op.stats()
        assert rc == 0 and info[0]["k"] == k
        ys[mode] = y
    monkeypatch.delenv("OV_BASIS_CAP_BYTES", raising=False)
    assert stats["stored"]["regen_steps"] == 0 and stats["auto_capped"]["regen_steps"] == k
    assert rel(ys["auto_capped"][0], ys["stored"][0]) < 1e-12
