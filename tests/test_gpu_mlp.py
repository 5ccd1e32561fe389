"""Learned sizing on the GPU: forward and gradient kernels against the oracle MLP,
training, and the a-posteriori guard around the prediction."""
import numpy as np
import pytest

import ovinputs as oi
from gpu_util import rel
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ov():
    import paper_0910_2918_gb300 as ov

    return ov


def test_forward_matches_oracle(ov):
    rng = np.random.default_rng(0)
    theta = omlp.init_params(3).astype(np.float32)
    X = rng.standard_normal((257, 16)).astype(np.float32)
    y = ov.ov_mlp_forward(theta, X)
    yref, _ = omlp.forward(theta.astype(np.float64), X.astype(np.float64))
    assert np.abs(y - yref).max() <= 1e-4 * max(1.0, np.abs(yref).max())


def test_gradient_matches_oracle(ov):
    rng = np.random.default_rng(1)
    theta = (omlp.init_params(4) * 0.5).astype(np.float32)
    X = rng.standard_normal((300, 16)).astype(np.float32)
    Y = rng.standard_normal((300, 2)).astype(np.float32)
    loss, g = ov.ov_mlp_loss_grad(theta, X, Y)
    lref, gref = omlp.loss_grad(theta.astype(np.float64), X.astype(np.float64), Y.astype(np.float64))
    assert abs(loss - lref) <= 1e-5 * abs(lref)
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)


def test_training_fits_a_smooth_map(ov):
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (1024, 16)).astype(np.float32)
    Y = np.stack([np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2], np.cos(X[:, 3]) - X[:, 4] ** 2], 1).astype(np.float32)
    theta0 = omlp.init_params(5).astype(np.float32)
    l0 = ov.ov_mlp_loss_grad(theta0, X, Y)[0]
    theta, hist = ov.ov_mlp_train(theta0, X, Y, epochs=300, batch=128, lr=3e-3, seed=7)
    assert hist[-1] < 0.05 * l0
    # the returned parameters reproduce the reported loss
    assert ov.ov_mlp_loss_grad(theta, X, Y)[0] == pytest.approx(float(hist[-1]), rel=1e-4)
    # deterministic given the seed
    theta2, hist2 = ov.ov_mlp_train(theta0, X, Y, epochs=300, batch=128, lr=3e-3, seed=7)
    assert np.array_equal(theta, theta2)


def test_adam_training_matches_oracle_steps(ov):
    """Three full-batch epochs of the GPU training loop (forward, backward and Adam
    kernels, beta 0.9 / 0.999, eps 1e-8) from a fixed theta equal three oracle steps
    (loss_grad, then adam_step with t = 1, 2, 3) element by element. At t = 1 Adam moves
    every parameter by about lr; at t = 2, 3 the bias corrections and both moments shape
    the step, so a wrong beta or correction moves theta by O(lr) = 1e-2, far above the
    bound. The bound, 1e-6 absolute plus 1e-5 relative, is ~15x the float-vs-double
    difference of the same three steps computed in numpy float32 (7e-8)."""
    rng = np.random.default_rng(5)
    theta0 = (omlp.init_params(3) * 0.5).astype(np.float32)
    X = rng.standard_normal((96, 16)).astype(np.float32)
    Y = rng.standard_normal((96, 2)).astype(np.float32)
    lr = 1e-2
    theta, hist = ov.ov_mlp_train(theta0, X, Y, epochs=3, batch=0, lr=lr, seed=1)
    th = theta0.astype(np.float64)
    m, v = np.zeros_like(th), np.zeros_like(th)
    for t in (1, 2, 3):
        _, g = omlp.loss_grad(th, X.astype(np.float64), Y.astype(np.float64))
        th, m, v = omlp.adam_step(th, g, m, v, t, lr)
    d = np.abs(theta.astype(np.float64) - th)
    assert np.all(d <= 1e-6 + 1e-5 * np.abs(th)), (float(d.max()), int(np.argmax(d)))
    # every parameter with a nonzero gradient moved by about lr at t = 1
    assert np.abs(th - theta0).max() > 2 * lr
    # the reported loss is the loss of the returned parameters
    assert omlp.loss(theta.astype(np.float64), X.astype(np.float64), Y.astype(np.float64)) == pytest.approx(
        float(hist[-1]), rel=1e-4)


def _constant_predictor(k_pred, l_pred):
    """Zero weights with biases (log k, log l): predicts the same (k, l) for every input."""
    th = np.zeros(5378, dtype=np.float32)
    th[5376] = np.log(k_pred)
    th[5377] = np.log(l_pred)
    return th


@pytest.mark.parametrize("k_pred,l_pred", [(40.0, 8.0), (330.0, 100.0)])
def test_guard_keeps_the_answer_when_the_prediction_is_wrong(ov, k_pred, l_pred):
    """A short k or a small l must not change the answer: checks continue past a short
    prediction and l grows until the inner estimate meets tol."""
    dims = (6, 6, 6, 6)
    U = oi.gauge_field(dims, "near_unit", 0, eps=0.3)
    x = oi.gaussian_source(dims, 1).reshape(1, -1)
    y0 = np.zeros_like(x)
    with ov.Overlap(dims, U, -1.6, 0.2, "fp64", opts=ov.make_opts(check_interval=10)) as op:
        rc0, i0 = op.sign_apply(x, y0, 1e-9, 800, 120)
    y1 = np.zeros_like(x)
    with ov.Overlap(dims, U, -1.6, 0.2, "fp64", opts=ov.make_opts(check_interval=10)) as op:
        op.set_sizer(_constant_predictor(k_pred, l_pred), 8, 120)
        rc1, i1 = op.sign_apply(x, y1, 1e-9, 800, 120)
    assert rc0 == 0 and rc1 == 0
    assert i1[0]["err_est"] <= 1e-9
    assert rel(y1[0], y0[0]) < 5e-9


def test_coefficients_readback(ov):
    from oracle import dirac, krylov

    dims = (4, 4, 4, 4)
    U = oi.gauge_field(dims, "haar", 0)
    x = oi.gaussian_source(dims, 1)
    with ov.Overlap(dims, U, -1.5, 0.3, "fp64", opts=ov.make_opts(k_fixed=20)) as op:
        y = np.zeros((1, x.size), complex)
        op.sign_apply(x.reshape(1, -1).copy(), y, 0, 20, 20)
        a, b, g = op.coefficients(0, 20)
    o = krylov.Outer(lambda v: dirac.A_apply(U, v, dims, -1.5, 0.3), lambda v: dirac.AH_apply(U, v, dims, -1.5, 0.3),
                     x, False)
    for _ in range(20):
        o.step()
    assert np.allclose(a, o.alpha, atol=1e-12)
    assert np.allclose(b, o.beta[:20], atol=1e-12)
    assert np.allclose(g, o.gamma[:20], atol=1e-12)


def test_trained_sizer_gain_on_held_out_problems(ov):
    """The trained network (committed parameters, records from the method itself) against
    the method without it, on held-out problems of the training family: the same
    tolerance is met with far fewer stopping checks and less time."""
    import time

    from paper_0910_2918_gb300 import sizer

    theta = sizer.load(sizer.DEFAULT_PARAMS)
    probs = oi.training_problems(2004)[2000:]
    checks = {0: 0, 1: 0}
    secs = {0: 0.0, 1: 0.0}
    for p in probs:
        U = oi.gauge_field(p["dims"], p["kind"], p["gauge_seed"], eps=p["eps"])
        x = oi.problem_source(p).reshape(1, -1)
        ys = {}
        for sized in (0, 1):
            y = np.zeros_like(x)
            with ov.Overlap(p["dims"], U, p["m_w"], p["mu"], "df64", opts=ov.make_opts(check_interval=10)) as op:
                if sized:
                    op.set_sizer(theta, 8, 120)
                op.sign_apply(x, y, 1e-8, 1000, 120)  # warm-up (and autotune)
                op.reset_stats()
                t0 = time.perf_counter()
                rc, info = op.sign_apply(x, y, 1e-8, 1000, 120)
                secs[sized] += time.perf_counter() - t0
                checks[sized] += op.stats()["checks"]
            assert rc == 0 and info[0]["err_est"] <= 1e-8
            ys[sized] = y[0]
        # both meet the estimate; the estimate is not a bound, so the two answers agree to
        # a few times tol
        assert rel(ys[1], ys[0]) < 2e-7
    assert checks[1] * 3 <= checks[0]
    assert secs[1] < secs[0]


def test_learned_sizing_at_24c48_two_pass(ov):
    """Evaluation workload of the learned sizing: 24^3 x 48, mu = 0.1, near-unit links
    (eps 0.3), m_w = -1.6, one Gaussian source, double-float vectors, two-pass
    recombination, tol 1e-8. The sized run meets the tolerance with fewer checks than the
    unsized one, and both agree with the FP64 path."""
    import time

    import torch

    from paper_0910_2918_gb300 import sizer

    dims = (24, 24, 24, 48)
    U = oi.gauge_field(dims, "near_unit", 0, eps=0.3)
    x = torch.from_numpy(oi.gaussian_source(dims, 1).reshape(1, -1)).cuda()
    res = {}
    for sized in (0, 1):
        y = torch.zeros_like(x)
        opts = ov.make_opts(check_interval=10, recombination=1)
        with ov.Overlap(dims, torch.from_numpy(U).cuda(), -1.6, 0.1, "df64", opts=opts) as op:
            if sized:
                op.set_sizer(sizer.load(sizer.DEFAULT_PARAMS), 8, 120)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, info = op.sign_apply(x, y, 1e-8, 1000, 120)
            torch.cuda.synchronize()
            res[sized] = (y.clone(), info[0], op.stats(), time.perf_counter() - t0)
        assert rc == 0 and info[0]["err_est"] <= 1e-8
    yr = torch.zeros_like(x)
    with ov.Overlap(dims, torch.from_numpy(U).cuda(), -1.6, 0.1, "fp64",
                    opts=ov.make_opts(check_interval=20, check_schedule=1, recombination=1)) as op:
        op.sign_apply(x, yr, 1e-10, 1000, 120)
    for sized in (0, 1):
        err = float(torch.linalg.norm(res[sized][0] - yr) / torch.linalg.norm(yr))
        assert err < 1e-7, (sized, err)
    assert res[1][2]["checks"] < res[0][2]["checks"]
    assert res[1][3] < res[0][3]


def test_prediction_beyond_k_max_keeps_a_final_baseline(ov):
    """A predicted k* beyond k_max puts the first check one interval before k_max, so the
    check at k_max has a baseline estimate and converged runs report OK."""
    dims = (6, 6, 6, 6)
    U = oi.gauge_field(dims, "near_unit", 0, eps=0.3)
    x = oi.gaussian_source(dims, 1).reshape(1, -1)
    y = np.zeros_like(x)
    with ov.Overlap(dims, U, -1.6, 0.2, "fp64", opts=ov.make_opts(check_interval=10)) as op:
        op.set_sizer(_constant_predictor(5000.0, 80.0), 8, 120)
        rc, info = op.sign_apply(x, y, 1e-9, 600, 120)
        st = op.stats()
    assert rc == 0 and info[0]["status"] == 0 and info[0]["err_est"] <= 1e-9
    assert info[0]["k"] == 600 and st["checks"] >= 2
