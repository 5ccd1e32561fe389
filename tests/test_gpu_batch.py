"""A batch of lattices of uneven sizes in one launch per step (48 problems: 12 each of
4^4, 6^4, 6^3x12 and 8^4): every problem's answer equals its own single-lattice run and
the oracle."""
import numpy as np
import pytest

import ovinputs as oi
from gpu_util import links_for, oracle_sign, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ov():
    import paper_0910_2918_gb300 as ov

    return ov


def _problems(n):
    probs = oi.problem_batch_48()
    # keep the size mix with n problems: take every 48/n-th
    step = max(1, 48 // n)
    return probs[::step][:n]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_equals_single_runs(ov, prec):
    probs = _problems(8)
    Us = [oi.gauge_field(p["dims"], p["kind"], p["gauge_seed"], eps=p["eps"]) for p in probs]
    xs = [oi.gaussian_source(p["dims"], p["source_seed"]).reshape(1, -1) for p in probs]
    tol = 1e-10 if prec == "fp64" else 1e-6
    opts = ov.make_opts(check_interval=10, block_size=128)  # one reduction order on both sides
    hb = ov.ov_batch_create([p["dims"] for p in probs], Us, [p["m_w"] for p in probs], [p["mu"] for p in probs],
                            prec, opts=opts)
    try:
        ys = [np.zeros_like(x) for x in xs]
        rc, infos = ov.ov_batch_sign_apply(hb, xs, ys, tol, 1000, 100)
    finally:
        ov.ov_destroy(hb)
    for i, p in enumerate(probs):
        y1 = np.zeros_like(xs[i])
        with ov.Overlap(p["dims"], Us[i], p["m_w"], p["mu"], prec, opts=opts) as op:
            rc1, i1 = op.sign_apply(xs[i], y1, tol, 1000, 100)
        assert infos[i]["k"] == i1[0]["k"]
        assert np.array_equal(ys[i], y1), (i, rel(ys[i], y1))


def test_autotuned_block_size_changes_only_rounding(ov):
    """Block sizes 64, 128 and 256 change only the order of the reductions: the answers
    agree to rounding, and the tuner reports the size it chose."""
    dims = (6, 6, 6, 6)
    U = oi.gauge_field(dims, "near_unit", 3, eps=0.3)
    x = oi.gaussian_source(dims, 4).reshape(1, -1)
    ys = {}
    for bs in (64, 128, 256, 0):
        y = np.zeros_like(x)
        with ov.Overlap(dims, U, -1.5, 0.2, "df64", opts=ov.make_opts(k_fixed=120, block_size=bs)) as op:
            op.sign_apply(x, y, 0, 120, 110)
            ys[bs] = (y[0], op.stats()["block_size"])
    for bs in (64, 256, 0):
        assert rel(ys[bs][0], ys[128][0]) < 1e-11
    assert ys[0][1] in (64, 128, 256)


def test_batch_48_mixed_vs_oracle_sampled(ov):
    """The 48-problem workload (uneven lattices, Haar or near-unit links, mu in [0, 0.5])
    in float arithmetic: every problem converges (or reports it), and sampled problems
    agree with the FP64 oracle within the float bound."""
    probs = oi.problem_batch_48()
    Us = [oi.gauge_field(p["dims"], p["kind"], p["gauge_seed"], eps=p["eps"]) for p in probs]
    xs = [oi.gaussian_source(p["dims"], p["source_seed"]).reshape(1, -1) for p in probs]
    hb = ov.ov_batch_create([p["dims"] for p in probs], Us, [p["m_w"] for p in probs], [p["mu"] for p in probs],
                            "fp32", opts=ov.make_opts(check_interval=10))
    try:
        ys = [np.zeros_like(x) for x in xs]
        rc, infos = ov.ov_batch_sign_apply(hb, xs, ys, 1e-6, 1000, 100)
    finally:
        ov.ov_destroy(hb)
    assert all(i["status"] in (0, 1) for i in infos)
    assert sum(i["status"] == 0 for i in infos) >= 40
    for i in (1, 14, 27, 40):  # one of each lattice shape, near-unit links
        p = probs[i]
        if infos[i]["status"] != 0:
            continue
        yo, io = oracle_sign(links_for("fp32", Us[i]), p["dims"], p["m_w"], p["mu"], xs[i][0], k_max=1000,
                             l=100, tol=1e-9, check_interval=20)
        assert rel(ys[i][0], yo) < 1e-5


@pytest.mark.parametrize("mu", [0.0, 0.25])
def test_graph_replay_equals_plain_launches(ov, mu):
    """Runs of outer steps replayed from a captured CUDA graph (the kernels read the step
    index and their slots from device memory) give bitwise the same answer as one launch
    per kernel, for stored and two-pass recombination."""
    dims = (4, 6, 4, 6)
    U = oi.gauge_field(dims, "near_unit", 5, eps=0.35)
    x = np.stack([oi.gaussian_source(dims, 6), oi.gaussian_source(dims, 7)])
    out = {}
    for recomb in (0, 1):
        for g in (0, 8):
            y = np.zeros_like(x)
            opts = ov.make_opts(check_interval=10, graph_steps=g, block_size=128, recombination=recomb)
            with ov.Overlap(dims, U, -1.5, mu, "df64", opts=opts) as op:
                rc, info = op.sign_apply(x, y, 1e-10, 600, 100)
                st = op.stats()
            assert rc == 0
            out[(recomb, g)] = (y, st)
        assert np.array_equal(out[(recomb, 0)][0], out[(recomb, 8)][0])
        assert out[(recomb, 8)][1]["graph_launches"] > 0 and out[(recomb, 0)][1]["graph_launches"] == 0
    assert rel(out[(1, 8)][0], out[(0, 8)][0]) < 1e-12
