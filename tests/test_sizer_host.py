"""Host-side parts of the learned sizing (no GPU): the features read from the outer
coefficients, and the folding of feature and target scaling into the network's first and
last layers, checked against the oracle MLP."""
import numpy as np

from oracle import mlp


def test_fold_scaling_equals_normalise_evaluate_denormalise():
    from paper_0910_2918_gb300 import sizer

    rng = np.random.default_rng(3)
    theta = mlp.init_params(5).astype(np.float64)
    F = rng.standard_normal((40, 16)) * rng.uniform(0.1, 3.0, 16) + rng.uniform(-1, 1, 16)
    fm, fs = F.mean(0), F.std(0) + 1e-12
    tm, ts = np.array([5.6, 4.1]), np.array([0.4, 0.3])
    y_norm, _ = mlp.forward(theta, (F - fm) / fs)
    expect = y_norm * ts + tm
    folded = sizer.fold_scaling(theta, fm, fs, tm, ts)
    assert folded.dtype == np.float32 and folded.size == mlp.N_PARAMS
    got, _ = mlp.forward(folded.astype(np.float64), F)
    assert np.allclose(got, expect, rtol=1e-5, atol=1e-4)


def test_features_from_raw_coefficients():
    from paper_0910_2918_gb300 import sizer

    rng = np.random.default_rng(4)
    alpha = rng.standard_normal(16) + 1j * rng.standard_normal(16)
    beta = np.concatenate([[0.0], rng.uniform(0.1, 1.0, 16)]).astype(complex)
    gamma = np.concatenate([[0.0], rng.standard_normal(16) + 1j * rng.standard_normal(16)])
    raw = np.concatenate([alpha[:16], beta[1:17], gamma[1:17]])[None, :]
    f_raw = sizer.features_from_raw(raw)[0]
    f = sizer.features(alpha, beta)
    assert f.shape == (16,)
    assert np.array_equal(f_raw, f)
    assert np.array_equal(f[:6], alpha[:6].real) and np.array_equal(f[6:12], alpha[:6].imag)
    assert np.array_equal(f[12:], beta[1:5].real)


def test_committed_network_on_held_out_records():
    """The committed network on the held-out convergence records (records 2000 on; the
    network was trained on the first 2000): k* and l* predicted within the accuracy the
    training reported (median |log(k_pred / k*)| ~ 0.14)."""
    import os

    from paper_0910_2918_gb300 import sizer

    theta = sizer.load(sizer.DEFAULT_PARAMS)
    assert theta.dtype == np.float32 and theta.size == mlp.N_PARAMS and np.all(np.isfinite(theta))
    d = np.load(os.path.join(os.path.dirname(sizer.__file__), "data", "sizer_records.npz"))
    held = np.arange(len(d["k"])) >= 2000
    m = held & d["conv"].astype(bool)
    assert m.sum() >= 100
    y, _ = mlp.forward(theta.astype(np.float64), sizer.features_from_raw(d["raw"])[m])
    ek = np.abs(y[:, 0] - np.log(d["k"][m]))
    el = np.abs(y[:, 1] - np.log(d["l"][m]))
    assert np.median(ek) < 0.25 and np.quantile(ek, 0.9) < 0.6
    assert np.median(el) < 0.25


def test_rough_network_on_its_held_out_records():
    """The parameters trained with rough fields, on the held-out part of the records they
    were trained beside (the last 15% of the rough and large sets, records 2000 on of the
    near-unit set at k <= 1000): k* within a median |log(k_pred / k*)| of 0.25, also on
    the Haar lattices, where the near-unit parameters were never trained."""
    import os

    from paper_0910_2918_gb300 import sizer

    theta = sizer.load(sizer.ROUGH_PARAMS)
    assert theta.dtype == np.float32 and theta.size == mlp.N_PARAMS and np.all(np.isfinite(theta))
    base = os.path.join(os.path.dirname(sizer.__file__), "data")
    for name, cut in (("sizer_records_nu_k1000.npz", 2000), ("sizer_records_rough.npz", None),
                      ("sizer_records_large.npz", None)):
        d = np.load(os.path.join(base, name))
        n = len(d["k"])
        held = np.arange(n) >= (cut if cut is not None else int(0.85 * n))
        m = held & d["conv"].astype(bool)
        assert m.sum() >= 10
        y, _ = mlp.forward(theta.astype(np.float64), sizer.features_from_raw(d["raw"])[m])
        ek = np.abs(y[:, 0] - np.log(d["k"][m]))
        assert np.median(ek) < 0.25, (name, np.median(ek))


def test_feature_sets_of_the_ablation():
    """Each feature set of the comparison has 16 entries (the network's input), drawn from
    the first 16 outer coefficients as named."""
    from paper_0910_2918_gb300 import sizer

    rng = np.random.default_rng(5)
    alpha = rng.standard_normal(16) + 1j * rng.standard_normal(16)
    beta = np.concatenate([[0.0], rng.uniform(0.1, 1.0, 16)]).astype(complex)
    raw = np.concatenate([alpha, beta[1:17], np.zeros(16)])[None, :]
    for fs in sizer.FEATURE_SETS:
        assert sizer.features_from_raw(raw, fs).shape == (1, 16)
    f = sizer.features_from_raw(raw, "a8b8")[0]
    assert np.array_equal(f[:8], alpha[:8].real) and np.array_equal(f[8:], beta[1:9].real)
    f = sizer.features_from_raw(raw, "a4i4b8")[0]
    assert np.array_equal(f[4:8], alpha[:4].imag) and np.array_equal(f[8:], beta[1:9].real)
