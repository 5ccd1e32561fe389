"""Learned sizing of the Krylov dimensions: data from the method itself, training on the GPU.

A convergence record of one problem is (features, k*, l*):
  features  f = (Re alpha_1..alpha_6, Im alpha_1..alpha_6, beta_2..beta_5), the first
            outer coefficients (Im alpha carries the chemical potential, Re alpha and beta
            the Wilson mass; the set was chosen on held-out records among several);
  k*        the outer dimension at which the stopping rule stops (checks every dk
            steps, outer estimate ||c_k - [c_{k-dk}; 0]|| / ||c_k|| <= tol, with an
            inner dimension large enough to be exact);
  l*        the smallest inner dimension (multiple of 8) whose inner estimate at k* is
            <= tol.
All of it is computed by libov: one apply with k fixed gives the coefficients
(ov_get_coefficients), one batched ov_inner_sign over every prefix H_k gives the
stopping point, and a binary search on l gives l*. The network (16 -> 64 -> 64 -> 2,
ov_mlp_*) is trained on (f, log k*, log l*) with the library's own kernels; feature
and target scaling are folded into the first and last layer, so the device sees raw
coefficients.

    python -m paper_0910_2918_gb300.sizer --records N --out data.npz   # generate
    python -m paper_0910_2918_gb300.sizer --train data.npz --out sizer.npz

The two parameter sets in the package were made by (data/ holds the records)
    --train data/sizer_records.npz --out sizer_params.npz
    --records 2200 --k-max 1000; --records 300 --rough --k-max 1000;
    --records 120 --large --k-max 1000 (the three record files), then
    --train data/sizer_records_nu_k1000.npz --also data/sizer_records_rough.npz
            data/sizer_records_large.npz --ablation --out sizer_params_rough.npz
"""
import argparse
import os
import time

import numpy as np

from . import binding as B

L_GRID = list(range(8, 121, 8))


def features(alpha, beta):
    """f = (Re alpha_1..alpha_6, Im alpha_1..alpha_6, beta_2..beta_5)."""
    return np.concatenate([np.real(alpha[:6]), np.imag(alpha[:6]), np.real(beta[1:5])]).astype(np.float64)


def _prefix_arrays(a, b, g, ks, ld):
    A = np.zeros((len(ks), ld), complex)
    Bm = np.zeros_like(A)
    G = np.zeros_like(A)
    for i, k in enumerate(ks):
        A[i, :k] = a[:k]
        Bm[i, 1:k] = b[1:k]
        G[i, 1:k] = g[1:k]
    return A, Bm, G


def convergence_record(dims, U, m_w, mu, x, tol=1e-8, k_max=600, dk=10, precision="df64"):
    """(features, k*, l*, converged) for one problem (see module docstring)."""
    opts = B.make_opts(k_fixed=k_max, recombination=B.OV_RECOMB_STORED)
    with B.Overlap(dims, U, m_w, mu, precision, opts=opts) as op:
        xs = np.ascontiguousarray(np.reshape(x, (1, -1)))
        y = np.zeros_like(xs)
        op.sign_apply(xs, y, tol, k_max, 8)
        a, b, g = op.coefficients(0, k_max)
        herm = mu == 0.0
        kk = len(a)
        ks = list(range(dk, kk + 1, dk))
        A, Bm, G = _prefix_arrays(a, b, g, ks, kk)
        rc, C, est_in, its = B.ov_inner_sign(op.h, ks, A, Bm, G, herm, 120)
        kstar, conv = ks[-1], False
        for i in range(1, len(ks)):
            ci = C[i, :ks[i]]
            cp = np.zeros_like(ci)
            cp[:ks[i - 1]] = C[i - 1, :ks[i - 1]]
            if np.linalg.norm(ci - cp) <= tol * np.linalg.norm(ci):
                kstar, conv = ks[i], True
                break
        # l*: smallest l on the grid with inner estimate <= tol at k* (binary search)
        A1, B1, G1 = _prefix_arrays(a, b, g, [kstar], kstar)
        lo, hi = 0, len(L_GRID) - 1
        while lo < hi:
            mid = (lo + hi) // 2
            l = min(L_GRID[mid], kstar)
            _, _, e, _ = B.ov_inner_sign(op.h, [kstar], A1, B1, G1, herm, l)
            if e[0] <= tol:
                hi = mid
            else:
                lo = mid + 1
        lstar = min(L_GRID[lo], kstar)
    return (features(a, b), kstar, lstar, conv,
            np.concatenate([a[:16], b[1:17], g[1:17]]).astype(np.complex128))


def features_from_raw(raw, fset="a6i6b4"):
    """Features from stored raw coefficients [alpha_1..16, beta_2..17, gamma_2..17]:
    a6i6b4 (the network's: Re alpha_1..6, Im alpha_1..6, beta_2..5), or for comparison
    a8b8 (the first 16 outer coefficients: Re alpha_1..8, beta_2..9), a4i4b8
    (Re alpha_1..4, Im alpha_1..4, beta_2..9), a8i8 (Re and Im alpha_1..8)."""
    raw = np.asarray(raw)
    a, b = raw[:, :16], raw[:, 16:32]
    parts = {"a6i6b4": [np.real(a[:, :6]), np.imag(a[:, :6]), np.real(b[:, :4])],
             "a8b8": [np.real(a[:, :8]), np.real(b[:, :8])],
             "a4i4b8": [np.real(a[:, :4]), np.imag(a[:, :4]), np.real(b[:, :8])],
             "a8i8": [np.real(a[:, :8]), np.imag(a[:, :8])]}[fset]
    return np.concatenate(parts, axis=1)


FEATURE_SETS = ["a6i6b4", "a8b8", "a4i4b8", "a8i8"]


def held_out_errors(theta, F, k, l):
    """Median and 90th percentile of |k_pred / k* - 1| and of |l_pred - l*|."""
    kp, lp = predict(theta, F)
    ek = np.abs(kp / k - 1.0)
    el = np.abs(lp - l)
    return {"k_rel_median": float(np.median(ek)), "k_rel_p90": float(np.percentile(ek, 90)),
            "l_abs_median": float(np.median(el)), "l_abs_p90": float(np.percentile(el, 90)),
            "k_under_20pct": float(np.mean(kp < 0.8 * k))}


def make_dataset(problems, tol=1e-8, k_max=600, log_every=50):
    import ovinputs as oi

    F, K, Lv, C, RAW = [], [], [], [], []
    t0 = time.time()
    for i, p in enumerate(problems):
        U = oi.gauge_field(p["dims"], p["kind"], p["gauge_seed"], eps=p["eps"])
        x = oi.problem_source(p)
        f, k, l, conv, raw = convergence_record(p["dims"], U, p["m_w"], p["mu"], x, tol, k_max)
        F.append(f)
        RAW.append(raw)
        K.append(k)
        Lv.append(l)
        C.append(conv)
        if log_every and (i + 1) % log_every == 0:
            print(f"records {i + 1}/{len(problems)} ({time.time() - t0:.0f} s)", flush=True)
    return dict(F=np.array(F), raw=np.array(RAW), k=np.array(K), l=np.array(Lv), conv=np.array(C),
                mu=np.array([p["mu"] for p in problems]), eps=np.array([p["eps"] for p in problems]),
                m_w=np.array([p["m_w"] for p in problems]),
                V=np.array([int(np.prod(p["dims"])) for p in problems]))


def fold_scaling(theta, fm, fs, tm, ts):
    """Parameters acting on raw features and producing raw targets."""
    th = np.asarray(theta, dtype=np.float64).copy()
    W1 = th[0:1024].reshape(64, 16)
    b1 = th[1024:1088]
    W3 = th[5248:5376].reshape(2, 64)
    b3 = th[5376:5378]
    W1n = W1 / fs[None, :]
    b1n = b1 - W1n @ fm
    W3n = W3 * ts[:, None]
    b3n = b3 * ts + tm
    th[0:1024] = W1n.ravel()
    th[1024:1088] = b1n
    th[5248:5376] = W3n.ravel()
    th[5376:5378] = b3n
    return th.astype(np.float32)


def train(F, k, l, epochs=600, lr=2e-3, seed=1, batch=0, val_frac=0.15):
    """Train on (F, log k, log l) with early stopping on the last val_frac of the records;
    returns (theta for raw inputs/outputs, training losses, validation losses)."""
    from . import binding as BB

    F = np.asarray(F, dtype=np.float64)
    T = np.stack([np.log(k), np.log(l)], axis=1)
    nv = int(round(val_frac * len(F)))
    nt = len(F) - nv
    fm, fs = F[:nt].mean(0), F[:nt].std(0) + 1e-12
    tm, ts = T[:nt].mean(0), T[:nt].std(0) + 1e-12
    Xn = ((F - fm) / fs).astype(np.float32)
    Yn = ((T - tm) / ts).astype(np.float32)
    rng = np.random.default_rng(seed)
    theta0 = []
    for o, i in [(64, 16), (64, 64), (2, 64)]:
        lim = np.sqrt(6.0 / i)
        theta0.append(rng.uniform(-lim, lim, o * i))
        theta0.append(np.zeros(o))
    theta0 = np.concatenate(theta0).astype(np.float32)
    th, hist, vhist = BB.ov_mlp_train(theta0, Xn[:nt], Yn[:nt], epochs, batch, lr, seed, Xn[nt:], Yn[nt:])
    return fold_scaling(th, fm, fs, tm, ts), hist, vhist


def predict(theta, F):
    out = B.ov_mlp_forward(theta, np.asarray(F, dtype=np.float32))
    return np.exp(out[:, 0]), np.exp(out[:, 1])


def save(path, theta, **meta):
    np.savez(path, theta=np.asarray(theta, dtype=np.float32), **meta)


def load(path):
    d = np.load(path)
    return d["theta"]


_HERE = os.path.dirname(os.path.abspath(__file__))
# trained on the near-unit records (6^4 to 8^4, k <= 600): the parameters of the smooth
# fields of the 16^4 and 24^3 x 48 workloads
DEFAULT_PARAMS = os.path.join(_HERE, "sizer_params.npz")
# trained on near-unit records with k <= 1000, rough (Haar) and near-unit records of the
# 48-lattice batch's shapes, and near-unit records from 10^4 to 16^4: for ensembles with
# rough fields
ROUGH_PARAMS = os.path.join(_HERE, "sizer_params_rough.npz")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--records", type=int, default=0)
    ap.add_argument("--first", type=int, default=0)
    ap.add_argument("--train", default=None)
    ap.add_argument("--out", required=True)
    ap.add_argument("--epochs", type=int, default=600)
    ap.add_argument("--train-n", type=int, default=2000, help="use the first N records (the rest stay held out)")
    ap.add_argument("--rough", action="store_true",
                    help="records from training_problems_rough (Haar and near-unit links, the batch's shapes)")
    ap.add_argument("--large", action="store_true", help="records from training_problems_large (10^4 to 16^4)")
    ap.add_argument("--k-max", type=int, default=600, help="outer dimension of a record's run")
    ap.add_argument("--also", nargs="*", default=[],
                    help="more record files: their first 85%% join the training set, the rest the held-out set")
    ap.add_argument("--ablation", action="store_true", help="train every feature set, report held-out errors")
    args = ap.parse_args()
    if args.records:
        import ovinputs as oi

        gen = (oi.training_problems_rough if args.rough else
               oi.training_problems_large if args.large else oi.training_problems)
        probs = gen(args.first + args.records)[args.first:]
        d = make_dataset(probs, k_max=args.k_max)
        np.savez(args.out, **d)
        print(f"wrote {args.out}: converged {int(d['conv'].sum())}/{len(probs)}")
    if args.train:
        sets = [np.load(args.train)] + [np.load(f) for f in args.also]
        n = args.train_n
        parts_tr, parts_ho = [], []
        for i, d in enumerate(sets):
            cut = n if i == 0 else int(0.85 * len(d["k"]))
            m = d["conv"].astype(bool)
            idx = np.arange(len(m))
            parts_tr.append((d, idx[(idx < cut) & m]))
            parts_ho.append((d, idx[(idx >= cut) & m]))

        def gather(parts, fset):
            F = np.concatenate([features_from_raw(d["raw"], fset)[ix] for d, ix in parts])
            return F, np.concatenate([d["k"][ix] for d, ix in parts]), np.concatenate([d["l"][ix] for d, ix in parts])

        for fset in (FEATURE_SETS if args.ablation else ["a6i6b4"]):
            F, k, l = gather(parts_tr, fset)
            theta, hist, vhist = train(F, k, l, epochs=args.epochs)
            Fh, kh, lh = gather(parts_ho, fset)
            err = held_out_errors(theta, Fh, kh, lh) if len(kh) else {}
            print(f"features {fset}: {len(k)} training records, best validation loss {vhist.min():.4f} "
                  f"(epoch {int(vhist.argmin())}); held out ({len(kh)} records): {err}", flush=True)
            if fset == "a6i6b4":
                save(args.out, theta, loss=hist, val_loss=vhist, n_train=len(k))
                print(f"wrote {args.out}")


if __name__ == "__main__":
    main()
