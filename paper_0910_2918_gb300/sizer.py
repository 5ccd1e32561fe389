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


def features_from_raw(raw):
    """Features from stored raw coefficients [alpha_1..16, beta_2..17, gamma_2..17]."""
    raw = np.asarray(raw)
    return np.concatenate([np.real(raw[:, :6]), np.imag(raw[:, :6]), np.real(raw[:, 16:20])], axis=1)


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


DEFAULT_PARAMS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sizer_params.npz")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--records", type=int, default=0)
    ap.add_argument("--first", type=int, default=0)
    ap.add_argument("--train", default=None)
    ap.add_argument("--out", required=True)
    ap.add_argument("--epochs", type=int, default=600)
    ap.add_argument("--train-n", type=int, default=2000, help="use the first N records (the rest stay held out)")
    args = ap.parse_args()
    if args.records:
        import ovinputs as oi

        probs = oi.training_problems(args.first + args.records)[args.first:]
        d = make_dataset(probs)
        np.savez(args.out, **d)
        print(f"wrote {args.out}: converged {int(d['conv'].sum())}/{len(probs)}")
    if args.train:
        d = np.load(args.train)
        n = args.train_n
        m = d["conv"][:n].astype(bool)
        F = (features_from_raw(d["raw"]) if "raw" in d else d["F"])[:n]
        theta, hist, vhist = train(F[m], d["k"][:n][m], d["l"][:n][m], epochs=args.epochs)
        save(args.out, theta, loss=hist, val_loss=vhist, n_train=int(m.sum()))
        print(f"wrote {args.out}: best validation loss {vhist.min():.4f} (epoch {int(vhist.argmin())}) "
              f"on {int(m.sum())} records")


if __name__ == "__main__":
    main()
