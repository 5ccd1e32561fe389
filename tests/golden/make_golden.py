"""Write the stored expected values under tests/golden/ (run by hand; slow).

Every value written here comes from the CPU oracle (`oracle/`) on the seeded inputs of
`ovinputs/`; nothing else is called. The paper prints no worked example, so these
fixtures hold oracle results at sizes the oracle cannot finish inside a test run.

c3_16x16x16x16_mu0.2_sign.json
    y = sgn(gamma5 D_w(mu)) x by the nested method (Secs. 2-3) on the 16^4 lattice of
    the benchmark: near-unit links exp(i 0.3 H) (seed 0), mu = 0.2, m_w = -1.6,
    antiperiodic in t, spin-colour point sources at site 0 (index 3*spin + colour),
    FP64, l = 120, tol = 1e-11, a check every 25 steps. Stored per source: the stopping
    step k, the estimate, the coefficients alpha, beta, gamma of the outer process,
    ||y||, the projections <r_i, y> on four seeded Gaussian vectors r_i (seeds 101..104,
    `ovinputs.gaussian_source(dims, seed, normalize=False)`), and y at every site within
    distance 2 of the source plus 64 seeded random sites (all 12 components each).

    Also stored: the step at which the oracle's stopping rule stops at the benchmark's
    tolerances (l = 72, checks at 100 and every 25 steps), from the stored coefficients.

    python tests/golden/make_golden.py            # about 8 minutes per source, 6 GB RAM
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import ovinputs as oi  # noqa: E402
from oracle import dirac, krylov  # noqa: E402

C3 = dict(dims=(16, 16, 16, 16), eps=0.3, gauge_seed=0, mu=0.2, m_w=-1.6, l=120, tol=1e-11, check_interval=25,
          k_max=1000, sources=[0, 7], proj_seeds=[101, 102, 103, 104], n_random_sites=64, sample_seed=7)


def sample_sites(dims, n_random, seed):
    """Sites within lattice distance 2 of site 0 (periodic), then n_random others."""
    Lx, Ly, Lz, Lt = dims
    near = set()
    for dx in range(-2, 3):
        for dy in range(-2, 3):
            for dz in range(-2, 3):
                for dt in range(-2, 3):
                    if abs(dx) + abs(dy) + abs(dz) + abs(dt) <= 2:
                        near.add((dx % Lx) + Lx * ((dy % Ly) + Ly * ((dz % Lz) + Lz * (dt % Lt))))
    rng = np.random.Generator(np.random.PCG64(seed))
    V = Lx * Ly * Lz * Lt
    extra = [int(s) for s in rng.choice(V, n_random + len(near), replace=False) if s not in near][:n_random]
    return sorted(near) + extra


def c3():
    cfg = C3
    dims = cfg["dims"]
    U = oi.gauge_field(dims, "near_unit", cfg["gauge_seed"], eps=cfg["eps"])
    X = oi.point_sources_12(dims, site=0)
    sites = sample_sites(dims, cfg["n_random_sites"], cfg["sample_seed"])
    idx = np.array([12 * s + c for s in sites for c in range(12)])
    projs = [oi.gaussian_source(dims, sd, normalize=False) for sd in cfg["proj_seeds"]]
    out = dict(config={k: v for k, v in cfg.items()}, sites=sites, sources={})
    for r in cfg["sources"]:
        t0 = time.time()
        y, info = krylov.sign_apply(lambda v: dirac.A_apply(U, v, dims, cfg["m_w"], cfg["mu"]),
                                    lambda v: dirac.AH_apply(U, v, dims, cfg["m_w"], cfg["mu"]), X[r], False,
                                    cfg["k_max"], cfg["l"], cfg["tol"], check_interval=cfg["check_interval"])
        k = int(info["k"])
        out["sources"][str(r)] = dict(
            k=k, l=int(info["l"]), status=int(info["status"]), err_est=float(info["err_est"]),
            norm=float(np.linalg.norm(y)),
            proj=[[float(z.real), float(z.imag)] for z in (np.vdot(p, y) for p in projs)],
            alpha=[[float(z.real), float(z.imag)] for z in np.asarray(info["alpha"][:k], dtype=complex)],
            beta=[float(np.real(b)) for b in info["beta"][:k + 1]],
            gamma=[[float(z.real), float(z.imag)] for z in np.asarray(info["gamma"][:k + 1], dtype=complex)],
            y=[[float(z.real), float(z.imag)] for z in y[idx]],
            seconds=round(time.time() - t0, 1))
        print(f"source {r}: k={k} err_est={info['err_est']:.3e} status={info['status']} "
              f"({time.time() - t0:.0f} s)", flush=True)
    path = os.path.join(HERE, "c3_16x16x16x16_mu0.2_sign.json")
    with open(path, "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print("wrote", path)


def c3_stops(tols=(5e-9, 1e-8)):
    """Add to the C3 fixture, per source and tolerance, the step at which the oracle's
    stopping rule stops (l = 72, a check at 100 and then every 25 steps, as the benchmark
    schedules them): the outer estimate ||c_k - [c_{k-25}; 0]|| / ||c_k|| from the stored
    coefficients alone (the inner level needs only H_k)."""
    path = os.path.join(HERE, "c3_16x16x16x16_mu0.2_sign.json")
    g = json.load(open(path))
    for r, s in g["sources"].items():
        a = np.array([complex(*z) for z in s["alpha"]])
        b = np.array(s["beta"], dtype=complex)
        gm = np.array([complex(*z) for z in s["gamma"]])
        stops = {}
        for tol in tols:
            c_prev, k_stop = None, None
            for k in range(100, len(a) + 1, 25):
                H = krylov.tridiag(a[:k], b[:k + 1], gm[:k + 1])
                c, _, _, _ = krylov.nested_sign_e1(H, 72, False)
                if c_prev is not None:
                    cp = np.zeros_like(c)
                    cp[:len(c_prev)] = c_prev
                    if np.linalg.norm(c - cp) / np.linalg.norm(c) <= tol:
                        k_stop = k
                        break
                c_prev = c
            stops[f"{tol:g}"] = k_stop
        s["k_stop_l72_check100_25"] = stops
        print(f"source {r}: stops {stops}", flush=True)
    with open(path, "w") as f:
        json.dump(g, f, separators=(",", ":"))


if __name__ == "__main__":
    if "--stops-only" not in sys.argv:
        c3()
    c3_stops()
