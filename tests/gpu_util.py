"""Helpers for the GPU parity tests (host-side only)."""
import numpy as np

import ovinputs as oi
from oracle import dirac, krylov


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def oracle_ops(U, dims, m_w, mu):
    return (lambda v: dirac.A_apply(U, v, dims, m_w, mu), lambda v: dirac.AH_apply(U, v, dims, m_w, mu))


def oracle_sign(U, dims, m_w, mu, x, **kw):
    fA, fAH = oracle_ops(U, dims, m_w, mu)
    return krylov.sign_apply(fA, fAH, x, mu == 0.0, **kw)


def links_for(prec, U):
    """The operator a run of precision `prec` sees: FP32 rounds the links to float once;
    double-float keeps them as float pairs (2^-48 relative), i.e. the FP64 operator."""
    return oi.round_links_fp32(U) if prec == "fp32" else U
