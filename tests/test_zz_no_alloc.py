"""The allocation-free Roberts-Higham entry point (for callers whose device memory is
all reserved by their own pool, or that must avoid the synchronisation an allocation
can cause) agrees with the regular entry point, call after call.

This file is collected last so that a failure here, in a run that stops at the first
failure, comes after every other test has run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _matrices(rng, count, m):
    mats = []
    for _ in range(count):
        X = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
        ev = np.concatenate([rng.uniform(0.3, 3, m // 2), -rng.uniform(0.3, 3, m - m // 2)])
        ev = ev + 1j * rng.uniform(-1, 1, m)
        mats.append(X @ np.diag(ev) @ np.linalg.inv(X))
    return np.ascontiguousarray(np.stack(mats))


def test_noalloc_matches_regular_entry_point_twice():
    import torch

    import ovinputs as oi
    import paper_0910_2918_gb300 as ov

    dims = (2, 2, 2, 2)
    # the allocation-free entry point eliminates in FP64: compare with the regular entry
    # point in the same arithmetic
    h = ov.ov_create(dims, oi.gauge_field(dims, "unit", 0), -1.5, 0.0,
                     opts=ov.make_opts(inner_arith=ov.binding.OV_INNER_FP64))
    try:
        rng = np.random.default_rng(11)
        for count, m in ((3, 40), (2, 120)):  # two calls in a row, different shapes
            T = _matrices(rng, count, m)
            rc_ref, S_ref, its_ref = ov.ov_rh_sign(h, T)
            Td = torch.from_numpy(T).cuda()
            Sd = torch.full_like(Td, float("nan"))
            rc, its = ov.ov_rh_sign_noalloc(Td, Sd)
            assert rc == 0 and rc_ref == 0
            S = Sd.cpu().numpy()
            for i in range(count):
                assert np.linalg.norm(S[i] - S_ref[i]) / np.linalg.norm(S_ref[i]) < 1e-10
            assert np.array_equal(its, its_ref)
    finally:
        ov.ov_destroy(h)


def test_noalloc_rejects_sizes_beyond_its_limits():
    import torch

    import paper_0910_2918_gb300 as ov

    T = torch.zeros((65, 4, 4), dtype=torch.complex128, device="cuda")
    with pytest.raises(ov.OvError) as e:
        ov.ov_rh_sign_noalloc(T, torch.zeros_like(T))
    assert e.value.code == -7
    T = torch.zeros((1, 121, 121), dtype=torch.complex128, device="cuda")
    with pytest.raises(ov.OvError) as e:
        ov.ov_rh_sign_noalloc(T, torch.zeros_like(T))
    assert e.value.code == -7


def test_noalloc_reports_singular_and_iteration_cap():
    """Status handling read back by the host: an exactly singular matrix (all zeros: the
    first pivot is zero) and an iteration cap of 1 both return OV_ERR_RH_NOCONV, with the
    iterations used reported (never more than the cap)."""
    import torch

    import paper_0910_2918_gb300 as ov

    Z = torch.zeros((1, 8, 8), dtype=torch.complex128, device="cuda")
    rc, its = ov.ov_rh_sign_noalloc(Z, torch.zeros_like(Z))
    assert rc == ov.binding.OV_ERR_RH_NOCONV
    assert 1 <= its[0] <= 100
    T = torch.from_numpy(_matrices(np.random.default_rng(3), 2, 16)).cuda()
    rc, its = ov.ov_rh_sign_noalloc(T, torch.zeros_like(T), rh_maxit=1)
    assert rc == ov.binding.OV_ERR_RH_NOCONV
    assert list(its) == [1, 1]


def test_noalloc_binding_rejects_mismatched_buffers():
    """The binding refuses buffers the kernel would read or write out of bounds."""
    import torch

    import paper_0910_2918_gb300 as ov

    T = torch.zeros((2, 8, 6), dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):
        ov.ov_rh_sign_noalloc(T, torch.zeros_like(T))
    T = torch.zeros((2, 8, 8), dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):
        ov.ov_rh_sign_noalloc(T, torch.zeros((1, 8, 8), dtype=torch.complex128, device="cuda"))
    with pytest.raises(ValueError):
        ov.ov_rh_sign_noalloc(T[0], torch.zeros_like(T[0]))
