"""The C-ABI library builds, loads and exports every entry point include/ov.h declares
(no compute calls: this runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libov():
    from paper_0910_2918_gb300 import _build

    _build.build()
    import paper_0910_2918_gb300 as ov

    return ov.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ov.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ov_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("ov_create", "ov_sign_apply", "ov_apply", "ov_destroy", "ov_wilson_apply", "ov_inner_sign",
              "ov_rh_sign", "ov_strerror", "ov_default_opts", "ov_set_opts", "ov_version", "ov_get_stats",
              "ov_reset_stats"):
        assert n in names


def test_library_exports_every_declared_symbol(libov):
    missing = [n for n in declared_functions() if not hasattr(libov, n)]
    assert not missing, missing


def test_host_side_calls_without_device(libov):
    import paper_0910_2918_gb300 as ov

    assert ov.ov_strerror(0) == "ok"
    assert "breakdown" in ov.ov_strerror(-5)
    o = ov.ov_default_opts()
    assert o.check_interval == 10 and o.inner_dl == 4 and o.rh_maxit == 100


def test_argument_validation_before_device_use(libov):
    """m_w outside (-2, 0) is rejected before any device work (Sec. 1)."""
    import numpy as np

    import paper_0910_2918_gb300 as ov

    U = np.zeros((16, 4, 3, 3), dtype=np.complex128)
    with pytest.raises(ov.OvError) as e:
        ov.ov_create((2, 2, 2, 2), U, 0.5, 0.0)
    assert e.value.code == -1
    with pytest.raises(ov.OvError):
        ov.ov_create((2, 2, 1, 2), U, -1.0, 0.0)


def test_no_cpu_fallback_in_product_path():
    """The package and the CUDA sources never import or call the oracle."""
    pkg = os.path.join(ROOT, "paper_0910_2918_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
