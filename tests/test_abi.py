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


def test_default_options_match_the_header(libov):
    """The defaults ov_default_opts fills are the ones include/ov.h documents in brackets."""
    import paper_0910_2918_gb300 as ov

    o = ov.ov_default_opts()
    assert (o.first_check, o.recombination, o.k_fixed, o.check_schedule, o.block_size, o.graph_steps,
            o.timing) == (0, 2, 0, 0, 0, 8, 0)
    assert o.rh_tol == 1e-10 and o.breakdown_tol == 1e-14
    assert o.inner_arith == ov.binding.OV_INNER_DF64 and o.relax == 0.0 and o.overlap_checks == 1
    hdr = open(os.path.join(ROOT, "include", "ov.h")).read()
    for name, default in (("inner_arith", "[OV_INNER_DF64]"), ("overlap_checks", "[1]"), ("graph_steps", "[8]")):
        block = hdr[hdr.index("int " + name + ";"):]
        assert default in block[:block.index("*/")], name


def test_options_struct_layout_matches_the_header(libov):
    """The binding's ctypes mirror has the header's fields in the header's order."""
    import paper_0910_2918_gb300 as ov

    hdr = open(os.path.join(ROOT, "include", "ov.h")).read()
    body = hdr[hdr.index("typedef struct {\n  int check_interval;"):]
    body = body[:body.index("} ov_opts;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(?:int|double)\s+([a-z_]+)\s*;", body)
    assert fields == [f for f, _ in ov.binding.ov_opts._fields_]


@pytest.mark.parametrize("struct", ["ov_stats", "ov_info", "ov_geom"])
def test_result_struct_layouts_match_the_header(libov, struct):
    import paper_0910_2918_gb300 as ov

    hdr = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "ov.h")).read(), flags=re.S)
    end = hdr.index("} " + struct + ";")
    body = hdr[hdr.rindex("typedef struct {", 0, end):end]
    fields = []
    for decl in re.findall(r"\b(?:int|double|long long)\s+([^;]+);", body):
        fields += [f.strip().split("[")[0] for f in decl.split(",")]
    assert fields == [f for f, _ in getattr(ov.binding, struct)._fields_]
