"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/surfelwarp.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

import paper_1904_13073_gb300 as sw
from paper_1904_13073_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "surfelwarp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sw_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    try:
        B.build()
    except RuntimeError as exc:
        if "nvcc not found" in str(exc):
            pytest.skip("no CUDA toolkit")
        raise
    return B.LIB


def test_every_declared_symbol_is_exported(built):
    lib = ctypes.CDLL(built)
    declared = _declared()
    assert len(declared) >= 25
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(sw.exported_symbols()) == declared


def test_host_only_calls_work_without_gpu(built):
    p = sw.sw_params_default(640, 480, 570.0, 570.0, 320.0, 240.0, 1000, 64)
    assert p.lambda_ == 5.0 and p.fuse_normal == pytest.approx(0.85) and p.recent_frames == 2
    assert sw.sw_status_string(4) == "solver breakdown"
    with pytest.raises(sw.SwError) as e:
        sw.sw_params_default(0, 480, 1, 1, 1, 1, 1, 9)
    assert e.value.status == 1
    bad = sw.sw_params_default(640, 480, 570.0, 570.0, 320.0, 240.0, 1000, 4)
    with pytest.raises(sw.SwError) as e:
        sw.sw_create_stream(bad)
    assert e.value.status == 1 and "max_nodes" in str(e.value)


def test_graft_entry_build_imports_package(built):
    import __graft_entry__
    __graft_entry__.build()


def test_appending_and_visibility_parameters_are_checked_on_the_host(built):
    """Defaults follow Table 1 (ε, t_low_confid) and the readings (δ_nn,
    finite-difference step, visibility off, node extension on); values out of
    range are refused before any device work."""
    p = sw.sw_params_default(640, 480, 570.0, 570.0, 320.0, 240.0, 1000, 64)
    assert p.eps == pytest.approx(0.2) and p.t_low_confid == 30
    assert p.delta_nn == pytest.approx(0.3) and p.fd_step == pytest.approx(1e-3)
    assert p.visibility == 0 and p.extend_nodes == 1
    for field, value, word in (("visibility", 2, "visibility"), ("extend_nodes", -1, "extend_nodes"),
                               ("eps", 1.5, "appending"), ("eps", 0.0, "appending"),
                               ("delta_nn", -0.1, "appending"), ("fd_step", 0.0, "appending"),
                               ("precision", 7, "precision")):
        bad = sw.sw_params_default(640, 480, 570.0, 570.0, 320.0, 240.0, 1000, 64)
        setattr(bad, field, value)
        with pytest.raises(sw.SwError) as e:
            sw.sw_create_stream(bad)
        assert e.value.status == 1 and word in str(e.value), (field, str(e.value))


def test_block_inverse_hook_checks_its_arguments_on_the_host(built):
    """Zero blocks is a no-op and a negative count or a missing array is
    refused, both before any device work."""
    import ctypes
    lib = sw.lib()
    ok = (ctypes.c_int * 1)()
    assert lib.sw_debug_block_inverse(None, 0, 0, None, None) == 0
    assert lib.sw_debug_block_inverse(None, -1, 0, None, ok) == 1
    assert lib.sw_debug_block_inverse(None, 3, 1, None, ok) == 1
