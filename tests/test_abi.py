"""CPU-only checks of the C-ABI library: it builds, loads, exports every
function include/tpcg.h declares, and the binding covers them.  No compute
call is made (no GPU here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "tpcg.h")).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(tpcg_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2501_03377_gb300 import build

    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("tpcg_plan_create", "tpcg_plan_destroy", "tpcg_solve", "tpcg_precond_apply", "tpcg_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    import ctypes

    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_2501_03377_gb300 import binding

    assert sorted(_declared()) == sorted(binding.declared_symbols())


def test_strerror_and_argument_checks_without_gpu(libpath):
    from paper_2501_03377_gb300 import binding as b

    assert b.tpcg_strerror(0) == "ok"
    assert "unknown" in b.tpcg_strerror(12345)
    # argument validation happens before any CUDA call
    assert b.tpcg_plan_create(2, 8, 8, "PPN", (1, 1, 1), 0, 0)[0] == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_plan_create(8, 8, 2, "PPN", (1, 1, 1), 0, 0)[0] == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_plan_create(8, 8, 8, (0, 9, 0), (1, 1, 1), 0, 0)[0] == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_plan_create(8, 8, 8, "PPN", (1, 0, 1), 0, 0)[0] == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_plan_create(8, 8, 8, "PPN", (1, 1, 1), 7, 0)[0] == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_plan_create(300, 8, 8, "PPN", (1, 1, 1), b.TPCG_MIXED_BF16, 0)[0] == b.TPCG_ERR_UNSUPPORTED
    assert b.lib().tpcg_plan_destroy(None) == b.TPCG_ERR_INVALID_ARG


def test_binding_constants_match_header_defines():
    """Every #define TPCG_* of the header has the same value in the binding."""
    from paper_2501_03377_gb300 import binding as b

    txt = open(os.path.join(ROOT, "include", "tpcg.h")).read()
    defines = dict(re.findall(r"^#define\s+(TPCG_\w+)\s+(-?\d+)", txt, flags=re.M))
    assert len(defines) > 20
    missing = [k for k in defines if not hasattr(b, k)]
    assert not missing, missing
    wrong = {k: (v, getattr(b, k)) for k, v in defines.items() if getattr(b, k) != int(v)}
    assert not wrong, wrong


def test_new_entry_points_validate_before_any_cuda_call(libpath):
    from paper_2501_03377_gb300 import binding as b

    assert b.tpcg_plan_set_precond(None, b.TPCG_PRECOND_JACOBI, 3, 1.3) == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_efield(None, 0, None, 0, 0, 0) == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_solve_host_stream(None, [], [], 1e-10, 10, 0)[0] == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_plan_set_option(None, b.TPCG_OPT_DEFER_U, 1) == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_plan_set_option(None, b.TPCG_OPT_FUSE_G, 0) == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_plan_precond_launches(None)[0] == b.TPCG_ERR_INVALID_ARG
