"""The C-ABI library builds, loads and exports every entry point include/map.h declares
(no compute calls: this runs without a GPU)."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "map.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|long long|const char\*)\s+(map_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_abi():
    names = header_functions()
    for n in ("map_create_pool", "map_fill_ghosts", "map_step", "map_cfl_dt", "map_flag_refine",
              "map_read_block", "map_regrid", "map_conservation"):
        assert n in names


def test_library_exports_every_symbol():
    from paper_1204_5849_gb300 import _build
    path = _build.build()
    import ctypes
    lib = ctypes.CDLL(path)
    for n in header_functions():
        assert hasattr(lib, n), n
    from paper_1204_5849_gb300 import binding
    assert sorted(binding.exported_symbols()) == header_functions()


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1204_5849_gb300 import binding
    with pytest.raises(RuntimeError):
        binding._lib = None
        binding.load(str(tmp_path / "missing.so"))
    binding._lib = None


def test_pool_setters_reject_a_null_pool():
    """The host-side setters check their pool before touching CUDA (no GPU needed)."""
    import ctypes
    from paper_1204_5849_gb300 import _build
    lib = ctypes.CDLL(_build.build())
    assert lib.map_set_conduction_loop(None, 1) == -1          # MAP_EINVAL
    assert lib.map_test_fail_waits(None, 1) == -1
    assert lib.map_set_launch(None, 0, 0, 0) == -1
