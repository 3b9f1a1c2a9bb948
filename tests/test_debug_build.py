"""The AWPM_DEBUG_BOUNDS variant of the library compiles (no GPU: nvcc
cross-compiles for sm_103a)."""
import os
import shutil

import pytest


def test_debug_bounds_build_compiles(tmp_path):
    if shutil.which(os.environ.get("NVCC", "nvcc")) is None:
        pytest.skip("nvcc not available")
    from paper_1801_09809_gb300 import build
    lib = build.build_debug(str(tmp_path / "libawpm_debug.so"), str(tmp_path / "obj"))
    assert os.path.getsize(lib) > 0
