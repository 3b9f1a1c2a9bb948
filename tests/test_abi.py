"""The C-ABI library builds, loads and exports every declared entry point (no GPU)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "awpm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(awpm_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def built_lib():
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    from paper_1801_09809_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("awpm_create", "awpm_destroy", "awpm_improve", "awpm_improve_ctx",
                     "awpm_search", "awpm_strerror", "awpm_default_options", "awpm_submit",
                     "awpm_poll", "awpm_improve_batch"):
        assert required in names


def test_every_declared_symbol_is_exported(built_lib):
    for name in declared_functions():
        assert hasattr(built_lib, name), name


def test_binding_covers_the_header():
    from paper_1801_09809_gb300 import awpm
    bound = {s[0] for s in awpm.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_struct_layouts_match_header():
    """ctypes mirrors of awpm_options / awpm_stats have the C sizes."""
    from paper_1801_09809_gb300 import awpm
    # awpm_options: 4 x int32 + pointer + size_t + 2 x int32
    assert ctypes.sizeof(awpm.Options) == 16 + 8 + 8 + 8
    # awpm_problem: 2 x int32 + 5 pointers
    assert ctypes.sizeof(awpm.Problem) == 8 + 40
    # awpm_stats: 2 int32 + 5 int64 + 4 double + 2 int32
    assert ctypes.sizeof(awpm.Stats) == 8 + 40 + 32 + 8
    # awpm_greedy_stats: 2 int32 + 2 double + 2 int64
    assert ctypes.sizeof(awpm.GreedyStats) == 8 + 16 + 16
    # awpm_mcm_stats: 2 int32 + double + 2 int64
    assert ctypes.sizeof(awpm.McmStats) == 8 + 8 + 16


def test_host_only_entry_points(built_lib):
    from paper_1801_09809_gb300 import awpm
    awpm._lib_handle = None
    assert awpm.awpm_strerror(0) == "ok"
    assert "perfect" in awpm.awpm_strerror(2)
    o = awpm.Options()
    awpm.lib().awpm_default_options(ctypes.byref(o))
    assert o.device == -1 and o.max_iters == 0 and o.lookup == 0 and o.stream is None


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1801_09809_gb300 import awpm
    monkeypatch.setattr(awpm, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(awpm, "_lib_handle", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        awpm.lib()


def test_constants_match_header():
    """Every #define of the header has the same value in the binding (the
    error codes through the ERRORS table)."""
    from paper_1801_09809_gb300 import awpm
    defines = dict(re.findall(r"#define AWPM_(\w+) +(\d+)u?\b", open(HEADER).read()))
    assert defines
    for name, value in defines.items():
        if name.startswith("ERR_"):
            assert awpm.ERRORS[int(value)] == name[4:], name
        elif name == "OK":
            assert awpm.AWPM_OK == int(value)
        else:
            assert getattr(awpm, name) == int(value), name
