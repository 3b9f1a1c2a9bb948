"""Mapping of device error bits to public codes, and the code table of the
binding (no GPU: the host-side mapping is compiled with the C++ compiler)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1801_09809_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include "awpm_internal.h"
using namespace awpm;
int main() {
    const unsigned cases[] = {0u, kErrInvalid, kErrUnsorted, kErrNonfinite, kErrNotPerfect,
                              kErrInternal, kErrTimeout, kErrBounds, kErrInternal | kErrTimeout,
                              kErrNotPerfect | kErrTimeout, kErrUnsorted | kErrNonfinite,
                              kErrInvalid | kErrNotPerfect | kErrInternal, 1u << 20};
    for (unsigned c : cases) std::printf("%u %d\n", c, awpm_code_of_bits(c));
    return 0;
}
"""


def test_error_bits_map_to_codes(tmp_path):
    cuda_inc = "/usr/local/cuda/include"
    if shutil.which("g++") is None or not os.path.isdir(cuda_inc):
        pytest.skip("g++ or CUDA headers missing")
    src = tmp_path / "m.cpp"
    src.write_text(PROG)
    exe = tmp_path / "m"
    subprocess.check_call(["g++", "-std=c++17", "-I" + CSRC, "-I" + os.path.join(ROOT, "include"),
                           "-I" + cuda_inc, str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {int(a): int(b) for a, b in (l.split() for l in out if l.strip())}
    from paper_1801_09809_gb300 import awpm
    name = {v: k for k, v in awpm.ERRORS.items()}
    # validation classes first, then internal consistency, then bounded waits
    assert got[0] == name["OK"]
    assert got[1] == name["INVALID_ARG"]
    assert got[2] == name["UNSORTED_OR_DUP"]
    assert got[4] == name["NONFINITE"]
    assert got[8] == name["NOT_PERFECT"]
    assert got[16] == name["INTERNAL"]
    assert got[32] == name["TIMEOUT"]
    assert got[64] == name["INTERNAL"]
    assert got[16 | 32] == name["INTERNAL"]
    assert got[8 | 32] == name["NOT_PERFECT"]
    assert got[2 | 4] == name["UNSORTED_OR_DUP"]
    assert got[1 | 8 | 16] == name["INVALID_ARG"]
    assert got[1 << 20] == name["INTERNAL"]  # unknown bits are not a timeout


def test_binding_codes_match_header():
    import re
    text = open(os.path.join(ROOT, "include", "awpm.h")).read()
    from paper_1801_09809_gb300 import awpm
    for k, v in re.findall(r"#define AWPM_ERR_(\w+)\s+(\d+)", text):
        assert awpm.ERRORS[int(v)] == k, (k, v)
    assert awpm.ERRORS[0] == "OK"
