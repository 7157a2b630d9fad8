"""The C-ABI library builds, loads and exports every symbol include/bipm.h
declares, and the ctypes records match the C struct layouts (no GPU needed)."""

import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2606_26341_gb300 import bipm, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "bipm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bipm_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return bipm.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(bipm.EXPORTS)


def test_library_is_in_tree_and_built_for_sm103a():
    path = build.lib_path()
    assert os.path.exists(path)
    assert os.path.dirname(path).startswith(os.path.dirname(os.path.abspath(bipm.__file__)))


def test_ctypes_records_match_c_layout(lib):
    src = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "bipm.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu\n", sizeof(bipm_problem_desc), sizeof(bipm_options),
             sizeof(bipm_stats), sizeof(bipm_iterate), sizeof(bipm_result));
      printf("%zu %zu %zu\n", offsetof(bipm_iterate, mode), offsetof(bipm_iterate, mu),
             offsetof(bipm_iterate, theta_ref));
      printf("%zu %zu\n", offsetof(bipm_stats, obj), offsetof(bipm_stats, mu));
      return 0;
    }
    """
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    vals = [int(v) for v in out]
    assert vals[0] == ctypes.sizeof(bipm.ProblemDescC)
    assert vals[1] == ctypes.sizeof(bipm.OptionsC)
    assert vals[2] == ctypes.sizeof(bipm.StatsC)
    assert vals[3] == ctypes.sizeof(bipm.IterateC)
    assert vals[4] == ctypes.sizeof(bipm.ResultC) == bipm.RESULT_DTYPE.itemsize
    assert vals[5] == bipm.IterateC.mode.offset
    assert vals[6] == bipm.IterateC.mu.offset
    assert vals[7] == bipm.IterateC.theta_ref.offset
    assert vals[8] == bipm.StatsC.obj.offset
    assert vals[9] == bipm.StatsC.mu.offset


def test_invalid_arguments_fail_without_a_device(lib):
    # argument checks run before any CUDA call
    d = bipm.ProblemDescC(0, 10, 0.05, 1, 0, 0.0)
    h = ctypes.c_void_p()
    rc = lib.bipm_create_batch(ctypes.byref(d), 4, None, None, ctypes.byref(h))
    assert rc == -22
    assert b"n_quads" in lib.bipm_last_error()
    d = bipm.ProblemDescC(1, 10, -1.0, 1, 0, 0.0)
    assert lib.bipm_create_batch(ctypes.byref(d), 4, None, None, ctypes.byref(h)) == -22
    assert lib.bipm_solve(None) == -22
    assert lib.bipm_step(None, 1) == -22


def test_header_codes_match_the_binding():
    """Error codes and per-problem statuses of include/bipm.h equal the binding's."""
    text = open(HEADER).read()
    defs = {k: int(v) for k, v in re.findall(r"#define (BIPM_[A-Z0-9_]+) \(?(-?\d+)\)?", text)}
    assert defs["BIPM_EINVAL"] == bipm.EINVAL and defs["BIPM_ENOMEM"] == bipm.ENOMEM
    assert defs["BIPM_ECUDA"] == bipm.ECUDA and defs["BIPM_ESTATE"] == bipm.ESTATE
    assert defs["BIPM_ETIMEOUT"] == bipm.ETIMEOUT
    for name in ("RUNNING", "CONVERGED", "MAX_ITER", "RESTO_FAILED", "EVAL_ERROR", "TINY_STEP", "EMPTY",
                 "FP64_ESCALATION_FAILED"):
        assert defs["BIPM_" + name] == getattr(bipm, name), name
    assert set(bipm.STATUS_NAMES) == set(range(8))


def test_every_declaration_states_its_errors_or_source():
    """Each exported call's comment names where it comes from (a passage of the
    paper, or that the paper has no counterpart) or documents its errors."""
    text = open(HEADER).read()
    for name in declared_functions():
        i = re.search(r"^[a-z].*\b" + name + r"\(", text, flags=re.M).start()
        start = text.rfind("*/", 0, i)
        begin = text.rfind("/*", 0, start)
        comment = re.sub(r"\s*\n\s*\*\s*", " ", text[begin:start])
        assert ("Sec." in comment or "Eq." in comment or "Table" in comment or "no counterpart" in comment
                or "Errors" in comment or "as for" in comment), name
