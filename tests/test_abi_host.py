"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every entry point declared in include/tctf2r.h, the parameter struct
layout of the binding matches the header, and argument validation rejects bad
inputs before any device work."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tctf2r.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2005_09838_gb300 import build, tc
    build.build()
    return tc.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(tc_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tc_init", "tc_iterate", "tc_objective", "tc_free", "tc_result", "tc_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(tc_\w+)", out))
    assert set(declared_functions()) <= exported


def test_params_layout_matches_header(tmp_path):
    from paper_2005_09838_gb300 import tc
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "tctf2r.h"\n'
                   'int main(void){printf("%zu", sizeof(tc_params));'
                   + "".join(f'printf(" %zu", offsetof(tc_params, {f}));' for f, _ in tc.tc_params._fields_)
                   + "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(tc.tc_params)
    assert vals[1:] == [getattr(tc.tc_params, f).offset for f, _ in tc.tc_params._fields_]


@pytest.mark.parametrize("kw,status", [
    (dict(n1=0), "TC_ERR_ARG"),
    (dict(r=0), "TC_ERR_ARG"),
    (dict(r=33), "TC_ERR_ARG"),
    (dict(r=9), "TC_ERR_ARG"),       # r > n2 = 8
    (dict(mu=-1.0), "TC_ERR_ARG"),
    (dict(rho2=float("nan")), "TC_ERR_ARG"),
    (dict(precision=9), "TC_ERR_ARG"),
    (dict(flags=1), "TC_ERR_ARG"),               # single pass is for TC_TF32 / TC_BF16 only
    (dict(precision=2, flags=2), "TC_ERR_ARG"),  # unknown flag bit
    (dict(step=1, alpha=0.0), "TC_ERR_ARG"),     # scaled steps need alpha, beta > 0
    (dict(step=1, beta=float("inf")), "TC_ERR_ARG"),
    (dict(step=2), "TC_ERR_ARG"),
    (dict(eps=-1e-6), "TC_ERR_ARG"),
])
def test_invalid_arguments_are_rejected_on_the_host(lib, kw, status):
    from paper_2005_09838_gb300 import tc
    base = dict(n1=4, n2=8, n3=5, r=2)
    base.update({k: v for k, v in kw.items() if k in base})
    p = tc.make_params(**base, **{k: v for k, v in kw.items() if k not in base})
    buf = np.zeros(4 * 8 * 5, np.float32)
    with pytest.raises(tc.TCError) as ei:
        tc.Completion(p, buf, np.zeros(buf.size, np.uint8), buf)
    assert status in str(ei.value)


def test_missing_inputs_are_rejected(lib):
    from paper_2005_09838_gb300 import tc
    p = tc.make_params(4, 8, 5, 2)
    with pytest.raises(tc.TCError) as ei:
        tc.Completion(p, None, None, None)
    assert "TC_ERR_ARG" in str(ei.value)


def test_free_is_null_safe(lib):
    assert lib.tc_free(None) == 0
