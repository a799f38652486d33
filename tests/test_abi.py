"""The C ABI library builds, loads without a GPU, exports every function that
include/*.h declares, and the Python binding's structs match the C layout."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from paper_2103_15039_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(lsgcpd_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_entry_points():
    names = _declared_functions()
    for n in ("lsgcpd_create", "lsgcpd_destroy", "lsgcpd_preprocess", "lsgcpd_estep", "lsgcpd_mstep",
              "lsgcpd_register", "lsgcpd_last_error", "lsgcpd_params_default"):
        assert n in names


def test_library_loads_and_exports_every_declared_symbol():
    L = binding.lib()
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_params_default_on_cpu():
    p = binding.default_params()
    assert p.w == pytest.approx(0.1)
    assert p.knn_k == 10 and p.max_iters == 50 and p.newton_max == 20
    assert list(p.init_R) == [1, 0, 0, 0, 1, 0, 0, 0, 1]


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "lsgcpd.h"\n'
        "int main(void){\n"
        ' printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(lsgcpd_params), offsetof(lsgcpd_params, knn_k),'
        " offsetof(lsgcpd_params, precision), sizeof(lsgcpd_result), offsetof(lsgcpd_result, iters),"
        " offsetof(lsgcpd_result, ms_total));\n return 0; }\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    P, R = binding.Params, binding.Result
    assert vals == [ctypes.sizeof(P), P.knn_k.offset, P.precision.offset, ctypes.sizeof(R), R.iters.offset,
                    R.ms_total.offset]


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = binding.lib().lsgcpd_create(ctypes.byref(h), 0, 10, 10)
    assert rc == 3 and not h.value  # ECUDA, no context


def test_invalid_arguments_are_rejected_before_any_device_work():
    L = binding.lib()
    assert L.lsgcpd_create(None, 0, 1, 1) == 1
    h = ctypes.c_void_p()
    assert L.lsgcpd_create(ctypes.byref(h), 0, 0, 5) == 1
    assert L.lsgcpd_create(ctypes.byref(h), 0, 5, -1) == 1
    # capacity beyond the 2^30-unit limit of the plan tables (4.2e6 x 4.2e6 in 128 x 128 tiles)
    assert L.lsgcpd_create(ctypes.byref(h), 0, 4_200_000, 4_200_000) == 1
    assert not h.value
    assert L.lsgcpd_last_error(None) == b"null context"
