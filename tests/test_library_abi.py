"""CPU checks of the C-ABI library: it builds, loads without a GPU, exports
every function declared in include/*.h, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lq2d.h")
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


@pytest.fixture(scope="module")
def lib():
    from paper_2304_04980_gb300 import build, lq2d
    build.build()
    return lq2d.load()


def declared_functions():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lq2d_[a-z_]+)\s*\(", text)))


def test_header_declarations_are_exported(lib):
    names = declared_functions()
    assert len(names) >= 13
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_2304_04980_gb300 import lq2d
    assert sorted(lq2d.EXPORTED) == declared_functions()


def test_status_codes_match_header():
    from paper_2304_04980_gb300 import lq2d
    text = open(HEADER).read()
    codes = dict(re.findall(r"LQ2D_(E[A-Z]+|OK)\s*=\s*(\d+)", text))
    assert int(codes["OK"]) == lq2d.OK and int(codes["EINVAL"]) == lq2d.EINVAL
    assert int(codes["ENOTPD"]) == lq2d.ENOTPD and int(codes["ETIMEOUT"]) == lq2d.ETIMEOUT


def test_stats_struct_layout(tmp_path):
    """The binding's Stats mirrors lq2d_stats of include/lq2d.h: a C program
    compiled against the header prints the size and every field offset."""
    import shutil
    import subprocess
    from paper_2304_04980_gb300 import lq2d
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = [n for n, _ in lq2d.Stats._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lq2d.h"\nint main(void) {\n'
                   '  printf("%zu\\n", sizeof(lq2d_stats));\n' +
                   "".join('  printf("%%zu\\n", offsetof(lq2d_stats, %s));\n' % n for n in names) +
                   "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(lq2d.Stats)
    assert out[1:] == [getattr(lq2d.Stats, n).offset for n in names]


@pytest.mark.parametrize("dims", [(0, 4, 4, 2, 1), (4, 0, 4, 2, 1), (4, 4, 0, 2, 1), (4, 4, 4, 0, 1),
                                  (4, 4, 4, 9, 1), (4, 4, 4, 2, 0), (4, 4, 4, 2, 9)])
def test_bad_dimensions_rejected_without_gpu(lib, dims):
    from paper_2304_04980_gb300 import lq2d
    h = ctypes.c_void_p()
    code = lib.lq2d_create(ctypes.byref(h), *dims, None, None, None, None, None, None, None)
    assert code == lq2d.EINVAL and not h.value
    assert lq2d.last_error()


def test_non_finite_host_input_rejected_without_gpu(lib):
    from paper_2304_04980_gb300 import lq2d, synth
    g = synth.random_grid(2, 2, 3, 2, 1, seed=1)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in g.arrays()]
    arrs[2] = arrs[2].copy()
    arrs[2][0, 0, 0] = np.nan
    h = ctypes.c_void_p()
    code = lib.lq2d_create(ctypes.byref(h), g.K, g.N, g.T, g.n, g.m, *[a.ctypes.data for a in arrs])
    assert code == lq2d.EINVAL and "non-finite" in lq2d.last_error()


def test_null_handle_calls_fail_cleanly(lib):
    from paper_2304_04980_gb300 import lq2d
    assert lib.lq2d_solve(None, 1e-8, 2, 2, 10, None, None, None, None, None, None) == lq2d.EINVAL
    assert lib.lq2d_set_option(None, 1, 0.0) == lq2d.EINVAL
    lib.lq2d_destroy(None)
    assert lib.lq2d_autotune(None, 2, 2, 1, None, None, None) == lq2d.EINVAL


def test_warmstart_net_rejects_bad_arguments_without_gpu(lib):
    from paper_2304_04980_gb300 import lq2d
    h = ctypes.c_void_p()
    assert lib.lq2d_wsnet_create(ctypes.byref(h), 4, 4, 3, 9, 8, 2, 2, 1.0) == lq2d.EINVAL and not h.value
    assert lib.lq2d_wsnet_create(ctypes.byref(h), 4, 4, 3, 2, 8, 2, 2, -1.0) == lq2d.EINVAL and not h.value
    assert lib.lq2d_wsnet_create(ctypes.byref(h), 4, 4, 3, 2, 0, 2, 2, 1.0) == lq2d.EINVAL and not h.value
    assert lib.lq2d_wsnet_forward_device(None, 1, None, None, None, None) == lq2d.EINVAL
    assert lib.lq2d_wsnet_train_step_device(None, 1, None, None, None, 1e-3, None, None) == lq2d.EINVAL
    lib.lq2d_wsnet_destroy(None)
