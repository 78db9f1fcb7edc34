"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point declared in include/fvlb.h, and validates arguments before
touching CUDA."""
import ctypes
import os

import pytest

from paper_2506_13072_gb300 import fvlb as F


def test_exports_every_declared_symbol():
    names = F.header_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(F.lib, n), n


def _create(*args, force=None):
    h = ctypes.c_void_p()
    r = F.lib.fvlb_create(ctypes.byref(h), *args, force)
    return r, h


@pytest.mark.parametrize("args", [
    (7, 8, 8, 1, 0.8, 0.1, 10.0),      # unknown lattice
    (9, 0, 8, 1, 0.8, 0.1, 10.0),      # empty grid
    (19, 8, 8, 0, 0.8, 0.1, 10.0),     # empty grid (3D)
    (9, 8, 8, 1, 0.5, 0.1, 10.0),      # tau_s <= 1/2
    (9, 8, 8, 1, 0.8, -0.1, 10.0),     # eta_p < 0
    (9, 8, 8, 1, 0.8, 0.1, 0.0),       # lambda <= 0
    (9, 8, 8, 1, float("nan"), 0.1, 1.0),
])
def test_create_rejects_invalid_arguments(args):
    r, h = _create(*args)
    assert r == F.FVLB_EINVAL
    assert not h.value
    assert F.last_error()


def test_create_rejects_unknown_force():
    f = F.fvlb_force()
    f.kind = 9
    r, h = _create(9, 8, 8, 1, 0.8, 0.1, 10.0, force=ctypes.byref(f))
    assert r == F.FVLB_EINVAL


def test_null_handle_calls_fail_cleanly():
    assert F.lib.fvlb_step(None, 1) == F.FVLB_EINVAL
    assert F.lib.fvlb_set_walls(None, 1) == F.FVLB_EINVAL
    assert F.lib.fvlb_set_scheme(None, 1) == F.FVLB_EINVAL
    assert F.lib.fvlb_set_model(None, 1, 0.1) == F.FVLB_EINVAL
    assert F.lib.fvlb_conformation(None, None) == F.FVLB_EINVAL
    assert F.lib.fvlb_set_check_interval(None, 5) == F.FVLB_EINVAL
    assert F.lib.fvlb_status(None, 1) == F.FVLB_EINVAL
    assert F.lib.fvlb_destroy(None) == F.FVLB_OK
    assert isinstance(F.lib.fvlb_last_error(None), bytes)


def test_allocator_hooks_both_or_neither():
    a = F.ALLOC_FN(lambda n, c: None)
    assert F.lib.fvlb_set_allocator(a, F.FREE_FN(), None) == F.FVLB_EINVAL
    assert F.lib.fvlb_set_allocator(F.ALLOC_FN(), F.FREE_FN(), None) == F.FVLB_OK


def test_compact_full_roundtrip():
    import numpy as np

    rng = np.random.default_rng(0)
    for D in (2, 3):
        A = rng.normal(size=(4, D, D))
        A = A + np.swapaxes(A, -1, -2)
        assert np.array_equal(F.compact_to_full(F.full_to_compact(A)), A)


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No CPU fallback: importing the binding without the built CUDA library
    raises ImportError."""
    import shutil
    import subprocess
    import sys

    pkg = tmp_path / "paper_2506_13072_gb300"
    pkg.mkdir()
    src = os.path.join(os.path.dirname(F.__file__), "fvlb.py")
    shutil.copy(src, pkg / "fvlb.py")
    (pkg / "__init__.py").write_text("")
    code = "import paper_2506_13072_gb300.fvlb"
    r = subprocess.run([sys.executable, "-c", code], cwd=tmp_path, capture_output=True, text=True)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "not built" in r.stderr


def test_plain_c_program_links_and_calls(tmp_path):
    """The header is plain C (C99, -pedantic) and a C program links the
    library directly, without Python, and gets the documented statuses from
    calls that need no GPU."""
    import os
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.dirname(F.LIB_PATH)
    src = tmp_path / "t.c"
    src.write_text(
        '#include <stdio.h>\n#include "fvlb.h"\n'
        "int main(void) {\n"
        "  if (fvlb_destroy(NULL) != FVLB_OK) return 1;\n"
        "  if (fvlb_set_walls(NULL, 1u) != FVLB_EINVAL) return 2;\n"
        "  if (fvlb_step(NULL, 1) != FVLB_EINVAL) return 3;\n"
        "  if (fvlb_set_model(NULL, FVLB_MODEL_GIESEKUS, 0.1) != FVLB_EINVAL) return 4;\n"
        "  const char *m = fvlb_last_error(NULL);\n"
        "  if (!m || !m[0]) return 5;\n"
        '  printf("ok\\n");\n'
        "  return 0;\n}\n")
    exe = tmp_path / "t"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    f"-I{os.path.join(root, 'include')}", str(src), "-o", str(exe),
                    f"-L{libdir}", "-lfvlb", f"-Wl,-rpath,{libdir}"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
