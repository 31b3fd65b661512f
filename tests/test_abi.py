"""The C-ABI library builds for sm_103a and exports every symbol that
include/bkrylov.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bkrylov.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bk_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_0903_4936_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_0903_4936_gb300 import build
        build.build()
    return _lib.LIB_PATH


def test_header_and_binding_agree():
    from paper_0903_4936_gb300 import _lib
    assert _declared() == sorted(_lib.EXPORTED)


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(L, name), name


def test_status_strings_without_gpu(libpath):
    from paper_0903_4936_gb300 import _lib
    L = _lib.lib()
    for code in range(8):
        assert L.bk_status_string(code)
    assert L.bk_field_bytes(None, 12, 0) == 0


def test_struct_layouts_match_header():
    """The ctypes mirrors of bk_solve_params / bk_solve_info have the C sizes."""
    import subprocess
    import tempfile
    src = '#include "bkrylov.h"\n#include <stdio.h>\nint main(){printf("%zu %zu\\n", ' \
          'sizeof(bk_solve_params), sizeof(bk_solve_info));return 0;}\n'
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    from paper_0903_4936_gb300 import _lib
    assert int(out[0]) == ctypes.sizeof(_lib.SolveParams)
    assert int(out[1]) == ctypes.sizeof(_lib.SolveInfo)


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_0903_4936_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
