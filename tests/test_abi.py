"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/dd4dvar.h declares; the ctypes structs match the C layout."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dd4dvar.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2205_06649_gb300 import _abi
    return _abi, ctypes.CDLL(_abi.LIB_PATH)


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dd4dv_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = header_functions()
    assert "dd4dv_eval" in names and "dd4dv_run" in names and len(names) >= 25


def test_every_declared_symbol_is_exported(lib):
    _abi, cdll = lib
    missing = [n for n in header_functions() if not hasattr(cdll, n)]
    assert not missing, missing


def test_binding_has_a_prototype_for_every_entry_point(lib):
    _abi, _ = lib
    assert sorted(_abi.PROTOTYPES) == header_functions()


def test_struct_layouts_match_c(lib):
    _abi, _ = lib
    src = '#include <stdio.h>\n#include <stddef.h>\n#include "dd4dvar.h"\nint main(void){' \
          'printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(dd4dv_model), sizeof(dd4dv_decomp),' \
          'sizeof(dd4dv_solver), sizeof(dd4dv_stats), offsetof(dd4dv_decomp, mu),' \
          'offsetof(dd4dv_stats, dw_inf)); return 0;}'
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    got = [ctypes.sizeof(_abi.dd4dv_model), ctypes.sizeof(_abi.dd4dv_decomp),
           ctypes.sizeof(_abi.dd4dv_solver), ctypes.sizeof(_abi.dd4dv_stats),
           _abi.dd4dv_decomp.mu.offset, _abi.dd4dv_stats.dw_inf.offset]
    assert [int(x) for x in out] == got


def test_last_error_without_context_is_callable(lib):
    _abi, _ = lib
    from paper_2205_06649_gb300 import lib as L
    assert isinstance(L.dd4dv_last_error(None), bytes)


def test_create_rejects_bad_model_without_touching_the_gpu(lib):
    import paper_2205_06649_gb300 as dd
    with pytest.raises(dd.DD4DVError) as e:
        dd.Context(2, 1, 10.0, 4)
    assert e.value.status == -1


def test_package_refuses_to_import_without_the_library(tmp_path):
    """There is no CPU fallback: a copy of the package without the built
    library raises ImportError at import."""
    import shutil
    import subprocess
    import sys
    src = os.path.join(ROOT, "paper_2205_06649_gb300")
    dst = tmp_path / "paper_2205_06649_gb300"
    shutil.copytree(src, dst, ignore=shutil.ignore_patterns("*.so", "csrc", "__pycache__"))
    r = subprocess.run([sys.executable, "-c", "import paper_2205_06649_gb300"], cwd=tmp_path,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "libdd4dvar.so" in r.stderr
