"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dpmm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dpmm_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libdpmm():
    from paper_1812_10048_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["dpmm_init", "dpmm_sweep", "dpmm_split_merge", "dpmm_labels",
                     "dpmm_logml_forward", "dpmm_logml_backward", "dpmm_free", "dpmm_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(libdpmm):
    missing = [n for n in declared_functions() if not hasattr(libdpmm, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1812_10048_gb300 import _lib
    missing = [n for n in declared_functions() if n not in _lib.SIGNATURES]
    assert not missing, missing


def test_default_opts_without_gpu(libdpmm):
    from paper_1812_10048_gb300 import dpmm_default_opts
    o = dpmm_default_opts()
    assert o.kmax == 256 and o.split_q == 1 and o.seed == 42 and o.engine == 0


def test_python_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1812_10048_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.lib()


@pytest.mark.parametrize("struct", ["dpmm_opts", "dpmm_tuning"])
def test_struct_layout_matches_the_header(tmp_path, struct):
    """The ctypes mirrors of dpmm_opts and dpmm_tuning have the header's size
    and field offsets (a C program compiled against include/dpmm.h prints
    them)."""
    import shutil
    import subprocess
    from paper_1812_10048_gb300 import _lib
    cls = getattr(_lib, struct)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f[0] for f in cls._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'    printf("%s %zu\\n", "{f}", offsetof({struct}, {f}));\n' for f in fields)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "dpmm.h"\n'
                   'int main(void) {\n'
                   f'    printf("sizeof %zu\\n", sizeof({struct}));\n' + body +
                   '    return 0;\n}\n')
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    assert int(out["sizeof"]) == ctypes.sizeof(cls)
    for f in fields:
        assert int(out[f]) == getattr(cls, f).offset, f


def test_binding_argument_counts_match_the_prototypes():
    """Every prototype in include/dpmm.h has as many parameters as its ctypes
    signature (a wrong count would pass garbage through the C ABI)."""
    from paper_1812_10048_gb300 import _lib
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "include", "dpmm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = re.findall(r"\b(dpmm_\w+)\s*\(([^;{]*?)\)\s*;", text)
    assert len(protos) >= 30
    for name, params in protos:
        params = " ".join(params.split())
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert name in _lib.SIGNATURES, name
        assert len(_lib.SIGNATURES[name][1]) == n, (name, n, len(_lib.SIGNATURES[name][1]))
