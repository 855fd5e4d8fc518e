"""The C-ABI library loads without a GPU and exports every function that
include/*.h declares (no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2512_21180_gb300 import build
    build.build()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\(", src, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "sizeof", "return"):
                names.add(name)
    return sorted(names)


def test_header_declares_core_calls():
    names = declared_functions()
    for n in ("geometry_create", "geometry_destroy", "forward_project", "back_project", "cbct_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2512_21180_gb300 import _lib
    lib = _lib.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # every declared function has a binding signature
    unbound = [n for n in declared_functions() if n not in {**_lib.SIGNATURES, **_lib.EXTRA_SIGNATURES}]
    assert not unbound, unbound


def test_last_error_is_a_string_without_gpu():
    from paper_2512_21180_gb300 import _lib
    assert isinstance(_lib.load().cbct_last_error(), bytes)
