"""The C-ABI library builds for sm_103a, loads, and exports every function
the header declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_header_symbol(lib_built):
    Q = lib_built
    names = Q.header_functions()
    assert len(names) >= 25
    lib = ctypes.CDLL(Q.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_header_is_plain_c():
    """No torch or C++ types in the boundary: only plain pointers and sizes."""
    txt = open(os.path.join(ROOT, "include", "qtt_homog.h")).read()
    for bad in ("torch", "at::", "std::", "template", "Tensor"):
        assert bad not in txt
    assert 'extern "C"' in txt


def test_every_entry_point_cites_and_documents():
    """Each declaration in the header is preceded by a comment block."""
    txt = open(os.path.join(ROOT, "include", "qtt_homog.h")).read()
    body = txt[txt.index("typedef struct qtt_op* qtt_op_t;"):]
    decls = re.findall(r"\n((?:int|void|size_t|uint64_t|const char\*) [a-z_0-9]+\()", body)
    assert len(decls) >= 25
