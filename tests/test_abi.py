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


def test_context_setters_reject_a_null_context(lib_built):
    """The setters validate their context before touching it (host code only,
    no CUDA call), so they can be called here without a GPU."""
    lib = ctypes.CDLL(lib_built.LIB_PATH)
    calls = [("qtt_ctx_set_green_broadcast", (1,)), ("qtt_ctx_set_concurrency", (6,)),
             ("qtt_ctx_set_contraction", (0,)), ("qtt_ctx_set_factorization", (0,)),
             ("qtt_ctx_set_svd", (1, 6)), ("qtt_ctx_set_tt_svd", (ctypes.c_double(2e9),)),
             ("qtt_ctx_set_jacobi", (ctypes.c_double(1.0), 40)), ("qtt_ctx_set_profiling", (1,))]
    for name, args in calls:
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        assert f(None, *args) == lib_built.QTT_EINVAL, name


def test_native_zipup_sfft_matches_the_oracle(lib_built):
    """The library's host zip-up construction of the SFFT MPO (Sec. 4.2; no GPU)
    is S = P_rev F+ (the oracle's dense bit-reversed DFT) for n = 1..8, has the
    ranks of the oracle's circuit construction at 1e-12, and reaches the
    printed rank 10 at 1e-10 for n = 8 (Sec. 5.2)."""
    import numpy as np
    from oracle import qtt as oq
    Q = lib_built
    for n in range(1, 9):
        cores = Q.qtt_sfft_mpo_zipup(n, 1e-12)
        assert np.allclose(oq.tto_full(cores), oq.sfft_dense(n), atol=1e-13)
        assert [c.shape[0] for c in cores] == [c.shape[0] for c in oq.sfft_axis_mpo_zipup(n, 1e-12)]
    assert max(c.shape[0] for c in Q.qtt_sfft_mpo_zipup(8, 1e-10)) == 10
    import ctypes as C
    need = C.c_size_t()
    ranks = (C.c_int * 26)()
    assert Q.lib.qtt_sfft_mpo_zipup(25, 1e-12, ranks, None, 0, C.byref(need)) == Q.QTT_EINVAL
    big = Q.qtt_sfft_mpo_zipup(20, 1e-10)        # 2^20 points per axis, no dense matrix
    assert len(big) == 20 and max(c.shape[0] for c in big) <= 12
