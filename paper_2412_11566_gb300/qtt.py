"""Python binding of the C ABI in include/qtt_homog.h (argument marshalling
only; every step runs in the CUDA library).

Device memory for a context is one torch uint8 tensor handed to the library
as its workspace; the context's work is ordered on a torch CUDA stream. TT and
operator cores cross the boundary as lists of complex128 numpy arrays: a TT
core has shape (r_{k-1}, d_k, r_k); an operator core (a_{k-1}, d_out, d_in,
a_k), or (a_{k-1}, d, a_k) when raised-diagonal.

Importing this module loads ``libqtt_homog.so`` from the package directory and
raises ImportError if it has not been built (``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqtt_homog.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "qtt_homog.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
lib = C.CDLL(LIB_PATH)

QTT_OK, QTT_EINVAL, QTT_ENOMEM, QTT_ECUDA, QTT_ENAN, QTT_ETIMEOUT = 0, -1, -2, -3, -4, -5
QTT_WRANKCAP, QTT_WNOCONV = 1, 2
QTT_FP64, QTT_FP32 = 0, 1
QTT_CONTRACT_SIMT, QTT_CONTRACT_TF32X3, QTT_CONTRACT_TC = 0, 1, 2
QTT_FACTOR_NATIVE, QTT_FACTOR_FP64, QTT_FACTOR_FP64_ROUNDING = 0, 1, 2
(QTT_SCHEME_DIRECT, QTT_SCHEME_CENTERED, QTT_SCHEME_FORWARD, QTT_SCHEME_BACKWARD,
 QTT_SCHEME_HEX8R, QTT_SCHEME_STAGGERED) = range(6)
MAXC = 64

_p = C.c_void_p
_i = C.c_int
_d = C.c_double
_ip = C.POINTER(C.c_int)
_dp = C.POINTER(C.c_double)


class SolveParams(C.Structure):
    _fields_ = [("tol", _d), ("max_iter", _i), ("eps_tt", _d), ("rmax", _i), ("scheme", _i),
                ("oversample", _i)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", _i), ("residual", _d), ("max_rank", _i), ("rank_cap_hit", _i),
                ("imag_leak", _d), ("ms", _d)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def _sig(name, res, args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("qtt_ctx_create", _i, [C.POINTER(_p), _i, _p, _i, _p, C.c_size_t, C.c_uint64])
_sig("qtt_ctx_destroy", None, [_p])
_sig("qtt_last_error", C.c_char_p, [_p])
_sig("qtt_ctx_bytes_in_use", C.c_size_t, [_p])
_sig("qtt_ctx_bytes_peak", C.c_size_t, [_p])
_sig("qtt_ctx_launches", C.c_uint64, [_p])
_sig("qtt_ctx_set_profiling", _i, [_p, _i])
_sig("qtt_ctx_profile", _i, [_p, _i, _dp])
_sig("qtt_tt_create", _i, [_p, _i, _ip, _ip, _dp, C.POINTER(_p)])
_sig("qtt_tt_from_dense", _i, [_p, _i, _ip, _dp, _d, _i, C.POINTER(_p)])
_sig("qtt_tt_shape", _i, [_p, _ip, _ip, _ip])
_sig("qtt_tt_export", _i, [_p, _p, _dp])
_sig("qtt_tt_to_dense", _i, [_p, _p, _dp])
_sig("qtt_tt_free", None, [_p])
_sig("qtt_op_create", _i, [_p, _i, _ip, _ip, _ip, _ip, _dp, C.POINTER(_p)])
_sig("qtt_op_shape", _i, [_p, _ip, _ip, _ip, _ip, _ip])
_sig("qtt_op_export", _i, [_p, _p, _dp])
_sig("qtt_op_free", None, [_p])
_sig("qtt_from_phase_field", _i, [_p, C.POINTER(C.c_uint8), _ip, _i, _i, _dp, _dp, _dp, _d, _i,
                                   C.POINTER(_p)])
_sig("qtt_sfft_operator", _i, [_p, _i, _i, _d, C.POINTER(_p)])
_sig("qtt_rank_estimate", _i, [_p, C.POINTER(C.c_uint8), _ip, C.POINTER(C.c_uint8), _ip, _i, _i,
                               _dp, _dp, _d, _i, _dp])
_sig("qtt_gamma_operator", _i, [_p, _i, _d, _d, _i, _d, _i, C.POINTER(_p)])
_sig("qtt_op_apply", _i, [_p, _p, _p, _d, _i, _i, _i, C.POINTER(_p)])
_sig("sfft_apply", _i, [_p, _p, _d, _i, C.POINTER(_p)])
_sig("isfft_apply", _i, [_p, _p, _d, _i, C.POINTER(_p)])
_sig("gamma0_apply", _i, [_p, _ip, _d, _d, _i, _p, _d, _i, C.POINTER(_p)])
_sig("tt_round", _i, [_p, _p, _d, _i])
_sig("qtt_tt_dot", _i, [_p, _p, _p, _dp, _dp])
_sig("qtt_op_mean_apply", _i, [_p, _p, _p, _dp])
_sig("qtt_tt_dot_noalloc", _i, [_p, _p, _p, _dp, _dp])
_sig("qtt_from_phase_matrices", _i, [_p, C.POINTER(C.c_uint8), _ip, _i, _i, _dp, _d, _i,
                                      C.POINTER(_p)])
_sig("qtt_op_sandwich_mean", _i, [_p, _p, _p, _p, _dp, _dp])
_sig("ls_solve_ceff_grad", _i, [_p, _p, C.POINTER(C.c_uint8), _ip, _i, _dp, _dp, _i, _ip, _ip,
                                 C.POINTER(SolveParams), _dp, _dp, C.POINTER(SolveInfo)])
_sig("ls_solve_ops", _i, [_p, _p, _p, _p, _p, _dp, _dp, C.POINTER(SolveParams), _dp,
                          C.POINTER(SolveInfo)])
_sig("ls_solve", _i, [_p, _p, _dp, C.POINTER(SolveParams), _dp, C.POINTER(SolveInfo)])
_sig("qtt_ctx_set_concurrency", _i, [_p, _i])
_sig("qtt_ctx_set_jacobi", _i, [_p, _d, _i])
_sig("qtt_ctx_set_tt_svd", _i, [_p, _d])
_sig("qtt_ctx_set_contraction", _i, [_p, _i])
_sig("qtt_ctx_set_factorization", _i, [_p, _i])
_sig("qtt_ctx_set_svd", _i, [_p, _i, _i])
_sig("qtt_ctx_set_green_broadcast", _i, [_p, _i])
_sig("qtt_sfft_mpo_zipup", _i, [_i, _d, C.POINTER(_i), _dp, C.c_size_t, C.POINTER(C.c_size_t)])
_sig("qtt_contraction_bench", _i, [_p, _i, _i, _i, _i, _i, _dp, _dp])
_sig("ls_solve_ceff", _i, [_p, _p, C.POINTER(SolveParams), _ip, _i, _dp, C.POINTER(SolveInfo)])
_sig("ls_solve_batched", _i, [_p, _i, C.POINTER(_p), C.POINTER(SolveParams), _dp,
                             C.POINTER(SolveInfo)])
_sig("ls_solve_jobs", _i, [_p, _i, C.POINTER(_p), _ip, C.POINTER(SolveParams), _dp,
                          C.POINTER(SolveInfo)])


def header_functions(path: str = HEADER):
    """Names of the functions declared in the C header."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b([a-z_][a-z0-9_]*)\s*\(",
                                 txt, flags=re.M)) - {"if", "while", "for", "return"})


class QttError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"qtt error {code}: {msg}")
        self.code = code


def _ints(v):
    a = (C.c_int * max(1, len(v)))(*[int(x) for x in v])
    return a


def _cplx_flat(cores):
    return np.ascontiguousarray(np.concatenate(
        [np.asarray(c, dtype=np.complex128).reshape(-1) for c in cores]).view(np.float64))


class Context:
    """A library context on a CUDA device with a torch-allocated workspace."""

    def __init__(self, device: int = 0, precision: int = QTT_FP64, workspace_bytes: int = 1 << 30,
                 seed: int = 2412, stream=None):
        import torch
        self.torch = torch
        self.device = device
        self.precision = precision
        self.seed = seed
        self.ws = torch.empty(int(workspace_bytes), dtype=torch.uint8, device=f"cuda:{device}")
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = _p()
        rc = lib.qtt_ctx_create(C.byref(h), device, _p(self.stream.cuda_stream), precision,
                                _p(self.ws.data_ptr()), int(workspace_bytes), C.c_uint64(seed))
        if rc != 0:
            raise QttError(rc, "qtt_ctx_create failed")
        self.h = h

    def check(self, rc, allow_warn=True):
        if rc < 0 or (rc > 0 and not allow_warn):
            raise QttError(rc, lib.qtt_last_error(self.h).decode())
        return rc

    def close(self):
        """Destroy the context; handles still alive become inert (their
        device memory went with the workspace)."""
        if getattr(self, "h", None):
            lib.qtt_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bytes_in_use(self):
        return lib.qtt_ctx_bytes_in_use(self.h)

    def bytes_peak(self):
        return lib.qtt_ctx_bytes_peak(self.h)

    def launches(self):
        return lib.qtt_ctx_launches(self.h)

    def set_concurrency(self, loads: int):
        self.check(lib.qtt_ctx_set_concurrency(self.h, int(loads)))

    def set_jacobi(self, tol_scale: float = 1.0, max_sweeps_fp32: int = 40):
        self.check(lib.qtt_ctx_set_jacobi(self.h, float(tol_scale), int(max_sweeps_fp32)))

    def set_contraction(self, mode: int):
        """QTT_CONTRACT_SIMT, QTT_CONTRACT_TF32X3 or QTT_CONTRACT_TC (FP32 contexts)."""
        self.check(lib.qtt_ctx_set_contraction(self.h, int(mode)))

    def set_factorization(self, mode: int):
        """QTT_FACTOR_NATIVE or QTT_FACTOR_FP64 (FP32 contexts)."""
        self.check(lib.qtt_ctx_set_factorization(self.h, int(mode)))

    def set_green_broadcast(self, on: bool = True):
        """Plane Green operator for x1-broadcast stiffness operators (see
        qtt_ctx_set_green_broadcast)."""
        self.check(lib.qtt_ctx_set_green_broadcast(self.h, int(on)))

    def set_svd(self, precond: bool = True, refine_sweeps: int = 6):
        """FP64 SVD path for matrices beyond shared memory (see qtt_ctx_set_svd)."""
        self.check(lib.qtt_ctx_set_svd(self.h, int(precond), int(refine_sweeps)))

    def set_tt_svd(self, gram_threshold: float = 2e9):
        self.check(lib.qtt_ctx_set_tt_svd(self.h, float(gram_threshold)))

    def set_profiling(self, on: bool):
        self.check(lib.qtt_ctx_set_profiling(self.h, int(on)))

    def profile(self, reset: bool = False):
        """{class: (launches, total_ms, algorithmic_flops)} for gemm, qr, svd."""
        out = np.zeros(11)
        self.check(lib.qtt_ctx_profile(self.h, int(reset), out.ctypes.data_as(_dp)))
        d = {name: (int(out[3 * i]), float(out[3 * i + 1]), float(out[3 * i + 2]))
             for i, name in enumerate(("gemm", "qr", "svd"))}
        self.last_sweeps = float(out[9])
        self.last_tc_launches = int(out[10])
        return d

    # ------------------------------------------------------------ handles
    def tt(self, cores):
        dims = [c.shape[1] for c in cores]
        ranks = [c.shape[0] for c in cores] + [cores[-1].shape[2]]
        flat = _cplx_flat(cores)
        h = _p()
        self.check(lib.qtt_tt_create(self.h, len(cores), _ints(dims), _ints(ranks),
                                     flat.ctypes.data_as(_dp), C.byref(h)))
        return TT(self, h)

    def tt_from_dense(self, T, eps=0.0, rmax=1 << 30):
        """qtt_tt_from_dense: TT-SVD of a dense tensor on the device."""
        T = np.ascontiguousarray(T, dtype=np.complex128)
        flat = T.reshape(-1).view(np.float64)
        h = _p()
        self.check(lib.qtt_tt_from_dense(self.h, T.ndim, _ints(T.shape), flat.ctypes.data_as(_dp),
                                         eps, rmax, C.byref(h)))
        return TT(self, h)

    def op(self, cores, diag=None):
        L = len(cores)
        if diag is None:
            diag = [c.ndim == 3 for c in cores]
        dout = [c.shape[1] for c in cores]
        din = [c.shape[1] if dg else c.shape[2] for c, dg in zip(cores, diag)]
        ranks = [c.shape[0] for c in cores] + [cores[-1].shape[-1]]
        flat = _cplx_flat(cores)
        h = _p()
        self.check(lib.qtt_op_create(self.h, L, _ints(dout), _ints(din), _ints(ranks),
                                     _ints([int(d) for d in diag]), flat.ctypes.data_as(_dp),
                                     C.byref(h)))
        return Op(self, h)


class TT:
    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h

    def shape(self):
        L = C.c_int()
        dims = (C.c_int * MAXC)()
        ranks = (C.c_int * (MAXC + 1))()
        lib.qtt_tt_shape(self.h, C.byref(L), dims, ranks)
        return list(dims[:L.value]), list(ranks[:L.value + 1])

    def cores(self):
        dims, ranks = self.shape()
        tot = sum(ranks[k] * dims[k] * ranks[k + 1] for k in range(len(dims)))
        buf = np.empty(2 * tot, dtype=np.float64)
        self.ctx.check(lib.qtt_tt_export(self.ctx.h, self.h, buf.ctypes.data_as(_dp)))
        z = buf.view(np.complex128)
        out, off = [], 0
        for k in range(len(dims)):
            n = ranks[k] * dims[k] * ranks[k + 1]
            out.append(z[off:off + n].reshape(ranks[k], dims[k], ranks[k + 1]).copy())
            off += n
        return out

    def to_dense(self):
        """qtt_tt_to_dense: the full tensor (complex128, shape dims)."""
        dims, _ = self.shape()
        buf = np.empty(2 * int(np.prod(dims)), dtype=np.float64)
        self.ctx.check(lib.qtt_tt_to_dense(self.ctx.h, self.h, buf.ctypes.data_as(_dp)))
        return buf.view(np.complex128).reshape(dims)

    def free(self):
        if self.h and self.ctx.h:
            lib.qtt_tt_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Op:
    def __init__(self, ctx: Context, h, owned: bool = True):
        self.ctx, self.h, self.owned = ctx, h, owned

    def shape(self):
        L = C.c_int()
        a = [(C.c_int * (MAXC + 1))() for _ in range(4)]
        lib.qtt_op_shape(self.h, C.byref(L), a[0], a[1], a[2], a[3])
        n = L.value
        return list(a[0][:n]), list(a[1][:n]), list(a[2][:n + 1]), list(a[3][:n])

    def cores(self):
        dout, din, ranks, diag = self.shape()
        sizes = [ranks[k] * dout[k] * (1 if diag[k] else din[k]) * ranks[k + 1]
                 for k in range(len(dout))]
        buf = np.empty(2 * sum(sizes), dtype=np.float64)
        self.ctx.check(lib.qtt_op_export(self.ctx.h, self.h, buf.ctypes.data_as(_dp)))
        z = buf.view(np.complex128)
        out, off = [], 0
        for k, n in enumerate(sizes):
            shp = ((ranks[k], dout[k], ranks[k + 1]) if diag[k]
                   else (ranks[k], dout[k], din[k], ranks[k + 1]))
            out.append(z[off:off + n].reshape(shp).copy())
            off += n
        return out

    def free(self):
        if self.h and self.owned and self.ctx.h:
            lib.qtt_op_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------- entry points (C names)

def qtt_from_phase_field(ctx: Context, phase, n, E, nu, lame0=None, eps_tt=1e-6, rmax=1 << 30):
    ph = np.ascontiguousarray(phase, dtype=np.uint8)
    shape = list(ph.shape)
    # contiguous copies: a strided view's .ctypes pointer would skip entries
    Ea = np.ascontiguousarray(E, dtype=np.float64)
    nua = np.ascontiguousarray(nu, dtype=np.float64)
    l0 = None if lame0 is None else np.ascontiguousarray(lame0, dtype=np.float64)
    h = _p()
    ctx.check(lib.qtt_from_phase_field(ctx.h, ph.ctypes.data_as(C.POINTER(C.c_uint8)),
                                       _ints(shape), n, len(Ea), Ea.ctypes.data_as(_dp),
                                       nua.ctypes.data_as(_dp),
                                       None if l0 is None else l0.ctypes.data_as(_dp),
                                       eps_tt, rmax, C.byref(h)))
    return Op(ctx, h)


def qtt_rank_estimate(ctx: Context, phase_a, phase_b, n, E, nu, eps_tt=1e-6, n_target=None):
    """Applicability estimate (Sec. 5.2): largest stiffness-TTO rank of the same
    geometry at 2^n (phase_a) and 2^(n+1) (phase_b), the growth factor per
    order and the rank extrapolated to 2^n_target. Returns a dict."""
    a = np.ascontiguousarray(phase_a, dtype=np.uint8)
    b = np.ascontiguousarray(phase_b, dtype=np.uint8)
    Ea = np.ascontiguousarray(E, dtype=np.float64)
    nua = np.ascontiguousarray(nu, dtype=np.float64)
    out = np.zeros(4)
    nt = n + 1 if n_target is None else n_target
    ctx.check(lib.qtt_rank_estimate(ctx.h, a.ctypes.data_as(C.POINTER(C.c_uint8)),
                                    _ints(list(a.shape)), b.ctypes.data_as(C.POINTER(C.c_uint8)),
                                    _ints(list(b.shape)), n, len(Ea), Ea.ctypes.data_as(_dp),
                                    nua.ctypes.data_as(_dp), eps_tt, nt, out.ctypes.data_as(_dp)))
    return {"rank_n": int(out[0]), "rank_n1": int(out[1]), "growth": float(out[2]),
            "rank_target": float(out[3]), "n_target": nt}


def qtt_sfft_mpo_zipup(n, eps=1e-12):
    """The SFFT MPO of one axis from the QFT circuit by zip-up (host, no GPU):
    a list of complex cores (r, 2, 2, r')."""
    ranks = (_i * (n + 1))()
    need = C.c_size_t()
    rc = lib.qtt_sfft_mpo_zipup(int(n), float(eps), ranks, None, 0, C.byref(need))
    if rc != QTT_EINVAL or need.value == 0:
        raise QttError(rc, "qtt_sfft_mpo_zipup: sizing call failed")
    buf = np.empty(need.value, dtype=np.float64)
    rc = lib.qtt_sfft_mpo_zipup(int(n), float(eps), ranks, buf.ctypes.data_as(_dp), buf.size,
                                C.byref(need))
    if rc != QTT_OK:
        raise QttError(rc, "qtt_sfft_mpo_zipup failed")
    z = buf.view(np.complex128)
    out, off = [], 0
    for k in range(n):
        cnt = ranks[k] * 4 * ranks[k + 1]
        out.append(z[off:off + cnt].reshape(ranks[k], 2, 2, ranks[k + 1]).copy())
        off += cnt
    return out


def qtt_sfft_operator(ctx: Context, n, adjoint=False, eps=1e-14):
    h = _p()
    ctx.check(lib.qtt_sfft_operator(ctx.h, n, int(adjoint), eps, C.byref(h)))
    return Op(ctx, h)


def qtt_gamma_operator(ctx: Context, n, lam0, mu0, scheme=0, eps_tt=1e-6, rmax=1 << 30):
    h = _p()
    ctx.check(lib.qtt_gamma_operator(ctx.h, n, lam0, mu0, scheme, eps_tt, rmax, C.byref(h)))
    return Op(ctx, h)


def qtt_op_apply(ctx: Context, op: Op, x: TT, eps_tt, rmax, oversample=16, apply_id=0):
    h = _p()
    rc = ctx.check(lib.qtt_op_apply(ctx.h, op.h, x.h, eps_tt, rmax, oversample, apply_id,
                                    C.byref(h)))
    return TT(ctx, h), rc


def sfft_apply(ctx: Context, x: TT, eps_tt, rmax):
    h = _p()
    rc = ctx.check(lib.sfft_apply(ctx.h, x.h, eps_tt, rmax, C.byref(h)))
    return TT(ctx, h), rc


def isfft_apply(ctx: Context, x: TT, eps_tt, rmax):
    h = _p()
    rc = ctx.check(lib.isfft_apply(ctx.h, x.h, eps_tt, rmax, C.byref(h)))
    return TT(ctx, h), rc


def gamma0_apply(ctx: Context, n, lam0, mu0, x: TT, eps_tt, rmax, scheme=0):
    h = _p()
    rc = ctx.check(lib.gamma0_apply(ctx.h, _ints([n, n, n]), lam0, mu0, scheme, x.h, eps_tt, rmax,
                                    C.byref(h)))
    return TT(ctx, h), rc


def tt_round(ctx: Context, x: TT, eps_tt, rmax):
    return ctx.check(lib.tt_round(ctx.h, x.h, eps_tt, rmax))


def qtt_tt_dot(ctx: Context, a: TT, b: TT) -> complex:
    re, im = C.c_double(), C.c_double()
    ctx.check(lib.qtt_tt_dot(ctx.h, a.h, b.h, C.byref(re), C.byref(im)))
    return complex(re.value, im.value)


def qtt_tt_dot_noalloc(ctx: Context, a: TT, b: TT, stream=None) -> complex:
    """<a, b> through the entry point that allocates nothing (ranks <= 64)."""
    re, im = C.c_double(), C.c_double()
    s = ctx.stream if stream is None else stream
    ctx.check(lib.qtt_tt_dot_noalloc(a.h, b.h, _p(s.cuda_stream), C.byref(re), C.byref(im)))
    return complex(re.value, im.value)


def qtt_op_mean_apply(ctx: Context, op: Op, x: TT):
    dout = op.shape()[0][0]
    buf = np.zeros(2 * dout)
    ctx.check(lib.qtt_op_mean_apply(ctx.h, op.h, x.h, buf.ctypes.data_as(_dp)))
    return buf.view(np.complex128).copy()


def solve_params(tol=1e-6, max_iter=5000, eps_tt=1e-8, rmax=64, scheme=0, oversample=16):
    return SolveParams(tol, max_iter, eps_tt, rmax, scheme, oversample)


def ls_solve_ops(ctx: Context, dC: Op, S: Op, Sh: Op, G: Op, C0, E_voigt, params: SolveParams):
    C0a = np.ascontiguousarray(C0, dtype=np.float64).reshape(36)
    Ea = np.ascontiguousarray(E_voigt, dtype=np.float64)
    sig = np.zeros(12)
    info = SolveInfo()
    rc = ctx.check(lib.ls_solve_ops(ctx.h, dC.h, S.h, Sh.h, G.h, C0a.ctypes.data_as(_dp),
                                    Ea.ctypes.data_as(_dp), C.byref(params),
                                    sig.ctypes.data_as(_dp), C.byref(info)))
    return sig.view(np.complex128).copy(), info.as_dict(), rc


def ls_solve(ctx: Context, dC: Op, E_voigt, params: SolveParams):
    Ea = np.ascontiguousarray(E_voigt, dtype=np.float64)
    sig = np.zeros(12)
    info = SolveInfo()
    rc = ctx.check(lib.ls_solve(ctx.h, dC.h, Ea.ctypes.data_as(_dp), C.byref(params),
                                sig.ctypes.data_as(_dp), C.byref(info)))
    return sig.view(np.complex128).copy(), info.as_dict(), rc


def ls_solve_ceff(ctx: Context, dC: Op, params: SolveParams, loads=None):
    loads = list(range(6)) if loads is None else list(loads)
    Ceff = np.zeros(36)
    infos = (SolveInfo * len(loads))()
    rc = ctx.check(lib.ls_solve_ceff(ctx.h, dC.h, C.byref(params), _ints(loads), len(loads),
                                     Ceff.ctypes.data_as(_dp), infos))
    return Ceff.reshape(6, 6).T.copy(), [i.as_dict() for i in infos], rc


PLANE_STRAIN_VOIGT = (1, 2, 3)   # 3D Voigt (22, 33, 23) = 2D (11, 22, 12) of the section (x2, x3)


def ls_solve_ceff_plane_strain(ctx: Context, phase2d, n, E, nu, params: SolveParams,
                               lame0=None, eps_tt=1e-8, rmax=1 << 30):
    """Plane-strain C_eff (3 x 3, Voigt (11, 22, 12) with engineering shear) of a
    2D section of 2^n x 2^n pixels (the paper's 2D experiments, Sec. 5; the
    3-component Voigt form of Sec. 2). For isotropic phases the plane-strain
    problem is the 3D problem of the section extruded along x1: on an x1-
    invariant field the Green operator has n_1 = 0, so the out-of-plane strain
    components stay exactly zero under in-plane loads and the in-plane block
    of the 3D C_eff is the 2D one. This call therefore uploads the section as
    a (1, 2^n, 2^n) grid whose x1 axis is broadcast (no binary cores for it),
    builds (C - C0) with qtt_from_phase_field and runs ls_solve_ceff for the
    three in-plane unit loads; it computes nothing itself. Returns
    (C 3 x 3, infos of the three loads, worst status)."""
    ph = np.asarray(phase2d)
    N = 1 << n
    if ph.shape != (N, N):
        raise ValueError(f"plane strain: phase must be ({N}, {N}), got {ph.shape}")
    dC = qtt_from_phase_field(ctx, ph.reshape(1, N, N), n, E, nu, lame0, eps_tt, rmax)
    try:
        C6, infos, rc = ls_solve_ceff(ctx, dC, params, loads=PLANE_STRAIN_VOIGT)
    finally:
        dC.free()
    idx = list(PLANE_STRAIN_VOIGT)
    return C6[np.ix_(idx, idx)].copy(), infos, rc


def ls_solve_batched(ctx: Context, dCs, params: SolveParams):
    """C_eff of several microstructures: returns (array (items, 6, 6), infos
    as a list of items lists of 6 dicts, worst status)."""
    dCs = list(dCs)
    hs = (_p * len(dCs))(*[d.h.value if isinstance(d.h, _p) else d.h for d in dCs])
    Ceff = np.zeros(36 * len(dCs))
    infos = (SolveInfo * (6 * len(dCs)))()
    rc = ctx.check(lib.ls_solve_batched(ctx.h, len(dCs), hs, C.byref(params),
                                        Ceff.ctypes.data_as(_dp), infos))
    C6 = Ceff.reshape(len(dCs), 6, 6).transpose(0, 2, 1).copy()
    inf = [[infos[6 * i + k].as_dict() for k in range(6)] for i in range(len(dCs))]
    return C6, inf, rc


def ls_solve_jobs(ctx: Context, dCs, loads, params: SolveParams):
    """Unit-load solves (dC[j], load[j]): returns (sigma_bar array (njobs, 6)
    complex, infos list, worst status)."""
    dCs = list(dCs)
    hs = (_p * len(dCs))(*[d.h.value if isinstance(d.h, _p) else d.h for d in dCs])
    sig = np.zeros(12 * len(dCs))
    infos = (SolveInfo * len(dCs))()
    rc = ctx.check(lib.ls_solve_jobs(ctx.h, len(dCs), hs, _ints(loads), C.byref(params),
                                     sig.ctypes.data_as(_dp), infos))
    return sig.view(np.complex128).reshape(len(dCs), 6).copy(), [i.as_dict() for i in infos], rc


def qtt_contraction_bench(ctx: Context, mode: int, M: int, N: int, K: int, reps: int = 10):
    """(ms per launch, relative error vs FP64) of one complex M x N x K contraction."""
    ms, err = C.c_double(), C.c_double()
    ctx.check(lib.qtt_contraction_bench(ctx.h, int(mode), int(M), int(N), int(K), int(reps),
                                        C.byref(ms), C.byref(err)))
    return ms.value, err.value


def qtt_from_phase_matrices(ctx: Context, phase, n, mats, eps_tt=1e-6, rmax=1 << 30):
    ph = np.ascontiguousarray(phase, dtype=np.uint8)
    M = np.ascontiguousarray(np.asarray(mats, dtype=np.float64).reshape(-1, 36))
    h = _p()
    ctx.check(lib.qtt_from_phase_matrices(ctx.h, ph.ctypes.data_as(C.POINTER(C.c_uint8)),
                                          _ints(list(ph.shape)), n, M.shape[0],
                                          M.ctypes.data_as(_dp), eps_tt, rmax, C.byref(h)))
    return Op(ctx, h)


def qtt_op_sandwich_mean(ctx: Context, op: Op, y: TT, x: TT) -> complex:
    re, im = C.c_double(), C.c_double()
    ctx.check(lib.qtt_op_sandwich_mean(ctx.h, op.h, y.h, x.h, C.byref(re), C.byref(im)))
    return complex(re.value, im.value)


PARAM_E, PARAM_NU = 0, 1


def ls_solve_ceff_grad(ctx: Context, dC: Op, phase, E, nu, params: SolveParams, wrt):
    """C_eff (6x6) and dC_eff/dp for p in wrt = [(phase index, 'E' | 'nu'), ...]."""
    ph = np.ascontiguousarray(phase, dtype=np.uint8)
    Ea = np.ascontiguousarray(E, dtype=np.float64)
    nua = np.ascontiguousarray(nu, dtype=np.float64)
    pp = [int(p) for p, _ in wrt]
    pk = [PARAM_E if k == "E" else PARAM_NU for _, k in wrt]
    Ceff = np.zeros(36)
    dC_ = np.zeros(36 * max(1, len(wrt)))
    infos = (SolveInfo * 6)()
    rc = ctx.check(lib.ls_solve_ceff_grad(ctx.h, dC.h, ph.ctypes.data_as(C.POINTER(C.c_uint8)),
                                          _ints(list(ph.shape)), len(Ea), Ea.ctypes.data_as(_dp),
                                          nua.ctypes.data_as(_dp), len(wrt), _ints(pp), _ints(pk),
                                          C.byref(params), Ceff.ctypes.data_as(_dp),
                                          dC_.ctypes.data_as(_dp), infos))
    grads = [dC_[36 * q:36 * (q + 1)].reshape(6, 6).T.copy() for q in range(len(wrt))]
    return Ceff.reshape(6, 6).T.copy(), grads, [i.as_dict() for i in infos], rc


def make_ceff_function(ctx: Context, phase, n, params: SolveParams, eps_op=1e-6, rmax_op=1 << 30):
    """torch.autograd.Function computing C_eff (6x6 float64 tensor) from the
    phase parameters (E_0, nu_0, E_1, nu_1, ...) of a fixed microstructure;
    backward contracts the kept forward strains with dC/dp on the device."""
    import torch

    class CeffFunction(torch.autograd.Function):
        @staticmethod
        def forward(fctx, theta):
            th = theta.detach().cpu().double().numpy()
            E, nu = th[0::2].tolist(), th[1::2].tolist()
            dC = qtt_from_phase_field(ctx, phase, n, E, nu, None, eps_op, rmax_op)
            wrt = [(p, k) for p in range(len(E)) for k in ("E", "nu")]
            C, grads, _, _ = ls_solve_ceff_grad(ctx, dC, phase, E, nu, params, wrt)
            dC.free()
            fctx.save_for_backward(torch.from_numpy(np.stack(grads)))
            return torch.from_numpy(C).to(theta.device)

        @staticmethod
        def backward(fctx, grad_out):
            (G,) = fctx.saved_tensors
            g = grad_out.detach().cpu().double()
            return (G * g.unsqueeze(0)).sum(dim=(1, 2)).to(grad_out.device)

    return CeffFunction
