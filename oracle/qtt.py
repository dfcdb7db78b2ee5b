"""Oracle B: the SFFT-based homogenisation scheme (Alg. 2) on quantised tensor
trains, in plain numpy fp64/complex128. Test infrastructure only (see
``oracle/__init__.py``).

Data model (Sec. 3, eq. (tt_format) and (tto_format); Sec. 4.3):
  * A TT is a list of cores; core k has shape (r_{k-1}, d_k, r_k), r_0 = r_L = 1.
  * A TTO is a list of cores of shape (a_{k-1}, d_out, d_in, a_k).
  * Controlled QTT (Sec. 4.3): core 0 is the Voigt core (d = 6); the 3n binary
    cores (d = 2) follow, grouped by axis x1, x2, x3, most significant bit
    first (eq. (binary_discretization)).
  * A raised TTO (eq. (tt_to_tto)) has binary cores G(a, i, j, b) = C(a, i, b) d_ij.

Steps follow the paper's order. Readings where the paper is garbled or silent:
  * Rounding threshold (eq. (rounding_condition_tt)): the per-bond truncation
    threshold is delta = eps ||x|| / sqrt(L - 1) (the printed 1/sqrt(1-n) is the
    square root of a negative number); a bond keeps the smallest rank whose
    discarded tail sum of squared singular values is <= delta^2, at least 1 and
    at most r_max ("<=" discards ties).
  * Matrix-vector product: the paper uses an AMEn-adapted product (App. B); this
    oracle provides the exact contraction (Table 2, "contract") and a
    randomized sketch-and-orthogonalise product (successive randomized
    compression), followed by rounding. Each right-to-left sketch environment
    is replaced by an orthonormal basis of its range before it enters the next
    one (orthonormal_range): the unnormalised environments are products of
    random cores whose condition number grows ~10x per core (6e6 after six
    cores at 16^3), which single precision cannot carry. Zip-up (SVD truncation on the fly without
    the right environment) was measured to lose 15-30 % of the product on the
    Green operator already at n = 3 and is not used.
  * SFFT: S = P_rev F+ per axis, F+[k, x] = N^-1/2 exp(+2 pi i k x / N), P_rev
    reverses the n output bits (the QFT without its swap network, Sec. 4.1). The
    MPO is obtained by TT-SVD of the dense matrix with core b carrying the pair
    (output bit b, input bit b); the paper's Zip-Up construction (Sec. 4.2) yields
    the same operator.
  * Momentum convention (Sec. 4.3): Gamma is evaluated on bit-reversed indices and
    conjugated: Gamma_S(k') = conj(Gamma(xi(rev k'))), xi in {-N/2+1, ..., N/2}.
"""
from __future__ import annotations

import math

import numpy as np

from . import dense, dense2d

# ------------------------------------------------------------------ helpers


def truncation_rank(s: np.ndarray, delta2: float, rmax: int):
    """Smallest k in [1, rmax] with sum_{i >= k} s_i^2 <= delta2 (s descending).
    Returns (k, cap_hit) where cap_hit says r_max cut more than delta2 allows."""
    s2 = np.asarray(s, dtype=np.float64) ** 2
    tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])  # tail[k] = sum_{i>=k}
    k = len(s2)
    for j in range(1, len(s2) + 1):
        if tail[j] <= delta2:
            k = j
            break
    k = max(1, k)
    cap_hit = k > rmax
    return min(k, rmax), cap_hit


def _svd(M):
    return np.linalg.svd(M, full_matrices=False)


def tt_ranks(cores):
    return [c.shape[0] for c in cores] + [cores[-1].shape[-1]]


# ------------------------------------------------------------------ TT basics


def tt_svd(T: np.ndarray, eps: float, rmax: int = 1 << 30):
    """TT-SVD of a dense tensor (Sec. 3 and App. D): sequential truncated SVDs
    of the unfoldings, left to right, with per-bond threshold eps||T||/sqrt(L-1)."""
    dims = T.shape
    L = len(dims)
    delta2 = (eps * np.linalg.norm(T)) ** 2 / max(L - 1, 1)
    cores = []
    r = 1
    M = np.asarray(T).reshape(r * dims[0], -1)
    for k in range(L - 1):
        U, s, Vh = _svd(M)
        kk, _ = truncation_rank(s, delta2, rmax)
        cores.append(U[:, :kk].reshape(r, dims[k], kk))
        M = (s[:kk, None] * Vh[:kk]).reshape(kk * dims[k + 1], -1)
        r = kk
    cores.append(M.reshape(r, dims[-1], 1))
    return cores


def tt_svd_randomized(T: np.ndarray, eps: float, rmax: int = 1 << 30, oversample: int = 8,
                      seed: int = 0):
    """TT-SVD with randomized SVDs of the unfoldings (App. D: the preprocessing
    that scales to large grids), left to right. At each bond the unfolding M
    (P x c) is sketched as Y = M Omega with a Gaussian Omega of k + oversample
    columns; Q = orth(Y), and the SVD of the small Q^H M gives the bond. k starts
    at 8 and doubles until the discarded tail of Q^H M's spectrum plus the part
    of M outside range(Q) is within the per-bond threshold
    eps ||T|| / sqrt(L - 1) (or k reaches min(P, c)); then the rank is chosen
    by the tail rule and capped at rmax, as in tt_svd."""
    rng = np.random.default_rng(seed)
    dims = T.shape
    L = len(dims)
    delta2 = (eps * np.linalg.norm(T)) ** 2 / max(L - 1, 1)
    cores = []
    M = T.reshape(dims[0], -1).astype(np.complex128)
    r = 1
    for j in range(L - 1):
        M = M.reshape(r * dims[j], -1)
        P, c = M.shape
        k = min(8, P, c)
        while True:
            Om = rng.standard_normal((c, min(k + oversample, c))) \
                + 1j * rng.standard_normal((c, min(k + oversample, c)))
            Q, _ = np.linalg.qr(M @ Om)
            B = Q.conj().T @ M
            outside = np.linalg.norm(M - Q @ B) ** 2      # energy outside range(Q)
            U, S, Vh = _svd(B)
            kk, _ = truncation_rank(S, max(delta2 - outside, 0.0), rmax)
            if (outside <= 0.25 * delta2 and kk < Q.shape[1]) or k >= min(P, c):
                break
            k = min(2 * k, P, c)
        cores.append((Q @ U[:, :kk]).reshape(r, dims[j], kk))
        M = S[:kk, None] * Vh[:kk]
        r = kk
    cores.append(M.reshape(r, dims[-1], 1))
    return cores


def tt_full(cores) -> np.ndarray:
    """Dense tensor of a TT (eq. (tt_format))."""
    out = cores[0]
    for c in cores[1:]:
        out = np.tensordot(out, c, axes=([out.ndim - 1], [0]))
    return out.reshape(out.shape[1:-1])


def tt_dot(a, b) -> complex:
    """<a, b> = sum conj(a) b by a left-to-right transfer-matrix sweep."""
    E = np.ones((1, 1), dtype=np.complex128)
    for A, B in zip(a, b):
        # E'[p, q] = sum_{r, s, i} conj(A[r, i, p]) E[r, s] B[s, i, q]
        E = np.einsum("rip,rs,siq->pq", A.conj(), E, B)
    return complex(E[0, 0])


def left_orthogonalize(cores):
    """QR sweep left to right (Sec. 3, rounding: orthogonalisation). Returns the
    new cores (0..L-2 left-orthonormal) and the norm (= ||last core||_F)."""
    cores = [c.astype(np.complex128, copy=True) for c in cores]
    for k in range(len(cores) - 1):
        r0, d, r1 = cores[k].shape
        Q, R = np.linalg.qr(cores[k].reshape(r0 * d, r1))
        cores[k] = Q.reshape(r0, d, Q.shape[1])
        cores[k + 1] = np.tensordot(R, cores[k + 1], axes=([1], [0]))
    return cores, float(np.linalg.norm(cores[-1]))


def tt_norm(cores) -> float:
    """||x||_F via orthogonalisation (no cancellation for small differences)."""
    return left_orthogonalize(cores)[1]


def tt_round(cores, eps: float, rmax: int, assume_left_orth: bool = False):
    """TT rounding (Sec. 3, eq. (rounding_condition_tt)): left-to-right QR
    orthogonalisation, then a right-to-left sweep of truncated SVDs.
    Result is right-orthogonal (cores 1..L-1 have orthonormal rows).
    Returns (cores, cap_hit)."""
    if assume_left_orth:
        cores = [c.copy() for c in cores]
        nrm = float(np.linalg.norm(cores[-1]))
    else:
        cores, nrm = left_orthogonalize(cores)
    L = len(cores)
    delta2 = (eps * nrm) ** 2 / max(L - 1, 1)
    cap = False
    for k in range(L - 1, 0, -1):
        r0, d, r1 = cores[k].shape
        U, s, Vh = _svd(cores[k].reshape(r0, d * r1))
        kk, hit = truncation_rank(s, delta2, rmax)
        cap |= hit
        cores[k] = Vh[:kk].reshape(kk, d, r1)
        cores[k - 1] = np.tensordot(cores[k - 1], U[:, :kk] * s[:kk], axes=([2], [0]))
    return cores, cap


def tt_add(a, b, alpha=1.0, beta=1.0):
    """alpha a + beta b as a TT of rank r(a) + r(b) (Table 2, "x + y")."""
    L = len(a)
    out = []
    for k in range(L):
        A, B = a[k], b[k]
        if k == 0:
            out.append(np.concatenate([alpha * A, beta * B], axis=2))
        elif k == L - 1:
            out.append(np.concatenate([A, B], axis=0))
        else:
            ra0, d, ra1 = A.shape
            rb0, _, rb1 = B.shape
            C = np.zeros((ra0 + rb0, d, ra1 + rb1), dtype=np.complex128)
            C[:ra0, :, :ra1] = A
            C[ra0:, :, ra1:] = B
            out.append(C)
    return out


def tt_right_orthogonalize(cores):
    """LQ sweep right to left: cores 1..L-1 get orthonormal rows."""
    cores = [c.astype(np.complex128, copy=True) for c in cores]
    for k in range(len(cores) - 1, 0, -1):
        r0, d, r1 = cores[k].shape
        Q, R = np.linalg.qr(cores[k].reshape(r0, d * r1).conj().T)
        cores[k] = Q.conj().T.reshape(Q.shape[1], d, r1)
        cores[k - 1] = np.tensordot(cores[k - 1], R.conj().T, axes=([2], [0]))
    return cores


# ------------------------------------------------------------------ operators


def raise_tt(cores):
    """Raise a TT to a diagonal TTO, G(a, i, j, b) = C(a, i, b) delta_ij (eq. (tt_to_tto))."""
    out = []
    for C in cores:
        r0, d, r1 = C.shape
        G = np.zeros((r0, d, d, r1), dtype=np.complex128)
        for i in range(d):
            G[:, i, i, :] = C[:, i, :]
        out.append(G)
    return out


def tto_full(op) -> np.ndarray:
    """Dense matrix (prod d_out) x (prod d_in) of a TTO (eq. (tto_format))."""
    out = op[0]                                   # (1, o, i, a)
    for W in op[1:]:
        out = np.tensordot(out, W, axes=([out.ndim - 1], [0]))
    out = out.reshape(out.shape[1:-1])            # (o1, i1, o2, i2, ...)
    L = len(op)
    perm = [2 * k for k in range(L)] + [2 * k + 1 for k in range(L)]
    out = out.transpose(perm)
    do = int(np.prod([W.shape[1] for W in op]))
    di = int(np.prod([W.shape[2] for W in op]))
    return out.reshape(do, di)


def tto_adjoint(op):
    """A^H: swap the in/out legs of every core and conjugate."""
    return [W.transpose(0, 2, 1, 3).conj() for W in op]


def tto_apply_exact(op, x):
    """Exact matrix-vector product (Table 2, "contract"): cores
    Y_k[(a, s), i, (b, s')] = sum_j W_k[a, i, j, b] X_k[s, j, s'], rank r(A) r(x)."""
    out = []
    for W, X in zip(op, x):
        a0, do, di, a1 = W.shape
        s0, _, s1 = X.shape
        Y = np.einsum("aijb,sjt->asibt", W, X)
        out.append(Y.reshape(a0 * s0, do, a1 * s1))
    return out


# ---------------------------------------------------------------- random sketches

PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85
SKETCH_TAG = 0x5EC7C0DE
MASK32 = 0xFFFFFFFF


def philox4x32(ctr, key, rounds: int = 10):
    """Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
    "Parallel random numbers: as easy as 1, 2, 3", SC'11), vectorised over
    uint64 arrays holding 32-bit words. ctr: 4 arrays, key: 2 ints."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK32 for c in ctr)
    k0 = np.uint64(key[0] & MASK32)
    k1 = np.uint64(key[1] & MASK32)
    for _ in range(rounds):
        p0 = np.uint64(PHILOX_M0) * c0
        p1 = np.uint64(PHILOX_M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK32)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK32)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + np.uint64(PHILOX_W0)) & np.uint64(MASK32)
        k1 = (k1 + np.uint64(PHILOX_W1)) & np.uint64(MASK32)
    return c0, c1, c2, c3


def _u32_to_unit(x):
    """32-bit word -> (int32(x) + 1/2) * 2^-31, exactly representable, in (-1, 1)."""
    x = np.asarray(x, dtype=np.uint64).astype(np.int64)
    x = np.where(x >= (1 << 31), x - (1 << 32), x)
    return (x.astype(np.float64) + 0.5) * 2.0 ** -31


def sketch_core(seed: int, apply_id: int, core: int, shape):
    """Random complex sketch core of the given shape, entries with real and
    imaginary parts uniform in (-1, 1). Entry e (row-major flat index) of core
    `core` in product number `apply_id` uses Philox counter
    (e >> 1, core, apply_id, SKETCH_TAG) and key (seed low, seed high); even e
    takes words (0, 1), odd e words (2, 3) as (real, imaginary)."""
    size = int(np.prod(shape))
    e = np.arange(size, dtype=np.uint64)
    w = philox4x32((e >> np.uint64(1), np.full(size, core), np.full(size, apply_id),
                    np.full(size, SKETCH_TAG)), (seed & MASK32, (seed >> 32) & MASK32))
    odd = (e & np.uint64(1)).astype(bool)
    re = np.where(odd, w[2], w[0])
    im = np.where(odd, w[3], w[1])
    return (_u32_to_unit(re) + 1j * _u32_to_unit(im)).reshape(shape)


SKETCH_DROP_TAU = 1e-11  # relative Cholesky pivot below which a sketch column is dropped


def orthonormal_range(P: np.ndarray, tau: float = SKETCH_DROP_TAU):
    """Q = P M with orthonormal columns spanning range(P), followed by zero
    columns: Cholesky factorisation R^H R = Pi^T (P^H P) Pi with diagonal
    pivoting (step j takes the largest remaining diagonal entry, the first one
    on ties), stopped when that entry is at or below tau * max_i (P^H P)_ii;
    the k steps taken give Q[:, :k] = (P Pi)[:, :k] R^{-1} and Q[:, k:] = 0.
    Pivoting keeps R^{-1} bounded where columns of P are nearly dependent.
    Returns (Q, M)."""
    G = P.conj().T @ P
    L = G.shape[0]
    A = G.astype(np.complex128, copy=True)
    perm = np.arange(L)
    ref = float(np.max(np.real(np.diag(G)))) if L else 0.0
    k = 0
    for j in range(L):
        dia = np.real(np.diag(A))[j:]
        p = j + int(np.argmax(dia))
        if not dia[p - j] > tau * ref:
            break
        A[[j, p], :] = A[[p, j], :]
        A[:, [j, p]] = A[:, [p, j]]
        perm[[j, p]] = perm[[p, j]]
        d = float(np.real(A[j, j]))
        A[j, j] = math.sqrt(d)
        A[j, j + 1:] = A[j, j + 1:] / math.sqrt(d)
        A[j + 1:, j + 1:] -= np.outer(A[j, j + 1:].conj(), A[j, j + 1:])
        k = j + 1
    R = np.triu(A[:k, :k])
    Rinv = np.zeros((k, k), dtype=np.complex128)
    for j in range(k):
        e = np.zeros(k, dtype=np.complex128)
        e[j] = 1.0
        Rinv[:, j] = (e - Rinv[:, :j] @ R[:j, j]) / R[j, j]
    M = np.zeros((L, L), dtype=np.complex128)
    M[perm[:k], :k] = Rinv
    return P @ M, M


def sketch_ranks(op, x, ell: int):
    """Sketch bond sizes: min(ell, exact product rank, left and right grid dims)."""
    L = len(op)
    dims = [W.shape[1] for W in op]
    out = []
    for k in range(L - 1):
        left = int(np.prod(dims[:k + 1]))
        right = int(np.prod(dims[k + 1:]))
        out.append(min(ell, op[k].shape[3] * x[k].shape[2], left, right))
    return out


def tto_apply_sketched(op, x, ell: int, seed: int, apply_id: int):
    """Compressed matrix-vector product by successive randomized compression:
      1. right-to-left: sketch the exact product's right parts with a random TT
         Omega of ranks ell_k,  Psi_k[a, s, p] = sum W_k[a, o, i, b] X_k[s, i, t]
         Psi_{k+1}[b, t, q] Omega_k[p, o, q], each Psi_k then replaced by an
         orthonormal basis of its range (orthonormal_range);
      2. left-to-right: with carry C[r, a, s], form T[r, o, b, t] = sum C W_k X_k,
         Z = T Psi_{k+1} ((r o) x ell_k), Q = orth(Z) by Householder QR, keep Q as
         output core k and carry Q^H T.
    No truncation by tolerance happens here (the rounding that follows does it).
    Output cores 0..L-2 are left-orthonormal."""
    L = len(op)
    ells = sketch_ranks(op, x, ell)
    psi = [None] * (L + 1)
    psi[L] = np.ones((1, 1, 1), dtype=np.complex128)
    for k in range(L - 1, 0, -1):
        W, X = op[k], x[k]
        Om = sketch_core(seed, apply_id, k, (ells[k - 1], W.shape[1], 1 if k == L - 1 else ells[k]))
        # XP[s, i, b, q] = sum_t X[s, i, t] Psi[b, t, q]
        XP = np.einsum("sit,btq->sibq", X, psi[k + 1])
        # U[s, i, b, p] = sum_q XP[s, i, b, q] Om[p, o, q]  (o kept)  -> [s, i, b, o, p]
        U = np.einsum("sibq,poq->sibop", XP, Om)
        P = np.einsum("aoib,sibop->asp", W, U)
        Q, _ = orthonormal_range(P.reshape(-1, P.shape[2]))
        psi[k] = Q.reshape(P.shape)
    C = np.ones((1, 1, 1), dtype=np.complex128)
    out = []
    for k in range(L):
        W, X = op[k], x[k]
        CX = np.einsum("ras,sjt->rajt", C, X)
        T = np.einsum("rajt,aojb->robt", CX, W)
        r, do, a1, s1 = T.shape
        if k == L - 1:
            out.append(T.reshape(r, do, a1 * s1))
            break
        Z = np.einsum("robt,btp->rop", T, psi[k + 1]).reshape(r * do, -1)
        Q, Rz = np.linalg.qr(Z)
        # a dropped sketch direction is an exactly zero column of Z, and a
        # residual column at the rounding-noise floor (|R_jj|^2 <= eps^2
        # ||Z||_F^2) carries nothing either; the QR's direction for such a
        # column is arbitrary and is removed
        dead = np.abs(np.diag(Rz)) ** 2 <= (2.220446049250313e-16 ** 2) * np.vdot(Z, Z).real
        Q[:, dead] = 0
        out.append(Q.reshape(r, do, Q.shape[1]))
        C = np.einsum("mr,rbt->mbt", Q.conj().T, T.reshape(r * do, a1, s1))
    return out


def tto_apply_amen(op, x, eps: float, rmax: int = 1 << 30, y0=None, kick: int = 4,
                   sweeps: int = 20, seed: int = 0, tol_change: float = None):
    """Compressed product y ~ A x by the AMEn-adapted scheme of App. B.

    y minimises ||y - A x|| core by core. With the other cores of y orthonormal
    (left of core k and right of it), the local minimiser is the Galerkin
    projection y_k = Y_{<k}^H (A x) Y_{>k}^H, formed from left and right
    environments of the projections of A x onto y's frames. After each local
    update the core is truncated (SVD at eps / sqrt(L - 1), rank cap rmax) and
    enriched: an approximate residual z ~ A x - y, a TT of rank `kick` kept
    up to date by the same projections onto its own frames, gives the
    residual projected onto y's left frame and z's right frame; these columns
    are appended to the core, a QR re-orthonormalises it, and the remainder
    moves into core k + 1 (the Galerkin correction that adapts the rank).
    Sweeps go left to right, each preceded by a right orthogonalisation of y
    and z, until the relative change of y between two sweeps is below
    tol_change (eps by default). Ends with a TT rounding at (eps, rmax).
    Returns (y, sweeps done). op: cores (a, o, i, a'); x: cores (s, i, t)."""
    L = len(op)
    rng = np.random.default_rng(seed)
    dims = [W.shape[1] for W in op]
    tol_change = eps if tol_change is None else tol_change

    def rand_tt(r):
        rk = [1] + [r] * (L - 1) + [1]
        return [(rng.standard_normal((rk[k], dims[k], rk[k + 1]))
                 + 1j * rng.standard_normal((rk[k], dims[k], rk[k + 1]))) for k in range(L)]

    y = [c.astype(np.complex128) for c in (rand_tt(2) if y0 is None else y0)]
    z = rand_tt(kick)
    d2 = 1.0 / max(L - 1, 1)
    td = np.tensordot

    # The contractions below take x's core, then A's core, then the frame's:
    # the rank r(A) r(x) product core is never formed.
    def right_env(F, W, X, R):
        """sum conj(F[p, o, u]) W[a, o, i, b] X[s, i, t] R[u, b, t] -> [p, a, s]"""
        A2 = td(td(X, R, axes=([2], [2])), W, axes=([1, 3], [2, 3]))    # (s, u, a, o)
        return td(F.conj(), A2, axes=([1, 2], [3, 1])).transpose(0, 2, 1)

    def left_apply(Lenv, W, X):
        """sum Lenv[p, a, s] W[a, o, i, b] X[s, i, t] -> [p, o, b, t]"""
        C2 = td(td(Lenv, X, axes=([2], [0])), W, axes=([1, 2], [0, 2]))  # (p, t, o, b)
        return C2.transpose(0, 2, 3, 1)

    def frame_overlap_right(Z, Y, R):
        """sum conj(Z[q, o, v]) Y[p, o, u] R[v, u] -> [q, p]"""
        return td(Z.conj(), td(Y, R, axes=([2], [1])), axes=([1, 2], [1, 2]))

    prev = None
    done = 0
    for sw in range(sweeps):
        y = tt_right_orthogonalize(y)
        z = tt_right_orthogonalize(z)
        # right environments: projections of A x and of y onto the right frames
        Ry = [None] * (L + 1)
        Rz = [None] * (L + 1)
        Rzy = [None] * (L + 1)
        Ry[L] = np.ones((1, 1, 1), dtype=np.complex128)
        Rz[L] = np.ones((1, 1, 1), dtype=np.complex128)
        Rzy[L] = np.ones((1, 1), dtype=np.complex128)
        for k in range(L - 1, 0, -1):
            Ry[k] = right_env(y[k], op[k], x[k], Ry[k + 1])
            Rz[k] = right_env(z[k], op[k], x[k], Rz[k + 1])
            Rzy[k] = frame_overlap_right(z[k], y[k], Rzy[k + 1])
        Ly = np.ones((1, 1, 1), dtype=np.complex128)
        Lz = np.ones((1, 1, 1), dtype=np.complex128)
        Lzy = np.ones((1, 1), dtype=np.complex128)
        for k in range(L):
            W, X = op[k], x[k]
            LWX = left_apply(Ly, W, X)                                  # (p, o, b, t)
            yk = td(LWX, Ry[k + 1], axes=([2, 3], [1, 2]))              # Galerkin core
            if k == L - 1:
                y[k] = yk
                break
            p, o, u = yk.shape
            U, S, Vh = _svd(yk.reshape(p * o, u))
            nrm2 = float(np.sum(S ** 2))
            kk, _ = truncation_rank(S, eps * eps * nrm2 * d2, rmax)
            yt = ((U[:, :kk] * S[:kk]) @ Vh[:kk]).reshape(p, o, u)     # truncated core
            # residual z_k = proj_z(A x) - proj_z(y), then orthonormalised
            LzWX = left_apply(Lz, W, X)                                 # (q, o, b, t)
            zk = (td(LzWX, Rz[k + 1], axes=([2, 3], [1, 2]))
                  - td(td(Lzy, yt, axes=([1], [0])), Rzy[k + 1], axes=([2], [1])))
            qz, _ = np.linalg.qr(zk.reshape(-1, zk.shape[2]))
            z[k] = qz.reshape(zk.shape[0], o, qz.shape[1])
            # enrichment: the residual on y's left frame and z's right frame
            ek = (td(LWX, Rz[k + 1], axes=([2, 3], [1, 2]))
                  - td(yt, Rzy[k + 1], axes=([2], [1])))
            Q, _ = np.linalg.qr(np.concatenate([U[:, :kk], ek.reshape(p * o, -1)], axis=1))
            y[k] = Q.reshape(p, o, Q.shape[1])
            carry = Q.conj().T @ yt.reshape(p * o, u)                   # r_new x u
            y[k + 1] = td(carry, y[k + 1], axes=([1], [0]))
            # left environments with the new cores
            Ly = td(y[k].conj(), LWX, axes=([0, 1], [0, 1]))            # (x, b, t)
            Lz = td(z[k].conj(), LzWX, axes=([0, 1], [0, 1]))
            Lzy = td(z[k].conj(), td(Lzy, y[k], axes=([1], [0])), axes=([0, 1], [0, 1]))
        done = sw + 1
        if prev is not None:
            change = tt_norm(tt_add(y, prev, 1.0, -1.0)) / max(tt_norm(y), 1e-300)
            if change < tol_change:
                break
        prev = [c.copy() for c in y]
    y, _ = tt_round(y, eps, rmax)
    return y, done


def tto_sandwich_mean(op, x):
    """Mean over the grid of (A x) without forming A x: the binary cores are
    contracted with the averaging vector (1/2, 1/2). Returns the Voigt vector
    mean_x sum_J A[I, J](x) x[J](x) (Sec. 2, the C_eff average)."""
    W0, X0 = op[0], x[0]                         # (1, 6, 6, a1), (1, 6, s1)
    V = np.einsum("ijb,jt->ibt", W0[0], X0[0])   # (6, a1, s1)
    for W, X in zip(op[1:], x[1:]):
        # V'[I, b, t] = sum_{a, s, i, j} V[I, a, s] W[a, i, j, b] X[s, j, t] / 2
        V = 0.5 * np.einsum("Ias,aijb,sjt->Ibt", V, W, X)
    return V[:, 0, 0]


# ------------------------------------------------------------------ SFFT MPO


def bit_reverse(k: int, n: int) -> int:
    return int(format(k, f"0{n}b")[::-1], 2)


def sfft_dense(n: int) -> np.ndarray:
    """S = P_rev F+ on one axis: S[k', x] = N^-1/2 exp(2 pi i rev(k') x / N)."""
    N = 1 << n
    rev = np.array([bit_reverse(k, n) for k in range(N)])
    x = np.arange(N)
    return np.exp(2j * np.pi * np.outer(rev, x) / N) / math.sqrt(N)


def matrix_to_mpo(M: np.ndarray, n: int, eps: float, rmax: int = 1 << 30):
    """TT-SVD of a 2^n x 2^n matrix with core b carrying (out bit b, in bit b),
    MSB first. Returns cores (f, 2, 2, f')."""
    T = M.reshape((2,) * n + (2,) * n)
    perm = [v for b in range(n) for v in (b, n + b)]
    T = T.transpose(perm).reshape((4,) * n)
    cores = tt_svd(T, eps, rmax)
    return [c.reshape(c.shape[0], 2, 2, c.shape[2]) for c in cores]


def sfft_axis_mpo(n: int, eps: float = 1e-12):
    """The SFFT (reduced QFT) of one axis as an MPO (Sec. 4.1-4.2), by TT-SVD of
    the dense matrix. The default accuracy 1e-12 gives the circuit's own ranks
    (sfft_axis_mpo_zipup) with the DFT reproduced to ~1e-14; at 1e-14, the
    SVD's noise level, rounding-noise directions pass the threshold (n = 8:
    ranks up to 127 instead of 12)."""
    return matrix_to_mpo(sfft_dense(n), n, eps)


def qft_circuit_gates(n: int):
    """The reduced QFT circuit of Sec. 4.1 (Hadamard and controlled-phase gates,
    without the SWAP network) on n qubits, qubit b carrying bit b of the input
    index MSB first, as gate MPOs in the order they act: for qubit q, H on q,
    then cP(pi / 2^(m - q)) between q and every less significant qubit m > q.
    Each cP is split, as Sec. 4.2 describes, into a copy tensor on q (bond
    index = the bit of q) and a phase tensor on m (identity for bond 0,
    P(theta) for bond 1), with identity pass-through cores between them.
    Gate MPO cores have the layout (r, out, in, r')."""
    I2 = np.eye(2, dtype=np.complex128)
    H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)

    def single(q, U):
        g = [I2.reshape(1, 2, 2, 1) for _ in range(n)]
        g[q] = U.reshape(1, 2, 2, 1)
        return g

    def cphase(q, m, theta):
        g = [I2.reshape(1, 2, 2, 1) for _ in range(n)]
        copy = np.zeros((1, 2, 2, 2), dtype=np.complex128)
        for a in range(2):
            copy[0, a, a, a] = 1.0
        g[q] = copy
        for s in range(q + 1, m):
            w = np.zeros((2, 2, 2, 2), dtype=np.complex128)
            for a in range(2):
                w[a, :, :, a] = I2
            g[s] = w
        ph = np.zeros((2, 2, 2, 1), dtype=np.complex128)
        ph[0, :, :, 0] = I2
        ph[1, :, :, 0] = np.diag([1.0, np.exp(1j * theta)])
        g[m] = ph
        return g

    gates = []
    for q in range(n):
        gates.append(single(q, H))
        for m in range(q + 1, n):
            gates.append(cphase(q, m, math.pi / (1 << (m - q))))
    return gates


def mpo_zipup(G, W, eps: float):
    """G W (W acts first) by the zip-up sweep of Sec. 4.2: left to right, the
    carried factor is contracted with the site's two cores, the result is
    reshaped to (carried rank x out x in, bond of G x bond of W), split by an
    SVD truncated at relative accuracy eps, and the left factor is kept as the
    site's core while S V^H moves on to the next site."""
    n = len(W)
    carry = np.ones((1, 1, 1), dtype=np.complex128)       # (R, g, w)
    cores = []
    for b in range(n):
        T = np.einsum("Rgw,gomh,wmiv->Roihv", carry, G[b], W[b])
        R, o, i, h, v = T.shape
        if b == n - 1:
            cores.append(T.reshape(R, o, i, h * v))
            break
        U, S, Vh = np.linalg.svd(T.reshape(R * o * i, h * v), full_matrices=False)
        k = max(1, int(np.sum(S > eps * S[0]))) if S[0] > 0 else 1
        cores.append(U[:, :k].reshape(R, o, i, k))
        carry = (S[:k, None] * Vh[:k]).reshape(k, h, v)
    return cores


def sfft_axis_mpo_zipup(n: int, eps: float = 1e-14):
    """The SFFT MPO of one axis built the way Sec. 4.2 builds it: the reduced QFT
    circuit's gates applied one after the other to the identity MPO by zip-up
    sweeps, then one TT rounding at eps (the cores as a TT with mode size 4)
    to reach the minimal ranks."""
    I2 = np.eye(2, dtype=np.complex128)
    op = [I2.reshape(1, 2, 2, 1) for _ in range(n)]
    for g in qft_circuit_gates(n):
        op = mpo_zipup(g, op, 1e-15)
    flat = [c.reshape(c.shape[0], 4, c.shape[3]) for c in op]
    flat, _ = tt_round(flat, eps, 1 << 30)
    return [c.reshape(c.shape[0], 2, 2, c.shape[2]) for c in flat]


def sfft_operator(n: int, eps: float = 1e-12, adjoint: bool = False):
    """3D SFFT TTO on the controlled QTT: identity Voigt core, then the axis
    MPOs of x1, x2, x3 joined by rank-1 bonds (Sec. 4.3). adjoint -> S^H = S^-1."""
    ax = sfft_axis_mpo(n, eps)
    op = [np.eye(6, dtype=np.complex128).reshape(1, 6, 6, 1)] + ax + ax + ax
    return tto_adjoint(op) if adjoint else op


# ------------------------------------------------------------------ Green operator


def axis_frequencies_bitrev(n: int) -> np.ndarray:
    """xi(rev k') for k' = 0..N-1 with the paper's representatives
    {-N/2+1, ..., N/2} (App. A)."""
    N = 1 << n
    k = np.array([bit_reverse(kp, n) for kp in range(N)])
    return np.where(k <= N // 2, k, k - N).astype(np.float64)


def gamma_field_sfft(n: int, lam0: float, mu0: float, scheme: str = "direct") -> np.ndarray:
    """Dense Voigt Green field in the SFFT momentum convention (Sec. 4.3):
    G[I, J, k'1, k'2, k'3] = conj(Gamma_V[I, J](xi(rev k'1), xi(rev k'2), xi(rev k'3))),
    Nyquist-symmetrised as in App. A (see oracle.dense). Real for the Direct,
    Centered and Hex8R schemes; complex for Forward, Backward and the
    staggered grid, whose Gamma(-xi) = conj(Gamma(xi)) makes the conjugate the
    operator of the opposite transform sign."""
    f = axis_frequencies_bitrev(n)
    N = 1 << n
    out = np.empty((6, 6, N, N, N), dtype=np.complex128)
    X2, X3 = np.meshgrid(f, f, indexing="ij")
    for a in range(N):
        xi = np.stack([np.full_like(X2, f[a]), X2, X3], axis=-1)
        out[:, :, a] = np.moveaxis(dense.green_voigt_symmetrised(xi, lam0, mu0, N, scheme),
                                   (-2, -1),
                                   (0, 1))
    return np.conj(out)


def controlled_field_to_tto(F: np.ndarray, n: int, eps: float, rmax: int):
    """(6, 6, N, N, N) Voigt-matrix field -> raised TTO: TT-SVD of the
    (36, 2, ..., 2) tensor, Voigt core reshaped to (1, 6, 6, a1), binary cores raised."""
    T = F.reshape((36,) + (2,) * (3 * n))
    cores = tt_svd(T.astype(np.complex128), eps, rmax)
    c0 = cores[0].reshape(1, 6, 6, cores[0].shape[2])
    return [c0] + raise_tt(cores[1:])


def gamma_qtt(n: int, lam0: float, mu0: float, eps: float, rmax: int = 1 << 30,
              scheme: str = "direct"):
    """Gamma_hat^0 of a discretisation scheme (one of oracle.dense.SCHEMES, the
    App. A table) as a raised TTO in the SFFT momentum convention."""
    return controlled_field_to_tto(gamma_field_sfft(n, lam0, mu0, scheme), n, eps, rmax)


def gamma_qtt_plane(n: int, lam0: float, mu0: float, eps: float, rmax: int = 1 << 30,
                    scheme: str = "direct"):
    """Gamma_hat^0 restricted to the plane xi_1 = 0, tensored with the identity
    on the x1 cores: Voigt core and x2, x3 cores from the TT-SVD of the
    (6, 6, N, N) plane field (SFFT convention), then n identity cores
    delta(a, a') I_2 inserted after the Voigt core. On x1-invariant fields,
    whose SFFT lives at xi_1 = 0 only, it acts as gamma_qtt does (Sec. 4.3,
    broadcast axes)."""
    full = gamma_field_sfft(n, lam0, mu0, scheme)   # (6, 6, N1, N2, N3), N1 bit-reversed
    plane = full[:, :, 0]                             # rev(0) = 0: xi_1 = 0
    T = plane.reshape((36,) + (2,) * (2 * n))
    cores = tt_svd(T.astype(np.complex128), eps, rmax)
    c0 = cores[0].reshape(1, 6, 6, cores[0].shape[2])
    r1 = c0.shape[3]
    ident = np.einsum("ab,ij->aijb", np.eye(r1), np.eye(2)).astype(np.complex128)
    return [c0] + [ident.copy() for _ in range(n)] + raise_tt(cores[1:])


# ------------------------------------------------------------------ stiffness operator


def stiffness_qtt(phase: np.ndarray, n: int, E, nu, lame0, eps: float, rmax: int = 1 << 30):
    """(C(x) - C0) as a raised TTO (Sec. 4.3): the Voigt-matrix field
    sum_p (C_p - C0) chi_p(x) compressed by TT-SVD, Voigt core (1, 6, 6, a1)."""
    N = 1 << n
    ph = np.broadcast_to(phase, (N, N, N))
    C0 = dense.stiffness_voigt(*lame0)
    F = np.zeros((6, 6, N, N, N))
    for p, (e, v) in enumerate(zip(E, nu)):
        dC = dense.stiffness_voigt(*dense.lame(e, v)) - C0
        F += dC[:, :, None, None, None] * (ph == p)[None, None]
    return controlled_field_to_tto(F, n, eps, rmax)


def e_tt(n: int, E_voigt):
    """Rank-1 mean strain TT (Sec. 4.3): Voigt core E scaled by sqrt(2)^{3n},
    binary cores (1, 1)/sqrt(2) (right-orthonormal)."""
    c0 = (np.asarray(E_voigt, dtype=np.complex128) * math.sqrt(2.0) ** (3 * n)).reshape(1, 6, 1)
    b = np.full((1, 2, 1), 1.0 / math.sqrt(2.0), dtype=np.complex128)
    return [c0] + [b.copy() for _ in range(3 * n)]


def to_voigt_field(cores, n: int) -> np.ndarray:
    """Dense (6, N, N, N) field of a controlled QTT."""
    N = 1 << n
    return tt_full(cores).reshape(6, N, N, N)


# ------------------------------------------------------------------ Alg. 2


def ls_solve(dC, G, S, Sh, E_voigt, n: int, tol: float, eps: float, rmax: int,
             max_iter: int = 5000, oversample: int = 16, seed: int = 2412, lame0=None,
             e_field=None, c0=None):
    """Alg. 2 (SFFT-based homogenisation), one unit load:
        tau_m   = round((C - C0) eps_m)
        tauh_m  = round(S tau_m)
        epsh_m  = round(Gamma_hat tauh_m)
        eps_m+1 = round(E - S^-1 epsh_m)
    each product by randomized sketching with sketch rank rmax + oversample
    (product number 4 (m - 1) + j for the j-th product of iteration m), each
    rounding at (eps, rmax); stop when ||eps_m+1 - eps_m||_F / ||E||_F < tol.
    sigma_bar = C0 E + mean((C - C0) eps_final) (Sec. 2, C_eff paragraph).
    Returns dict(eps, sigma_bar, iters, history, max_rank, cap_hit).
    e_field / c0: the mean-strain TT and the reference Voigt stiffness for a
    Voigt form other than the 3D one (the 2D plane-strain operators below);
    by default e_tt(n, E_voigt) and the 3D stiffness of lame0."""
    Ett = e_tt(n, E_voigt) if e_field is None else e_field
    normE = tt_norm(Ett)
    ell = rmax + oversample
    x = Ett
    hist = []
    cap = False
    maxr = 1
    it = 0
    for it in range(1, max_iter + 1):
        t0 = 4 * (it - 1)
        tau, h1 = tt_round(tto_apply_sketched(dC, x, ell, seed, t0), eps, rmax, assume_left_orth=True)
        tauh, h2 = tt_round(tto_apply_sketched(S, tau, ell, seed, t0 + 1), eps, rmax,
                            assume_left_orth=True)
        epsh, h3 = tt_round(tto_apply_sketched(G, tauh, ell, seed, t0 + 2), eps, rmax,
                            assume_left_orth=True)
        y = tto_apply_sketched(Sh, epsh, ell, seed, t0 + 3)
        xn, h4 = tt_round(tt_add(Ett, y, 1.0, -1.0), eps, rmax)
        cap |= h1 | h2 | h3 | h4
        maxr = max(maxr, *tt_ranks(tau), *tt_ranks(tauh), *tt_ranks(epsh), *tt_ranks(xn))
        rel = tt_norm(tt_add(xn, x, 1.0, -1.0)) / normE
        hist.append(rel)
        x = xn
        if rel < tol:
            break
    sig = tto_sandwich_mean(dC, x)
    if c0 is not None:
        sig = sig + np.asarray(c0) @ np.asarray(E_voigt, dtype=np.float64)
    elif lame0 is not None:
        sig = sig + dense.stiffness_voigt(*lame0) @ np.asarray(E_voigt, dtype=np.float64)
    return dict(eps=x, sigma_bar=sig, iters=it, history=hist, max_rank=maxr, cap_hit=cap)


# ------------------------------------------------------------------ 2D (plane strain)
# The paper's 2D form (Sec. 2: 3-component Voigt vectors, 3 x 3 stiffness; a
# controlled QTT whose Voigt core has d = 3, Sec. 4.3) on a 2^n x 2^n grid:
# L = 2n + 1 cores, x1 bits then x2 bits, most significant first.


def _field_to_tto(F: np.ndarray, bits: int, eps: float, rmax: int):
    """(v, v, 2^bits...) Voigt-matrix field -> raised TTO with Voigt core (1, v, v, a1)."""
    v = F.shape[0]
    cores = tt_svd(F.reshape((v * v,) + (2,) * bits).astype(np.complex128), eps, rmax)
    c0 = cores[0].reshape(1, v, v, cores[0].shape[2])
    return [c0] + raise_tt(cores[1:])


def sfft_operator_2d(n: int, eps: float = 1e-12, adjoint: bool = False):
    """2D SFFT TTO: 3 x 3 identity Voigt core, then the axis MPO of x1 and x2."""
    ax = sfft_axis_mpo(n, eps)
    op = [np.eye(3, dtype=np.complex128).reshape(1, 3, 3, 1)] + ax + ax
    return tto_adjoint(op) if adjoint else op


def gamma_qtt_2d(n: int, lam0: float, mu0: float, eps: float, rmax: int = 1 << 30,
                 scheme: str = "direct"):
    """2D Green TTO in the SFFT convention: conj(Gamma_V) of oracle.dense2d at the
    bit-reversed frequencies, Nyquist rule included."""
    f = axis_frequencies_bitrev(n)
    X1, X2 = np.meshgrid(f, f, indexing="ij")
    G = dense2d.green2_symmetrised(np.stack([X1, X2], axis=-1), lam0, mu0, 1 << n, scheme)
    return _field_to_tto(np.conj(np.moveaxis(G, (-2, -1), (0, 1))), 2 * n, eps, rmax)


def stiffness_qtt_2d(phase: np.ndarray, n: int, E, nu, lame0, eps: float, rmax: int = 1 << 30):
    """(C(x) - C0) of a 2^n x 2^n section in plane strain as a raised TTO."""
    C0 = dense2d.stiffness_voigt2(*lame0)
    F = np.zeros((3, 3) + phase.shape)
    for p, (e, v) in enumerate(zip(E, nu)):
        F += (dense2d.stiffness_voigt2(*dense2d.lame(e, v)) - C0)[:, :, None, None] * (phase == p)
    return _field_to_tto(F, 2 * n, eps, rmax)


def e_tt_2d(n: int, E_voigt3):
    """Rank-1 mean strain TT in 2D: Voigt core E sqrt(2)^(2n), binary cores (1, 1)/sqrt(2)."""
    c0 = (np.asarray(E_voigt3, dtype=np.complex128) * math.sqrt(2.0) ** (2 * n)).reshape(1, 3, 1)
    b = np.full((1, 2, 1), 1.0 / math.sqrt(2.0), dtype=np.complex128)
    return [c0] + [b.copy() for _ in range(2 * n)]


def phase_matrices_qtt(phase: np.ndarray, n: int, mats, eps: float, rmax: int = 1 << 30):
    """Raised TTO of the Voigt-matrix field sum_p mats[p] [phase == p]."""
    N = 1 << n
    ph = np.broadcast_to(phase, (N, N, N))
    F = np.zeros((6, 6, N, N, N))
    for p, M in enumerate(mats):
        F += np.asarray(M)[:, :, None, None, None] * (ph == p)[None, None]
    return controlled_field_to_tto(F, n, eps, rmax)


def tto_sandwich_bilinear_mean(op, y, x):
    """mean over the grid of sum_{I,J} y_I(x) A[I, J](x) x_J(x) (bilinear, no
    conjugation), by a transfer sweep over the cores with the binary cores
    averaged by (1/2, 1/2)."""
    W0, X0, Y0 = op[0], x[0], y[0]
    # V[s, a, t] = sum_{I, J} Y0[0, I, s] W0[0, I, J, a] X0[0, J, t]
    V = np.einsum("Is,IJa,Jt->sat", Y0[0], W0[0], X0[0])
    for W, X, Y in zip(op[1:], x[1:], y[1:]):
        V = 0.5 * np.einsum("sat,sib,aijc,tjd->bcd", V, Y, W, X)
    return complex(V[0, 0, 0])
