"""Pins of Oracle B (the QTT/SFFT scheme, Alg. 2) against what the paper and
the mathematics fix: exact TT round trips, the rounding error bound, the
raised-TTO/Hadamard identity (App. C), the product rank (Table 2), the SFFT as
a bit-reversed unitary DFT and its printed MPO rank, the momentum-space
convention (the QTT pipeline equals the dense FFT pipeline), the Philox
known-answer vectors, and cross-checks of the two oracles."""
import json
import os

import numpy as np
import pytest

from oracle import dense, qtt as oq
from paper_2412_11566_gb300 import synth
from tests._helpers import random_tt

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_tt_svd_roundtrip_exact():
    rng = np.random.default_rng(0)
    T = rng.standard_normal((6, 2, 2, 2, 2, 2)) + 1j * rng.standard_normal((6, 2, 2, 2, 2, 2))
    cores = oq.tt_svd(T, 0.0)
    assert rel(oq.tt_full(cores), T) < 1e-14
    # full ranks of a random tensor
    assert oq.tt_ranks(cores) == [1, 6, 12, 8, 4, 2, 1]


@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-6])
def test_rounding_error_bound(eps):
    rng = np.random.default_rng(1)
    x = random_tt(rng, [6, 2, 2, 2, 2, 2, 2], [1, 5, 8, 9, 8, 6, 3, 1])
    full = oq.tt_full(x)
    y, cap = oq.tt_round(x, eps, 1000)
    assert not cap
    assert rel(oq.tt_full(y), full) <= eps * (1 + 1e-10)
    # result is right-orthogonal
    for c in y[1:]:
        M = c.reshape(c.shape[0], -1)
        assert np.allclose(M @ M.conj().T, np.eye(M.shape[0]), atol=1e-12)
    # rounding of an exact low-rank TT with redundant rank is lossless
    z, _ = oq.tt_round(oq.tt_add(x, x, 1.0, 1.0), 1e-12, 1000)
    assert rel(oq.tt_full(z), 2 * full) < 1e-12
    assert oq.tt_ranks(z) == oq.tt_ranks(oq.tt_round(x, 1e-12, 1000)[0])


def test_rank_cap_flag():
    rng = np.random.default_rng(2)
    x = random_tt(rng, [6, 2, 2, 2, 2], [1, 6, 10, 4, 2, 1])
    y, cap = oq.tt_round(x, 1e-12, 3)
    assert cap and max(oq.tt_ranks(y)) == 3


def test_raised_tto_is_hadamard():
    """App. C: contracting the raised TTO of a with b gives a (.) b."""
    rng = np.random.default_rng(3)
    dims = [2, 2, 2, 2, 2]
    a = random_tt(rng, dims, [1, 2, 3, 3, 2, 1])
    b = random_tt(rng, dims, [1, 3, 2, 4, 2, 1])
    c = oq.tto_apply_exact(oq.raise_tt(a), b)
    assert rel(oq.tt_full(c), oq.tt_full(a) * oq.tt_full(b)) < 1e-14
    # Table 2: exact product rank r(A) r(x)
    assert oq.tt_ranks(c) == [ra * rb for ra, rb in zip(oq.tt_ranks(a), oq.tt_ranks(b))]


def test_exact_product_equals_dense_matvec():
    rng = np.random.default_rng(4)
    op = [rng.standard_normal(s) + 1j * rng.standard_normal(s)
          for s in [(1, 3, 2, 2), (2, 2, 3, 3), (3, 2, 2, 1)]]
    x = random_tt(rng, [2, 3, 2], [1, 2, 2, 1])
    y = oq.tto_apply_exact(op, x)
    assert rel(oq.tt_full(y).reshape(-1), oq.tto_full(op) @ oq.tt_full(x).reshape(-1)) < 1e-14


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_sfft_is_bit_reversed_unitary_dft(n):
    """S = P_rev F+ (Sec. 4.1): bit-reversed output of the +i DFT, unitary."""
    N = 1 << n
    S = oq.sfft_dense(n)
    rng = np.random.default_rng(n)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    rev = [oq.bit_reverse(k, n) for k in range(N)]
    assert np.allclose(S @ x, (np.fft.ifft(x) * np.sqrt(N))[rev], atol=1e-12)
    assert np.allclose(S.conj().T @ S, np.eye(N), atol=1e-12)
    mpo = oq.sfft_axis_mpo(n, 1e-14)
    assert np.allclose(oq.tto_full(mpo), S, atol=1e-12)


def test_sfft_mpo_rank_printed_value():
    """The (I)SFFT TTO rank converges to 10 for n >= 8 at accuracy 1e-10."""
    g = json.load(open(os.path.join(GOLD, "paper_values.json")))["sfft_mpo_rank"]
    for n in (8, 9):
        mpo = oq.sfft_axis_mpo(n, g["delta_acc"])
        assert max(c.shape[0] for c in mpo) == g["value"]
    # the full QFT (with the reordering) is not low rank: the reduced form matters
    n = 8
    N = 1 << n
    full_dft = np.exp(2j * np.pi * np.outer(np.arange(N), np.arange(N)) / N) / np.sqrt(N)
    assert max(c.shape[0] for c in oq.matrix_to_mpo(full_dft, n, 1e-10)) > 2 * g["value"]


@pytest.mark.parametrize("n", [1, 2, 4, 6, 8])
def test_sfft_zipup_circuit_equals_dense_and_ranks(n):
    """Sec. 4.2: the reduced QFT circuit (Hadamards and controlled phases split
    into copy and phase tensors) taken to an MPO by zip-up sweeps is the SFFT
    S = P_rev F+ of Sec. 4.1 (and so the momentum convention of Sec. 4.3
    follows from the circuit), and the TT-SVD MPO of the dense matrix at the
    solver's accuracy 1e-12 has exactly the circuit MPO's ranks."""
    z = oq.sfft_axis_mpo_zipup(n, 1e-12)
    assert np.allclose(oq.tto_full(z), oq.sfft_dense(n), atol=1e-13)
    assert [c.shape[0] for c in z] == [c.shape[0] for c in oq.sfft_axis_mpo(n, 1e-12)]
    assert max(c.shape[0] for c in z) <= 1 << (n // 2)


def test_sfft_zipup_printed_rank_and_planted_gate_mistakes():
    """The circuit construction reaches the printed SFFT rank (10 at 1e-10 for
    n = 8, Sec. 5.2); dropping one controlled phase or flipping the phase sign
    gives a different operator."""
    g = json.load(open(os.path.join(GOLD, "paper_values.json")))["sfft_mpo_rank"]
    z = oq.sfft_axis_mpo_zipup(8, g["delta_acc"])
    assert max(c.shape[0] for c in z) == g["value"]
    n = 4
    I2 = np.eye(2, dtype=np.complex128)
    gates = oq.qft_circuit_gates(n)
    for bad in (gates[:2] + gates[3:],
                [[np.conj(c) for c in gt] for gt in gates]):
        op = [I2.reshape(1, 2, 2, 1) for _ in range(n)]
        for gt in bad:
            op = oq.mpo_zipup(gt, op, 1e-15)
        assert not np.allclose(oq.tto_full(op), oq.sfft_dense(n), atol=1e-6)


def test_sfft_3d_operator_and_inverse():
    n = 2
    N = 1 << n
    S = oq.tto_full(oq.sfft_operator(n))
    Sh = oq.tto_full(oq.sfft_operator(n, adjoint=True))
    assert np.allclose(Sh @ S, np.eye(S.shape[0]), atol=1e-12)
    rng = np.random.default_rng(7)
    f = rng.standard_normal((6, N, N, N)) + 1j * rng.standard_normal((6, N, N, N))
    rev = [oq.bit_reverse(k, n) for k in range(N)]
    ref = (np.fft.ifftn(f, axes=(1, 2, 3)) * N ** 1.5)[:, rev][:, :, rev][:, :, :, rev]
    assert np.allclose((S @ f.reshape(-1)).reshape(f.shape), ref, atol=1e-12)


@pytest.mark.parametrize("n", [2, 3])
def test_momentum_convention_matches_dense_pipeline(n):
    """S^H Gamma_S S equals ifft(Gamma(xi) fft(.)) of the dense scheme: the
    bit reversal and conjugation of Sec. 4.3 reproduce the FFT scheme's Green
    operator (with numpy's Nyquist representative)."""
    N = 1 << n
    lam0, mu0 = 2.0, 1.0
    rng = np.random.default_rng(n)
    tau = rng.standard_normal((6, N, N, N)) + 1j * rng.standard_normal((6, N, N, N))
    f = dense.frequencies(N)
    XI = np.stack(np.meshgrid(f, f, f, indexing="ij"), -1)
    d = np.fft.ifftn(np.einsum("abcIJ,Jabc->Iabc", dense.green_voigt_symmetrised(XI, lam0, mu0, N),
                               np.fft.fftn(tau, axes=(1, 2, 3))), axes=(1, 2, 3))
    S = oq.tto_full(oq.sfft_operator(n))
    Sh = oq.tto_full(oq.sfft_operator(n, adjoint=True))
    G = oq.gamma_field_sfft(n, lam0, mu0)
    v = (S @ tau.reshape(-1)).reshape(tau.shape)
    w = np.einsum("IJabc,Jabc->Iabc", G, v)
    q = (Sh @ w.reshape(-1)).reshape(tau.shape)
    assert np.abs(q - d).max() < 1e-12 * np.abs(d).max()
    # and the compressed Green TTO reproduces the field
    Gt = oq.tto_full(oq.gamma_qtt(n, lam0, mu0, 1e-13))
    assert np.allclose(np.diag(Gt[:N ** 3, :N ** 3]), G[0, 0].reshape(-1), atol=1e-11)


def test_gamma_separability():
    """App. D: Gamma = (1/mu0) Gamma1 - beta0 Gamma2 with Lame-independent parts."""
    n = 2
    g_a = oq.gamma_field_sfft(n, 1.0, 1.0)
    g_b = oq.gamma_field_sfft(n, 3.0, 0.5)
    # beta0 for each, recover Gamma1, Gamma2 from two parameter sets and predict a third
    b = lambda l, m: (l + m) / (m * (l + 2 * m))
    A = np.array([[1 / 1.0, -b(1.0, 1.0)], [1 / 0.5, -b(3.0, 0.5)]])
    coef = np.linalg.solve(A, np.stack([g_a.reshape(-1), g_b.reshape(-1)]))
    g_c = oq.gamma_field_sfft(n, 0.7, 2.2)
    pred = (1 / 2.2) * coef[0] - b(0.7, 2.2) * coef[1]
    assert np.allclose(pred, g_c.reshape(-1), atol=1e-12)


def test_philox_known_answers():
    kat = json.load(open(os.path.join(GOLD, "philox_kat.json")))["vectors"]
    for v in kat:
        ctr = [np.array([int(h, 16)], dtype=np.uint64) for h in v["ctr"]]
        key = [int(h, 16) for h in v["key"]]
        out = oq.philox4x32(ctr, key)
        assert ["%08x" % int(w[0]) for w in out] == v["out"]


def test_sketch_core_values():
    s = oq.sketch_core(2412, 3, 5, (3, 2, 4))
    assert s.shape == (3, 2, 4)
    assert np.all(np.abs(s.real) < 1) and np.all(np.abs(s.imag) < 1)
    # exactly representable values: (int32 + 1/2) 2^-31
    assert np.all(((s.real * 2 ** 31 - 0.5) % 1) == 0)
    assert not np.allclose(s, oq.sketch_core(2412, 3, 6, (3, 2, 4)))


def test_sketched_product_exact_with_full_sketch():
    n = 2
    rng = np.random.default_rng(9)
    G = oq.gamma_qtt(n, 2.0, 1.0, 1e-13)
    x = oq.tt_round(random_tt(rng, [6] + [2] * (3 * n), [1, 4, 6, 5, 6, 4, 2, 1]), 1e-14, 100)[0]
    ref = oq.tto_full(G) @ oq.tt_full(x).reshape(-1)
    y = oq.tto_apply_sketched(G, x, 10 ** 4, 1, 0)
    assert rel(oq.tt_full(y).reshape(-1), ref) < 1e-11
    # output cores 0..L-2 left-orthonormal, up to exactly zero columns where a
    # sketch direction was dependent on the others
    for c in y[:-1]:
        M = c.reshape(-1, c.shape[2])
        G = M.conj().T @ M
        live = np.linalg.norm(M, axis=0) > 0
        assert np.allclose(G, np.diag(live.astype(float)), atol=1e-11)


def _random_op(rng, dims, ranks):
    return [rng.standard_normal((ranks[k], d, d, ranks[k + 1]))
            + 1j * rng.standard_normal((ranks[k], d, d, ranks[k + 1])) for k, d in enumerate(dims)]


def _tto_sum(a, b):
    """a + b as a TTO of rank r(a) + r(b) (block-diagonal cores)."""
    L = len(a)
    out = []
    for k, (A, B) in enumerate(zip(a, b)):
        if k == 0:
            out.append(np.concatenate([A, B], axis=3))
        elif k == L - 1:
            out.append(np.concatenate([A, B], axis=0))
        else:
            C = np.zeros((A.shape[0] + B.shape[0],) + A.shape[1:3] + (A.shape[3] + B.shape[3],),
                         dtype=np.complex128)
            C[:A.shape[0], :, :, :A.shape[3]] = A
            C[A.shape[0]:, :, :, A.shape[3]:] = B
            out.append(C)
    return out


def _below_rank_case():
    """A product whose formal rank (Table 2: a s = 12) is twice its true rank
    (6): the operator is A + A/2 written with rank 4, the TT has rank 3."""
    dims = [6] + [2] * 9
    rng = np.random.default_rng(3)
    A = _random_op(rng, dims, [1] + [2] * 9 + [1])
    A2 = _tto_sum(A, [W * (0.5 if k == 0 else 1.0) for k, W in enumerate(A)])
    x = random_tt(rng, dims, [1] + [3] * 9 + [1])
    y = oq.tt_full(oq.tto_apply_exact(A2, x)).reshape(-1)
    return A2, x, y


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_sketched_product_below_formal_rank_is_exact():
    """Sketch rank ell = 6 is half the product's formal rank but equal to its
    true rank: the randomized compression must recover the exact product (the
    sketch spans the range of each right unfolding, and every live direction is
    kept). A dropped live column of the orthonormalised environment, or an
    environment that does not span the product's right range, fails here
    (both planted in test_sketched_pin_catches_planted_mistakes)."""
    A2, x, y = _below_rank_case()
    assert oq.tt_ranks(oq.tto_apply_exact(A2, x))[5] == 12
    assert oq.tt_ranks(oq.tt_round(oq.tto_apply_exact(A2, x), 1e-14, 10 ** 9)[0])[5] == 6
    for ell in (6, 8):
        ys = oq.tto_apply_sketched(A2, x, ell, 11, 2)
        assert _rel(oq.tt_full(ys).reshape(-1), y) < 1e-12


def test_sketched_product_quasi_optimal():
    """Below the true rank (flat spectra: a random TT through the Green
    operator) the sketched product is within 2x the error of the TT-SVD
    rounding of the exact product at half the sketch rank (measured at most
    1.4x over seeds 0-3 and ell in {8, 12, 16, 24}), and, being a TT of ranks
    <= ell, no better than the optimal rank-ell error, which the TT-SVD
    rounding exceeds by at most sqrt(L - 1) (Sec. 3, rounding bound)."""
    n = 3
    G = oq.gamma_qtt(n, 2.0, 1.0, 1e-12)
    dims = [6] + [2] * (3 * n)
    L = len(dims)
    for seed in range(2):
        rng = np.random.default_rng(seed)
        x = random_tt(rng, dims, [1] + [6] * (L - 1) + [1])
        yc = oq.tto_apply_exact(G, x)
        y = oq.tt_full(yc).reshape(-1)
        for ell in (8, 16, 24):
            e_sk = _rel(oq.tt_full(oq.tto_apply_sketched(G, x, ell, 7 + seed, 3)).reshape(-1), y)
            e_half = _rel(oq.tt_full(oq.tt_round(yc, 0.0, ell // 2)[0]).reshape(-1), y)
            e_full = _rel(oq.tt_full(oq.tt_round(yc, 0.0, ell)[0]).reshape(-1), y)
            assert e_full / np.sqrt(L - 1) <= e_sk <= 2.0 * e_half, (seed, ell, e_sk, e_half)


def test_sketched_pin_catches_planted_mistakes(monkeypatch):
    """Plant two mistakes in the oracle's sketched product and check that the
    below-rank pin fails: (1) the orthonormalised environment loses its last
    live column; (2) the environment is replaced by an orthonormal basis of an
    unrelated space of the same size."""
    A2, x, y = _below_rank_case()
    good = oq.orthonormal_range

    def dropped(P, tau=oq.SKETCH_DROP_TAU):
        Q, M = good(P, tau)
        k = int(np.sum(np.linalg.norm(Q, axis=0) > 0.5))
        Q, M = Q.copy(), M.copy()
        Q[:, k - 1] = 0
        M[:, k - 1] = 0
        return Q, M

    def unrelated(P, tau=oq.SKETCH_DROP_TAU):
        r = np.random.default_rng(P.shape[0] * 31 + P.shape[1])
        Z = r.standard_normal(P.shape) + 1j * r.standard_normal(P.shape)
        return np.linalg.qr(Z)[0], np.eye(P.shape[1])

    for bad in (dropped, unrelated):
        monkeypatch.setattr(oq, "orthonormal_range", bad)
        ys = oq.tto_apply_sketched(A2, x, 6, 11, 2)
        assert _rel(oq.tt_full(ys).reshape(-1), y) > 1e-3, bad.__name__
    monkeypatch.setattr(oq, "orthonormal_range", good)


def test_orthonormal_range_is_pivoted_qr():
    # full column rank: Q is the thin-QR factor, with real positive diagonal
    # in R, of P with its columns in the pivot order (numpy's QR of the
    # permuted matrix, column phases moved into R)
    rng = np.random.default_rng(31)
    P = (rng.standard_normal((40, 10)) + 1j * rng.standard_normal((40, 10))) * np.arange(1, 11)
    Q, M = oq.orthonormal_range(P)
    assert np.allclose(Q.conj().T @ Q, np.eye(10), atol=1e-12)
    # recover the pivot order: column j of Q uses P's columns perm[0..j]
    order = []
    for j in range(10):
        nz = set(np.flatnonzero(np.abs(M[:, j]) > 0).tolist())
        new_cols = nz - set(order)
        assert len(new_cols) == 1
        order.append(new_cols.pop())
    assert order[0] == 9          # largest column norm first
    Qn, Rn = np.linalg.qr(P[:, order])
    ph = np.diag(Rn) / np.abs(np.diag(Rn))
    assert np.allclose(Q, Qn * ph[None, :], atol=1e-12)
    assert np.allclose(Q @ (Q.conj().T @ P), P, atol=1e-11)


def test_orthonormal_range_drops_dependent_columns():
    rng = np.random.default_rng(32)
    P = rng.standard_normal((30, 9)) + 1j * rng.standard_normal((30, 9))
    P[:, 3] = 2 * P[:, 0] - (1 - 1j) * P[:, 1]
    P[:, 7] = 0
    Q, M = oq.orthonormal_range(P)
    # rank 7: seven orthonormal columns, then exactly zero ones
    assert np.allclose(Q[:, :7].conj().T @ Q[:, :7], np.eye(7), atol=1e-12)
    assert np.all(Q[:, 7:] == 0) and np.all(M[:, 7:] == 0)
    # same range: P is reproduced by its projection onto Q
    assert np.allclose(Q @ (Q.conj().T @ P), P, atol=1e-11)


def test_orthonormal_range_ill_conditioned():
    # singular values 1 .. 1e-4: Gram condition 1e8, orthogonality to ~eps 1e8
    rng = np.random.default_rng(33)
    U, _ = np.linalg.qr(rng.standard_normal((50, 12)) + 1j * rng.standard_normal((50, 12)))
    V, _ = np.linalg.qr(rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12)))
    P = U @ np.diag(np.logspace(0, -4, 12)) @ V
    Q, M = oq.orthonormal_range(P)
    assert np.allclose(Q.conj().T @ Q, np.eye(12), atol=1e-6)
    assert np.allclose(Q @ (Q.conj().T @ P), P, atol=1e-12)
    # pivoting bounds the inverse factor: |M| stays within 1/sigma_min scale
    assert np.abs(M).max() < 1e6


def test_e_tt_and_mean():
    n = 2
    Ev = np.array([1.0, -2.0, 0.5, 0.0, 3.0, 0.0])
    E = oq.e_tt(n, Ev)
    F = oq.to_voigt_field(E, n)
    assert np.allclose(F, Ev[:, None, None, None] * np.ones((1, 4, 4, 4)))
    assert np.isclose(oq.tt_norm(E), np.linalg.norm(Ev) * 8)
    for c in E[1:]:
        M = c.reshape(c.shape[0], -1)
        assert np.allclose(M @ M.conj().T, 1)
    ph = synth.centred_sphere(n, 0.3)
    dC = oq.stiffness_qtt(ph, n, (1.0, 3.0), (0.3, 0.2), (1.0, 0.7), 1e-13)
    rng = np.random.default_rng(5)
    x = random_tt(rng, [6] + [2] * 6, [1, 6, 5, 4, 6, 4, 2, 1])
    ref = (oq.tto_full(dC) @ oq.tt_full(x).reshape(-1)).reshape(6, -1).mean(axis=1)
    assert np.allclose(oq.tto_sandwich_mean(dC, x), ref, atol=1e-12)


def test_stiffness_qtt_is_the_field():
    n = 2
    ph = synth.centred_sphere(n, 0.35)
    E, nu = (1.0, 5.0), (0.3, 0.25)
    lam0 = dense.reference_lame(E, nu)
    dC = oq.stiffness_qtt(ph, n, E, nu, lam0, 1e-13)
    M = oq.tto_full(dC)
    C0 = dense.stiffness_voigt(*lam0)
    ncell = 64
    for cell in (0, 21, 42):
        p = ph.reshape(-1)[cell]
        ref = dense.stiffness_voigt(*dense.lame(E[p], nu[p])) - C0
        block = M[cell::ncell, cell::ncell]
        assert np.allclose(block, ref, atol=1e-12)
    # with the mean reference medium C_A - C0 = -(C_B - C0): Voigt bond rank 1;
    # any other reference medium gives rank 2
    assert dC[0].shape[3] == 1
    assert oq.stiffness_qtt(ph, n, E, nu, (1.0, 0.7), 1e-13)[0].shape[3] == 2


@pytest.mark.parametrize("n,load", [(2, 0), (2, 3), (3, 1)])
def test_qtt_oracle_matches_dense_oracle(n, load):
    """The two oracles (Alg. 1 and Alg. 2) agree when no truncation bites."""
    ph = synth.centred_sphere(n, 0.3)
    E, nu = (1.0, 6.0), (0.3, 0.25)
    lam0 = dense.reference_lame(E, nu)
    dC = oq.stiffness_qtt(ph, n, E, nu, lam0, 1e-13)
    G = oq.gamma_qtt(n, *lam0, 1e-13)
    S, Sh = oq.sfft_operator(n), oq.sfft_operator(n, adjoint=True)
    Ev = np.eye(6)[load]
    r = oq.ls_solve(dC, G, S, Sh, Ev, n, 1e-300, 1e-13, 1000, max_iter=12, lame0=lam0)
    d = dense.basic_scheme(ph, E, nu, Ev, tol=1e-300, max_iter=12)
    assert np.allclose(r["history"], d["history"], rtol=1e-7)
    assert np.abs(r["sigma_bar"] - d["sigma_bar"]).max() < 1e-10
    assert np.abs(oq.to_voigt_field(r["eps"], n) - d["eps"]).max() < 1e-10


def test_laminate_qtt_low_rank_and_exact():
    """A laminate's strain stays rank-1 per layer pattern: the QTT solve
    reproduces the closed-form laminate stiffness with small ranks."""
    from tests.test_oracle_dense import laminate_closed_form
    n = 3
    ph1 = synth.laminate(n, 2)
    E, nu = (9.0, 1.5), (0.3, 0.2)
    lam0 = dense.reference_lame(E, nu)
    dC = oq.stiffness_qtt(ph1, n, E, nu, lam0, 1e-12)
    G = oq.gamma_qtt(n, *lam0, 1e-12)
    S, Sh = oq.sfft_operator(n), oq.sfft_operator(n, adjoint=True)
    ref = laminate_closed_form(ph1.reshape(-1), E, nu)
    for load in (2, 3):
        r = oq.ls_solve(dC, G, S, Sh, np.eye(6)[load], n, 1e-11, 1e-12, 64, lame0=lam0)
        assert np.allclose(r["sigma_bar"].real, ref[:, load], atol=1e-8 * np.abs(ref).max())
        assert r["max_rank"] <= 16


def test_pin_catches_missing_bit_reversal(monkeypatch):
    """Plant a mistake: SFFT without the bit reversal. The DFT pin fails."""
    monkeypatch.setattr(oq, "bit_reverse", lambda k, n: k)
    with pytest.raises(AssertionError):
        test_sfft_is_bit_reversed_unitary_dft.__wrapped__(3) if hasattr(
            test_sfft_is_bit_reversed_unitary_dft, "__wrapped__") else _sfft_check(3)


def _sfft_check(n):
    N = 1 << n
    S = oq.sfft_dense(n)
    x = np.arange(N) + 1j
    rev = [int(format(k, f"0{n}b")[::-1], 2) for k in range(N)]
    assert np.allclose(S @ x, (np.fft.ifft(x) * np.sqrt(N))[rev], atol=1e-12)


def test_qtt_oracle_matches_dense_oracle_centered():
    """Oracle B with the Centered-scheme Green TTO against oracle A with the
    Centered scheme (App. A table), 4^3 sphere, load e11."""
    n = 2
    ph = synth.centred_sphere(n, 0.3)
    E, nu = (1.0, 10.0), (0.3, 0.3)
    lam0 = dense.reference_lame(E, nu)
    dC = oq.stiffness_qtt(ph, n, E, nu, lam0, 1e-12)
    G = oq.gamma_qtt(n, *lam0, 1e-12, scheme="centered")
    S, Sh = oq.sfft_operator(n), oq.sfft_operator(n, adjoint=True)
    Ev = np.eye(6)[0]
    b = oq.ls_solve(dC, G, S, Sh, Ev, n, 1e-11, 1e-12, 1000, lame0=lam0, seed=2412)
    a = dense.basic_scheme(ph, E, nu, Ev, tol=1e-11, scheme="centered")
    assert np.abs(b["sigma_bar"] - a["sigma_bar"]).max() < 1e-8 * np.abs(a["sigma_bar"]).max()


def _asymmetric_phase(n):
    N = 1 << n
    return (np.random.default_rng(31).random((N, N, N)) < 0.4).astype(np.uint8)


@pytest.mark.parametrize("scheme", ["forward", "hex8r", "staggered"])
def test_qtt_oracle_matches_dense_oracle_other_schemes(scheme):
    """Oracle B with the Green TTO of the Forward, Hex8R and staggered schemes
    (App. A table; complex for Forward and staggered, whose SFFT-side field is
    the conjugate) against oracle A with the same scheme, on a seeded 4^3
    two-phase field without mirror symmetry, load e11 and the shear load e23."""
    n = 2
    ph = _asymmetric_phase(n)
    E, nu = (1.0, 10.0), (0.3, 0.3)
    lam0 = dense.reference_lame(E, nu)
    dC = oq.stiffness_qtt(ph, n, E, nu, lam0, 1e-12)
    G = oq.gamma_qtt(n, *lam0, 1e-12, scheme=scheme)
    S, Sh = oq.sfft_operator(n), oq.sfft_operator(n, adjoint=True)
    for k in (0, 3):
        Ev = np.eye(6)[k]
        b = oq.ls_solve(dC, G, S, Sh, Ev, n, 1e-11, 1e-12, 1000, lame0=lam0, seed=2412)
        a = dense.basic_scheme(ph, E, nu, Ev, tol=1e-11, scheme=scheme)
        assert np.abs(b["sigma_bar"] - a["sigma_bar"]).max() < 1e-8 * np.abs(a["sigma_bar"]).max()


def test_qtt_complex_scheme_needs_the_conjugate():
    """Planted mistake: the staggered Green field without the SFFT-convention
    conjugation is the operator of the mirrored grid, which the dense
    comparison detects on a field without mirror symmetry."""
    n = 2
    ph = _asymmetric_phase(n)
    E, nu = (1.0, 10.0), (0.3, 0.3)
    lam0 = dense.reference_lame(E, nu)
    dC = oq.stiffness_qtt(ph, n, E, nu, lam0, 1e-12)
    F = np.conj(oq.gamma_field_sfft(n, *lam0, "staggered"))
    G = oq.controlled_field_to_tto(F, n, 1e-12, 1 << 30)
    S, Sh = oq.sfft_operator(n), oq.sfft_operator(n, adjoint=True)
    Ev = np.eye(6)[3]
    b = oq.ls_solve(dC, G, S, Sh, Ev, n, 1e-11, 1e-12, 1000, lame0=lam0, seed=2412)
    a = dense.basic_scheme(ph, E, nu, Ev, tol=1e-11, scheme="staggered")
    assert np.abs(b["sigma_bar"] - a["sigma_bar"]).max() > 1e-6 * np.abs(a["sigma_bar"]).max()


@pytest.mark.parametrize("scheme", ["direct", "staggered"])
def test_plane_green_on_broadcast_geometry(scheme):
    """Sec. 4.3, broadcast axes: on a geometry broadcast along x1 the strain is
    x1-invariant, its SFFT lives at xi_1 = 0, and Gamma(0, xi_2, xi_3) (x) I on
    the x1 cores gives the same solve as the full Green operator; on a field
    that varies along x1 it does not (it is not the same operator)."""
    n = 2
    ph = synth.section_3d(synth.circle2d(n, 0.3, centre=(0.4, 0.55)))   # (1, N, N)
    E, nu = (1.0, 20.0), (0.3, 0.25)
    lam0 = dense.reference_lame(E, nu)
    dC = oq.stiffness_qtt(synth.broadcast_dense(ph, n), n, E, nu, lam0, 1e-12)
    S, Sh = oq.sfft_operator(n), oq.sfft_operator(n, adjoint=True)
    Gf = oq.gamma_qtt(n, *lam0, 1e-12, scheme=scheme)
    Gp = oq.gamma_qtt_plane(n, *lam0, 1e-12, scheme=scheme)
    assert max(oq.tt_ranks(Gp)) < max(oq.tt_ranks(Gf))
    for k in (0, 3):
        Ev = np.eye(6)[k]
        a = oq.ls_solve(dC, Gf, S, Sh, Ev, n, 0.0, 1e-12, 1000, max_iter=12, lame0=lam0)
        b = oq.ls_solve(dC, Gp, S, Sh, Ev, n, 0.0, 1e-12, 1000, max_iter=12, lame0=lam0)
        assert np.abs(a["sigma_bar"] - b["sigma_bar"]).max() < 1e-9 * np.abs(a["sigma_bar"]).max()
        assert np.allclose(a["history"], b["history"], rtol=1e-7, atol=1e-12)
    ph3 = synth.sphere_field(n, [(0.3, 0.4, 0.55)], [0.3])
    dC3 = oq.stiffness_qtt(ph3, n, E, nu, lam0, 1e-12)
    a = oq.ls_solve(dC3, Gf, S, Sh, np.eye(6)[0], n, 0.0, 1e-12, 1000, max_iter=3, lame0=lam0)
    b = oq.ls_solve(dC3, Gp, S, Sh, np.eye(6)[0], n, 0.0, 1e-12, 1000, max_iter=3, lame0=lam0)
    assert np.abs(a["sigma_bar"] - b["sigma_bar"]).max() > 1e-4 * np.abs(a["sigma_bar"]).max()


def test_randomized_tt_svd_matches_tt_svd():
    """App. D's randomized TT-SVD: on an exact-rank TT it finds the same ranks
    as the TT-SVD at 1e-12 and 1e-6; on the 16^3 Green field it meets the
    TT-SVD's error bound eps ||T|| with at most one more rank per bond."""
    rng = np.random.default_rng(3)
    ranks = [1, 4, 6, 8, 8, 8, 8, 8, 8, 8, 6, 4, 2, 1]
    T = oq.tt_full(random_tt(rng, [6] + [2] * 12, ranks)).reshape([6] + [2] * 12)
    for eps in (1e-12, 1e-6):
        b = oq.tt_svd_randomized(T, eps, seed=1)
        assert oq.tt_ranks(b) == oq.tt_ranks(oq.tt_svd(T, eps))
        assert np.linalg.norm(oq.tt_full(b).reshape(T.shape) - T) < 1e-12 * np.linalg.norm(T)
    G = oq.gamma_field_sfft(4, 1.3, 0.7).reshape((36,) + (2,) * 12).astype(np.complex128)
    for eps in (1e-2, 1e-4, 1e-6):
        a, b = oq.tt_svd(G, eps), oq.tt_svd_randomized(G, eps, seed=2)
        err = np.linalg.norm(oq.tt_full(b).reshape(G.shape) - G) / np.linalg.norm(G)
        assert err <= eps
        assert all(rb <= ra + 1 for ra, rb in zip(oq.tt_ranks(a), oq.tt_ranks(b)))
