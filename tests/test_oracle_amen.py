"""Pins of the oracle's AMEn-adapted product (App. B) and its comparison with
the successive randomized compression the CUDA path uses (Sec. 3, Table 2),
on random operators and on the Green product of an actual LS iteration."""
import numpy as np
import pytest

from oracle import dense, qtt as oq
from paper_2412_11566_gb300 import synth
from tests._helpers import random_tt


def _random_op(rng, L, r):
    ra = [1] + [r] * (L - 1) + [1]
    return [rng.standard_normal((ra[k], 2, 2, ra[k + 1]))
            + 1j * rng.standard_normal((ra[k], 2, 2, ra[k + 1])) for k in range(L)]


def test_amen_exact_when_rank_suffices():
    """From a random rank-2 start, the enrichment grows y to the product's exact
    rank (2 x 3 = 6) and the Galerkin sweeps reach A x to rounding."""
    rng = np.random.default_rng(1)
    L = 8
    op = _random_op(rng, L, 2)
    x = random_tt(rng, [2] * L, [1] + [3] * (L - 1) + [1])
    ref = oq.tt_full(oq.tto_apply_exact(op, x))
    y, sweeps = oq.tto_apply_amen(op, x, 1e-12)
    assert np.linalg.norm(oq.tt_full(y) - ref) < 1e-12 * np.linalg.norm(ref)
    assert max(oq.tt_ranks(y)) <= 6 and sweeps <= 4


def test_amen_truncated_within_tolerance():
    """At eps = 1e-3 the result is within the rounding tolerance of A x (App. B's
    local truncation plus the final rounding), with no more rank than the
    rounded exact product."""
    rng = np.random.default_rng(2)
    L = 10
    op = _random_op(rng, L, 3)
    x = random_tt(rng, [2] * L, [1] + [4] * (L - 1) + [1])
    ex = oq.tto_apply_exact(op, x)
    ref = oq.tt_full(ex)
    eps = 1e-3
    y, _ = oq.tto_apply_amen(op, x, eps, kick=6)
    assert np.linalg.norm(oq.tt_full(y) - ref) <= 3 * eps * np.linalg.norm(ref)
    yr, _ = oq.tt_round(ex, eps, 1 << 30)
    assert max(oq.tt_ranks(y)) <= max(oq.tt_ranks(yr)) + 2


@pytest.fixture(scope="module")
def green_product_case():
    """Gamma_hat tauh at the sixth iteration of the 8^3 sphere (contrast 10,
    eps 1e-6, r_max 128), the product of the fifth as the warm start, and the
    dense A x from the dense Green field."""
    n, eps, rmax = 3, 1e-6, 128
    ph = synth.centred_sphere(n, 0.3)
    E, nu = (1.0, 10.0), (0.3, 0.3)
    lam0 = dense.reference_lame(E, nu)
    dC = oq.stiffness_qtt(ph, n, E, nu, lam0, eps)
    G = oq.gamma_qtt(n, *lam0, eps)
    S, Sh = oq.sfft_operator(n), oq.sfft_operator(n, adjoint=True)
    ell = rmax + 16

    def tauh_of(x):
        tau, _ = oq.tt_round(oq.tto_apply_sketched(dC, x, ell, 1, 0), eps, rmax, assume_left_orth=True)
        th, _ = oq.tt_round(oq.tto_apply_sketched(S, tau, ell, 1, 1), eps, rmax, assume_left_orth=True)
        return th

    x5 = oq.ls_solve(dC, G, S, Sh, np.eye(6)[0], n, 0.0, eps, rmax, max_iter=5)["eps"]
    x6 = oq.ls_solve(dC, G, S, Sh, np.eye(6)[0], n, 0.0, eps, rmax, max_iter=6)["eps"]
    th5, th6 = tauh_of(x5), tauh_of(x6)
    warm, _ = oq.tt_round(oq.tto_apply_sketched(G, th5, ell, 5, 2), eps, rmax, assume_left_orth=True)
    N = 1 << n
    yd = np.einsum("IJxyz,Jxyz->Ixyz", oq.gamma_field_sfft(n, *lam0),
                   oq.tt_full(th6).reshape(6, N, N, N))
    return dict(G=G, x=th6, warm=warm, yd=yd, eps=eps, rmax=rmax, ell=ell)


def _err(c, yd):
    return np.linalg.norm(oq.tt_full(c).reshape(yd.shape) - yd) / np.linalg.norm(yd)


def test_amen_and_sketched_agree_on_the_green_product(green_product_case):
    """On the Green product of an LS iteration, AMEn and the successive
    randomized compression reach the same accuracy (the rounding floor, below
    eps) at the same rank. From the previous iteration's product AMEn needs one
    sweep; from a cold rank-2 start it needs several (the rank grows by at
    most `kick` per sweep)."""
    c = green_product_case
    G, x, yd, eps, rmax = c["G"], c["x"], c["yd"], c["eps"], c["rmax"]
    ys, _ = oq.tt_round(oq.tto_apply_sketched(G, x, c["ell"], 7, 3), eps, rmax,
                        assume_left_orth=True)
    e_s = _err(ys, yd)
    assert e_s < eps
    yw, sw = oq.tto_apply_amen(G, x, eps, rmax, y0=[a.copy() for a in c["warm"]], kick=4,
                               sweeps=1, tol_change=0.0)
    assert _err(yw, yd) < 1.5 * e_s and max(oq.tt_ranks(yw)) == max(oq.tt_ranks(ys))
    cold = [_err(oq.tto_apply_amen(G, x, eps, rmax, kick=4, sweeps=s, tol_change=0.0)[0], yd)
            for s in (1, 4, 16)]
    assert cold[0] > 0.1 and cold[1] > 1e-3 and cold[2] < 1.5 * e_s


def test_sketched_product_quasi_optimal_in_the_truncating_regime():
    """The regime between the exact case and the flat spectrum: on the Green
    product of an 8^3 LS iteration, truncated to ranks 8, 16 and 24 (errors
    3e-1 to 2e-2), the sketched product (sketch rank r + 16, then rounding to
    r) is within 10 % of the TT-SVD of the dense A x at the same rank for every
    one of 8 seeds, and so is AMEn."""
    n = 3
    ph = synth.centred_sphere(n, 0.3)
    E, nu = (1.0, 10.0), (0.3, 0.3)
    lam0 = dense.reference_lame(E, nu)
    dC = oq.stiffness_qtt(ph, n, E, nu, lam0, 1e-10)
    G = oq.gamma_qtt(n, *lam0, 1e-10)
    S, Sh = oq.sfft_operator(n), oq.sfft_operator(n, adjoint=True)
    x = oq.ls_solve(dC, G, S, Sh, np.eye(6)[0], n, 0.0, 1e-10, 500, max_iter=6)["eps"]
    tau, _ = oq.tt_round(oq.tto_apply_sketched(dC, x, 400, 1, 0), 1e-10, 500, assume_left_orth=True)
    th, _ = oq.tt_round(oq.tto_apply_sketched(S, tau, 400, 1, 1), 1e-10, 500, assume_left_orth=True)
    N = 1 << n
    yd = np.einsum("IJxyz,Jxyz->Ixyz", oq.gamma_field_sfft(n, *lam0),
                   oq.tt_full(th).reshape(6, N, N, N))
    for r in (8, 16, 24):
        opt = _err(oq.tt_svd(yd.reshape((6,) + (2,) * (3 * n)).astype(np.complex128), 1e-14, r), yd)
        assert 1e-2 < opt < 0.5
        for seed in range(8):
            ys, _ = oq.tt_round(oq.tto_apply_sketched(G, th, r + 16, seed, 3), 1e-14, r,
                                assume_left_orth=True)
            assert _err(ys, yd) <= 1.1 * opt, (r, seed)
        ya, _ = oq.tto_apply_amen(G, th, 1e-14, r, kick=8, sweeps=12)
        assert _err(ya, yd) <= 1.1 * opt
