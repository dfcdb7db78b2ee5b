"""The plain-method FP64 workload: one centred sphere r = 0.25 L with E 10 in
a matrix E 1 (nu 0.3 both), load e11, stop tolerance 1e-6, eps_tt 1e-8.

  * At 32^3 (n = 5, 16 cores) with r_max 64, on the oracle's own operators:
    sigma_bar within 1e-8 of the QTT oracle (Alg. 2 with the same Philox
    sketches) after the same number of iterations. At this rank cap the
    iteration cannot reach 1e-6: the converged dense strain of this geometry
    has QTT rank 354 at eps 1e-8 (245 at 1e-4), measured from the dense
    oracle's solution, so both sides level off at the cap's truncation error
    (a residual of ~3e-2). The cap cuts from the first iteration on (the
    Green TTO alone has rank 240 here), inside a flat part of the spectrum:
    which 64 directions survive then depends on rounding-level differences,
    and the two sides drift apart over the iterations (measured on the GPU:
    6e-9 in sigma_bar after 2 iterations, 1 % in the residual after 8). The
    comparison is taken after the first iteration, and its bound is set by
    the truncation's own condition: perturbing the oracle's Green cores by
    1e-15 (relative, random) moves its first-iteration sigma_bar by 3.8e-9,
    so no implementation can be held to 1e-10 here; the bound is 1e-8.
  * The same geometry and settings at 16^3 (n = 4), where r_max 128 is the
    full rank of every bond: converged to 1e-6 through the public path
    (operators built on the device from the phase field), C_eff column e11
    within 1e-4 of the dense FFT scheme (Alg. 1)."""
import numpy as np
import pytest

from oracle import dense, qtt as oq
from paper_2412_11566_gb300 import synth
from tests._helpers import to_lib_op

pytestmark = pytest.mark.gpu

SEED = 2412


@pytest.fixture(scope="module")
def Q(lib_built):
    return lib_built


def test_c1_vs_qtt_oracle(Q):
    w = synth.sphere32_fp64()
    lam0 = dense.reference_lame(w.E, w.nu)
    dC = oq.stiffness_qtt(w.phase, w.n, w.E, w.nu, lam0, 1e-12)
    G = oq.gamma_qtt(w.n, *lam0, 1e-12)
    S, Sh = oq.sfft_operator(w.n), oq.sfft_operator(w.n, adjoint=True)
    C0 = dense.stiffness_voigt(*lam0)
    Ev = np.eye(6)[0]
    m = 1
    ref = oq.ls_solve(dC, G, S, Sh, Ev, w.n, 1e-300, w.eps_tt, w.rmax, max_iter=m, lame0=lam0,
                      seed=SEED)
    # a stop tolerance above the first residual (0.36): both sides stop after
    # the first iteration
    assert ref["history"][0] < 0.5
    tol = 0.5
    ctx = Q.Context(0, Q.QTT_FP64, 8 << 30, seed=SEED)
    try:
        dc, dd = to_lib_op(dC)
        gc, gd = to_lib_op(G)
        sig, info, rc = Q.ls_solve_ops(ctx, ctx.op(dc, dd), ctx.op(S), ctx.op(Sh),
                                       ctx.op(gc, gd), C0, Ev,
                                       Q.solve_params(tol, 500, w.eps_tt, w.rmax))
        assert info["iters"] == m
        assert abs(info["residual"] - ref["history"][-1]) < 1e-7 * ref["history"][-1]
        assert np.abs(sig - ref["sigma_bar"]).max() < 1e-8 * np.abs(ref["sigma_bar"]).max()
    finally:
        ctx.close()


def test_c1_geometry_full_rank_vs_dense_oracle(Q):
    n = 4
    ph = synth.centred_sphere(n, 0.25)
    w = synth.sphere32_fp64()
    ctx = Q.Context(0, Q.QTT_FP64, 8 << 30, seed=SEED)
    try:
        dC = Q.qtt_from_phase_field(ctx, ph, n, w.E, w.nu, None, w.eps_tt, 128)
        C, infos, rc = Q.ls_solve_ceff(ctx, dC, Q.solve_params(w.tol, 300, w.eps_tt, 128),
                                       loads=[0])
        Cd, imag, its = dense.ceff(ph, w.E, w.nu, tol=w.tol, loads=[0])
        assert infos[0]["residual"] < w.tol
        assert np.abs(C[:, 0] - Cd[:, 0]).max() < 1e-4 * np.abs(Cd[:, 0]).max()
    finally:
        ctx.close()
