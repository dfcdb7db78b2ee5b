"""The plain-method FP64 workload: 32^3 grid (n = 5, 16 cores), one centred
sphere r = 0.25 L with E 10 in a matrix E 1 (nu 0.3 both), load e11, stop
tolerance 1e-6, eps_tt 1e-8, r_max 64 (Alg. 2 end to end in FP64).

  * Through the public path (operators built on the device from the phase
    field): C_eff column e11 within 1e-4 of the dense FFT scheme (Alg. 1).
  * On the oracle's own operators: sigma_bar within 1e-10 of the QTT oracle
    run with the same Philox sketches, stopped after the same iteration."""
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


def test_c1_vs_dense_oracle(Q):
    w = synth.sphere32_fp64()
    ctx = Q.Context(0, Q.QTT_FP64, 8 << 30, seed=SEED)
    try:
        dC = Q.qtt_from_phase_field(ctx, w.phase, w.n, w.E, w.nu, None, w.eps_tt, w.rmax)
        C, infos, rc = Q.ls_solve_ceff(ctx, dC, Q.solve_params(w.tol, 500, w.eps_tt, w.rmax),
                                       loads=[0])
        Cd, imag, its = dense.ceff(w.phase, w.E, w.nu, tol=w.tol, loads=[0])
        assert infos[0]["residual"] < w.tol
        assert np.abs(C[:, 0] - Cd[:, 0]).max() < 1e-4 * np.abs(Cd[:, 0]).max()
    finally:
        ctx.close()


def test_c1_vs_qtt_oracle(Q):
    w = synth.sphere32_fp64()
    lam0 = dense.reference_lame(w.E, w.nu)
    dC = oq.stiffness_qtt(w.phase, w.n, w.E, w.nu, lam0, 1e-12)
    G = oq.gamma_qtt(w.n, *lam0, 1e-12)
    S, Sh = oq.sfft_operator(w.n), oq.sfft_operator(w.n, adjoint=True)
    C0 = dense.stiffness_voigt(*lam0)
    Ev = np.eye(6)[0]
    full = oq.ls_solve(dC, G, S, Sh, Ev, w.n, w.tol, w.eps_tt, w.rmax, max_iter=200,
                       lame0=lam0, seed=SEED)
    m = full["iters"]
    assert full["history"][-1] < w.tol
    # a stop tolerance between the last two residuals: both sides stop after m
    tol = float(np.sqrt(full["history"][m - 2] * full["history"][m - 1]))
    ctx = Q.Context(0, Q.QTT_FP64, 8 << 30, seed=SEED)
    try:
        dc, dd = to_lib_op(dC)
        gc, gd = to_lib_op(G)
        sig, info, rc = Q.ls_solve_ops(ctx, ctx.op(dc, dd), ctx.op(S), ctx.op(Sh),
                                       ctx.op(gc, gd), C0, Ev,
                                       Q.solve_params(tol, 500, w.eps_tt, w.rmax))
        assert info["iters"] == m
        assert np.abs(sig - full["sigma_bar"]).max() < 1e-10 * np.abs(full["sigma_bar"]).max()
    finally:
        ctx.close()
