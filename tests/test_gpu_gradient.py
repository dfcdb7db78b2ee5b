"""GPU gradient of C_eff with respect to the phase parameters (E, nu per
phase): the sandwich contraction against the oracle, the full gradient
against the oracle's energy form (itself pinned against central differences
of the dense scheme), and the torch.autograd.Function against central
differences of the GPU's own C_eff."""
import numpy as np
import pytest

from oracle import dense, qtt as oq
from paper_2412_11566_gb300 import synth
from tests._helpers import random_tt, to_lib_op

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q(lib_built):
    return lib_built


@pytest.fixture(scope="module")
def ctx64(Q):
    c = Q.Context(0, Q.QTT_FP64, 1 << 30, seed=2412)
    yield c
    c.close()


def test_sandwich_matches_oracle(Q, ctx64):
    n = 2
    rng = np.random.default_rng(4)
    ph = synth.centred_sphere(n, 0.3)
    mats = [rng.standard_normal((6, 6)), rng.standard_normal((6, 6))]
    op = oq.phase_matrices_qtt(ph, n, mats, 1e-13)
    dims = [6] + [2] * (3 * n)
    x = random_tt(rng, dims, [1, 6, 5, 4, 6, 4, 2, 1])
    y = random_tt(rng, dims, [1, 3, 6, 5, 3, 4, 2, 1])
    ref = oq.tto_sandwich_bilinear_mean(op, y, x)
    gop = Q.qtt_from_phase_matrices(ctx64, ph, n, np.stack(mats), 1e-13)
    got = Q.qtt_op_sandwich_mean(ctx64, gop, ctx64.tt(y), ctx64.tt(x))
    assert abs(got - ref) < 1e-11 * abs(ref)
    # and the device-built operator is the oracle's field
    cores, diag = to_lib_op(op)
    assert abs(Q.qtt_op_sandwich_mean(ctx64, ctx64.op(cores, diag), ctx64.tt(y), ctx64.tt(x)) - ref) \
        < 1e-11 * abs(ref)


def test_gradient_matches_oracle_energy_form(Q, ctx64):
    n = 2
    ph = synth.centred_sphere(n, 0.3)
    E, nu = [1.0, 10.0], [0.3, 0.25]
    lame0 = dense.reference_lame(E, nu)
    fields = {k: dense.basic_scheme(ph, E, nu, np.eye(6)[k], tol=1e-13, lame0=lame0)["eps"]
              for k in range(6)}
    wrt = [(0, "E"), (1, "E"), (0, "nu"), (1, "nu")]
    ref = dense.ceff_gradient_energy(ph, E, nu, fields, wrt)
    dC = Q.qtt_from_phase_field(ctx64, ph, n, E, nu, None, 1e-12)
    C, grads, infos, rc = Q.ls_solve_ceff_grad(ctx64, dC, ph, E, nu,
                                               Q.solve_params(1e-300, 200, 1e-12, 64), wrt)
    Cd, _, _ = dense.ceff(ph, E, nu, tol=1e-13, lame0=lame0)
    assert np.abs(C - Cd).max() < 1e-8 * np.abs(Cd).max()
    for q, key in enumerate(wrt):
        assert np.abs(grads[q] - ref[key]).max() < 1e-7 * np.abs(ref[key]).max(), key


def test_autograd_function_matches_central_differences(Q, ctx64):
    import torch
    n = 2
    ph = synth.centred_sphere(n, 0.3)
    # a fixed iteration count (the stop test's FP64 inner-product residual has
    # a ~1e-8 floor, so a tiny tolerance would stop the FD solves on noise)
    params = Q.solve_params(1e-300, 200, 1e-12, 64)
    fn = Q.make_ceff_function(ctx64, ph, n, params, eps_op=1e-12)
    theta = torch.tensor([1.0, 0.3, 10.0, 0.25], dtype=torch.float64, requires_grad=True)
    C = fn.apply(theta)
    w = torch.from_numpy(np.random.default_rng(1).standard_normal((6, 6)))
    (C * w).sum().backward()
    g = theta.grad.numpy()
    # directional central difference of the GPU C_eff along a random parameter
    # direction, with the reference medium held fixed at the base point's mean
    lame0 = dense.reference_lame([1.0, 10.0], [0.3, 0.25])
    th0 = theta.detach().numpy()
    v = np.random.default_rng(2).standard_normal(4) * np.abs(th0)
    h = 1e-4
    ctx64.set_concurrency(6)
    vals = []
    for s in (+1, -1):
        t = th0 + s * h * v
        dC = Q.qtt_from_phase_field(ctx64, ph, n, t[0::2], t[1::2], lame0, 1e-12)
        Cs, _, _ = Q.ls_solve_ceff(ctx64, dC, params)
        vals.append((Cs * w.numpy()).sum())
    ctx64.set_concurrency(1)
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(g @ v - fd) < 1e-6 * max(1.0, abs(fd))


def test_gradient_matches_oracle_energy_form_8cubed(Q):
    """The same check at 8^3 (a 0.35 L sphere, contrast 10), where ranks are
    no longer trivial: dC_eff/dp for (E, nu) of both phases within 1e-6 of the
    oracle's energy form on the dense scheme's converged strains."""
    n = 3
    ph = synth.centred_sphere(n, 0.35)
    E, nu = [1.0, 10.0], [0.3, 0.25]
    lame0 = dense.reference_lame(E, nu)
    fields = {k: dense.basic_scheme(ph, E, nu, np.eye(6)[k], tol=1e-13, lame0=lame0)["eps"]
              for k in range(6)}
    wrt = [(0, "E"), (1, "E"), (0, "nu"), (1, "nu")]
    ref = dense.ceff_gradient_energy(ph, E, nu, fields, wrt)
    ctx = Q.Context(0, Q.QTT_FP64, 8 << 30, seed=2412)
    try:
        dC = Q.qtt_from_phase_field(ctx, ph, n, E, nu, None, 1e-12)
        ctx.set_concurrency(6)
        C, grads, infos, rc = Q.ls_solve_ceff_grad(ctx, dC, ph, E, nu,
                                                   Q.solve_params(1e-300, 150, 1e-12, 256), wrt)
    finally:
        ctx.close()
    for q, key in enumerate(wrt):
        assert np.abs(grads[q] - ref[key]).max() < 1e-6 * np.abs(ref[key]).max(), key
