"""Pins of the gradient of C_eff (the energy form used by the adjoint
path): against central finite differences of the dense scheme, and the QTT
oracle's sandwich contraction against the dense energy form."""
import numpy as np
import pytest

from oracle import dense, qtt as oq
from paper_2412_11566_gb300 import synth


def solve_fields(ph, E, nu, tol, lame0):
    return {k: dense.basic_scheme(ph, E, nu, np.eye(6)[k], tol=tol, lame0=lame0)["eps"]
            for k in range(6)}


@pytest.mark.parametrize("p,wrt", [(0, "E"), (1, "E"), (0, "nu"), (1, "nu")])
def test_energy_gradient_matches_central_differences(p, wrt):
    ph = synth.centred_sphere(2, 0.3)
    E, nu = [1.0, 10.0], [0.3, 0.25]
    lame0 = dense.reference_lame(E, nu)       # fixed while differentiating
    fields = solve_fields(ph, E, nu, 1e-13, lame0)
    G = dense.ceff_gradient_energy(ph, E, nu, fields, [(p, wrt)])[(p, wrt)]
    vals = {"E": E, "nu": nu}
    base = vals[wrt][p]
    h = 1e-4 * abs(base)
    Cs = []
    for s in (+1, -1):
        v = list(vals[wrt])
        v[p] = base + s * h
        kw = dict(E=E, nu=nu)
        kw[wrt] = v
        C, _, _ = dense.ceff(ph, kw["E"], kw["nu"], tol=1e-13, lame0=lame0)
        Cs.append(C)
    fd = (Cs[0] - Cs[1]) / (2 * h)
    assert np.abs(G - fd).max() < 1e-6 * max(1.0, np.abs(fd).max())
    assert np.abs(G - G.T).max() < 1e-9 * np.abs(G).max()


def test_qtt_sandwich_matches_dense_energy_form():
    n = 2
    ph = synth.centred_sphere(n, 0.3)
    E, nu = [1.0, 10.0], [0.3, 0.25]
    lame0 = dense.reference_lame(E, nu)
    fields = solve_fields(ph, E, nu, 1e-12, lame0)
    ref = dense.ceff_gradient_energy(ph, E, nu, fields, [(1, "E")])[(1, "E")]
    D = dense.stiffness_voigt_derivative(E[1], nu[1], "E")
    op = oq.phase_matrices_qtt(ph, n, [np.zeros((6, 6)), D], 1e-13)
    tts = {k: oq.tt_svd(fields[k].reshape((6,) + (2,) * (3 * n)), 1e-14) for k in range(6)}
    G = np.array([[oq.tto_sandwich_bilinear_mean(op, tts[l], tts[k]).real for k in range(6)]
                  for l in range(6)])
    assert np.abs(G - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("scheme", ["staggered", "forward", "hex8r", "centered"])
def test_energy_gradient_holds_for_every_scheme(scheme):
    """Every scheme's Green operator is the projector of a discrete variational
    problem (Gamma_V = B (B^H C0 B)^-1 B^H), so C_eff is an energy minimum and
    dC_eff/dp = <eps_l^T dC/dp eps_k> holds for each of them: checked against
    central differences on a 4^3 field without mirror symmetry."""
    ph = (np.random.default_rng(17).random((4, 4, 4)) < 0.4).astype(np.uint8)
    E, nu = [1.0, 10.0], [0.3, 0.25]
    lame0 = dense.reference_lame(E, nu)
    fields = {k: dense.basic_scheme(ph, E, nu, np.eye(6)[k], tol=1e-13, lame0=lame0,
                                    scheme=scheme)["eps"] for k in range(6)}
    G = dense.ceff_gradient_energy(ph, E, nu, fields, [(1, "E")])[(1, "E")]
    h = 1e-4 * E[1]
    Cp, _, _ = dense.ceff(ph, [E[0], E[1] + h], nu, tol=1e-13, lame0=lame0, scheme=scheme)
    Cm, _, _ = dense.ceff(ph, [E[0], E[1] - h], nu, tol=1e-13, lame0=lame0, scheme=scheme)
    fd = (Cp - Cm) / (2 * h)
    assert np.abs(G - fd).max() < 1e-6 * max(1.0, np.abs(fd).max())
