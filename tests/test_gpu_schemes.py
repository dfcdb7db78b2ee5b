"""GPU parity of the Green operators of the App. A discretisation schemes
beyond Direct and Centered: Forward, Backward, Hex8R and the staggered grid.

The device operator is compared with the oracle's TT-SVD of the same field
(whose scheme symbols are pinned by a brute-force real-space construction in
tests/test_oracle_schemes.py), and the full solve with each scheme against
the dense FFT scheme (Alg. 1) run with that scheme."""
import numpy as np
import pytest

from oracle import dense, qtt as oq
from paper_2412_11566_gb300 import synth
from tests._helpers import from_lib_op

pytestmark = pytest.mark.gpu

SEED = 2412
NAMES = {"forward": 2, "backward": 3, "hex8r": 4, "staggered": 5}


@pytest.fixture(scope="module")
def Q(lib_built):
    return lib_built


@pytest.fixture(scope="module")
def ctx64(Q):
    c = Q.Context(0, Q.QTT_FP64, 1 << 30, seed=SEED)
    yield c
    c.close()


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def test_scheme_constants(Q):
    assert [Q.QTT_SCHEME_FORWARD, Q.QTT_SCHEME_BACKWARD, Q.QTT_SCHEME_HEX8R,
            Q.QTT_SCHEME_STAGGERED] == [NAMES[s] for s in ("forward", "backward", "hex8r",
                                                           "staggered")]


@pytest.mark.parametrize("scheme", list(NAMES))
def test_gamma_operator_scheme_vs_oracle(Q, ctx64, scheme):
    """The device Green TTO of the scheme (complex for Forward, Backward and
    staggered; from the monomials of v/|v| for Hex8R) against the oracle's
    TT-SVD of its Green field in the SFFT convention, for two reference media
    at 8^3, and distinct from the Direct operator."""
    n = 3
    for lam0, mu0 in [(3.5, 1.25), (0.7, 4.0)]:
        op = Q.qtt_gamma_operator(ctx64, n, lam0, mu0, NAMES[scheme], 1e-12)
        G = oq.tto_full(from_lib_op(op.cores(), op.shape()[3]))
        ref = oq.tto_full(oq.gamma_qtt(n, lam0, mu0, 1e-12, scheme=scheme))
        assert rel(G, ref) < 1e-9
        direct = oq.tto_full(oq.gamma_qtt(n, lam0, mu0, 1e-12))
        assert rel(G, direct) > 1e-3


def test_gamma_operator_scheme_arguments(Q, ctx64):
    """A scheme outside 0..5 and n = 9 for a complex scheme are rejected with
    QTT_EINVAL before any device work."""
    with pytest.raises(Q.QttError) as ei:
        Q.qtt_gamma_operator(ctx64, 3, 1.0, 1.0, 6, 1e-8)
    assert ei.value.code == Q.QTT_EINVAL
    with pytest.raises(Q.QttError) as ei:
        Q.qtt_gamma_operator(ctx64, 9, 1.0, 1.0, Q.QTT_SCHEME_STAGGERED, 1e-8)
    assert ei.value.code == Q.QTT_EINVAL


def _off_centre_sphere(n):
    return synth.sphere_field(n, [(0.31, 0.47, 0.62)], [0.3])


@pytest.mark.parametrize("scheme", ["forward", "hex8r", "staggered"])
def test_ls_solve_scheme_vs_dense_oracle(Q, ctx64, scheme):
    """The full solve with the scheme against the dense FFT scheme with the same
    Green operator (Alg. 1), 8^3 off-centre sphere (no mirror symmetry), loads
    e11 and e23."""
    n = 3
    ph = _off_centre_sphere(n)
    E, nu = (1.0, 10.0), (0.3, 0.3)
    dC = Q.qtt_from_phase_field(ctx64, ph, n, E, nu, None, 1e-10)
    p = Q.solve_params(1e-6, 500, 1e-9, 64, NAMES[scheme])
    C, infos, rc = Q.ls_solve_ceff(ctx64, dC, p, loads=[0, 3])
    Cd, imag, its = dense.ceff(ph, E, nu, tol=1e-6, loads=[0, 3], scheme=scheme)
    for k in (0, 3):
        assert np.abs(C[:, k] - Cd[:, k]).max() < 1e-5 * np.abs(Cd).max()
