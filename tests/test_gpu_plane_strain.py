"""GPU parity of the 2D (plane-strain) entry against the 2D dense oracle
(oracle/dense2d.py, written on its own and pinned in tests/test_oracle_2d.py),
on a pixel disk off the centre (the paper's 2D Circle geometry) and a random
two-phase section."""
import numpy as np
import pytest

from oracle import dense2d

pytestmark = [
    pytest.mark.gpu,
    pytest.mark.xfail(strict=False, reason="not yet run on a GPU: a failure here is reported "
                                           "without stopping the rest of the suite"),
]

SEED = 2412


@pytest.fixture(scope="module")
def Q(lib_built):
    return lib_built


@pytest.fixture(scope="module")
def ctx64(Q):
    c = Q.Context(0, Q.QTT_FP64, 1 << 30, seed=SEED)
    yield c
    c.close()


def _disk(n, centre=(0.42, 0.57), radius=0.3):
    N = 1 << n
    c = (np.arange(N) + 0.5) / N
    d1 = c[:, None] - centre[0]
    d2 = c[None, :] - centre[1]
    d1 -= np.round(d1)
    d2 -= np.round(d2)
    return (d1 ** 2 + d2 ** 2 <= radius ** 2).astype(np.uint8)


@pytest.mark.parametrize("n,scheme,geometry", [(4, "direct", "disk"),
                                                (3, "staggered", "random")])
def test_plane_strain_vs_2d_oracle(Q, ctx64, n, scheme, geometry):
    N = 1 << n
    ph = (_disk(n) if geometry == "disk"
          else (np.random.default_rng(21).random((N, N)) < 0.4).astype(np.uint8))
    E, nu = (1.0, 10.0), (0.3, 0.3)
    code = {"direct": Q.QTT_SCHEME_DIRECT, "staggered": Q.QTT_SCHEME_STAGGERED}[scheme]
    p = Q.solve_params(1e-6, 500, 1e-9, 64, code)
    C2, infos, rc = Q.ls_solve_ceff_plane_strain(ctx64, ph, n, E, nu, p, eps_tt=1e-10)
    ref, imag, its = dense2d.ceff2(ph, E, nu, tol=1e-6, scheme=scheme)
    assert imag < 1e-10
    assert np.abs(C2 - ref).max() < 1e-5 * np.abs(ref).max()
