"""GPU: the plane Green operator for x1-broadcast stiffness operators
(qtt_ctx_set_green_broadcast; Sec. 4.3 on broadcast axes). Solves with it
must match solves with the full Green operator and the dense oracle; solves
on geometries without that broadcast must be unaffected by the setting. The
identity behind it is pinned on the CPU in
tests/test_oracle_qtt.py::test_plane_green_on_broadcast_geometry."""
import json
import os

import numpy as np
import pytest

from oracle import dense
from paper_2412_11566_gb300 import synth

pytestmark = [
    pytest.mark.gpu,
    pytest.mark.xfail(strict=False, reason="not yet run on a GPU: a failure here is reported "
                                           "without stopping the rest of the suite"),
]

SEED = 2412
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def Q(lib_built):
    return lib_built


def _solve(Q, phase, n, E, nu, scheme, broadcast, loads):
    ctx = Q.Context(0, Q.QTT_FP64, 1 << 30, seed=SEED)
    try:
        ctx.set_green_broadcast(broadcast)
        dC = Q.qtt_from_phase_field(ctx, phase, n, E, nu, None, 1e-10)
        p = Q.solve_params(1e-6, 500, 1e-9, 128, scheme)
        C, infos, rc = Q.ls_solve_ceff(ctx, dC, p, loads=loads)
        dC.free()
        return C
    finally:
        ctx.close()


@pytest.mark.parametrize("scheme_name", ["direct", "staggered"])
def test_plane_green_matches_full_green_on_broadcast_geometry(Q, scheme_name):
    n = 4
    ph = synth.section_3d(synth.circle2d(n, 0.3, centre=(0.4, 0.55)))   # (1, N, N)
    E, nu = (1.0, 10.0), (0.3, 0.25)
    scheme = {"direct": Q.QTT_SCHEME_DIRECT, "staggered": Q.QTT_SCHEME_STAGGERED}[scheme_name]
    loads = [0, 3]
    Cp = _solve(Q, ph, n, E, nu, scheme, True, loads)
    Cf = _solve(Q, ph, n, E, nu, scheme, False, loads)
    Cd, _, _ = dense.ceff(ph, E, nu, tol=1e-6, loads=loads, scheme=scheme_name)
    for k in loads:
        assert np.abs(Cp[:, k] - Cf[:, k]).max() < 1e-5 * np.abs(Cf[:, k]).max()
        assert np.abs(Cp[:, k] - Cd[:, k]).max() < 1e-5 * np.abs(Cd[:, k]).max()


def test_plane_green_setting_leaves_other_geometries_alone(Q):
    n = 3
    ph = synth.sphere_field(n, [(0.3, 0.4, 0.55)], [0.3])
    E, nu = (1.0, 10.0), (0.3, 0.3)
    a = _solve(Q, ph, n, E, nu, Q.QTT_SCHEME_DIRECT, True, [0])
    b = _solve(Q, ph, n, E, nu, Q.QTT_SCHEME_DIRECT, False, [0])
    # same operators and sketches; only the order of atomic FP64 sums may differ
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(b).max())


@pytest.mark.skipif(os.environ.get("QTT_RUN_2048") != "1",
                    reason="the 2048^3 QTT-only configuration: set QTT_RUN_2048=1 (about 200 GB "
                           "of workspace; minutes per load)")
def test_lamfib2048_load_e11(Q):
    """The 2048^3 laminate-with-fibres configuration (contrast 100, tol 1e-4,
    eps_tt 1e-6, r_max 256), load e11, through the plane Green operator,
    against the stored dense-oracle column (the dense scheme on the reduced
    (1, 2048, 2048) grid)."""
    w = synth.by_name("lamfib2048")
    ref = json.load(open(os.path.join(GOLD, "lamfib2048_ceff_tol0.0001.json")))["columns"]["0"]
    ctx = Q.Context(0, Q.QTT_FP64, 200 << 30, seed=SEED)
    try:
        ctx.set_green_broadcast(True)
        dC = Q.qtt_from_phase_field(ctx, w.phase, w.n, w.E, w.nu, None, w.eps_tt, w.rmax)
        C, infos, rc = Q.ls_solve_ceff(ctx, dC, Q.solve_params(w.tol, 600, w.eps_tt, w.rmax, 0, 16),
                                       loads=[0])
        dC.free()
    finally:
        ctx.close()
    r = np.asarray(ref["sigma_bar_re"])
    assert infos[0]["residual"] < w.tol
    assert np.abs(C[:, 0] - r).max() <= 1e-4 * np.abs(r).max()
