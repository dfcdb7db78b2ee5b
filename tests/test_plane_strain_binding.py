"""Host logic of the plane-strain entry (ls_solve_ceff_plane_strain) on the
CPU: the two C-ABI calls it composes are replaced by recorders that answer
with the 3D oracle, so the test checks the grid it uploads (the section
extruded along a broadcast x1 axis), the loads it asks for, the block it
returns and the handle it frees, against the 2D oracle."""
import numpy as np
import pytest

from oracle import dense, dense2d


class _FakeOp:
    def __init__(self, phase, E, nu):
        self.phase, self.E, self.nu, self.freed = phase, E, nu, False

    def free(self):
        self.freed = True


def test_plane_strain_composition(lib_built, monkeypatch):
    Q = lib_built
    calls = {}

    def fake_from_phase(ctx, phase, n, E, nu, lame0=None, eps_tt=1e-6, rmax=1 << 30):
        calls["phase"] = np.array(phase)
        calls["op"] = _FakeOp(np.array(phase), E, nu)
        return calls["op"]

    def fake_solve(ctx, dC, params, loads=None):
        calls["loads"] = list(loads)
        C, _, _ = dense.ceff(dC.phase, dC.E, dC.nu, tol=1e-12, loads=loads)
        return C, [{"status": 0}] * len(loads), 0

    monkeypatch.setattr(Q, "qtt_from_phase_field", fake_from_phase)
    monkeypatch.setattr(Q, "ls_solve_ceff", fake_solve)
    n = 3
    ph = (np.random.default_rng(12).random((8, 8)) < 0.35).astype(np.uint8)
    E, nu = (1.0, 15.0), (0.3, 0.2)
    C2, infos, rc = Q.ls_solve_ceff_plane_strain(None, ph, n, E, nu, params=None)
    assert calls["phase"].shape == (1, 8, 8) and np.array_equal(calls["phase"][0], ph)
    assert calls["loads"] == [1, 2, 3] and calls["op"].freed
    ref, _, _ = dense2d.ceff2(ph, E, nu, tol=1e-12)
    assert np.allclose(C2, ref, atol=1e-10 * np.abs(ref).max())
    assert len(infos) == 3 and rc == 0
    with pytest.raises(ValueError):
        Q.ls_solve_ceff_plane_strain(None, ph[:, :4], n, E, nu, params=None)
