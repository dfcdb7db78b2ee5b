"""The paper's geometry families (Sec. 5.1 and App. F) as seeded phase fields:
shapes, volume fractions, periodicity, determinism, and the symmetry the 2D
plane-strain C_eff of a symmetric section must have (2D oracle)."""
import numpy as np
import pytest

from oracle import dense2d
from paper_2412_11566_gb300 import synth


def test_shapes_and_fractions():
    n = 4
    assert synth.laminate2d(n).shape == (16, 16) and synth.laminate2d(n).mean() == 0.5
    assert np.all(synth.laminate2d(n) == synth.laminate2d(n)[0])     # layers normal to axis 2
    assert synth.square2d(n).mean() == 0.25
    assert synth.checkerboard2d(n).mean() == 0.5 and synth.checkerboard3d(n).mean() == 0.5
    assert synth.box3d(n).mean() == 0.125
    assert abs(synth.circle2d(6).mean() - np.pi * 0.09) < 0.01
    assert synth.section_3d(synth.circle2d(n)).shape == (1, 16, 16)
    for f in (synth.spots2d, synth.voronoi2d, synth.voronoi3d):
        a, b = f(n), f(n)
        assert a.dtype == np.uint8 and set(np.unique(a)) <= {0, 1} and np.array_equal(a, b)
        assert 0.05 < a.mean() < 0.95
    E, nu = synth.paper_materials()
    assert E == (4.0 / 3.0, 29.0 / 3.0) and nu == (1.0 / 3.0, 1.0 / 3.0)


def test_periodic_wrap():
    """A disk centred on the cell corner is split over the four corners."""
    a = synth.circle2d(5, 0.2, centre=(0.0, 0.0))
    assert a[0, 0] and a[-1, -1] and a[0, -1] and a[-1, 0] and not a[16, 16]
    assert np.array_equal(a, a[::-1, ::-1])


@pytest.mark.parametrize("make", [synth.square2d, synth.circle2d, synth.checkerboard2d])
@pytest.mark.parametrize("scheme", ["centered", "hex8r"])
def test_symmetric_sections_give_symmetric_ceff(make, scheme):
    """Sections symmetric under swapping their axes and under reflections have
    C11 = C22 and no normal-shear coupling in plane strain with the centred
    schemes (2D oracle, paper materials)."""
    ph = make(3)
    E, nu = synth.paper_materials()
    C, imag, _ = dense2d.ceff2(ph, E, nu, tol=1e-10, scheme=scheme)
    assert imag < 1e-12
    assert abs(C[0, 0] - C[1, 1]) < 1e-8 * C[0, 0]
    assert abs(C[0, 2]) < 1e-8 * C[0, 0] and abs(C[1, 2]) < 1e-8 * C[0, 0]


def test_direct_scheme_nyquist_corner_coupling_decays():
    """With the Direct scheme the App. A Nyquist rule (average with all Nyquist
    components negated at once) leaves the normal-shear coupling of Gamma at
    the bins where both components are Nyquist, so a mirror-symmetric square
    shows a small coupling C13 that falls by > 4x per doubling of N."""
    E, nu = synth.paper_materials()
    c = []
    for n in (3, 4, 5):
        C, _, _ = dense2d.ceff2(synth.square2d(n), E, nu, tol=1e-10, loads=[2])
        c.append(abs(C[0, 2] / C[2, 2]))
    assert 1e-5 < c[0] < 1e-3 and c[1] < c[0] / 4 and c[2] < c[1] / 4
