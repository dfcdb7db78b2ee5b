"""Pins of the oracle's discretisation schemes (App. A table of divergence
operators: Direct, Centered, Forward, Backward, Hex8R, staggered grid).

The anchor that does not go through the oracle's momentum-space formulas is a
brute-force real-space construction on tiny periodic grids: the strain
operator D of each scheme assembled from shift matrices (forward, backward,
centred and corner-averaged differences), the Green operator as
D (D^T C0 D)^+ D^T by a dense pseudo-inverse, applied to a random
polarisation and compared with the oracle's FFT application. A slip in a
symbol's sign or direction, in the staggered placement of normal and shear
strains, in a Voigt factor or in the Nyquist handling changes the operator
on these grids and fails it."""
import numpy as np
import pytest
import scipy.fft as sfft

from oracle import dense
from paper_2412_11566_gb300 import synth
from tests._helpers import laminate_closed_form

STENCIL_SCHEMES = ("centered", "forward", "backward", "hex8r", "staggered")


def shift_matrix(shape, a):
    """(S u)(x) = u(x + e_a) on a periodic grid, as a V x V matrix."""
    V = int(np.prod(shape))
    idx = np.arange(V).reshape(shape)
    tgt = np.roll(idx, -1, axis=a)
    S = np.zeros((V, V))
    S[idx.ravel(), tgt.ravel()] = 1.0
    return S


def axis_stencils(shape, scheme):
    """Per-axis difference matrices for the normal and the shear strains."""
    V = int(np.prod(shape))
    I = np.eye(V)
    S = [shift_matrix(shape, a) for a in range(3)]
    fwd = [S[a] - I for a in range(3)]
    bwd = [I - S[a].T for a in range(3)]
    if scheme == "forward":
        return fwd, fwd
    if scheme == "backward":
        return bwd, bwd
    if scheme == "staggered":
        return fwd, bwd
    if scheme == "centered":
        cen = [0.5 * (S[a] - S[a].T) for a in range(3)]
        return cen, cen
    if scheme == "hex8r":
        # strain at the cell corner: the difference along a averaged over the
        # four cell edges parallel to a
        out = []
        for a in range(3):
            M = 0.25 * fwd[a]
            for b in range(3):
                if b != a:
                    M = M @ (I + S[b])
            out.append(M)
        return out, out
    raise ValueError(scheme)


def strain_matrix(shape, scheme):
    """D (6V x 3V): engineering Voigt strain of a displacement field, blocks
    [I][m] of V x V; eps_aa = Dn_a u_a, 2 eps_ab = Ds_b u_a + Ds_a u_b."""
    V = int(np.prod(shape))
    Dn, Ds = axis_stencils(shape, scheme)
    D = np.zeros((6 * V, 3 * V))
    blk = lambda I, m: (slice(I * V, (I + 1) * V), slice(m * V, (m + 1) * V))
    for a in range(3):
        D[blk(a, a)] = Dn[a]
    for I, (a, b) in enumerate(dense.VOIGT[3:], start=3):
        D[blk(I, a)] = Ds[b]
        D[blk(I, b)] = Ds[a]
    return D


def green_real_space(shape, scheme, lam0, mu0):
    D = strain_matrix(shape, scheme)
    V = int(np.prod(shape))
    C0 = np.kron(dense.stiffness_voigt(lam0, mu0), np.eye(V))
    K = D.T @ C0 @ D
    return D @ np.linalg.pinv(K, rcond=1e-10, hermitian=True) @ D.T


def green_fourier_apply(tau, scheme, lam0, mu0):
    shape = tau.shape[1:]
    G = dense.green_field(shape, lam0, mu0, scheme=scheme)
    th = sfft.fftn(tau, axes=(1, 2, 3))
    eh = dense._apply_green(th, G)
    eh[:, 0, 0, 0] = 0.0
    return sfft.ifftn(eh, axes=(1, 2, 3))


@pytest.mark.parametrize("shape", [(4, 4, 4), (2, 4, 6), (1, 4, 6)])
@pytest.mark.parametrize("scheme", STENCIL_SCHEMES)
def test_green_equals_real_space_operator(scheme, shape):
    """Oracle Gamma (momentum space, Nyquist rule included) equals the real-space
    operator of the scheme's difference stencil on every mode of the grid."""
    rng = np.random.default_rng(7)
    lam0, mu0 = 1.9, 0.8
    tau = rng.standard_normal((6,) + shape)
    ref = (green_real_space(shape, scheme, lam0, mu0) @ tau.ravel()).reshape(tau.shape)
    got = green_fourier_apply(tau, scheme, lam0, mu0)
    assert np.abs(got.imag).max() < 1e-12
    assert np.allclose(got.real, ref, atol=1e-11 * np.abs(ref).max())


def test_real_space_check_catches_planted_mistakes(monkeypatch):
    """Swapping forward and backward differences, or taking the staggered
    shear strains with forward differences, fails the real-space comparison."""
    shape = (4, 4, 4)
    rng = np.random.default_rng(8)
    tau = rng.standard_normal((6,) + shape)
    lam0, mu0 = 1.9, 0.8
    ref_f = (green_real_space(shape, "forward", lam0, mu0) @ tau.ravel()).reshape(tau.shape)
    ref_s = (green_real_space(shape, "staggered", lam0, mu0) @ tau.ravel()).reshape(tau.shape)
    orig = dense.difference_symbols
    monkeypatch.setattr(dense, "difference_symbols", lambda xi, N: orig(xi, N)[::-1])
    bad = green_fourier_apply(tau, "forward", lam0, mu0).real
    assert not np.allclose(bad, ref_f, atol=1e-6 * np.abs(ref_f).max())
    monkeypatch.setattr(dense, "difference_symbols", orig)
    monkeypatch.setattr(dense, "gradient_symbol",
                        lambda xi, N, s: dense._voigt_symbol(*([orig(xi, N)[0]] * 2)))
    bad = green_fourier_apply(tau, "staggered", lam0, mu0).real
    assert not np.allclose(bad, ref_s, atol=1e-6 * np.abs(ref_s).max())


def test_symbol_form_equals_closed_form():
    """Gamma_V = B (B^H C0 B)^-1 B^H with B built from k = i v equals the Direct
    closed form at v; with the Hex8R operator written out from the table as
    (i/4) tan(q_j/2) prod_l (1 + e^{i q_l}) it equals the closed form at the
    oracle's scheme_vector (off the Nyquist planes, where tan is finite)."""
    rng = np.random.default_rng(9)
    N = 16
    for _ in range(30):
        lam0, mu0 = rng.uniform(0.1, 5), rng.uniform(0.1, 5)
        v = rng.standard_normal(3)
        B = dense._voigt_symbol(1j * v, 1j * v)
        assert np.allclose(dense.green_voigt_from_symbol(B, lam0, mu0),
                           dense.green_voigt_direct(v, lam0, mu0), atol=1e-12)
        xi = rng.integers(-N // 2 + 1, N // 2, size=3).astype(float)
        if not xi.any():
            continue
        q = 2 * np.pi * xi / N
        kH = 0.25j * np.tan(q / 2) * np.prod(1 + np.exp(1j * q))
        got = dense.green_voigt_from_symbol(dense._voigt_symbol(kH, kH), lam0, mu0)
        ref = dense.green_voigt_direct(dense.scheme_vector(xi, N, "hex8r"), lam0, mu0)
        assert np.allclose(got, ref, atol=1e-10)


@pytest.mark.parametrize("scheme", dense.SCHEMES)
def test_green_projector_hermitian_real_preserving(scheme):
    """On an 8 x 8 x 6 grid: Gamma_V C0 Gamma_V = Gamma_V (for the Direct scheme
    off its Nyquist planes, where the App. A rule averages two projectors),
    Gamma_V is Hermitian, Gamma(0) = 0, and Gamma(-xi mod N) = conj(Gamma(xi))
    on every mode, Nyquist planes included."""
    shape = (8, 8, 6)
    lam0, mu0 = 2.3, 0.7
    C0 = dense.stiffness_voigt(lam0, mu0)
    G = np.stack(dense.green_field(shape, lam0, mu0, scheme=scheme))   # (N1, N2, N3, 6, 6)
    assert np.all(G[0, 0, 0] == 0)
    keep = np.ones(shape, dtype=bool)
    if scheme == "direct":
        for a, N in enumerate(shape):
            sl = [slice(None)] * 3
            sl[a] = N // 2
            keep[tuple(sl)] = False
    assert np.allclose((G @ C0 @ G)[keep], G[keep], atol=1e-12)
    assert np.allclose(G, np.conj(np.swapaxes(G, -1, -2)), atol=1e-13)
    mirror = G[np.ix_(*[(-np.arange(N)) % N for N in shape])]
    assert np.allclose(mirror, np.conj(G), atol=1e-13)


def test_backward_is_conjugate_forward_and_limits():
    """Backward = conj(Forward) at every mode (k- = -conj(k+)); at low
    frequency every scheme approaches the Direct operator (consistency)."""
    shape = (8, 8, 8)
    gf = np.stack(dense.green_field(shape, 1.0, 1.0, scheme="forward"))
    gb = np.stack(dense.green_field(shape, 1.0, 1.0, scheme="backward"))
    assert np.allclose(gb, np.conj(gf), atol=1e-13)
    assert np.abs(gf.imag).max() > 1e-2
    xi = np.array([1.0, -2.0, 1.0])
    ref = dense.green_voigt_direct(xi, 1.2, 0.9)
    for scheme in dense.SCHEMES:
        err = [np.abs(dense.green_voigt(xi, 1.2, 0.9, N, scheme) - ref).max() for N in (256, 512)]
        assert err[1] < 1e-2 and (scheme == "direct" or err[1] < 0.6 * err[0])


@pytest.mark.parametrize("scheme", dense.SCHEMES)
def test_laminate_closed_form_every_scheme(scheme):
    """Layers normal to x3: every scheme's fixed point is the exact laminate
    C_eff (the strain depends on x3 only; for the Centered scheme the two
    layers hold equal numbers of even and odd planes), with a real strain."""
    n = 3
    ph1 = synth.laminate(n, 2)
    ph = synth.broadcast_dense(ph1, n)
    E, nu = (9.0, 1.5), (0.3, 0.2)
    C, imag, _ = dense.ceff(ph, E, nu, tol=1e-13, scheme=scheme)
    ref = laminate_closed_form(ph1.reshape(-1), E, nu)
    assert np.allclose(C, ref, atol=1e-9 * np.abs(ref).max())
    assert imag < 1e-12


def test_schemes_differ_on_an_inclusion():
    """On a sphere the schemes give distinct C_eff columns, Forward and Backward
    the same one (mirror images on a mirror-symmetric geometry), each with a
    real mean stress."""
    ph = synth.centred_sphere(3, 0.3)
    E, nu = (1.0, 10.0), (0.3, 0.3)
    cols = {}
    for scheme in dense.SCHEMES:
        C, imag, _ = dense.ceff(ph, E, nu, tol=1e-10, loads=[0], scheme=scheme)
        assert imag < 1e-10
        cols[scheme] = C[:, 0]
    scale = np.abs(cols["direct"]).max()
    assert np.allclose(cols["forward"], cols["backward"], atol=1e-8 * scale)
    names = [s for s in dense.SCHEMES if s != "backward"]
    for i, a in enumerate(names):
        for b in names[i + 1:]:
            assert np.abs(cols[a] - cols[b]).max() > 1e-4 * scale, (a, b)
