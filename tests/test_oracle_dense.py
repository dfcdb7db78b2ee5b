"""Pins of Oracle A (the dense FFT basic scheme, Alg. 1) against facts the
paper and the mathematics fix: the Green operator's definition and projector
identities, a brute-force DFT, exact solutions (homogeneous medium, laminate),
the LU solution of the discrete Lippmann-Schwinger system, and the Voigt,
Reuss and Hashin-Shtrikman bounds. Each check is chosen so that a plausible
slip in the oracle (a dropped term, a wrong sign, a Voigt factor, a transposed
operand) fails it."""
import json
import os

import numpy as np
import pytest

from oracle import dense
from paper_2412_11566_gb300 import synth
from tests._helpers import laminate_closed_form

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def sym_tensor_from_voigt_strain(e):
    """Engineering-shear Voigt strain -> symmetric 3x3 tensor."""
    t = np.zeros((3, 3), dtype=np.result_type(e, float))
    for I, (i, j) in enumerate(dense.VOIGT):
        v = e[I] if I < 3 else e[I] / 2
        t[i, j] = v
        t[j, i] = v
    return t


def voigt_of_stress(s):
    return np.array([s[i, j] for (i, j) in dense.VOIGT])


def voigt_of_strain(t):
    return np.array([t[i, j] * dense.WEIGHT[I] for I, (i, j) in enumerate(dense.VOIGT)])


def test_paper_material_lame():
    g = json.load(open(os.path.join(GOLD, "paper_values.json")))["materials_2d"]
    lam1, mu1 = dense.lame(g["E1"], g["nu1"])
    lam2, mu2 = dense.lame(g["E2"], g["nu2"])
    # nu = 1/3: lambda = 3E/4, mu = 3E/8 -> exact rationals
    assert np.isclose(lam1, 7.25) and np.isclose(mu1, 3.625)
    assert np.isclose(lam2, 1.0) and np.isclose(mu2, 0.5)


def test_voigt_stiffness_matches_tensor():
    rng = np.random.default_rng(0)
    lam, mu = 2.3, 0.7
    C = dense.stiffness_tensor(lam, mu)
    CV = dense.stiffness_voigt(lam, mu)
    for _ in range(5):
        ev = rng.standard_normal(6)
        eps = sym_tensor_from_voigt_strain(ev)
        sig = np.einsum("ijkl,kl->ij", C, eps)
        assert np.allclose(CV @ ev, voigt_of_stress(sig))
        # energy density sigma : eps = sigma_V . eps_V
        assert np.isclose(np.sum(sig * eps), (CV @ ev) @ ev)


def green_from_definition(xi, lam0, mu0):
    """eq. (orig_green_eshelby): [q_i (q_m C0_mjkn q_n)^-1 q_l]_sym by a
    matrix inverse of the acoustic tensor and explicit symmetrisation."""
    C0 = dense.stiffness_tensor(lam0, mu0)
    K = np.einsum("m,mjkn,n->jk", xi, C0, xi)
    Ninv = np.linalg.inv(K)
    g = np.einsum("i,jk,l->ijkl", xi, Ninv, xi)
    g = 0.5 * (g + g.transpose(1, 0, 2, 3))
    g = 0.5 * (g + g.transpose(0, 1, 3, 2))
    return g


def test_green_closed_form_equals_definition():
    rng = np.random.default_rng(1)
    for _ in range(20):
        xi = rng.standard_normal(3) * rng.uniform(0.1, 10)
        lam0, mu0 = rng.uniform(0.1, 5), rng.uniform(0.1, 5)
        assert np.allclose(dense.green_tensor_direct(xi, lam0, mu0),
                           green_from_definition(xi, lam0, mu0), atol=1e-12)
    assert np.all(dense.green_tensor_direct(np.zeros(3), 1.0, 1.0) == 0)


def test_green_projector_identities():
    rng = np.random.default_rng(2)
    lam0, mu0 = 1.7, 0.9
    C0 = dense.stiffness_tensor(lam0, mu0)
    for _ in range(10):
        xi = rng.standard_normal(3)
        G = dense.green_tensor_direct(xi, lam0, mu0)
        # Gamma C0 Gamma = Gamma
        GCG = np.einsum("ijkl,klmn,mnpq->ijpq", G, C0, G)
        assert np.allclose(GCG, G, atol=1e-12)
        # Gamma C0 sym(xi (x) u) = sym(xi (x) u): compatible strains pass through
        u = rng.standard_normal(3)
        e = 0.5 * (np.outer(xi, u) + np.outer(u, xi))
        assert np.allclose(np.einsum("ijkl,klmn,mn->ij", G, C0, e), e, atol=1e-12)
        # Gamma tau = 0 for equilibrated tau (tau xi = 0)
        B = rng.standard_normal((3, 3))
        P = np.eye(3) - np.outer(xi, xi) / (xi @ xi)
        tau = P @ (B + B.T) @ P
        assert np.allclose(np.einsum("ijkl,kl->ij", G, tau), 0, atol=1e-12)


def test_green_voigt_form():
    rng = np.random.default_rng(3)
    lam0, mu0 = 1.3, 0.6
    for _ in range(5):
        xi = rng.standard_normal(3)
        G = dense.green_tensor_direct(xi, lam0, mu0)
        GV = dense.green_voigt_direct(xi, lam0, mu0)
        B = rng.standard_normal((3, 3))
        tau = B + B.T
        eps = np.einsum("ijkl,kl->ij", G, tau)
        assert np.allclose(GV @ voigt_of_stress(tau), voigt_of_strain(eps))


@pytest.mark.parametrize("N", [4, 8, 16])
def test_fft_against_brute_force_dft(N):
    """The FFT of the oracle equals the O(N^2) DFT per axis on grids up to 16^3."""
    import scipy.fft as sfft
    rng = np.random.default_rng(N)
    f = rng.standard_normal((2, N, N, N)) + 1j * rng.standard_normal((2, N, N, N))
    x = np.arange(N)
    F = np.exp(-2j * np.pi * np.outer(x, x) / N)
    ref = np.einsum("ai,bj,ck,zijk->zabc", F, F, F, f)
    assert np.allclose(sfft.fftn(f, axes=(1, 2, 3)), ref, atol=1e-9 * np.abs(ref).max())
    back = sfft.ifftn(ref, axes=(1, 2, 3))
    assert np.allclose(back, f, atol=1e-12 * np.abs(f).max())


def test_homogeneous_medium_exact():
    """C(x) = C1 everywhere: C_eff = C1 for any reference medium."""
    ph = synth.centred_sphere(3, 0.3)
    E, nu = (2.0, 2.0), (0.25, 0.25)
    C, imag, iters = dense.ceff(ph, E, nu, tol=1e-12, lame0=(0.7, 0.4))
    assert np.allclose(C, dense.stiffness_voigt(*dense.lame(2.0, 0.25)), atol=1e-12)
    assert max(iters) <= 2


def test_laminate_closed_form():
    n = 3
    ph1 = synth.laminate(n, 2)                 # (1, 1, 8): layers normal to x3
    ph = synth.broadcast_dense(ph1, n)
    E, nu = (9.0, 1.5), (0.3, 0.2)
    C, imag, iters = dense.ceff(ph, E, nu, tol=1e-13)
    ref = laminate_closed_form(ph1.reshape(-1), E, nu)
    assert np.allclose(C, ref, atol=1e-9 * np.abs(ref).max())
    # the simple isotropic forms along and across the layers
    lm = [dense.lame(e, v) for e, v in zip(E, nu)]
    assert np.isclose(C[2, 2], 1 / np.mean([1 / (l + 2 * m) for l, m in lm]))
    assert np.isclose(C[3, 3], 1 / np.mean([1 / m for _, m in lm]))
    assert np.isclose(C[5, 5], np.mean([m for _, m in lm]))


def test_fixed_point_equals_lu_solution():
    """On a 4^3 two-phase grid the converged iterate solves the discrete LS
    system (I + Gamma * (C - C0)) eps = E, assembled as a dense 384 x 384
    matrix from an explicit DFT matrix and solved by LU."""
    n = 2
    N = 1 << n
    ph = synth.centred_sphere(n, 0.3)
    E, nu = (1.0, 8.0), (0.3, 0.2)
    lam0, mu0 = dense.reference_lame(E, nu)
    C0 = dense.stiffness_voigt(lam0, mu0)
    Cs = [dense.stiffness_voigt(*dense.lame(e, v)) for e, v in zip(E, nu)]
    ncell = N ** 3
    x = np.arange(N)
    F1 = np.exp(-2j * np.pi * np.outer(x, x) / N)
    F = np.kron(np.kron(F1, F1), F1)                   # (ncell, ncell), C-order cells
    Finv = F.conj().T / ncell
    f = dense.frequencies(N)
    XI = np.stack(np.meshgrid(f, f, f, indexing="ij"), -1).reshape(-1, 3)
    GV = dense.green_voigt_symmetrised(XI, lam0, mu0, N)  # (ncell, 6, 6)
    # Gamma* as a (6 ncell) x (6 ncell) matrix acting on [I][cell] ordering
    Gop = np.zeros((6 * ncell, 6 * ncell), dtype=complex)
    for I in range(6):
        for J in range(6):
            Gop[I * ncell:(I + 1) * ncell, J * ncell:(J + 1) * ncell] = Finv @ np.diag(GV[:, I, J]) @ F
    dC = np.zeros((6 * ncell, 6 * ncell))
    phf = ph.reshape(-1)
    for c in range(ncell):
        M = Cs[phf[c]] - C0
        for I in range(6):
            for J in range(6):
                dC[I * ncell + c, J * ncell + c] = M[I, J]
    A = np.eye(6 * ncell) + Gop @ dC
    for k in (0, 4):
        Ev = np.eye(6)[k]
        rhs = np.repeat(Ev, ncell).astype(complex)
        eps_lu = np.linalg.solve(A, rhs).reshape(6, N, N, N)
        r = dense.basic_scheme(ph, E, nu, Ev, tol=1e-14, max_iter=20000)
        assert np.abs(r["eps"] - eps_lu).max() < 1e-11


def test_bounds_and_symmetry_sphere():
    n = 3
    ph = synth.centred_sphere(n, 0.35)
    E, nu = (1.0, 10.0), (0.3, 0.3)
    C, imag, iters = dense.ceff(ph, E, nu, tol=1e-10)
    Cs = [dense.stiffness_voigt(*dense.lame(e, v)) for e, v in zip(E, nu)]
    frac = np.array([np.mean(ph == p) for p in range(2)])
    voigt = frac[0] * Cs[0] + frac[1] * Cs[1]
    reuss = np.linalg.inv(frac[0] * np.linalg.inv(Cs[0]) + frac[1] * np.linalg.inv(Cs[1]))
    Cs_sym = 0.5 * (C + C.T)
    assert np.linalg.eigvalsh(voigt - Cs_sym).min() > 0
    assert np.linalg.eigvalsh(Cs_sym - reuss).min() > -1e-9
    # symmetric and cubic (centred sphere, even grid)
    assert np.abs(C - C.T).max() < 1e-6 * np.abs(C).max()
    assert np.isclose(C[0, 0], C[1, 1], rtol=1e-6) and np.isclose(C[1, 1], C[2, 2], rtol=1e-6)
    assert np.isclose(C[3, 3], C[4, 4], rtol=1e-6) and np.isclose(C[4, 4], C[5, 5], rtol=1e-6)
    # Hashin-Shtrikman bulk bounds for the effective bulk modulus
    K = [e / (3 * (1 - 2 * v)) for e, v in zip(E, nu)]
    G = [e / (2 * (1 + v)) for e, v in zip(E, nu)]
    Keff = C[:3, :3].sum() / 9.0
    lo, hi = (0, 1) if K[0] < K[1] else (1, 0)
    hs = lambda a, b: K[a] + frac[b] / (1 / (K[b] - K[a]) + 3 * frac[a] / (3 * K[a] + 4 * G[a]))
    assert hs(lo, hi) * (1 - 1e-3) <= Keff <= hs(hi, lo) * (1 + 1e-3)


def test_nyquist_symmetrisation_keeps_fields_real():
    """App. A: the symmetrised operator satisfies Gamma(xi) = Gamma(-xi mod N)
    on the discrete spectrum, so a real polarisation gives a real strain."""
    N = 4
    f = dense.frequencies(N)
    XI = np.stack(np.meshgrid(f, f, f, indexing="ij"), -1)
    G = dense.green_voigt_symmetrised(XI, 1.3, 0.7, N)
    idx = (-np.arange(N)) % N
    partner = G[idx][:, idx][:, :, idx]
    assert np.allclose(G, partner, atol=1e-14)
    ph = synth.centred_sphere(2, 0.3)
    r = dense.basic_scheme(ph, (1.0, 10.0), (0.3, 0.25), np.eye(6)[3], tol=1e-12)
    assert np.abs(r["eps"].imag).max() < 1e-13
    # without the symmetrisation the aliased pairs disagree at Nyquist modes
    raw = dense.green_voigt_direct(XI, 1.3, 0.7)
    assert np.abs(raw - raw[idx][:, idx][:, :, idx]).max() > 1e-3


def test_pin_catches_dropped_green_term(monkeypatch):
    """Plant a mistake (drop the n_i n_j n_k n_l term of Gamma) in the oracle:
    the definition pin and the projector pin must both fail."""
    orig = dense.green_tensor_direct

    def broken(xi, lam0, mu0):
        n = np.asarray(xi, dtype=float) / np.linalg.norm(xi)
        beta0 = (lam0 + mu0) / (mu0 * (lam0 + 2 * mu0))
        return orig(xi, lam0, mu0) + beta0 * np.einsum("i,j,k,l->ijkl", n, n, n, n)

    monkeypatch.setattr(dense, "green_tensor_direct", broken)
    with pytest.raises(AssertionError):
        test_green_closed_form_equals_definition()
    with pytest.raises(AssertionError):
        test_green_projector_identities()


def test_broadcast_grid_equals_full_grid():
    """A field constant along x1 has Fourier content only at xi_1 = 0, so the
    basic scheme on the (1, N, N) grid is the basic scheme on the (N, N, N)
    grid restricted to those modes: same iterates, same sigma_bar. This holds
    only if the Nyquist symmetrisation (App. A) is taken per axis with that
    axis' own extent (a slip that uses N_1 = 1 for all axes moves sigma_bar by
    7e-2 on this random phase field)."""
    n = 3
    N = 1 << n
    rng = np.random.default_rng(5)
    ph1 = (rng.random((1, N, N)) < 0.3).astype(np.uint8)   # broadcast x1
    ph = synth.broadcast_dense(ph1, n)
    E, nu = (1.0, 20.0), (0.3, 0.25)
    for k in (0, 3, 4):
        a = dense.basic_scheme(ph1, E, nu, np.eye(6)[k], tol=0.0, max_iter=8)
        b = dense.basic_scheme(ph, E, nu, np.eye(6)[k], tol=0.0, max_iter=8)
        assert np.allclose(a["sigma_bar"], b["sigma_bar"], rtol=0, atol=1e-12)
        assert np.allclose(a["history"], b["history"], rtol=1e-10, atol=1e-14)
        assert np.allclose(a["eps"][:, 0], b["eps"][:, 0], atol=1e-12)


def green_from_definition_complex(k, lam0, mu0):
    """eq. (orig_green_eshelby) for a complex divergence operator k (App. A
    table): [k_i (k_m^* C0_mjkn k_n)^-1 k_l^*]_sym with a Hermitian acoustic
    tensor, by a matrix inverse and explicit symmetrisation."""
    C0 = dense.stiffness_tensor(lam0, mu0)
    K = np.einsum("m,mjkn,n->jk", k.conj(), C0, k)
    g = np.einsum("i,jk,l->ijkl", k, np.linalg.inv(K), k.conj())
    g = 0.5 * (g + g.transpose(1, 0, 2, 3))
    g = 0.5 * (g + g.transpose(0, 1, 3, 2))
    return g


def test_centered_green_equals_definition():
    """Centered scheme, k_j = i sin(q_j): the definition with that complex k
    is real and equals the Direct closed form at s = sin(q), which is how the
    oracle evaluates it; Nyquist components give s_j = 0 exactly."""
    rng = np.random.default_rng(11)
    N = 16
    for _ in range(20):
        xi = rng.integers(-N // 2 + 1, N // 2 + 1, size=3).astype(float)
        if not np.any(np.sin(2 * np.pi * xi / N) != 0):
            continue
        lam0, mu0 = rng.uniform(0.1, 5), rng.uniform(0.1, 5)
        k = 1j * np.sin(2 * np.pi * xi / N)
        ref = green_from_definition_complex(k, lam0, mu0)
        assert np.abs(ref.imag).max() < 1e-12
        got = dense.green_tensor_direct(dense.scheme_vector(xi, N, "centered"), lam0, mu0)
        assert np.allclose(got, ref.real, atol=1e-12)
    v = dense.scheme_vector(np.array([N / 2, 0.0, -N / 2]), N, "centered")
    assert np.all(v == 0)


def test_centered_scheme_homogeneous_and_distinct():
    """The Centered scheme keeps the homogeneous-medium exactness (C_eff = C1)
    and gives a different C_eff than the Direct scheme on an inclusion."""
    n = 3
    ph = np.zeros((8, 8, 8), dtype=np.uint8)
    E, nu = (3.0, 3.0), (0.3, 0.3)
    C, _, _ = dense.ceff(ph, E, nu, tol=1e-12, lame0=(1.0, 1.2), scheme="centered")
    assert np.allclose(C, dense.stiffness_voigt(*dense.lame(3.0, 0.3)), atol=1e-10)
    ph = synth.centred_sphere(n, 0.3)
    E, nu = (1.0, 10.0), (0.3, 0.3)
    Cc, _, _ = dense.ceff(ph, E, nu, tol=1e-10, loads=[0], scheme="centered")
    Cd, _, _ = dense.ceff(ph, E, nu, tol=1e-10, loads=[0])
    assert np.abs(Cc[:, 0] - Cd[:, 0]).max() > 1e-3 * np.abs(Cd[:, 0]).max()
