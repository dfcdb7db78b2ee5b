"""Oracle A: dense FFT-based homogenisation (the basic scheme, Alg. 1), fp64.

Test infrastructure only (see ``oracle/__init__.py``).

Conventions (readings of the paper, each stated once here):
  * Voigt order (11, 22, 33, 23, 13, 12). Strains carry engineering shear
    (gamma = 2 eps), stresses do not, so sigma_V = C_V eps_V (Sec. 2, Voigt
    paragraph).
  * Reference medium C0: isotropic with the arithmetic mean of the smallest and
    largest phase Lame parameters (the paper does not state C0).
  * Fourier transform: numpy's forward FFT (exp(-2 pi i k x / N)) with numpy's
    frequency representatives (Nyquist at -N/2). This is the same discrete
    operator as the SFFT scheme's exp(+2 pi i k x / N) transform with the
    paper's representatives {-N/2+1, ..., N/2} (App. A) and the conjugated
    momentum-space operator (Sec. 4.3).
  * Nyquist symmetrisation (App. A): the step's stated purpose is the symmetry
    Gamma(q)* = Gamma(-q) that keeps the strain real. For an even N the
    partner of a Nyquist mode is its alias -q mod N, i.e. q with its Nyquist
    components negated, so at those modes Gamma is replaced by the average of
    Gamma(xi) and Gamma(xi with its Nyquist components negated). This makes
    the discrete operator real-preserving and self-adjoint (iterates stay
    real; C_eff is the energy form).
  * Stop test (Alg. 1): ||eps_{m+1} - eps_m||_F / ||E field||_F < tol, with the
    unweighted Euclidean norm over voxels and Voigt components.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

# Voigt index I -> tensor pair (i, j); weight 2 on shear components.
VOIGT = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
WEIGHT = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])


def lame(E: float, nu: float):
    """Lame parameters of an isotropic phase from Young's modulus and Poisson ratio."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def stiffness_tensor(lam: float, mu: float) -> np.ndarray:
    """Isotropic C_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk)."""
    d = np.eye(3)
    return (lam * np.einsum("ij,kl->ijkl", d, d)
            + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))


def stiffness_voigt(lam: float, mu: float) -> np.ndarray:
    """6x6 Voigt stiffness acting on engineering strain (Sec. 2, Voigt notation)."""
    C = stiffness_tensor(lam, mu)
    return np.array([[C[i, j, k, l] for (k, l) in VOIGT] for (i, j) in VOIGT])


def reference_lame(E, nu):
    """(lam0, mu0): arithmetic mean of min and max phase Lame parameters."""
    lm = [lame(e, v) for e, v in zip(E, nu)]
    lams = [a for a, _ in lm]
    mus = [b for _, b in lm]
    return 0.5 * (min(lams) + max(lams)), 0.5 * (min(mus) + max(mus))


def green_tensor_direct(xi: np.ndarray, lam0: float, mu0: float) -> np.ndarray:
    """Gamma^0_ijkl(xi) of the Direct scheme (k = i q, App. A Table) for an
    isotropic C0, from eq. (orig_green_eshelby) worked out in closed form:

      Gamma_ijkl = (d_ik n_j n_l + d_il n_j n_k + d_jk n_i n_l + d_jl n_i n_k)/(4 mu0)
                   - (lam0 + mu0)/(mu0 (lam0 + 2 mu0)) n_i n_j n_k n_l,
    with n = xi/|xi|, and Gamma(0) = 0.  xi: (..., 3) array. Returns (..., 3,3,3,3)."""
    xi = np.asarray(xi, dtype=np.float64)
    r2 = np.sum(xi * xi, axis=-1)
    zero = r2 == 0
    nrm = np.sqrt(np.where(zero, 1.0, r2))
    n = xi / nrm[..., None]
    d = np.eye(3)
    t1 = (np.einsum("ik,...j,...l->...ijkl", d, n, n) + np.einsum("il,...j,...k->...ijkl", d, n, n)
          + np.einsum("jk,...i,...l->...ijkl", d, n, n) + np.einsum("jl,...i,...k->...ijkl", d, n, n))
    beta0 = (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0))
    t2 = np.einsum("...i,...j,...k,...l->...ijkl", n, n, n, n)
    g = t1 / (4.0 * mu0) - beta0 * t2
    g[zero] = 0.0
    return g


def green_voigt_direct(xi: np.ndarray, lam0: float, mu0: float) -> np.ndarray:
    """Voigt form Gamma_V[I, J] = w_I w_J Gamma_{i_I j_I k_J l_J} (..., 6, 6),
    mapping a Voigt stress-like polarisation to an engineering strain."""
    g = green_tensor_direct(xi, lam0, mu0)
    out = np.empty(g.shape[:-4] + (6, 6))
    for I, (i, j) in enumerate(VOIGT):
        for J, (k, l) in enumerate(VOIGT):
            out[..., I, J] = WEIGHT[I] * WEIGHT[J] * g[..., i, j, k, l]
    return out


SCHEMES = ("direct", "centered", "forward", "backward", "hex8r", "staggered")

# Schemes whose divergence operator is k = c(q) v(q) with a factor c common to
# the three components and a real vector v: Gamma is homogeneous of degree 0
# in k, so it is the Direct closed form at v (real, even in v).
REAL_SCHEMES = ("direct", "centered", "hex8r")


def _axis_extents(N) -> np.ndarray:
    return np.broadcast_to(np.asarray(N, dtype=np.float64), (3,))


def _cos_sin(xi: np.ndarray, N, frac: float):
    """cos and sin of frac * 2 pi xi_a / N_a, with the values at xi = 0 and at
    the Nyquist component (2 |xi_a| = N_a) set exactly (sin(pi) = 0,
    cos(pi / 2) = 0) so that the symbols there are exactly real or zero."""
    Nv = _axis_extents(N)
    t = frac * 2.0 * np.pi * xi / Nv
    c, s = np.cos(t), np.sin(t)
    nyq = 2.0 * np.abs(xi) == Nv
    if frac == 1.0:
        s = np.where(nyq, 0.0, s)
        c = np.where(nyq, -1.0, c)
    else:
        c = np.where(nyq, 0.0, c)
        s = np.where(nyq, np.sign(xi), s)
    return c, s


def scheme_vector(xi: np.ndarray, N, scheme: str = "direct") -> np.ndarray:
    """The real vector v whose direction enters the Green operator of a scheme
    with k = c(q) v (App. A table of divergence operators k(q), q_a = 2 pi
    xi_a / N_a).
      Direct:   k = i q, v = xi / N_a (prop. to q). App. A defines q for
                cubic grids only; on a grid with unequal N_a the voxels are read
                as unit cubes (the reading the difference stencils make), so
                q_a = 2 pi xi_a / N_a on every axis.
      Centered: k = i sin(q), v_a = sin(q_a); inserting k = i s into eq.
                (orig_green_eshelby) gives k_i (.)^-1 k_l^* = s_i (.)^-1 s_l
                and s C0 s as the acoustic tensor, i.e. the Direct closed
                form at s. At a Nyquist component sin(pi) = 0 exactly.
      Hex8R:    k_j = (i/4) tan(q_j/2) prod_l (1 + e^{i q_l}) (the rotated
                scheme of the table's source; its printed sum over l is read
                as this product), = 2 i e^{i sum_l q_l / 2} v_j with
                v_j = sin(q_j/2) prod_{l != j} cos(q_l/2). v = 0 (Gamma = 0)
                where two components sit at the Nyquist frequency."""
    xi = np.asarray(xi, dtype=np.float64)
    if scheme == "direct":
        return xi / _axis_extents(N)
    if scheme == "centered":
        return _cos_sin(xi, N, 1.0)[1]
    if scheme == "hex8r":
        c, s = _cos_sin(xi, N, 0.5)
        return np.stack([s[..., 0] * c[..., 1] * c[..., 2],
                         c[..., 0] * s[..., 1] * c[..., 2],
                         c[..., 0] * c[..., 1] * s[..., 2]], axis=-1)
    raise ValueError(scheme)


def difference_symbols(xi: np.ndarray, N):
    """Forward and backward difference symbols of the App. A table under
    numpy's transform (u(x + e_a) -> e^{+i q_a} u_hat):
    k+_a = e^{i q_a} - 1, k-_a = -(e^{-i q_a} - 1) = 1 - e^{-i q_a}.
    Both are real (-2 and +2) at a Nyquist component."""
    c, s = _cos_sin(np.asarray(xi, dtype=np.float64), N, 1.0)
    return (c - 1.0) + 1j * s, (1.0 - c) + 1j * s


def _voigt_symbol(k_normal: np.ndarray, k_shear: np.ndarray) -> np.ndarray:
    """(..., 6, 3) matrix B with eps_hat_V = B u_hat: normal strains
    eps_aa = k_normal_a u_a, engineering shears 2 eps_ab = k_shear_b u_a +
    k_shear_a u_b (Voigt order 11, 22, 33, 23, 13, 12)."""
    shape = k_normal.shape[:-1]
    B = np.zeros(shape + (6, 3), dtype=np.complex128)
    for a in range(3):
        B[..., a, a] = k_normal[..., a]
    for I, (a, b) in enumerate(VOIGT[3:], start=3):
        B[..., I, a] = k_shear[..., b]
        B[..., I, b] = k_shear[..., a]
    return B


def gradient_symbol(xi: np.ndarray, N, scheme: str) -> np.ndarray:
    """B(q) (..., 6, 3) of the strain operator of a complex scheme (App. A
    table): Forward and Backward use k+ resp. k- for every component; the
    staggered grid (the table's dual scheme) takes its normal strains with
    forward and its shear strains with backward differences."""
    kp, km = difference_symbols(xi, N)
    if scheme == "forward":
        return _voigt_symbol(kp, kp)
    if scheme == "backward":
        return _voigt_symbol(km, km)
    if scheme == "staggered":
        return _voigt_symbol(kp, km)
    raise ValueError(scheme)


def green_voigt_from_symbol(B: np.ndarray, lam0: float, mu0: float) -> np.ndarray:
    """eq. (orig_green_eshelby) in Voigt form for a strain operator B(q):
    Gamma_V = B (B^H C0_V B)^-1 B^H (the 3 x 3 acoustic tensor B^H C0_V B is
    Hermitian positive definite where B != 0); Gamma_V = 0 where B = 0. It
    maps a Voigt stress-like polarisation to an engineering strain: the
    displacement solving B^H (C0_V B u + tau) = 0 gives eps = -Gamma_V tau."""
    C0 = stiffness_voigt(lam0, mu0)
    Bh = np.conj(np.swapaxes(B, -1, -2))
    K = Bh @ C0 @ B
    zero = np.sum(np.abs(B) ** 2, axis=(-2, -1)) == 0
    K = np.where(zero[..., None, None], np.eye(3), K)
    G = B @ np.linalg.solve(K, Bh)
    return np.where(zero[..., None, None], 0.0, G)


def green_voigt(xi: np.ndarray, lam0: float, mu0: float, N, scheme: str = "direct"):
    """Gamma_V(xi) of a scheme before the Nyquist rule: the Direct closed form
    at scheme_vector for the real schemes, green_voigt_from_symbol for the
    complex ones (complex output)."""
    if scheme in REAL_SCHEMES:
        return green_voigt_direct(scheme_vector(xi, N, scheme), lam0, mu0)
    return green_voigt_from_symbol(gradient_symbol(xi, N, scheme), lam0, mu0)


def green_voigt_symmetrised(xi: np.ndarray, lam0: float, mu0: float, N,
                            scheme: str = "direct") -> np.ndarray:
    """Gamma_V with the Nyquist symmetrisation of App. A: at modes with a
    component |xi_a| = N_a/2 (the Nyquist frequency of an even axis of N_a
    points) the value is the average of Gamma_V(xi) and Gamma_V at xi with
    those components negated (its aliased partner -xi mod N); elsewhere
    Gamma_V(xi). N is one extent for a cubic grid or the three extents
    (N_1, N_2, N_3); an axis of extent 1 has no Nyquist mode. For the
    Centered, Forward, Backward, Hex8R and staggered schemes the two values
    coincide (their symbols at a Nyquist component are equal at +-N_a/2, or
    differ only by a sign that Gamma does not see), so the rule changes only
    the Direct scheme."""
    xi = np.asarray(xi, dtype=np.float64)
    half = _axis_extents(N) / 2.0
    nyq = (np.abs(xi) == half) & (half >= 1.0)
    flip = np.where(nyq, -xi, xi)
    return 0.5 * (green_voigt(xi, lam0, mu0, N, scheme)
                  + green_voigt(flip, lam0, mu0, N, scheme))


def frequencies(N: int) -> np.ndarray:
    """Integer frequencies xi of numpy's FFT bins (Nyquist at -N/2); q = 2 pi xi / N."""
    return np.fft.fftfreq(N, d=1.0 / N)


def _stiffness_field_apply(phase, Cs, field):
    """sum_J C(x)[I, J] field[J](x) for a phase-indexed list of 6x6 matrices."""
    out = np.zeros_like(field)
    for p, Cp in enumerate(Cs):
        mask = phase == p
        if not mask.any():
            continue
        out[:, mask] = Cp @ field[:, mask]
    return out


def green_field(shape, lam0, mu0, slabs=None, scheme="direct"):
    """Gamma_V at every frequency of an (N1, N2, N3) grid, symmetrised at the
    Nyquist modes of each axis: a list over xi_1 of (N2, N3, 6, 6) slabs.
    Computed once per solve (it depends on the grid and C0 only). slabs: the
    xi_1 bin indices to compute (all by default)."""
    N1, N2, N3 = shape
    f1, f2, f3 = frequencies(N1), frequencies(N2), frequencies(N3)
    x2, x3 = np.meshgrid(f2, f3, indexing="ij")
    out = []
    for a in (range(N1) if slabs is None else slabs):
        xi = np.stack([np.full_like(x2, f1[a]), x2, x3], axis=-1)
        out.append(green_voigt_symmetrised(xi, lam0, mu0, (N1, N2, N3), scheme))
    return out


def _apply_green(tau_hat, G):
    """eps_hat[I] = sum_J Gamma_V[I, J](xi) tau_hat[J], slab by slab in xi_1."""
    out = np.empty_like(tau_hat)
    for a in range(tau_hat.shape[1]):
        out[:, a] = np.einsum("yzIJ,Jyz->Iyz", G[a], tau_hat[:, a])
    return out


def basic_scheme(phase, E, nu, E_voigt, tol=1e-6, max_iter=5000, lame0=None, workers=-1,
                 eps0=None, green=None, scheme="direct"):
    """Alg. 1 (FFT-based homogenisation) on a dense (N1, N2, N3) phase grid.

    Iterates eps_{m+1} = E - IFFT[Gamma_hat FFT[(C - C0) eps_m]] from eps_0 = E
    until ||eps_{m+1} - eps_m||_F / ||E||_F < tol (Alg. 1; LS eq.
    (lippmann_schwinger) and its Fourier form). Returns a dict with the final
    strain field (6, N1, N2, N3) complex, the mean stress sigma_bar = <C eps>
    (Sec. 2, C_eff paragraph), the iteration count and the residual history.
    green: the slabs of green_field(phase.shape, lam0, mu0), when the caller
    already holds them (they are computed here otherwise)."""
    phase = np.asarray(phase)
    lam0, mu0 = reference_lame(E, nu) if lame0 is None else lame0
    C0 = stiffness_voigt(lam0, mu0)
    Cs = [stiffness_voigt(*lame(e, v)) for e, v in zip(E, nu)]
    dCs = [C - C0 for C in Cs]
    Ev = np.asarray(E_voigt, dtype=np.float64)
    shape = phase.shape
    Eb = np.broadcast_to(Ev[:, None, None, None], (6,) + shape).astype(np.complex128)
    eps = Eb.copy() if eps0 is None else np.asarray(eps0, dtype=np.complex128).copy()
    normE = np.linalg.norm(Ev) * np.sqrt(float(np.prod(shape)))
    G = green_field(shape, lam0, mu0, scheme=scheme) if green is None else green
    hist = []
    it = 0
    for it in range(1, max_iter + 1):
        tau = _stiffness_field_apply(phase, dCs, eps)
        tau_hat = sfft.fftn(tau, axes=(1, 2, 3), workers=workers)
        eps_hat = _apply_green(tau_hat, G)
        eps_hat[:, 0, 0, 0] = 0.0
        eps_new = Eb - sfft.ifftn(eps_hat, axes=(1, 2, 3), workers=workers)
        rel = np.linalg.norm(eps_new - eps) / normE
        hist.append(rel)
        eps = eps_new
        if rel < tol:
            break
    sig = _stiffness_field_apply(phase, Cs, eps).reshape(6, -1).mean(axis=1)
    return dict(eps=eps, sigma_bar=sig, iters=it, history=hist, lame0=(lam0, mu0))


def ceff(phase, E, nu, tol=1e-6, max_iter=5000, lame0=None, loads=range(6), scheme="direct"):
    """C_eff column by column from unit Voigt loads E = e_k (Sec. 2). Returns
    (Ceff real 6x6 with column k = Re sigma_bar(e_k), max |Im sigma_bar|, iters)."""
    C = np.zeros((6, 6))
    imag = 0.0
    iters = []
    for k in loads:
        e = np.zeros(6)
        e[k] = 1.0
        r = basic_scheme(phase, E, nu, e, tol=tol, max_iter=max_iter, lame0=lame0, scheme=scheme)
        C[:, k] = r["sigma_bar"].real
        imag = max(imag, float(np.abs(r["sigma_bar"].imag).max()))
        iters.append(r["iters"])
    return C, imag, iters


def stiffness_voigt_derivative(E: float, nu: float, wrt: str) -> np.ndarray:
    """d C_V / d E or d C_V / d nu of an isotropic phase (chain rule through
    lam(E, nu), mu(E, nu))."""
    d = 1.0 - 2.0 * nu
    if wrt == "E":
        dlam = nu / ((1.0 + nu) * d)
        dmu = 1.0 / (2.0 * (1.0 + nu))
    elif wrt == "nu":
        dlam = E * (1.0 + 2.0 * nu * nu) / ((1.0 + nu) ** 2 * d ** 2)
        dmu = -E / (2.0 * (1.0 + nu) ** 2)
    else:
        raise ValueError(wrt)
    return stiffness_voigt(dlam, dmu)


def ceff_gradient_energy(phase, E, nu, eps_fields, params):
    """dC_eff / dp from converged strain fields (one per unit load, Sec. 2):
    at the fixed point of the LS equation the strains minimise the energy over
    E + compatible fields, so  dC_eff[l][k]/dp = < eps_l^T (dC/dp) eps_k >  with
    dC/dp non-zero only in the phase p refers to. params: list of
    (phase index, 'E' or 'nu'). eps_fields: dict k -> (6, N1, N2, N3).
    Returns {param: 6x6 array}."""
    out = {}
    loads = sorted(eps_fields)
    for (p, wrt) in params:
        D = stiffness_voigt_derivative(E[p], nu[p], wrt)
        mask = (np.asarray(phase) == p)
        G = np.zeros((6, 6))
        for k in loads:
            De = np.zeros_like(eps_fields[k])
            De[:, mask] = D @ eps_fields[k][:, mask]
            for l in loads:
                G[l, k] = np.mean(np.sum(eps_fields[l] * De, axis=0)).real
        out[(p, wrt)] = G
    return out
