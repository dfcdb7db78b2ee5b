"""Oracle A in 2D: the dense FFT basic scheme (Alg. 1) on an (N1, N2) grid in
plane strain, fp64.

Test infrastructure only (see ``oracle/__init__.py``). Written on its own,
without oracle.dense's Green operator, so that the two can be compared.

Readings of the paper (Sec. 2, Voigt paragraph: 3-component Voigt vectors and
a 3 x 3 stiffness in 2D):
  * Voigt order (11, 22, 12); strains carry engineering shear 2 eps_12,
    stresses do not.
  * Plane strain: an isotropic phase of Lame parameters (lam, mu) has the 2D
    stiffness [[lam + 2 mu, lam, 0], [lam, lam + 2 mu, 0], [0, 0, mu]] (the
    in-plane block of the 3D one), and the reference medium C0 is the
    arithmetic mean of the smallest and largest phase Lame parameters, as in
    3D. The 2D C_eff is then the in-plane block of the 3D C_eff of the same
    section extruded along the third axis.
  * Green operator (App. A, eq. (orig_green_eshelby)) for the scheme's strain
    symbol B(q) (3 x 2, eps_hat_V = B u_hat): Gamma_V = B (B^H C0 B)^-1 B^H,
    0 where B = 0. Divergence operators from App. A's table per axis, with
    q_a = 2 pi xi_a / N_a and numpy's transform (u(x + e_a) -> e^{i q_a}):
      direct    k = i q            centered  k = i sin q
      forward   k+ = e^{iq} - 1    backward  k- = 1 - e^{-iq}
      staggered normal strains with k+, shear strain with k-
      hex8r     the rotated scheme in 2D, k_j = c(q) v_j with a common factor
                c and v_j = sin(q_j/2) cos(q_l/2) (l != j)
    with sin q = 0, cos q = -1 exactly at a Nyquist component and
    cos(q/2) = 0 there.
  * Nyquist symmetrisation (App. A): at a mode with a Nyquist component,
    Gamma is the average of its values at xi and at xi with those components
    negated (its aliased partner).
  * Stop test: ||eps_{m+1} - eps_m||_F / ||E field||_F < tol.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

SCHEMES = ("direct", "centered", "forward", "backward", "hex8r", "staggered")


def lame(E: float, nu: float):
    return E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), E / (2.0 * (1.0 + nu))


def stiffness_voigt2(lam: float, mu: float) -> np.ndarray:
    """Plane-strain Voigt stiffness acting on (eps11, eps22, 2 eps12)."""
    return np.array([[lam + 2 * mu, lam, 0.0], [lam, lam + 2 * mu, 0.0], [0.0, 0.0, mu]])


def reference_lame(E, nu):
    lm = [lame(e, v) for e, v in zip(E, nu)]
    return (0.5 * (min(a for a, _ in lm) + max(a for a, _ in lm)),
            0.5 * (min(b for _, b in lm) + max(b for _, b in lm)))


def _axis_symbols(x: np.ndarray, N: float, scheme: str):
    """(normal, shear) symbol of one axis at integer frequencies x."""
    nyq = 2.0 * np.abs(x) == N
    q = 2.0 * np.pi * x / N
    c = np.where(nyq, -1.0, np.cos(q))
    s = np.where(nyq, 0.0, np.sin(q))
    kp = (c - 1.0) + 1j * s
    km = (1.0 - c) + 1j * s
    if scheme == "direct":
        return 1j * q, 1j * q
    if scheme == "centered":
        return 1j * s, 1j * s
    if scheme == "forward":
        return kp, kp
    if scheme == "backward":
        return km, km
    if scheme == "staggered":
        return kp, km
    raise ValueError(scheme)


def strain_symbol2(xi: np.ndarray, N, scheme: str) -> np.ndarray:
    """B(q) (..., 3, 2): eps11 = kn_1 u1, eps22 = kn_2 u2,
    2 eps12 = kt_2 u1 + kt_1 u2."""
    xi = np.asarray(xi, dtype=np.float64)
    Nv = np.broadcast_to(np.asarray(N, dtype=np.float64), (2,))
    if scheme == "hex8r":
        nyq = 2.0 * np.abs(xi) == Nv
        h = np.pi * xi / Nv
        sh = np.where(nyq, np.sign(xi), np.sin(h))
        ch = np.where(nyq, 0.0, np.cos(h))
        v = np.stack([sh[..., 0] * ch[..., 1], ch[..., 0] * sh[..., 1]], axis=-1)
        kn = kt = 1j * v
    else:
        a = [_axis_symbols(xi[..., j], Nv[j], scheme) for j in range(2)]
        kn = np.stack([a[0][0], a[1][0]], axis=-1)
        kt = np.stack([a[0][1], a[1][1]], axis=-1)
    B = np.zeros(xi.shape[:-1] + (3, 2), dtype=np.complex128)
    B[..., 0, 0] = kn[..., 0]
    B[..., 1, 1] = kn[..., 1]
    B[..., 2, 0] = kt[..., 1]
    B[..., 2, 1] = kt[..., 0]
    return B


def green2(xi: np.ndarray, lam0: float, mu0: float, N, scheme: str = "direct") -> np.ndarray:
    """Gamma_V(xi) (..., 3, 3) of the scheme before the Nyquist rule."""
    B = strain_symbol2(xi, N, scheme)
    C0 = stiffness_voigt2(lam0, mu0)
    Bh = np.conj(np.swapaxes(B, -1, -2))
    K = Bh @ C0 @ B
    zero = np.sum(np.abs(B) ** 2, axis=(-2, -1)) == 0
    K = np.where(zero[..., None, None], np.eye(2), K)
    G = B @ np.linalg.solve(K, Bh)
    return np.where(zero[..., None, None], 0.0, G)


def green2_symmetrised(xi: np.ndarray, lam0: float, mu0: float, N, scheme: str = "direct"):
    """green2 with the Nyquist rule of App. A (average with the aliased partner)."""
    xi = np.asarray(xi, dtype=np.float64)
    half = np.broadcast_to(np.asarray(N, dtype=np.float64), (2,)) / 2.0
    nyq = (np.abs(xi) == half) & (half >= 1.0)
    flip = np.where(nyq, -xi, xi)
    return 0.5 * (green2(xi, lam0, mu0, N, scheme) + green2(flip, lam0, mu0, N, scheme))


def green_field2(shape, lam0, mu0, scheme="direct") -> np.ndarray:
    """Gamma_V at every frequency of an (N1, N2) grid: (N1, N2, 3, 3)."""
    f1 = np.fft.fftfreq(shape[0], d=1.0 / shape[0])
    f2 = np.fft.fftfreq(shape[1], d=1.0 / shape[1])
    X1, X2 = np.meshgrid(f1, f2, indexing="ij")
    return green2_symmetrised(np.stack([X1, X2], axis=-1), lam0, mu0, shape, scheme)


def basic_scheme2(phase, E, nu, E_voigt, tol=1e-6, max_iter=5000, lame0=None, scheme="direct"):
    """Alg. 1 on an (N1, N2) phase grid in plane strain; returns the final strain
    (3, N1, N2), sigma_bar = <C eps>, the iteration count and the residuals."""
    phase = np.asarray(phase)
    lam0, mu0 = reference_lame(E, nu) if lame0 is None else lame0
    C0 = stiffness_voigt2(lam0, mu0)
    Cs = [stiffness_voigt2(*lame(e, v)) for e, v in zip(E, nu)]
    shape = phase.shape
    Ev = np.asarray(E_voigt, dtype=np.float64)
    Eb = np.broadcast_to(Ev[:, None, None], (3,) + shape).astype(np.complex128)
    eps = Eb.copy()
    normE = np.linalg.norm(Ev) * np.sqrt(float(np.prod(shape)))
    G = green_field2(shape, lam0, mu0, scheme)

    def stiff(mats, f):
        out = np.zeros_like(f)
        for p, M in enumerate(mats):
            m = phase == p
            out[:, m] = M @ f[:, m]
        return out

    dCs = [M - C0 for M in Cs]
    hist = []
    it = 0
    for it in range(1, max_iter + 1):
        th = sfft.fftn(stiff(dCs, eps), axes=(1, 2))
        eh = np.einsum("xyIJ,Jxy->Ixy", G, th)
        eh[:, 0, 0] = 0.0
        new = Eb - sfft.ifftn(eh, axes=(1, 2))
        rel = np.linalg.norm(new - eps) / normE
        hist.append(rel)
        eps = new
        if rel < tol:
            break
    sig = stiff(Cs, eps).reshape(3, -1).mean(axis=1)
    return dict(eps=eps, sigma_bar=sig, iters=it, history=hist, lame0=(lam0, mu0))


def ceff2(phase, E, nu, tol=1e-6, max_iter=5000, lame0=None, loads=range(3), scheme="direct"):
    """Plane-strain C_eff (3 x 3) column by column from unit loads; returns
    (C, max |Im sigma_bar|, iterations per load)."""
    C = np.zeros((3, 3))
    imag = 0.0
    its = []
    for k in loads:
        r = basic_scheme2(phase, E, nu, np.eye(3)[k], tol, max_iter, lame0, scheme)
        C[:, k] = r["sigma_bar"].real
        imag = max(imag, float(np.abs(r["sigma_bar"].imag).max()))
        its.append(r["iters"])
    return C, imag, its
