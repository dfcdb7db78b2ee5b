"""Shared test helpers: conversions between oracle operator cores and the
library's core layout, seeded random TTs and the exact C_eff of a laminate."""
import numpy as np

from oracle import dense


def to_lib_op(op_cores):
    """Oracle TTO (all cores 4-D) -> library cores: binary cores of a raised
    operator (diagonal in (d_out, d_in)) become (a, d, a')."""
    out, diag = [], []
    for k, W in enumerate(op_cores):
        a0, do, di, a1 = W.shape
        if k > 0 and do == di:
            D = np.einsum("aiib->aib", W)
            off = W.copy()
            for i in range(do):
                off[:, i, i, :] = 0
            if np.abs(off).max() == 0:
                out.append(D)
                diag.append(True)
                continue
        out.append(W)
        diag.append(False)
    return out, diag


def from_lib_op(cores, diag):
    out = []
    for c, dg in zip(cores, diag):
        if dg:
            a0, d, a1 = c.shape
            W = np.zeros((a0, d, d, a1), dtype=np.complex128)
            for i in range(d):
                W[:, i, i, :] = c[:, i, :]
            out.append(W)
        else:
            out.append(c)
    return out


def random_tt(rng, dims, ranks, scale=1.0):
    cores = []
    for k, d in enumerate(dims):
        shp = (ranks[k], d, ranks[k + 1])
        cores.append(scale * (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)))
    return cores


def laminate_closed_form(ph1d, E, nu):
    """Exact C_eff of layers normal to x3 (normal n = {33, 23, 13} = Voigt
    {2, 3, 4}, tangential t = {11, 22, 12} = Voigt {0, 1, 5})."""
    Cs = [dense.stiffness_voigt(*dense.lame(e, v)) for e, v in zip(E, nu)]
    n_idx, t_idx = [2, 3, 4], [0, 1, 5]
    frac = np.array([np.mean(ph1d == p) for p in range(len(E))])
    avg = lambda f: sum(w * f(C) for w, C in zip(frac, Cs))
    Cnn_inv = lambda C: np.linalg.inv(C[np.ix_(n_idx, n_idx)])
    Cstar_nn = np.linalg.inv(avg(Cnn_inv))
    Cstar_tn = avg(lambda C: C[np.ix_(t_idx, n_idx)] @ Cnn_inv(C)) @ Cstar_nn
    A = avg(lambda C: C[np.ix_(t_idx, t_idx)]
            - C[np.ix_(t_idx, n_idx)] @ Cnn_inv(C) @ C[np.ix_(n_idx, t_idx)])
    Cstar_tt = A + avg(lambda C: C[np.ix_(t_idx, n_idx)] @ Cnn_inv(C)) @ Cstar_nn @ \
        avg(lambda C: Cnn_inv(C) @ C[np.ix_(n_idx, t_idx)])
    out = np.zeros((6, 6))
    out[np.ix_(n_idx, n_idx)] = Cstar_nn
    out[np.ix_(t_idx, n_idx)] = Cstar_tn
    out[np.ix_(n_idx, t_idx)] = Cstar_tn.T
    out[np.ix_(t_idx, t_idx)] = Cstar_tt
    return out
