"""Shared test helpers: conversions between oracle operator cores and the
library's core layout, and seeded random TTs."""
import numpy as np


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
