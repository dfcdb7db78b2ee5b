"""Seeded synthetic microstructures (voxel phase fields) and material tables.

This module is shared by the CUDA path, the oracle and the tests. It holds no
arithmetic of the homogenisation method: it only draws geometry (which voxel
belongs to which phase) and lists the per-phase (E, nu) pairs of each workload.

Phase fields are uint8 arrays of shape (N1, N2, N3) in C order (x3 fastest);
0 is the matrix, 1 the inclusion phase. An axis of extent 1 is a broadcast
axis (the field is constant along it). Voxel (i, j, k) is sampled at its centre
((i+1/2)/N, (j+1/2)/N, (k+1/2)/N) of the unit cell, with periodic distances.

The shapes follow the paper's geometry families (spheres/boxes, Sec. 5.1;
fibres and laminates, App. F), at the sizes of the benchmark workloads.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    """A named synthetic workload: geometry, materials and solver settings."""
    name: str
    n: int                      # bits per axis, N = 2**n
    phase: np.ndarray           # uint8 (N1, N2, N3); extent 1 = broadcast axis
    E: tuple                    # Young's modulus per phase
    nu: tuple                   # Poisson ratio per phase
    tol: float                  # stop-test tolerance delta_tol
    eps_tt: float               # TT rounding accuracy
    rmax: int                   # TT rank cap
    loads: tuple = (0, 1, 2, 3, 4, 5)  # Voigt unit load cases to solve


def _centres(N: int) -> np.ndarray:
    return (np.arange(N, dtype=np.float64) + 0.5) / N


def _periodic(d: np.ndarray) -> np.ndarray:
    return d - np.round(d)


def sphere_field(n: int, centres, radii) -> np.ndarray:
    """Union of balls (periodic) on a 2^n grid; centres/radii in cell units."""
    N = 1 << n
    c = _centres(N)
    out = np.zeros((N, N, N), dtype=np.uint8)
    for (cx, cy, cz), r in zip(centres, radii):
        dx = _periodic(c - cx) ** 2
        dy = _periodic(c - cy) ** 2
        dz = _periodic(c - cz) ** 2
        inside = (dx[:, None, None] + dy[None, :, None] + dz[None, None, :]) <= r * r
        out[inside] = 1
    return out


def centred_sphere(n: int, radius: float) -> np.ndarray:
    return sphere_field(n, [(0.5, 0.5, 0.5)], [radius])


def random_spheres(n: int, count: int, rmin: float, rmax: float, seed: int,
                   max_tries: int = 100000):
    """Non-overlapping spheres: centres U[0,1)^3, radii U(rmin, rmax).

    Rejection sampling keeps every pair at periodic distance >= r_i + r_j + one
    voxel. Returns (phase, centres, radii)."""
    N = 1 << n
    rng = np.random.default_rng(seed)
    centres, radii = [], []
    tries = 0
    while len(centres) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("sphere packing failed")
        c = rng.random(3)
        r = rng.uniform(rmin, rmax)
        ok = True
        for c2, r2 in zip(centres, radii):
            d = np.linalg.norm(_periodic(c - np.asarray(c2)))
            if d < r + r2 + 1.0 / N:
                ok = False
                break
        if ok:
            centres.append(tuple(c))
            radii.append(r)
    return sphere_field(n, centres, radii), centres, radii


def random_fibres(n: int, seed: int, max_tries: int = 1000):
    """Aligned circular fibres along x3 (broadcast axis: shape (N, N, 1)).

    count ~ U{4..8}, volume fraction phi ~ U(0.3, 0.5), equal radius
    r = sqrt(phi / (count * pi)); centres U[0,1)^2 with periodic distance
    >= 2r + one voxel. If packing fails after max_tries the count is reduced.
    Contrast ~ U(5, 50). Returns (phase, info dict)."""
    N = 1 << n
    rng = np.random.default_rng(seed)
    count = int(rng.integers(4, 9))
    phi = float(rng.uniform(0.3, 0.5))
    contrast = float(rng.uniform(5.0, 50.0))
    while True:
        r = math.sqrt(phi / (count * math.pi))
        centres = []
        tries = 0
        while len(centres) < count and tries < max_tries:
            tries += 1
            c = rng.random(2)
            if all(np.linalg.norm(_periodic(c - np.asarray(c2))) >= 2 * r + 1.0 / N for c2 in centres):
                centres.append(tuple(c))
        if len(centres) == count:
            break
        count -= 1
        if count == 0:
            raise RuntimeError("fibre packing failed")
    c = _centres(N)
    out = np.zeros((N, N, 1), dtype=np.uint8)
    for cx, cy in centres:
        d2 = _periodic(c - cx)[:, None] ** 2 + _periodic(c - cy)[None, :] ** 2
        out[d2 <= r * r, 0] = 1
    return out, dict(count=count, phi=phi, radius=r, contrast=contrast, centres=centres)


def laminate(n: int, layers: int = 2, stiff_first: bool = True) -> np.ndarray:
    """Layers normal to x3 on voxel faces; layer j is stiff when j is even
    (stiff_first) and matrix otherwise. Shape (1, 1, N): broadcast x1, x2."""
    N = 1 << n
    idx = (np.arange(N) * layers) // N
    stiff = (idx % 2 == 0) if stiff_first else (idx % 2 == 1)
    return stiff.astype(np.uint8).reshape(1, 1, N)


def laminate_with_fibres(n: int, radius: float = 0.06, offset=(0.0, 1.0 / 16),
                         layer_offset: float = 0.0) -> np.ndarray:
    """8 layers normal to x3 (stiff in layers 0, 2, 4, 6, the layer pattern
    shifted by layer_offset along x3) plus a 4x4 lattice of stiff fibres along
    x1 centred at ((j+1/2)/4 + offset[0], (k+1/2)/4 + offset[1]) in (x2, x3),
    radius `radius` L. Shape (1, N, N): broadcast x1. The defaults are the
    large QTT-only workload's geometry."""
    N = 1 << n
    c = _centres(N)
    lay = ((np.floor((c - layer_offset) * 8).astype(np.int64) % 2) == 0)
    out = np.broadcast_to(lay[None, :], (N, N)).copy()
    for j in range(4):
        for k in range(4):
            cy, cz = (j + 0.5) / 4 + offset[0], (k + 0.5) / 4 + offset[1]
            d2 = _periodic(c - cy)[:, None] ** 2 + _periodic(c - cz)[None, :] ** 2
            out |= d2 <= radius ** 2
    return out.astype(np.uint8).reshape(1, N, N)


# ------------------------------------------------ the paper's geometry families
# Sec. 5.1 (Fig. geometries: Laminate, Square, Circle) and App. F (Checkerboard,
# Spots, Voronoi), as 2D sections of shape (N, N) and in the paper's two 3D
# generalisations: extruded along x1 (section_3d: Pillar, Circular Pillar,
# reduced Checkerboard, Fibres) or the same in every direction (Box, Sphere,
# Checkerboard 3D, Voronoi 3D). The paper gives no sizes; the defaults below
# are ours: square side L/2, circle radius 0.3 L, 2 x 2 checkerboard tiles,
# 8 spots of radius 0.08 L, 16 Voronoi seeds.

PAPER_MATERIALS = ((29.0 / 3.0, 4.0 / 3.0), (1.0 / 3.0, 1.0 / 3.0))
"""(E, nu) of the geometry figures: grey phase E = 29/3 GPa, white E = 4/3 GPa,
nu = 1/3 for both (phase 1 = grey, phase 0 = white: E = (4/3, 29/3))."""


def paper_materials():
    """(E, nu) per phase index (0 = white matrix, 1 = grey inclusion)."""
    (e_grey, e_white), (nu_grey, nu_white) = PAPER_MATERIALS
    return (e_white, e_grey), (nu_white, nu_grey)


def laminate2d(n: int, layers: int = 2) -> np.ndarray:
    """Layers normal to the section's second axis, stiff first: (N, N)."""
    N = 1 << n
    return np.ascontiguousarray(np.broadcast_to(laminate(n, layers).reshape(1, N), (N, N)))


def square2d(n: int, side: float = 0.5) -> np.ndarray:
    """Centred square inclusion of the given side (in L): (N, N)."""
    c = _centres(1 << n)
    inside = np.abs(c - 0.5) < side / 2
    return (inside[:, None] & inside[None, :]).astype(np.uint8)


def circle2d(n: int, radius: float = 0.3, centre=(0.5, 0.5)) -> np.ndarray:
    """Disk inclusion (periodic distance): (N, N)."""
    c = _centres(1 << n)
    d2 = _periodic(c - centre[0])[:, None] ** 2 + _periodic(c - centre[1])[None, :] ** 2
    return (d2 <= radius * radius).astype(np.uint8)


def checkerboard2d(n: int, tiles: int = 2) -> np.ndarray:
    """tiles x tiles alternating squares: (N, N)."""
    N = 1 << n
    t = (np.arange(N) * tiles) // N
    return ((t[:, None] + t[None, :]) % 2).astype(np.uint8)


def spots2d(n: int, count: int = 8, radius: float = 0.08, seed: int = 2412) -> np.ndarray:
    """count disks of equal radius at seeded uniform centres, allowed to
    overlap (union): (N, N)."""
    rng = np.random.default_rng(seed)
    out = np.zeros((1 << n, 1 << n), dtype=np.uint8)
    for cx, cy in rng.random((count, 2)):
        out |= circle2d(n, radius, (cx, cy))
    return out


def voronoi2d(n: int, seeds: int = 16, seed: int = 2412) -> np.ndarray:
    """Periodic Voronoi tessellation of seeded uniform points; a cell belongs to
    phase (index of its point) mod 2: (N, N)."""
    rng = np.random.default_rng(seed)
    pts = rng.random((seeds, 2))
    c = _centres(1 << n)
    d2 = (_periodic(c[:, None, None] - pts[None, None, :, 0]) ** 2
          + _periodic(c[None, :, None] - pts[None, None, :, 1]) ** 2)
    return (np.argmin(d2, axis=2) % 2).astype(np.uint8)


def section_3d(section: np.ndarray) -> np.ndarray:
    """A 2D section extruded along x1: shape (1, N, N) with x1 broadcast."""
    return np.ascontiguousarray(section[None])


def box3d(n: int, side: float = 0.5) -> np.ndarray:
    """Centred cube inclusion (the Square seen from every direction)."""
    c = _centres(1 << n)
    inside = np.abs(c - 0.5) < side / 2
    return (inside[:, None, None] & inside[None, :, None] & inside[None, None, :]).astype(np.uint8)


def checkerboard3d(n: int, tiles: int = 2) -> np.ndarray:
    """tiles^3 alternating cubes."""
    N = 1 << n
    t = (np.arange(N) * tiles) // N
    return ((t[:, None, None] + t[None, :, None] + t[None, None, :]) % 2).astype(np.uint8)


def voronoi3d(n: int, seeds: int = 16, seed: int = 2412) -> np.ndarray:
    """Periodic 3D Voronoi tessellation, phase = (index of the point) mod 2."""
    rng = np.random.default_rng(seed)
    pts = rng.random((seeds, 3))
    c = _centres(1 << n)
    best = np.full((1 << n,) * 3, np.inf)
    lab = np.zeros((1 << n,) * 3, dtype=np.int64)
    for i, (px, py, pz) in enumerate(pts):
        d2 = (_periodic(c - px)[:, None, None] ** 2 + _periodic(c - py)[None, :, None] ** 2
              + _periodic(c - pz)[None, None, :] ** 2)
        closer = d2 < best
        best = np.where(closer, d2, best)
        lab = np.where(closer, i, lab)
    return (lab % 2).astype(np.uint8)


def broadcast_dense(phase: np.ndarray, n: int) -> np.ndarray:
    """Expand broadcast axes of a phase field to the full (N, N, N) grid."""
    N = 1 << n
    return np.ascontiguousarray(np.broadcast_to(phase, (N, N, N)))


# ---------------------------------------------------------------- workloads

def sphere32_fp64() -> Workload:
    """32^3 grid, one centred sphere r = 0.25 L; matrix E=1, nu=0.3; sphere
    E=10, nu=0.3; load e11; tol 1e-6; eps_tt 1e-8; r_max 64."""
    return Workload("sphere32", 5, centred_sphere(5, 0.25), (1.0, 10.0), (0.3, 0.3),
                    1e-6, 1e-8, 64, loads=(0,))


def spheres256(n: int = 8, seed: int = 2412) -> Workload:
    """8 non-overlapping spheres, radius U(0.05, 0.12) L, seeded centres;
    matrix E=1, nu=0.3; spheres E=20, nu=0.25; 6 loads; tol 1e-4; eps_tt 1e-6;
    r_max 128."""
    ph, _, _ = random_spheres(n, 8, 0.05, 0.12, seed)
    return Workload(f"spheres{1 << n}", n, ph, (1.0, 20.0), (0.3, 0.25), 1e-4, 1e-6, 128)


def lamfib256(n: int = 8) -> Workload:
    """8 layers normal to x3 plus a 4x4 lattice of fibres along x1 (the
    geometry of laminate_with_fibres, broadcast x1) on a 2^n grid; matrix
    E=1, nu=0.3; layers and fibres E=20, nu=0.25; 6 loads; tol 1e-4; eps_tt
    1e-6; r_max 128."""
    return Workload(f"lamfib{1 << n}", n, laminate_with_fibres(n), (1.0, 20.0), (0.3, 0.25),
                    1e-4, 1e-6, 128)


def lamfib_family(n: int = 8, items: int = 64, base_seed: int = 2412):
    """Laminate-with-fibres microstructures for batched C_eff: the large
    QTT-only workload's arrangement (layers and lattice as in
    laminate_with_fibres' defaults) with item i's fibre radius drawn (seed
    base_seed + i) from U(0.045, 0.075) L; materials and solver settings as
    lamfib256. Every item is periodic with period L/4 in x2 and x3."""
    out = []
    for i in range(items):
        rng = np.random.default_rng(base_seed + i)
        r = float(rng.uniform(0.045, 0.075))
        out.append(Workload(f"lamfib{1 << n}_{i}", n, laminate_with_fibres(n, r),
                            (1.0, 20.0), (0.3, 0.25), 1e-4, 1e-6, 128))
    return out


def by_name(name: str) -> Workload:
    """The named workloads of the benchmark and the stored C_eff columns."""
    table = {"spheres256": spheres256, "lamfib256": lamfib256,
             "lamfib2048": laminate_fibres2048}
    return table[name]()


def fibre_batch(items: int = 64, base_seed: int = 2413):
    """Batch of aligned-fibre microstructures, n ~ U{6,7,8,9} per item."""
    out = []
    for i in range(items):
        rng = np.random.default_rng(base_seed + i)
        n = int(rng.integers(6, 10))
        ph, info = random_fibres(n, base_seed + i)
        out.append(Workload(f"fibres{i}", n, ph, (1.0, info["contrast"]), (0.3, 0.25),
                            1e-4, 1e-6, 128))
    return out


def sphere128_grad() -> Workload:
    """128^3 centred sphere at volume fraction 0.15 (r = 0.3296 L), contrast 10."""
    r = (3 * 0.15 / (4 * math.pi)) ** (1.0 / 3.0)
    return Workload("sphere128", 7, centred_sphere(7, r), (1.0, 10.0), (0.3, 0.25),
                    1e-4, 1e-6, 128)


def laminate_fibres2048(n: int = 11) -> Workload:
    """The large QTT-only configuration: laminate_with_fibres on 2048^3
    (broadcast x1), matrix E=1, inclusions E=100, nu 0.3; tol 1e-4, eps_tt
    1e-6, r_max 256."""
    return Workload(f"lamfib{1 << n}", n, laminate_with_fibres(n), (1.0, 100.0), (0.3, 0.3),
                    1e-4, 1e-6, 256)
