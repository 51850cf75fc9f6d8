"""Seeded synthetic inputs for the FETI solvers: tile meshes, SIMP densities,
Dirichlet masks and nodal loads.

This module only *describes* state problems (array shapes, random fields,
boundary masks).  It holds none of the solver's arithmetic: no stiffness,
no tearing, no dual operator.  Both the CPU oracle and the CUDA path consume
these descriptions, so a parity test feeds both sides bit-identical inputs.

Conventions shared by every consumer (they are the library's public input
format, not a method choice):

* A problem is a regular grid of ``tiles`` subdomains (modules), each a
  regular grid of ``elems`` unit square (2D) or unit cube (3D) elements.
* Global elements are numbered lexicographically with x fastest, then y,
  then z; global nodes likewise on the (n_el + 1)-per-axis node grid.
* ``rho``: float64 [n_elements], the SIMP relative density of each element.
* ``dirichlet``: uint8 [n_nodes * dim], 1 where that DOF is fixed to zero;
  DOF ``dim * node + d``.
* ``f``: float64 [n_nodes * dim], the global nodal load vector.

The paper's own benchmark geometries (the laminated academic problems and
the modular MBB-beam snapshots, Section 4) are not available; the seeded
random fields below stand in for them with the same structure: fixed regular
modular partitioning and stiffness contrast that reaches the interfaces.  The
academic problems also get stand-ins built from the section's prose only
(laminated beam, laminated grid, grid of stiff inclusions; the material
values and exact geometry are readings).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Tuple

import numpy as np

__all__ = [
    "Problem", "tile_problem", "gaussian_field", "binary_patterns",
    "config1", "config2", "config3", "config4", "config5",
    "layered_beam", "layered_grid", "inclusion_grid", "multiplier_pairs", "multiplier_block",
]


@dataclasses.dataclass
class Problem:
    """One linear-elastic state problem on a tile grid (see module doc)."""

    name: str
    dim: int
    tiles: Tuple[int, ...]
    elems: Tuple[int, ...]
    E0: float
    Emin: float
    nu: float
    p: float
    rho: np.ndarray
    dirichlet: np.ndarray
    f: np.ndarray

    @property
    def n_el_axis(self) -> Tuple[int, ...]:
        return tuple(t * e for t, e in zip(self.tiles, self.elems))

    @property
    def n_node_axis(self) -> Tuple[int, ...]:
        return tuple(n + 1 for n in self.n_el_axis)

    @property
    def n_elements(self) -> int:
        return int(np.prod(self.n_el_axis))

    @property
    def n_nodes(self) -> int:
        return int(np.prod(self.n_node_axis))

    @property
    def n_dofs(self) -> int:
        return self.n_nodes * self.dim

    @property
    def n_subdomains(self) -> int:
        return int(np.prod(self.tiles))

    def node_id(self, *ijk: int) -> int:
        nn = self.n_node_axis
        if self.dim == 2:
            return ijk[0] + nn[0] * ijk[1]
        return ijk[0] + nn[0] * (ijk[1] + nn[1] * ijk[2])


def _empty_bc(dim, tiles, elems):
    nn = [t * e + 1 for t, e in zip(tiles, elems)]
    n_nodes = int(np.prod(nn))
    return nn, np.zeros(n_nodes * dim, np.uint8), np.zeros(n_nodes * dim, np.float64)


def tile_problem(name, dim, tiles, elems, rho, *, bc="clamped_left", E0=1.0,
                 Emin=1e-6, nu=0.3, p=3.0) -> Problem:
    """Wrap a density field with one of the boundary-condition recipes.

    ``clamped_left``: every node on x = 0 is fixed in all directions; a unit
    point load acts in -y (2D) or -z (3D) at the middle node of the x = max
    edge (2D) or face (3D).
    ``mbb``: the two bottom corner nodes (x = 0 and x = max at y = 0) are
    fixed in x and y; a unit -y load acts at the midspan node of the top edge.
    """
    tiles = tuple(int(t) for t in tiles)
    elems = tuple(int(e) for e in elems)
    nn, dmask, f = _empty_bc(dim, tiles, elems)
    def nid(*ijk):
        if dim == 2:
            return ijk[0] + nn[0] * ijk[1]
        return ijk[0] + nn[0] * (ijk[1] + nn[1] * ijk[2])
    if bc == "clamped_left":
        if dim == 2:
            for j in range(nn[1]):
                n = nid(0, j)
                dmask[2 * n:2 * n + 2] = 1
            f[2 * nid(nn[0] - 1, (nn[1] - 1) // 2) + 1] = -1.0
        else:
            for k in range(nn[2]):
                for j in range(nn[1]):
                    n = nid(0, j, k)
                    dmask[3 * n:3 * n + 3] = 1
            f[3 * nid(nn[0] - 1, (nn[1] - 1) // 2, (nn[2] - 1) // 2) + 2] = -1.0
    elif bc == "traction_right":
        # clamped x = 0 edge; uniform traction on the x = max edge with a unit
        # tensile normal (+x) and a unit tangential (-y) resultant, lumped to
        # the edge nodes by the trapezoidal rule (end nodes carry half)
        assert dim == 2
        for j in range(nn[1]):
            n = nid(0, j)
            dmask[2 * n:2 * n + 2] = 1
        h = 1.0 / (nn[1] - 1)
        for j in range(nn[1]):
            w = h * (0.5 if j in (0, nn[1] - 1) else 1.0)
            n = nid(nn[0] - 1, j)
            f[2 * n] += w
            f[2 * n + 1] -= w
    elif bc == "mbb":
        assert dim == 2
        for n in (nid(0, 0), nid(nn[0] - 1, 0)):
            dmask[2 * n:2 * n + 2] = 1
        f[2 * nid((nn[0] - 1) // 2, nn[1] - 1) + 1] = -1.0
    else:
        raise ValueError(bc)
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
    assert rho.size == int(np.prod([t * e for t, e in zip(tiles, elems)]))
    return Problem(name, dim, tiles, elems, float(E0), float(Emin), float(nu), float(p),
                   rho, dmask, f)


def gaussian_field(shape, sigma, rng) -> np.ndarray:
    """Smoothed Gaussian random field mapped to (0, 1).

    White noise -> periodic Gaussian filter of standard deviation ``sigma``
    (in elements, applied in Fourier space) -> standardise -> standard normal
    CDF.  Returned with axis 0 = x (so ``.ravel(order='F')`` is the global
    lexicographic element order).
    """
    noise = rng.standard_normal(shape)
    freqs = [np.fft.fftfreq(n) for n in shape]
    grids = np.meshgrid(*freqs, indexing="ij")
    k2 = sum(g * g for g in grids)
    kernel = np.exp(-2.0 * (math.pi ** 2) * (sigma ** 2) * k2)
    field = np.real(np.fft.ifftn(np.fft.fftn(noise) * kernel))
    field = (field - field.mean()) / max(field.std(), 1e-300)
    from scipy.special import ndtr
    return ndtr(field)


def _assemble_tiles(tile_fields: List[np.ndarray], tiles, elems) -> np.ndarray:
    """Place per-tile element fields (axis 0 = x) into the global lexicographic array."""
    dim = len(tiles)
    full = np.empty(tuple(t * e for t, e in zip(tiles, elems)), np.float64)
    for s, fld in enumerate(tile_fields):
        idx = np.unravel_index(s, tiles, order="F")
        sl = tuple(slice(i * e, (i + 1) * e) for i, e in zip(idx, elems))
        full[sl] = fld
    return full.ravel(order="F") if dim else full


def binary_patterns(n_patterns, elems, sigma, rng, lo=1e-3, hi=1.0):
    """Binary module patterns: smoothed field thresholded at 0.5 -> {lo, hi}."""
    return [np.where(gaussian_field(tuple(elems), sigma, rng) >= 0.5, hi, lo)
            for _ in range(n_patterns)]


def config1(seed: int = 0) -> Problem:
    """2x2 subdomains of 8x8 Q4, rho ~ U[0,1] i.i.d., Emin = 1e-6."""
    rng = np.random.Generator(np.random.PCG64(seed))
    tiles, elems = (2, 2), (8, 8)
    rho = rng.uniform(0.0, 1.0, size=16 * 16)
    return tile_problem("2x2 tiles of 8x8 Q4, iid U[0,1]", 2, tiles, elems, rho, Emin=1e-6)


def config2(tiles: int = 16, elems: int = 32, n_patterns: int = 4, seed: int = 1,
            sigma: float = 4.0) -> Problem:
    """Modular tiles: each subdomain carries one of ``n_patterns`` seeded binary
    patterns (rho in {1e-3, 1}), Emin = 0 so the contrast after p = 3 is 1e9."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pats = binary_patterns(n_patterns, (elems, elems), sigma, rng)
    choice = rng.integers(0, n_patterns, size=tiles * tiles)
    rho = _assemble_tiles([pats[c] for c in choice], (tiles, tiles), (elems, elems))
    return tile_problem(f"{tiles}x{tiles} tiles of {elems}x{elems} Q4, {n_patterns} binary modules",
                        2, (tiles, tiles), (elems, elems), rho, Emin=0.0)


def config3(n_problems: int = 64, seed: int = 3, tile_range=(4, 24), elem_range=(16, 48),
            sigma: float = 8.0) -> List[Problem]:
    """Many independent 2D state problems of uneven size (batching workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for q in range(n_problems):
        t = int(rng.integers(tile_range[0], tile_range[1] + 1))
        e = int(rng.integers(elem_range[0], elem_range[1] + 1))
        fld = gaussian_field((t * e, t * e), sigma, rng)
        rho = np.where(fld >= 0.5, 1.0, 0.0).ravel(order="F")
        out.append(tile_problem(f"batch[{q}] {t}x{t} tiles of {e}x{e}", 2, (t, t), (e, e), rho,
                                Emin=1e-6))
    return out


def config4(tiles: int = 8, elems: int = 8, seed: int = 4, sigma: float = 8.0) -> Problem:
    """3D H8: tiles^3 subdomains of elems^3 elements, smoothed field clipped to [1e-3, 1].

    The field is rounded to a multiple of 2^-20 before clipping: the FFT and the
    normal CDF may differ in their last bits between machines, and the rounding
    makes the densities (and their hash) the same on every host."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = tiles * elems
    fld = np.clip(np.round(gaussian_field((n, n, n), sigma, rng) * 2.0 ** 20) * 2.0 ** -20, 1e-3, 1.0)
    return tile_problem(f"{tiles}^3 tiles of {elems}^3 H8, smoothed field", 3,
                        (tiles,) * 3, (elems,) * 3, fld.ravel(order="F"), Emin=0.0)


def config5(tiles: int = 32, elems: int = 64, volfrac: float = 0.4) -> Problem:
    """MBB-type beam for the compliance / sensitivity loop: uniform start density."""
    n = tiles * elems
    rho = np.full(n * n, volfrac)
    return tile_problem(f"MBB beam {tiles}x{tiles} tiles of {elems}x{elems}", 2, (tiles, tiles),
                        (elems, elems), rho, bc="mbb", Emin=1e-6)


# ---- stand-ins for the academic problems of Section 4 ---------------------------
# Regular partitions built from the prose only (the figure with the geometry and
# the material values is not available): element moduli E = rho (p = 1, Emin = 0)
# with rho in {contrast^-1, 1}; clamped left edge, tensile and tangential
# traction on the right edge.

def _layers(elems: int, layers: int, contrast: float) -> np.ndarray:
    """One square module of ``layers`` horizontal laminae (stiff, compliant, ...)."""
    y = (np.arange(elems) + 0.5) / elems
    lam = np.minimum((y * layers).astype(int), layers - 1)
    row = np.where(lam % 2 == 0, 1.0, 1.0 / contrast)
    return np.tile(row[None, :], (elems, 1))          # axis 0 = x


def _inclusion(elems: int, frac: float, contrast: float) -> np.ndarray:
    """A compliant square module with a centred stiff square inclusion of side frac * elems."""
    c = (np.arange(elems) + 0.5) / elems
    inside = np.abs(c - 0.5) < frac / 2
    return np.where(inside[:, None] & inside[None, :], 1.0, 1.0 / contrast)


def _academic(name, tiles, elems, module, contrast):
    rho = _assemble_tiles([module] * (tiles[0] * tiles[1]), tiles, (elems, elems))
    return tile_problem(name, 2, tiles, (elems, elems), rho, bc="traction_right", E0=1.0, Emin=0.0, p=1.0)


def layered_beam(elems: int = 14, layers: int = 7, contrast: float = 1e3, n: int = 9) -> Problem:
    """A beam of ``n`` square subdomains in a row, each of ``layers`` alternating
    stiff / compliant laminae running along the beam (the jumps reach every
    interface)."""
    return _academic(f"laminated beam 1x{n}, {layers} layers, contrast {contrast:g}", (n, 1), elems,
                     _layers(elems, layers, contrast), contrast)


def layered_grid(elems: int = 16, layers: int = 8, contrast: float = 1e3, n: int = 3) -> Problem:
    """An n x n grid of the same laminated modules (interior cross points).  With
    an even number of laminae a module starts stiff and ends compliant, so the
    horizontal interfaces and the cross points join a compliant lamina to a
    stiff one."""
    return _academic(f"laminated {n}x{n} grid, {layers} layers, contrast {contrast:g}", (n, n), elems,
                     _layers(elems, layers, contrast), contrast)


def inclusion_grid(elems: int = 16, frac: float = 0.5, contrast: float = 1e3, n: int = 4) -> Problem:
    """An n x n grid of compliant modules, each with a centred stiff inclusion
    (homogeneous material along every interface)."""
    return _academic(f"{n}x{n} grid with stiff inclusions, contrast {contrast:g}", (n, n), elems,
                     _inclusion(elems, frac, contrast), contrast)


# ---- seeded test blocks on a multiplier space ------------------------------------
# Two implementations may number and orient the multipliers differently.  A row
# is identified by the (subdomain, local DOF) copies it joins, so test blocks are
# generated from that identity (not from the row's position) and every row is
# multiplied by the sign its implementation gives the canonically first copy:
# B^T X is then the same interface vector on both sides.

_SM_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """The SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
    pseudorandom number generators", OOPSLA 2014) applied to uint64 arrays."""
    with np.errstate(over="ignore"):
        z = x + _SM_GAMMA
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def multiplier_pairs(layout: np.ndarray):
    """Canonical identity of each multiplier row.

    ``layout``: int [n, 6] rows (s1, dof1, sign1, s2, dof2, sign2), s2 = -1 for a
    single-subdomain row.  Returns (keys int64 [n, 4] = the two (s, dof) copies in
    increasing order, (-1, -1) for a missing second copy; sign float64 [n] = the
    row's sign on its first key copy)."""
    L = np.asarray(layout, dtype=np.int64)
    a = L[:, 0:2]
    b = L[:, 3:5]
    has_b = L[:, 3] >= 0
    swap = has_b & ((b[:, 0] < a[:, 0]) | ((b[:, 0] == a[:, 0]) & (b[:, 1] < a[:, 1])))
    first = np.where(swap[:, None], b, a)
    second = np.where(swap[:, None], a, b)
    second = np.where(has_b[:, None], second, -1)
    keys = np.concatenate([first, second], axis=1)
    sign = np.where(swap, L[:, 5], L[:, 2]).astype(np.float64)
    return keys, sign


def multiplier_block(keys: np.ndarray, sign: np.ndarray, m: int, seed: int, col0: int = 0) -> np.ndarray:
    """Test block X [n, m] on a multiplier space: X[l, j] = sign[l] * U(keys[l], col0 + j)
    with U uniform in [-1, 1) from SplitMix64 of the seed, the row's canonical key and
    the column -- the same values whatever order either implementation gives its rows."""
    k = np.asarray(keys, dtype=np.int64).astype(np.uint64)
    h = _splitmix64(np.full(k.shape[0], np.uint64(seed)))
    for c in range(4):
        h = _splitmix64(h ^ k[:, c])
    out = np.empty((k.shape[0], m), np.float64)
    for j in range(m):
        z = _splitmix64(h ^ np.uint64(((col0 + j) * int(_SM_GAMMA)) & 0xFFFFFFFFFFFFFFFF))
        out[:, j] = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0
    return out * np.asarray(sign, np.float64)[:, None]
