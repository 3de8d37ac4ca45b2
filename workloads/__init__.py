"""Seeded synthetic inputs: the problem generators of arXiv:2202.12309 Sec. 4.1.

The paper's Parthenon-hydro runs three problem generators (a linear wave, a
spherical blast wave, Kelvin-Helmholtz) and times uniform and static/adaptive
multilevel meshes built from them (Sec. 5).  No dataset is involved.  This
module builds the initial *conserved* state of such problems on any list of
leaf blocks, from cell-centre coordinates and a counter-based random generator,
so that the result does not depend on how the mesh is split into blocks.

It is the one module that the CUDA path's tests/bench and the CPU oracle both
use.  It holds no step of the numerical method (no reconstruction, flux,
update, time step, ghost exchange or refinement arithmetic): only the initial
data, written as conserved variables U = (rho, rho v, E) with
E = p/(gamma-1) + rho |v|^2 / 2, which is how each problem is defined.

Random numbers: SplitMix64 (Steele, Lea & Flood 2014; Vigna's public
reference), keyed by (seed, level, global cell index) for per-cell noise and by
(seed, stream, counter) for per-problem parameters.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

NVAR = 5
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """SplitMix64 output function applied to the state x (uint64, vectorised)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def to_unit(z):
    """Top 53 bits of a uint64 as a double in [0, 1)."""
    return (np.asarray(z, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def cell_uniform(seed: int, level: int, I, J, K):
    """Uniform [0,1) draw for the cell with global indices (I,J,K) at `level`."""
    with np.errstate(over="ignore"):
        key = (np.uint64(seed) * np.uint64(0x100000001B3)) ^ (np.uint64(level) << np.uint64(60))
        lin = ((np.asarray(K, np.uint64) << np.uint64(40)) | (np.asarray(J, np.uint64) << np.uint64(20))
               | np.asarray(I, np.uint64))
        return to_unit(splitmix64(splitmix64(key ^ lin)))


def stream_uniform(seed: int, stream: int, count: int):
    """`count` uniform [0,1) draws from stream `stream` of `seed`."""
    with np.errstate(over="ignore"):
        base = splitmix64(np.uint64(seed) ^ (np.uint64(stream) << np.uint64(32)))
        ctr = base + np.arange(count, dtype=np.uint64) * _GOLDEN
    return to_unit(splitmix64(ctr))


@dataclasses.dataclass
class Geometry:
    """Block geometry: nx cells per block, nb root blocks, domain [xmin, xmax]."""
    nx: Tuple[int, int, int]
    nb: Tuple[int, int, int]
    xmin: Tuple[float, float, float] = (-0.5, -0.5, -0.5)
    xmax: Tuple[float, float, float] = (0.5, 0.5, 0.5)

    def dx(self, d: int, level: int) -> float:
        return (self.xmax[d] - self.xmin[d]) / float((self.nb[d] * self.nx[d]) << level)


def uniform_leaves(geo: Geometry) -> np.ndarray:
    """Level-0 leaves of a uniform mesh, (level, lx1, lx2, lx3) per row, in
    x1-fastest order.  Callers that need the tree's Z-order take the leaf list
    from the mesh itself."""
    rows = [(0, i, j, k) for k in range(geo.nb[2]) for j in range(geo.nb[1]) for i in range(geo.nb[0])]
    return np.asarray(rows, dtype=np.int64)


def _block_cells(geo: Geometry, leaf):
    """Global indices and cell-centre coordinates (each shaped n3,n2,n1)."""
    lev, l1, l2, l3 = (int(v) for v in leaf)
    idx = []
    xs = []
    for d, l in enumerate((l1, l2, l3)):
        g = l * geo.nx[d] + np.arange(geo.nx[d], dtype=np.int64)
        idx.append(g)
        xs.append(geo.xmin[d] + (g.astype(np.float64) + 0.5) * geo.dx(d, lev))
    K, J, I = np.meshgrid(idx[2], idx[1], idx[0], indexing="ij")
    z, y, x = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return lev, (I, J, K), (x, y, z)


def _alloc(geo: Geometry, leaves) -> np.ndarray:
    return np.zeros((len(leaves), NVAR, geo.nx[2], geo.nx[1], geo.nx[0]), dtype=np.float64)


def blast(geo: Geometry, leaves, gamma: float = 5.0 / 3.0, seed: int = 0, center=(0.0, 0.0, 0.0),
          radius: float = 0.1, rho0: float = 1.0, noise: float = 0.01, p0: float = 0.1,
          p_in: float = 100.0) -> np.ndarray:
    """Spherical blast wave: rho = rho0 (1 + noise (2u-1)), v = 0, p = p0, and
    p = p_in where |x - center| < radius (strict).  noise=0 gives the
    noise-free, mirror-symmetric variant."""
    U = _alloc(geo, leaves)
    for b, leaf in enumerate(leaves):
        lev, (I, J, K), (x, y, z) = _block_cells(geo, leaf)
        rho = rho0 * np.ones_like(x)
        if noise != 0.0:
            u = cell_uniform(seed, lev, I, J, K)
            rho = rho0 * (1.0 + noise * (2.0 * u - 1.0))
        r2 = (x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2
        p = np.where(r2 < radius * radius, p_in, p0)
        U[b, 0] = rho
        U[b, 4] = p / (gamma - 1.0)
    return U


def linear_wave(geo: Geometry, leaves, gamma: float = 5.0 / 3.0, seed: int = 0, amp: float = 1e-4,
                kvec=(1, 0, 0), rho0: float = 1.0, p0: float = 0.6, phase=None) -> np.ndarray:
    """Linear sound wave on (rho0, p0): rho = rho0 (1 + A cos phi),
    v = A c cos phi k_hat, p = p0 + A rho0 c^2 cos phi, phi = 2 pi k.x + phi0,
    c = sqrt(gamma p0 / rho0); phi0 is seeded unless given."""
    if phase is None:
        phase = 2.0 * math.pi * float(stream_uniform(seed, 1, 1)[0])
    c = math.sqrt(gamma * p0 / rho0)
    kn = math.sqrt(sum(float(k) ** 2 for k in kvec))
    khat = [float(k) / kn for k in kvec]
    U = _alloc(geo, leaves)
    for b, leaf in enumerate(leaves):
        _, _, (x, y, z) = _block_cells(geo, leaf)
        ph = 2.0 * math.pi * (kvec[0] * x + kvec[1] * y + kvec[2] * z) + phase
        cp = np.cos(ph)
        rho = rho0 * (1.0 + amp * cp)
        vel = [amp * c * cp * khat[d] for d in range(3)]
        p = p0 + amp * rho0 * c * c * cp
        U[b, 0] = rho
        for d in range(3):
            U[b, 1 + d] = rho * vel[d]
        U[b, 4] = p / (gamma - 1.0) + 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)
    return U


def sod_doubled(geo: Geometry, leaves, gamma: float = 1.4, x_if: float = 0.25, left=(1.0, 0.0, 1.0),
                right=(0.125, 0.0, 0.1)) -> np.ndarray:
    """Sod shock tube made periodic by doubling: the `left` state (rho, v1, p)
    inside |x1| < x_if, the `right` state outside; both interfaces evolve as
    independent (mirrored) Sod problems until their waves meet."""
    U = _alloc(geo, leaves)
    for b, leaf in enumerate(leaves):
        _, _, (x, _, _) = _block_cells(geo, leaf)
        inside = np.abs(x) < x_if
        rho = np.where(inside, left[0], right[0])
        v1 = np.where(inside, left[1], right[1])
        p = np.where(inside, left[2], right[2])
        U[b, 0] = rho
        U[b, 1] = rho * v1
        U[b, 4] = p / (gamma - 1.0) + 0.5 * rho * v1 * v1
    return U


def sod(geo: Geometry, leaves, gamma: float = 1.4, x_if: float = 0.0, left=(1.0, 0.0, 1.0),
        right=(0.125, 0.0, 0.1)) -> np.ndarray:
    """Sod shock tube along x1: the `left` state (rho, v1, p) for x1 < x_if,
    the `right` state for x1 >= x_if (for domains with non-periodic x1
    boundaries)."""
    U = _alloc(geo, leaves)
    for b, leaf in enumerate(leaves):
        _, _, (x, _, _) = _block_cells(geo, leaf)
        inside = x < x_if
        rho = np.where(inside, left[0], right[0])
        v1 = np.where(inside, left[1], right[1])
        p = np.where(inside, left[2], right[2])
        U[b, 0] = rho
        U[b, 1] = rho * v1
        U[b, 4] = p / (gamma - 1.0) + 0.5 * rho * v1 * v1
    return U


def kelvin_helmholtz(geo: Geometry, leaves, gamma: float = 1.4, seed: int = 0, amp: float = 0.01,
                     rho_in: float = 2.0, rho_out: float = 1.0, shear: float = 0.5, p0: float = 2.5,
                     half_width: float = 0.25) -> np.ndarray:
    """Kelvin-Helmholtz shear layers (the paper's adaptive-refinement problem
    generator, Sec. 4.1): rho = rho_in, v1 = +shear inside |x2| < half_width,
    rho = rho_out, v1 = -shear outside; p = p0; seeded perturbations
    amp (u - 1/2) on v1 and v2 in every cell (two independent draws)."""
    U = _alloc(geo, leaves)
    for b, leaf in enumerate(leaves):
        lev, (I, J, K), (x, y, z) = _block_cells(geo, leaf)
        inside = np.abs(y) < half_width
        rho = np.where(inside, rho_in, rho_out)
        v1 = np.where(inside, shear, -shear) + amp * (cell_uniform(seed, lev, I, J, K) - 0.5)
        v2 = amp * (cell_uniform(seed + 1, lev, I, J, K) - 0.5)
        U[b, 0] = rho
        U[b, 1] = rho * v1
        U[b, 2] = rho * v2
        U[b, 4] = p0 / (gamma - 1.0) + 0.5 * rho * (v1 * v1 + v2 * v2)
    return U


def _modes(kmax: int = 2):
    ks = []
    for a in range(-kmax, kmax + 1):
        for b in range(-kmax, kmax + 1):
            for c in range(-kmax, kmax + 1):
                if (a, b, c) != (0, 0, 0) and a * a + b * b + c * c <= kmax * kmax:
                    ks.append((a, b, c))
    return ks


def smooth_random_density(geo: Geometry, leaves, gamma: float = 5.0 / 3.0, seed: int = 0,
                          amp: float = 0.1, p0: float = 0.6) -> np.ndarray:
    """rho = 1 + amp * sum_k a_k cos(2 pi k.x + phi_k) over integer k with
    0 < |k| <= 2, a_k uniform in [-1,1]/#modes and phi_k uniform in [0, 2 pi)
    from `seed`; v = 0, p = p0."""
    ks = _modes(2)
    draws = stream_uniform(seed, 7, 2 * len(ks))
    a = (2.0 * draws[: len(ks)] - 1.0) / len(ks)
    ph = 2.0 * math.pi * draws[len(ks):]
    U = _alloc(geo, leaves)
    for b, leaf in enumerate(leaves):
        _, _, (x, y, z) = _block_cells(geo, leaf)
        rho = np.ones_like(x)
        for m, (k1, k2, k3) in enumerate(ks):
            rho = rho + amp * a[m] * np.cos(2.0 * math.pi * (k1 * x + k2 * y + k3 * z) + ph[m])
        U[b, 0] = rho
        U[b, 4] = p0 / (gamma - 1.0)
    return U


def density_target(geo: Geometry, leaves, seed: int) -> np.ndarray:
    """Target density field for the adjoint loss: the smooth random density of
    another seed, shaped [block, n3, n2, n1]."""
    return smooth_random_density(geo, leaves, seed=seed)[:, 0].copy()


@dataclasses.dataclass
class BatchMember:
    n: int          # cells per dimension (cubic)
    block: int      # block edge
    center: Tuple[float, float, float]
    p_in: float
    seed: int


def batch_members(seed: int, nsim: int = 64, sizes: Sequence[int] = (32, 64, 96, 128),
                  blocks: Sequence[int] = (16, 32)) -> List[BatchMember]:
    """Independent blast-wave problems: n uniform in `sizes`, block edge uniform
    in `blocks` (only those that divide n), centre uniform in [-0.3, 0.3]^3,
    p_in log-uniform in [10, 100]."""
    u = stream_uniform(seed, 11, 6 * nsim).reshape(nsim, 6)
    out = []
    for s in range(nsim):
        n = int(sizes[min(int(u[s, 0] * len(sizes)), len(sizes) - 1)])
        ok = [bk for bk in blocks if n % bk == 0]
        bk = int(ok[min(int(u[s, 1] * len(ok)), len(ok) - 1)])
        c = tuple(float(-0.3 + 0.6 * u[s, 2 + d]) for d in range(3))
        p_in = float(10.0 ** (1.0 + u[s, 5]))
        out.append(BatchMember(n=n, block=bk, center=c, p_in=p_in, seed=seed * 1000 + s))
    return out
