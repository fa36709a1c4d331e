"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds none of the method's arithmetic: it only names workloads (grid,
domain, boundary mode) and samples right-hand sides on the box lattice.  Both the
CUDA library and the oracle decide for themselves which lattice nodes are unknowns.

Right-hand side: the paper's rho comes from a particle bunch deposited on the grid
(Sec. 4); a synthetic Gaussian bunch rho = exp(-1/2 sum((x_i - c_i)/sigma_i)^2)
(peak 1, epsilon_0 = 1) stands in for it.  The centre jitter is drawn from
splitmix64 (Steele, Lea, Flood 2014: add 0x9E3779B97F4A7C15, then two xor-shift /
multiply rounds with 0xBF58476D1CE4E5B9 and 0x94D049BB133111EB, xor-shift 31).
"""
from dataclasses import dataclass, field
from typing import Tuple

import numpy as np

CONSTANT, LINEAR, QUADRATIC = 0, 1, 2
Z_ROBIN, Z_DIRICHLET = 0, 1

_M64 = (1 << 64) - 1


def splitmix64(state: int):
    """One splitmix64 step: returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & _M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return state, z ^ (z >> 31)


def uniform(seed: int, count: int, lo: float, hi: float):
    """`count` doubles uniform in [lo, hi) from splitmix64 seeded with `seed`."""
    out = []
    s = seed & _M64
    for _ in range(count):
        s, z = splitmix64(s)
        out.append(lo + (hi - lo) * ((z >> 11) * (1.0 / (1 << 53))))
    return out


@dataclass
class Grid:
    n: Tuple[int, int, int]
    h: Tuple[float, float, float]
    origin: Tuple[float, float, float]

    @property
    def nbox(self):
        return self.n[0] * self.n[1] * self.n[2]

    def axes(self):
        return [self.origin[d] + np.arange(self.n[d], dtype=np.float64) * self.h[d] for d in range(3)]


def cell_centred_grid(nx, ny=None, nz=None) -> Grid:
    """Unit box centred at 0 with h_i = 1/n_i and nodes at cell centres."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    h = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    return Grid((nx, ny, nz), h, tuple(-0.5 + hh / 2.0 for hh in h))


def vertex_grid(m) -> Grid:
    """Vertex-centred unit box [-1/2, 1/2]^3 with m intervals per axis (m+1 nodes)."""
    h = 1.0 / m
    return Grid((m + 1, m + 1, m + 1), (h, h, h), (-0.5, -0.5, -0.5))


@dataclass
class Domain:
    a: float
    b: float
    taper: float = 1.0
    cx: float = 0.0
    cy: float = 0.0
    zbc: int = Z_ROBIN
    symmetrize: int = 1


@dataclass
class Workload:
    name: str
    grid: Grid
    domain: Domain
    mode: int
    sigma: Tuple[float, float, float] = (0.1, 0.1, 0.2)
    centre: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    jitter: float = 0.02
    params: dict = field(default_factory=dict)


def gaussian_bunch(grid: Grid, centre, sigma, seed: int, jitter: float = 0.02):
    """rho on the whole box (x fastest), float64, centre jittered by U(-jitter, jitter)^3."""
    j = uniform(0x5EED0000 + seed, 3, -jitter, jitter) if jitter > 0 else [0.0, 0.0, 0.0]
    c = [centre[d] + j[d] for d in range(3)]
    x, y, z = grid.axes()
    gx = np.exp(-0.5 * ((x - c[0]) / sigma[0]) ** 2)
    gy = np.exp(-0.5 * ((y - c[1]) / sigma[1]) ** 2)
    gz = np.exp(-0.5 * ((z - c[2]) / sigma[2]) ** 2)
    rho = gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return np.ascontiguousarray(rho.reshape(-1))


def pipe_workload(n: int, mode: int = LINEAR) -> Workload:
    """Elliptic pipe (semi-axes 0.45 / 0.30) in an n^3 cell-centred box, off-centre bunch."""
    return Workload(f"elliptic_pipe_{n}^3", cell_centred_grid(n), Domain(0.45, 0.30), mode,
                    centre=(0.08, 0.04, 0.10), params=dict(max_coarse=4096))


def cylinder_workload(n: int = 32, mode: int = CONSTANT) -> Workload:
    """Circular pipe of radius 0.45 in an n^3 cell-centred box, centred bunch."""
    return Workload(f"cylinder_{n}^3", cell_centred_grid(n), Domain(0.45, 0.45), mode,
                    params=dict(max_coarse=1000, max_levels=3))


def taper_workload(nx, ny, nz, mode: int = LINEAR) -> Workload:
    """Circular pipe narrowing linearly from radius 0.45 to 0.30 along z."""
    return Workload(f"taper_{nx}x{ny}x{nz}", cell_centred_grid(nx, ny, nz),
                    Domain(0.45, 0.45, taper=0.30 / 0.45), mode)


def bunch_particles(grid: Grid, n: int, centre, sigma, seed: int, total_charge: float = 1.0):
    """Synthetic macro-particles of a Gaussian bunch: positions ~ N(centre, sigma) per axis
    (numpy PCG64, seed), kept when all 8 surrounding lattice nodes lie in the box; equal
    charges summing to total_charge.  Returns x, y, z, q (float64 arrays)."""
    rng = np.random.default_rng(seed)
    lo = np.array(grid.origin)
    hi = lo + (np.array(grid.n) - 1) * np.array(grid.h)
    out = []
    while sum(len(a) for a in out) < n:
        p = rng.normal(np.array(centre), np.array(sigma), size=(n, 3))
        p = p[np.all((p >= lo) & (p < hi), axis=1)]
        out.append(p)
    p = np.concatenate(out)[:n]
    q = np.full(n, total_charge / n)
    return p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(), q


def gaussian_bunch_torch(grid: Grid, centre, sigma, seed: int, jitter: float = 0.02, device="cuda"):
    """The same Gaussian bunch built with torch on the device (for large serving workloads)."""
    import torch
    j = uniform(0x5EED0000 + seed, 3, -jitter, jitter) if jitter > 0 else [0.0, 0.0, 0.0]
    c = [centre[d] + j[d] for d in range(3)]
    ax = [grid.origin[d] + torch.arange(grid.n[d], dtype=torch.float64, device=device) * grid.h[d]
          for d in range(3)]
    g = [torch.exp(-0.5 * ((ax[d] - c[d]) / sigma[d]) ** 2) for d in range(3)]
    return (g[2][:, None, None] * g[1][None, :, None] * g[0][None, None, :]).reshape(-1).contiguous()


@dataclass
class Request:
    rid: int
    arrival: float       # seconds after the start of the stream
    geometry: int        # index into the geometry table
    step: int            # PIC time step of this geometry (the bunch drifts +0.005 in z per step)
    seed: int


def serving_geometries(count: int = 20, seed: int = 7, sizes=(32, 48, 64, 96, 128, 160, 192, 256)):
    """`count` geometries: kind cycles cylinder / elliptic pipe / taper, grid drawn from `sizes`."""
    out = []
    s = seed & _M64
    for g in range(count):
        s, z = splitmix64(s)
        n = sizes[z % len(sizes)]
        kind = g % 3
        if kind == 0:
            w = cylinder_workload(n, LINEAR)
        elif kind == 1:
            w = pipe_workload(n, LINEAR)
        else:
            w = taper_workload(n, n, n, LINEAR)
        w.name = f"g{g}_{w.name}"
        out.append(w)
    return out


def serving_requests(count: int = 10000, mean_gap_s: float = 0.002, ngeom: int = 20, seed: int = 99):
    """Poisson arrivals (exponential gaps) over `ngeom` geometries; each geometry's requests are
    consecutive time steps of one simulation."""
    import math
    out = []
    s = seed & _M64
    t = 0.0
    steps = [0] * ngeom
    for r in range(count):
        s, z1 = splitmix64(s)
        s, z2 = splitmix64(s)
        u = ((z1 >> 11) + 1) * (1.0 / ((1 << 53) + 1))
        t += -mean_gap_s * math.log(u)
        g = z2 % ngeom
        out.append(Request(r, t, g, steps[g], seed=1000 * g + steps[g]))
        steps[g] += 1
    return out


def batched_instances(count: int = 64, seed: int = 1234, lo: int = 48, hi: int = 160):
    """`count` instances with n_x, n_y, n_z drawn independently from U{lo..hi} (h_i = 1/n_i);
    geometry cycles cylinder / elliptic pipe / taper 0.45 -> 0.30."""
    out = []
    s = seed & _M64
    for k in range(count):
        n = []
        for _ in range(3):
            s, z = splitmix64(s)
            n.append(lo + z % (hi - lo + 1))
        grid = cell_centred_grid(*n)
        kind = k % 3
        if kind == 0:
            dom = Domain(0.45, 0.45)
        elif kind == 1:
            dom = Domain(0.45, 0.30)
        else:
            dom = Domain(0.45, 0.45, taper=0.30 / 0.45)
        out.append(Workload(f"b{k}_{n[0]}x{n[1]}x{n[2]}_k{kind}", grid, dom, LINEAR,
                            centre=(0.0, 0.0, 0.0)))
    return out
