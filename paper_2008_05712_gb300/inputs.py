"""Seeded synthetic inputs for the batched pair-interaction path.

This module is shared by the CUDA path's tests/benchmarks and by the CPU
oracle's tests.  It holds only input generation: particle and atom
distributions, the fixed-point MD input format, and random task lists.  It
contains none of the method's arithmetic (no tree, no interaction list, no
force law, no residency or packing logic).

All generators draw from ``numpy.random.Generator(PCG64(seed))`` and return
float32 arrays laid out as ``xyzm`` (x, y, z, mass) per particle, the layout
the device pool stores.

Workload shapes follow the paper's two applications (Section 4.1 N-body with
Barnes-Hut gravity on clustered particle sets; Section 4.2 cell/patch based
molecular dynamics with a cutoff).  The paper's own datasets (cube300, lambs)
are not available; these seeded distributions stand in for them.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 20080571

# Fixed-point resolution of the MD input format: local offsets are integer
# multiples of 2**-MD_FRAC_BITS.
MD_FRAC_BITS = 21
MD_SCALE = float(1 << MD_FRAC_BITS)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def plummer(n: int, seed: int, a: float = 1.0, total_mass: float = 1.0,
            xmax: float = 0.999) -> np.ndarray:
    """Plummer sphere of ``n`` equal-mass particles, float32 (n, 4) xyzm.

    Radius by inverse CDF of the Plummer cumulative mass profile,
    r = a (X^(-2/3) - 1)^(-1/2) with X uniform on (0, xmax]; the outer
    (1 - xmax) of the mass is truncated.  Directions are isotropic.
    """
    g = rng(seed)
    x = xmax * (1.0 - g.random(n))          # (0, xmax]
    r = a / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
    cos_t = g.uniform(-1.0, 1.0, n)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    phi = g.uniform(0.0, 2.0 * math.pi, n)
    out = np.empty((n, 4), dtype=np.float32)
    out[:, 0] = r * sin_t * np.cos(phi)
    out[:, 1] = r * sin_t * np.sin(phi)
    out[:, 2] = r * cos_t
    out[:, 3] = total_mass / n
    return out


def merger(n1: int, n2: int, seed: int, separation: float = 10.0) -> np.ndarray:
    """Two Plummer spheres on the x axis, equal particle mass (mass ratio
    n1:n2), scale radii 1 and (n2/n1)^(1/3) (equal central density), centre
    of mass at the origin.  float32 (n1+n2, 4)."""
    n = n1 + n2
    a2 = (n2 / n1) ** (1.0 / 3.0)
    p1 = plummer(n1, seed, a=1.0, total_mass=n1 / n)
    p2 = plummer(n2, seed + 1, a=a2, total_mass=n2 / n)
    x1 = -separation * n2 / n
    x2 = separation * n1 / n
    p1[:, 0] += np.float32(x1)
    p2[:, 0] += np.float32(x2)
    return np.concatenate([p1, p2], axis=0)


def drift(xyzm: np.ndarray, seed: int, sigma: float = 1e-3) -> np.ndarray:
    """Random displacement N(0, sigma) per axis; masses unchanged."""
    g = rng(seed)
    out = xyzm.copy()
    out[:, :3] += g.normal(0.0, sigma, (xyzm.shape[0], 3)).astype(np.float32)
    return out


class MDSystem:
    """Lennard-Jones fluid in the fixed-point cell format.

    Every atom carries an integer cell coordinate (cx, cy, cz) on an
    ``ncell``^3 periodic grid and a local offset u in [0, edge) that is an
    integer multiple of 2**-21 and therefore exact in float32.  ``edge`` is
    itself on the 2**-21 grid, and the box length is ``ncell * edge``.

    Attributes
    ----------
    cell : uint32 (n,)  linear cell index cx + ncell*(cy + ncell*cz)
    u    : float32 (n, 4) local offsets (ux, uy, uz, 1.0)
    U    : int64 (n, 3) local offsets in grid units (u * 2**21)
    edge : float  cell edge (exact float32 value)
    E    : int    cell edge in grid units
    ncell: int
    box  : float  ncell * edge
    """

    def __init__(self, cell, U, E, ncell):
        self.cell = cell
        self.U = U
        self.E = int(E)
        self.ncell = int(ncell)
        self.edge = self.E / MD_SCALE
        self.box = self.ncell * self.edge
        u = np.empty((cell.shape[0], 4), dtype=np.float32)
        u[:, :3] = (U / MD_SCALE).astype(np.float32)
        u[:, 3] = 1.0
        self.u = u

    @property
    def n(self):
        return int(self.cell.shape[0])


def fcc_lj(cells_per_axis: int, seed: int, density: float = 0.8442,
           jitter: float = 0.05, ncell: int = 42) -> MDSystem:
    """Jittered FCC lattice with 4 * cells_per_axis^3 atoms.

    Lattice constant (4/density)^(1/3).  The MD cell edge is put on the
    2**-21 grid (box length then becomes ncell * edge exactly); the lattice
    is laid out in that box, every coordinate gets Gaussian jitter of std
    ``jitter``, is wrapped periodically and snapped to the 2**-21 grid.
    """
    lat = (4.0 / density) ** (1.0 / 3.0)
    box0 = cells_per_axis * lat
    E = int(round(box0 / ncell * MD_SCALE))
    box_units = ncell * E                        # box length in grid units
    lat_units = box_units / cells_per_axis       # lattice constant, grid units
    base = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0],
                     [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    idx = np.arange(cells_per_axis)
    gx, gy, gz = np.meshgrid(idx, idx, idx, indexing="ij")
    corners = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1).astype(np.float64)
    pos = (corners[:, None, :] + base[None, :, :]).reshape(-1, 3)  # lattice units
    g = rng(seed)
    pos_units = pos * lat_units + g.normal(0.0, jitter, pos.shape) * MD_SCALE
    X = np.mod(np.rint(pos_units).astype(np.int64), box_units)
    C = X // E
    U = X - C * E
    cell = (C[:, 0] + ncell * (C[:, 1] + ncell * C[:, 2])).astype(np.uint32)
    return MDSystem(cell, U.astype(np.int64), E, ncell)


def lj_2d(cells_per_axis: int, seed: int, density: float = 0.7, jitter: float = 0.05,
          ncell: int = 16) -> MDSystem:
    """Planar Lennard-Jones system: a jittered square lattice of
    cells_per_axis^2 atoms at number density ``density`` (per unit area) in a
    periodic square of ``ncell`` x ``ncell`` cells, in the fixed-point cell
    format of MDSystem with z = 0 (cell index cx + ncell * cy)."""
    lat = (1.0 / density) ** 0.5
    box0 = cells_per_axis * lat
    E = int(round(box0 / ncell * MD_SCALE))
    box_units = ncell * E
    lat_units = box_units / cells_per_axis
    idx = np.arange(cells_per_axis)
    gx, gy = np.meshgrid(idx, idx, indexing="ij")
    pos = np.stack([gx.ravel(), gy.ravel()], axis=1).astype(np.float64) + 0.5
    g = rng(seed)
    pos_units = pos * lat_units + g.normal(0.0, jitter, pos.shape) * MD_SCALE
    X2 = np.mod(np.rint(pos_units).astype(np.int64), box_units)
    X = np.zeros((X2.shape[0], 3), np.int64)
    X[:, :2] = X2
    C = X // E
    C[:, 2] = 0
    U = X - C * E
    cell = (C[:, 0] + ncell * C[:, 1]).astype(np.uint32)
    return MDSystem(cell, U.astype(np.int64), E, ncell)


def md_displace(sys: MDSystem, seed: int, sigma: float) -> MDSystem:
    """Move every atom by N(0, sigma) per axis, re-wrapped into the box."""
    g = rng(seed)
    n = sys.n
    c = sys.cell.astype(np.int64)
    C = np.stack([c % sys.ncell, (c // sys.ncell) % sys.ncell,
                  c // (sys.ncell * sys.ncell)], axis=1)
    box_units = sys.ncell * sys.E
    X = C * sys.E + sys.U
    X = np.mod(X + np.rint(g.normal(0.0, sigma, (n, 3)) * MD_SCALE).astype(np.int64),
               box_units)
    C2 = X // sys.E
    U2 = X - C2 * sys.E
    cell = (C2[:, 0] + sys.ncell * (C2[:, 1] + sys.ncell * C2[:, 2])).astype(np.uint32)
    return MDSystem(cell, U2, sys.E, sys.ncell)


def loguniform_int(g: np.random.Generator, lo: int, hi: int, n: int) -> np.ndarray:
    """Integers floor(exp(U(log lo, log hi))), clipped to [lo, hi]."""
    v = np.floor(np.exp(g.uniform(math.log(lo), math.log(hi), n))).astype(np.int64)
    return np.clip(v, lo, hi)


def uneven_tasks(n_ids: int, n_tasks: int, seed: int, t_range=(8, 1024),
                 s_range=(16, 16384), run=32, order: np.ndarray | None = None):
    """Random gravity tasks over an id space of ``n_ids`` particles.

    Targets: a contiguous run of length nT (log-uniform on t_range) at a
    uniform random start in ``order`` (a permutation of ids; identity if
    None).  Sources: ceil(nS/run) contiguous runs of <= ``run`` ids at
    uniform random starts, truncated to nS (nS log-uniform on s_range).

    Returns (tgt_off uint64 (T+1), tgt_ids uint32, src_off uint64 (T+1),
    src_ids uint32).
    """
    g = rng(seed)
    if order is None:
        order = np.arange(n_ids, dtype=np.uint32)
    order = np.asarray(order, dtype=np.uint32)
    nt = loguniform_int(g, t_range[0], t_range[1], n_tasks)
    ns = loguniform_int(g, s_range[0], s_range[1], n_tasks)
    nt = np.minimum(nt, n_ids)
    tgt_off = np.zeros(n_tasks + 1, dtype=np.uint64)
    src_off = np.zeros(n_tasks + 1, dtype=np.uint64)
    tgt_off[1:] = np.cumsum(nt)
    src_off[1:] = np.cumsum(ns)
    tgt = np.empty(int(tgt_off[-1]), dtype=np.uint32)
    src = np.empty(int(src_off[-1]), dtype=np.uint32)
    tstart = g.integers(0, n_ids - nt + 1)
    for t in range(n_tasks):
        a = int(tgt_off[t])
        tgt[a:a + nt[t]] = order[tstart[t]:tstart[t] + nt[t]]
    for t in range(n_tasks):
        k = int(ns[t])
        nrun = (k + run - 1) // run
        starts = g.integers(0, n_ids - run + 1, nrun)
        ids = order[(starts[:, None] + np.arange(run)[None, :]).ravel()][:k]
        a = int(src_off[t])
        src[a:a + k] = ids
    return tgt_off, tgt, src_off, src


def random_id_batches(id_space: int, n_batches: int, per_batch: int, seed: int,
                      hot: float = 0.5):
    """Id reference traces for residency tests: each batch draws
    ``per_batch`` ids, a fraction ``hot`` from a small hot set (so ids recur
    across batches) and the rest uniformly; duplicates are kept."""
    g = rng(seed)
    hot_set = g.choice(id_space, size=max(1, id_space // 8), replace=False)
    out = []
    for _ in range(n_batches):
        nh = int(per_batch * hot)
        a = g.choice(hot_set, size=nh)
        b = g.integers(0, id_space, per_batch - nh)
        v = np.concatenate([a, b]).astype(np.uint32)
        g.shuffle(v)
        out.append(v)
    return out


def poisson_arrivals(n: int, rate: float, seed: int, producers: int = 16) -> np.ndarray:
    """Open-loop arrival schedule of ``n`` requests, uint64 nanoseconds.

    ``producers`` independent Poisson producers, each at ``rate/producers``
    requests per second (exponential inter-arrival times), merged in time
    order; the merged stream is Poisson at the aggregate ``rate``.  Returns
    the first ``n`` arrival times of the merged stream, non-decreasing.
    """
    g = rng(seed)
    per = rate / producers
    # enough arrivals per producer to cover the first n of the merge with
    # overwhelming probability
    k = int(n / producers + 8 * math.sqrt(n / producers) + 16)
    while True:
        gaps = g.exponential(1.0 / per, size=(producers, k))
        t = np.cumsum(gaps, axis=1).ravel()
        t.sort()
        horizon = np.cumsum(gaps, axis=1)[:, -1].min()
        if t.shape[0] >= n and t[n - 1] <= horizon:
            return np.round(t[:n] * 1e9).astype(np.uint64)
        k *= 2
