"""Seeded synthetic inputs shaped like the workloads of the topological Vicsek study.

This module only draws numbers: positions on the fixed-point grid, initial
headings and run parameters.  It holds none of the method's arithmetic
(neighbor selection, alignment, noise, advection), so both the CUDA path and
the CPU oracle can consume its output without sharing any code with each other.

Conventions used by every generator:

* positions are ``int32`` fixed-point grid coordinates ``pos_q`` in
  ``[0, L_q)`` per axis, where ``L_q = round(L * 2**F)`` and a real
  coordinate is ``pos_q * 2**-F``;
* headings are unit vectors stored as ``float32`` (``dir``); in 2D the
  angle ``theta`` they were drawn from is kept as well;
* all draws come from ``numpy.random.Generator(PCG64(seed))`` with
  ``seed = 1000 + workload index`` unless a seed is passed.

The paper (Sec. "Metric and topological flocking models") studies
self-propelled particles in a periodic domain whose neighbors are the k
nearest particles or the Delaunay/Voronoi neighbors; it names no dataset,
so every input here is synthetic.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

TWO_PI = 2.0 * math.pi


@dataclasses.dataclass
class Workload:
    """One periodic system plus the run parameters it is simulated with."""

    name: str
    dim: int
    pos_q: np.ndarray          # (N, dim) int32 in [0, box_q[a])
    dir: np.ndarray            # (N, dim) float32 unit headings
    theta: Optional[np.ndarray]  # (N,) float32 angles in [0, 2pi) (2D only)
    box_q: tuple               # L_q per axis (python ints)
    frac_bits: int
    rule: str = "knn"          # "knn" | "voronoi" | "metric"
    k: int = 7
    v0: float = 0.5
    dt: float = 1.0
    eta: float = 0.3
    seed: int = 1              # counter-based noise key
    noise: str = "angular"     # "angular" | "vectorial"
    steps: int = 50
    check_every: int = 1
    replica: int = 0

    @property
    def n(self) -> int:
        return int(self.pos_q.shape[0])

    @property
    def box_len(self) -> tuple:
        return tuple(b / float(1 << self.frac_bits) for b in self.box_q)

    @property
    def density(self) -> float:
        vol = 1.0
        for b in self.box_len:
            vol *= b
        return self.n / vol


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def box_q_for(length: float, frac_bits: int) -> int:
    """L_q = round(L * 2**F): the box edge in grid units."""
    lq = int(round(length * float(1 << frac_bits)))
    if lq < 1 or lq > (1 << 31):
        raise ValueError(f"box of {length} at F={frac_bits} gives L_q={lq}, outside [1, 2^31]")
    return lq


def quantize(x: np.ndarray, frac_bits: int, box_q: int) -> np.ndarray:
    """Real coordinates -> grid coordinates, wrapped into [0, L_q)."""
    q = np.floor(np.asarray(x, dtype=np.float64) * float(1 << frac_bits)).astype(np.int64)
    return np.mod(q, box_q).astype(np.int32)


def uniform_positions(rng: np.random.Generator, n: int, box_q: Sequence[int]) -> np.ndarray:
    """Independent uniform integers in [0, L_q) per axis."""
    cols = [rng.integers(0, int(b), size=n, dtype=np.int64) for b in box_q]
    return np.stack(cols, axis=1).astype(np.int32)


def headings_2d(rng: np.random.Generator, n: int):
    """theta ~ U[0, 2pi) in float32 and its unit vector rounded to float32."""
    theta = rng.uniform(0.0, TWO_PI, size=n).astype(np.float32)
    theta = np.where(theta >= np.float32(TWO_PI), np.float32(0.0), theta).astype(np.float32)
    t64 = theta.astype(np.float64)
    d = np.stack([np.cos(t64), np.sin(t64)], axis=1).astype(np.float32)
    return theta, d


def headings_3d(rng: np.random.Generator, n: int) -> np.ndarray:
    """Unit vectors uniform on the sphere, rounded to float32."""
    z = rng.uniform(-1.0, 1.0, size=n)
    ph = rng.uniform(0.0, TWO_PI, size=n)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(ph), s * np.sin(ph), z], axis=1).astype(np.float32)


def uniform_system(n: int, length: float, frac_bits: int, dim: int = 2, input_seed: int = 1000,
                   name: str = "uniform", **params) -> Workload:
    rng = _rng(input_seed)
    bq = box_q_for(length, frac_bits)
    box = (bq,) * dim
    pos = uniform_positions(rng, n, box)
    if dim == 2:
        theta, d = headings_2d(rng, n)
    else:
        theta, d = None, headings_3d(rng, n)
    return Workload(name=name, dim=dim, pos_q=pos, dir=d, theta=theta, box_q=box,
                    frac_bits=frac_bits, **params)


# ---------------------------------------------------------------------------
# The five workload shapes of the study (index 1..5)
# ---------------------------------------------------------------------------

def topological_small(seed: int = 1001) -> Workload:
    """2D kNN (k=7) flock: N=2048 uniform in a periodic square of L=45.25
    (density ~1), F=16, v0=0.5, dt=1, angular noise eta=0.3, 50 steps."""
    return uniform_system(2048, 45.25, 16, 2, seed, name="knn2d_N2048_L45.25_F16",
                          rule="knn", k=7, v0=0.5, dt=1.0, eta=0.3, seed=1,
                          steps=50, check_every=1)


def voronoi_mixed(eta: float = 0.1, seed: int = 1002) -> Workload:
    """2D Voronoi flock: N=65536, L=256 (density 1), F=16.  Left half x in
    [0,128): 32768 uniform points.  Right half: a stretched hexagonal lattice
    of 128 columns x 256 rows with unit spacing, odd rows offset by 1/2,
    plus Gaussian jitter sigma=0.1 per coordinate.  v0=0.3, 1000 steps."""
    rng = _rng(seed)
    L, F = 256.0, 16
    bq = box_q_for(L, F)
    half = 32768
    xl = rng.uniform(0.0, 128.0, size=half)
    yl = rng.uniform(0.0, 256.0, size=half)
    col, row = np.meshgrid(np.arange(128), np.arange(256), indexing="xy")
    col = col.ravel().astype(np.float64)
    row = row.ravel().astype(np.float64)
    xh = 128.0 + col + 0.25 + 0.5 * (row % 2) + rng.normal(0.0, 0.1, size=half)
    yh = row + 0.5 + rng.normal(0.0, 0.1, size=half)
    x = np.concatenate([xl, xh])
    y = np.concatenate([yl, yh])
    pos = np.stack([quantize(x, F, bq), quantize(y, F, bq)], axis=1)
    theta, d = headings_2d(rng, pos.shape[0])
    return Workload(name=f"voronoi2d_N65536_L256_F16_mixed_eta{eta}", dim=2, pos_q=pos, dir=d,
                    theta=theta, box_q=(bq, bq), frac_bits=F, rule="voronoi", k=0,
                    v0=0.3, dt=1.0, eta=eta, seed=1, steps=1000, check_every=100)


def clustered_large(n: int = 1 << 22, k: int = 7, n_clusters: int = 256, sigma: float = 4.0,
                    background: float = 0.2, seed: int = 1003) -> Workload:
    """2D kNN flock at scale: N=2^22 at density 1 (L=2048), F=20.  A mixture
    of 256 Gaussian clusters (sigma=4, centers uniform, 80% of the particles
    split as evenly as possible) and a 20% uniform background.  v0=0.5,
    eta=0.2, 200 steps.  A smaller ``n`` keeps density 1 (L=sqrt(n))."""
    rng = _rng(seed)
    F = 20
    L = math.sqrt(n)
    bq = box_q_for(L, F)
    n_bg = int(round(background * n))
    n_cl = n - n_bg
    centers = rng.uniform(0.0, L, size=(n_clusters, 2))
    per = np.full(n_clusters, n_cl // n_clusters, dtype=np.int64)
    per[: n_cl - per.sum()] += 1
    owner = np.repeat(np.arange(n_clusters), per)
    xy = centers[owner] + rng.normal(0.0, sigma, size=(n_cl, 2))
    bg = rng.uniform(0.0, L, size=(n_bg, 2))
    allxy = np.concatenate([xy, bg], axis=0)
    perm = rng.permutation(n)
    allxy = allxy[perm]
    pos = np.stack([quantize(allxy[:, 0], F, bq), quantize(allxy[:, 1], F, bq)], axis=1)
    theta, d = headings_2d(rng, n)
    return Workload(name=f"knn2d_N{n}_clustered{n_clusters}_F20_k{k}", dim=2, pos_q=pos, dir=d,
                    theta=theta, box_q=(bq, bq), frac_bits=F, rule="knn", k=k, v0=0.5,
                    dt=1.0, eta=0.2, seed=1, steps=200, check_every=50)


def uniform_large(n: int = 1 << 22, k: int = 7, seed: int = 1013) -> Workload:
    """The uniform counterpart of ``clustered_large`` (same N, F, box)."""
    w = uniform_system(n, math.sqrt(n), 20, 2, seed, name=f"knn2d_N{n}_uniform_F20_k{k}",
                       rule="knn", k=k, v0=0.5, dt=1.0, eta=0.2, seed=1, steps=200,
                       check_every=50)
    return w


def knn_3d(n: int = 1 << 20, k: int = 7, seed: int = 1023) -> Workload:
    """3D kNN flock: cubic periodic box at density 1, F=20, vectorial noise."""
    L = float(n) ** (1.0 / 3.0)
    return uniform_system(n, L, 20, 3, seed, name=f"knn3d_N{n}_F20_k{k}", rule="knn", k=k,
                          v0=0.5, dt=1.0, eta=0.2, seed=1, noise="vectorial", steps=200,
                          check_every=50)


def voronoi_3d(n: int = 1 << 18, seed: int = 1024, eta: float = 0.2) -> Workload:
    """3D Voronoi flock: cubic periodic box at density 1 (L = N^(1/3), 64 for
    N = 2^18), vectorial noise.  F = 15 keeps the box within 2^21 grid units
    (L_q = 2^21 at N = 2^18), the range of the exact 3D Voronoi predicates."""
    L = float(n) ** (1.0 / 3.0)
    F = 15
    while F > 0 and L * float(1 << F) > float(1 << 21):
        F -= 1
    return uniform_system(n, L, F, 3, seed, name=f"voronoi3d_N{n}_F{F}", rule="voronoi", k=0,
                          v0=0.5, dt=1.0, eta=eta, seed=1, noise="vectorial", steps=200,
                          check_every=50)


def replica_sizes(n_rep: int = 512, lo: int = 1024, hi: int = 65536, seed: int = 1004) -> np.ndarray:
    rng = _rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi), size=n_rep)
    return np.rint(np.exp(u)).astype(np.int64)


def replica_batch(n_rep: int = 512, k: int = 7, seed: int = 1004,
                  sizes: Optional[Sequence[int]] = None) -> List[Workload]:
    """Independent 2D kNN flocks, N_r log-uniform in [1024, 65536], each in
    its own periodic box at density 1 (L_r = sqrt(N_r)), F=16, eta swept
    linearly 0.05..0.6 across replicas, v0=0.5, 100 steps."""
    if sizes is None:
        sizes = replica_sizes(n_rep, seed=seed)
    rng = _rng(seed + 7919)
    out = []
    for r, nr in enumerate(sizes):
        nr = int(nr)
        eta = 0.05 + 0.55 * r / max(1, len(sizes) - 1)
        bq = box_q_for(math.sqrt(nr), 16)
        pos = uniform_positions(rng, nr, (bq, bq))
        theta, d = headings_2d(rng, nr)
        out.append(Workload(name=f"rep{r}", dim=2, pos_q=pos, dir=d, theta=theta,
                            box_q=(bq, bq), frac_bits=16, rule="knn", k=k, v0=0.5, dt=1.0,
                            eta=float(np.float32(eta)), seed=1, steps=100, check_every=100,
                            replica=r))
    return out


def precision_study(rule: str = "voronoi", n: int = 1 << 20, seed: int = 1005) -> Workload:
    """Uniform 2D flock at density 2 (L=sqrt(2^19)), F=20, eta=0.25, for the
    heading-summation precision study (Voronoi and kNN k=7)."""
    L = math.sqrt(n / 2.0)
    return uniform_system(n, L, 20, 2, seed, name=f"{rule}2d_N{n}_rho2_F20", rule=rule,
                          k=7 if rule == "knn" else 0, v0=0.5, dt=1.0, eta=0.25, seed=1,
                          steps=10000, check_every=1000)


# ---------------------------------------------------------------------------
# Small structured inputs used by the pins
# ---------------------------------------------------------------------------

def square_lattice(m: int, spacing_q: int, offset_q: int = 0) -> tuple:
    """m x m square lattice filling a periodic box of side m*spacing."""
    i, j = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    x = offset_q + i.ravel() * spacing_q
    y = offset_q + j.ravel() * spacing_q
    bq = m * spacing_q
    pos = np.stack([np.mod(x, bq), np.mod(y, bq)], axis=1).astype(np.int32)
    return pos, (bq, bq)


def stretched_hex_lattice(cols: int, rows: int, dx_q: int, dy_q: int) -> tuple:
    """Rows of spacing dx, odd rows shifted by dx/2, row pitch dy; periodic
    when ``rows`` is even.  dx_q must be even so the shift stays on the grid."""
    if dx_q % 2 or rows % 2:
        raise ValueError("dx_q and rows must be even for a periodic hex lattice")
    c, r = np.meshgrid(np.arange(cols), np.arange(rows), indexing="xy")
    x = c.ravel() * dx_q + (r.ravel() % 2) * (dx_q // 2)
    y = r.ravel() * dy_q
    box = (cols * dx_q, rows * dy_q)
    pos = np.stack([np.mod(x, box[0]), np.mod(y, box[1])], axis=1).astype(np.int32)
    return pos, box


def cubic_lattice(kind: str, m, spacing_q, offset_q=(0, 0, 0)) -> tuple:
    """Simple cubic ("sc"), body-centred ("bcc") or face-centred ("fcc")
    lattice of m = (mx, my, mz) conventional cells of edges spacing_q =
    (ax, ay, az) (even, so that the centring offsets a/2 stay on the grid),
    shifted by offset_q and wrapped into the periodic box (mx ax, my ay, mz az)."""
    m = (m,) * 3 if np.isscalar(m) else tuple(m)
    a = (spacing_q,) * 3 if np.isscalar(spacing_q) else tuple(spacing_q)
    if kind != "sc" and any(x % 2 for x in a):
        raise ValueError("centred lattices need even spacings")
    basis = {"sc": [(0, 0, 0)],
             "bcc": [(0, 0, 0), (1, 1, 1)],
             "fcc": [(0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1)]}[kind]
    k, j, i = np.meshgrid(np.arange(m[2]), np.arange(m[1]), np.arange(m[0]), indexing="ij")
    cells = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.int64)
    box = tuple(int(m[t] * a[t]) for t in range(3))
    pts = []
    for b in basis:
        off = np.array([b[t] * (a[t] // 2) + offset_q[t] for t in range(3)], dtype=np.int64)
        pts.append(cells * np.array(a, dtype=np.int64) + off)
    pos = np.concatenate(pts, axis=0)
    pos = np.mod(pos, np.array(box, dtype=np.int64)).astype(np.int32)
    return pos, box


def random_dirs(n: int, dim: int = 2, seed: int = 77) -> np.ndarray:
    rng = _rng(seed)
    if dim == 2:
        return headings_2d(rng, n)[1]
    return headings_3d(rng, n)
