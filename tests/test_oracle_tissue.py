"""Pins of the oracle's Voronoi tissue model (Sec. "Geometric models of dense
tissue": the energy of Eq. (vmEnergy) over the Voronoi cells; Sec. "Voronoi
model forces": F_i = -dE/dr_i by the chain rule through the vertices).

* cell areas against an independent exact construction: each cell clipped
  from its periodic box by the bisectors of every image of every other
  particle, in exact rationals (no triangulation), on tiny systems;
* the closed forms of a centred rectangular ("stretched hexagonal") lattice:
  area dx*dy, hexagon perimeter, zero force by inversion symmetry, and the
  energy N [KA (A - A0)^2 + KP (P - P0)^2];
* sum of areas = box area, sum of forces = 0 (translation invariance);
* forces against central finite differences of the oracle's own energy,
  which is recomputed from scratch (a fresh triangulation) at every shift,
  so a dropped neighbor-cell term, a wrong sign or a transposed Jacobian
  in the chain rule fails.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2103_10239_gb300 import workloads as W


def _clip(poly, a, b, c):
    """Keep the part of the convex polygon with a*x + b*y <= c (exact)."""
    out = []
    m = len(poly)
    for k in range(m):
        p, q = poly[k], poly[(k + 1) % m]
        fp = a * p[0] + b * p[1] - c
        fq = a * q[0] + b * q[1] - c
        if fp <= 0:
            out.append(p)
        if (fp < 0 < fq) or (fq < 0 < fp):
            t = fp / (fp - fq)
            out.append((p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1])))
    return out


def exact_cell(pos, box, i, reach=2):
    """Voronoi cell of particle i (relative to it) in exact rationals."""
    Lx, Ly = int(box[0]), int(box[1])
    hx, hy = Fraction(Lx, 2), Fraction(Ly, 2)
    poly = [(-hx, -hy), (hx, -hy), (hx, hy), (-hx, hy)]
    xi, yi = int(pos[i, 0]), int(pos[i, 1])
    for j in range(pos.shape[0]):
        for sy in range(-reach, reach + 1):
            for sx in range(-reach, reach + 1):
                if j == i and sx == 0 and sy == 0:
                    continue
                dx = int(pos[j, 0]) + sx * Lx - xi
                dy = int(pos[j, 1]) + sy * Ly - yi
                # points closer to 0 than to d: 2 d.x <= |d|^2
                poly = _clip(poly, Fraction(2 * dx), Fraction(2 * dy), Fraction(dx * dx + dy * dy))
    return poly


def _area_perim(poly):
    A = Fraction(0)
    P = 0.0
    for k in range(len(poly)):
        p, q = poly[k], poly[(k + 1) % len(poly)]
        A += (p[0] * q[1] - q[0] * p[1]) / 2
        P += math.sqrt(float((q[0] - p[0]) ** 2 + (q[1] - p[1]) ** 2))
    return A, P


@pytest.mark.parametrize("seed,n,L", [(1, 5, 3.0), (2, 9, 4.0), (3, 14, 5.0)])
def test_areas_and_perimeters_match_exact_clipping(seed, n, L):
    F = 12
    w = W.uniform_system(n, L, F, 2, input_seed=seed, rule="voronoi", k=0)
    area, perim, _, _ = oracle.tissue(w.pos_q, w.box_q, F, 1.0, 1.0, 1.0, 3.8, forces=False)
    s = 2.0 ** -F
    for i in range(n):
        A, P = _area_perim(exact_cell(w.pos_q, w.box_q, i))
        assert abs(area[i] - float(A) * s * s) <= 1e-12 * max(1.0, float(A) * s * s)
        assert abs(perim[i] - P * s) <= 1e-12 * max(1.0, P * s)


@pytest.mark.parametrize("dxq,dyq", [(65536, 56756), (65536, 40000), (65536, 90000)])
def test_centred_rectangular_lattice_closed_forms(dxq, dyq):
    """Rows of spacing dx, odd rows shifted by dx/2, row pitch dy (with
    dx/2 < dy and dx < 2 dy, the six neighbors are (+-dx, 0) and
    (+-dx/2, +-dy)): the cell is the hexagon with vertices (+-dx/2, +-y1),
    (0, +-y2), y1 = (dy^2 - dx^2/4)/(2 dy), y2 = (dy^2 + dx^2/4)/(2 dy)."""
    F = 16
    pos, box = W.stretched_hex_lattice(8, 10, dxq, dyq)
    dx, dy = dxq / 2.0 ** F, dyq / 2.0 ** F
    y1 = (dy * dy - dx * dx / 4) / (2 * dy)
    y2 = (dy * dy + dx * dx / 4) / (2 * dy)
    P_hex = 4 * y1 + 4 * math.hypot(dx / 2, y2 - y1)
    KA, KP, A0, P0 = 1.3, 0.7, 0.9, 3.6
    area, perim, e, f = oracle.tissue(pos, box, F, KA, KP, A0, P0)
    assert np.allclose(area, dx * dy, rtol=1e-13, atol=0)
    assert np.allclose(perim, P_hex, rtol=1e-13, atol=0)
    assert np.abs(f).max() < 1e-11
    n = pos.shape[0]
    assert e == pytest.approx(n * (KA * (dx * dy - A0) ** 2 + KP * (P_hex - P0) ** 2), rel=1e-12)
    _, _, e0, f0 = oracle.tissue(pos, box, F, KA, KP, dx * dy, P_hex)
    assert abs(e0) < 1e-20 and np.abs(f0).max() < 1e-12


def test_areas_tile_the_box_and_forces_sum_to_zero():
    F = 16
    w = W.uniform_system(400, 20.0, F, 2, input_seed=5, rule="voronoi", k=0)
    area, perim, e, f = oracle.tissue(w.pos_q, w.box_q, F, 1.0, 1.0, 1.0, 3.8)
    Lx, Ly = (b / 2.0 ** F for b in w.box_q)
    assert area.sum() == pytest.approx(Lx * Ly, rel=1e-12)
    assert np.abs(f.sum(axis=0)).max() < 1e-10 * np.abs(f).max() * 400
    assert e == pytest.approx(np.sum((area - 1.0) ** 2 + (perim - 3.8) ** 2), rel=1e-12)


@pytest.mark.parametrize("KA,KP,A0,P0", [(1.0, 1.0, 1.0, 3.8), (2.0, 0.0, 0.8, 0.0), (0.0, 1.0, 0.0, 3.2)])
def test_forces_are_minus_the_energy_gradient(KA, KP, A0, P0):
    """Central differences of the energy (new triangulation at each shift,
    delta = 8 grid units = 1.2e-4 length units) against the chain rule."""
    F = 16
    w = W.uniform_system(60, 7.7, F, 2, input_seed=3, rule="voronoi", k=0)
    pos = w.pos_q.astype(np.int64)
    _, _, _, f = oracle.tissue(pos, w.box_q, F, KA, KP, A0, P0)
    d = 8
    scale = np.abs(f).max()
    for i in [0, 5, 17, 33, 59]:
        for ax in range(2):
            pp = pos.copy()
            pm = pos.copy()
            pp[i, ax] = (pp[i, ax] + d) % w.box_q[ax]
            pm[i, ax] = (pm[i, ax] - d) % w.box_q[ax]
            ep = oracle.tissue(pp, w.box_q, F, KA, KP, A0, P0, forces=False)[2]
            em = oracle.tissue(pm, w.box_q, F, KA, KP, A0, P0, forces=False)[2]
            fd = -(ep - em) / (2 * d / 2.0 ** F)
            assert abs(fd - f[i, ax]) <= 2e-6 * scale, (i, ax, fd, f[i, ax])


def test_coincident_particles_are_rejected():
    w = W.uniform_system(30, 6.0, 16, 2, input_seed=7, rule="voronoi", k=0)
    pos = w.pos_q.copy()
    pos[3] = pos[4]
    with pytest.raises(RuntimeError):
        oracle.tissue(pos, w.box_q, 16, 1.0, 1.0, 1.0, 3.8)
