"""Tiny-input references in exact integer arithmetic -- TEST INFRASTRUCTURE ONLY.

These re-derive the neighbor relations by algorithms different from the C
oracle, to pin it:

* :func:`knn_brute` sorts every (squared distance, id) pair with Python ints.
* :func:`voronoi_brute` decides "i and j share a Voronoi edge of positive
  length" directly from the definition of the Voronoi cell as the set of
  points closer to i than to any other site (Sec. "Computational tools:
  Voronoi neighbor lists"): the bisector line of i and (an image of) j is
  clipped by every other site's half-plane, and the pair is kept iff a segment
  of positive length survives.  No triangulation is involved.
"""
from __future__ import annotations

from fractions import Fraction
from typing import List

import numpy as np


def min_image(d: int, L: int) -> int:
    if 2 * d > L:
        d -= L
    if 2 * d <= -L:
        d += L
    return d


def knn_brute(pos, box, k: int) -> List[List[int]]:
    pos = [tuple(int(c) for c in p) for p in np.asarray(pos)]
    box = [int(b) for b in box]
    out = []
    for i, pi in enumerate(pos):
        keyed = []
        for j, pj in enumerate(pos):
            if j == i:
                continue
            D = sum(min_image(pj[a] - pi[a], box[a]) ** 2 for a in range(len(box)))
            keyed.append((D, j))
        keyed.sort()
        out.append([j for _, j in keyed[:k]])
    return out


def _tiled_sites(pos, Lx: int, Ly: int, rx: int, ry: int):
    """All periodic images with shifts in [-rx, rx] x [-ry, ry] periods."""
    xs, ys, ids = [], [], []
    for sy in range(-ry, ry + 1):
        for sx in range(-rx, rx + 1):
            xs.append(pos[:, 0].astype(np.int64) + sx * Lx)
            ys.append(pos[:, 1].astype(np.int64) + sy * Ly)
            ids.append(np.arange(pos.shape[0]))
    return np.concatenate(xs), np.concatenate(ys), np.concatenate(ids)


def voronoi_brute(pos, box) -> List[List[int]]:
    """Voronoi neighbors by clipping bisectors (exact; O(N^3) on 25 N sites).

    Coincident particles form one site: they are each other's neighbors, and
    a coincident copy of a site clips nothing (its half-plane is the site's).

    Every site that can shape the cell of i lies within twice the cell's
    circumradius, which is at most half the box diagonal because the cell of
    i fits in the box-sized rectangle centred on i; the tiling below reaches
    one full diagonal beyond the box on every side.  Coordinates must stay
    below ~2^20 so that int64 products are exact in the vectorised pre-pass."""
    pos = np.asarray(pos, dtype=np.int64)
    Lx, Ly = int(box[0]), int(box[1])
    diag = (Lx * Lx + Ly * Ly) ** 0.5
    rx = int(np.ceil(diag / Lx)) + 1
    ry = int(np.ceil(diag / Ly)) + 1
    n = pos.shape[0]
    X, Y, ID = _tiled_sites(pos, Lx, Ly, rx, ry)
    res = []
    for i in range(n):
        xi, yi = int(pos[i, 0]), int(pos[i, 1])
        nbrs = set()
        ex = X - xi
        ey = Y - yi
        for c in range(X.shape[0]):
            j = int(ID[c])
            if int(ex[c]) == 0 and int(ey[c]) == 0:
                if j != i:
                    nbrs.add(j)  # a coincident particle: same site, a neighbor
                continue
            # bisector of i and site c: points m + t*d with m=(p_i+p_c)/2,
            # d = perp(p_c - p_i); keep-side of site e:
            #   2 x.(p_e - p_i) <= |p_e|^2 - |p_i|^2
            # with 2m = p_i + p_c this reads  t * a_e <= r_e  where
            #   a_e = 2 d.(p_e - p_i),  r_e = |p_e|^2 - |p_i|^2 - (p_i+p_c).(p_e - p_i)
            dxv, dyv = -int(ey[c]), int(ex[c])
            sx2, sy2 = xi + int(X[c]), yi + int(Y[c])
            a = 2 * (dxv * ex + dyv * ey)
            r = (X * X + Y * Y) - (xi * xi + yi * yi) - (sx2 * ex + sy2 * ey)
            mask = np.ones(X.shape[0], dtype=bool)
            mask[c] = False
            mask &= ~((ex == 0) & (ey == 0))
            a_m, r_m = a[mask], r[mask]
            if np.any((a_m == 0) & (r_m < 0)):
                continue  # a parallel site cuts the whole bisector away
            pos_a = a_m > 0
            neg_a = a_m < 0
            hi = None
            lo = None
            if np.any(pos_a):
                fr = r_m[pos_a] / a_m[pos_a]
                cand = np.nonzero(fr <= fr.min() * (1 - 1e-9) + np.abs(fr.min()) * 1e-9 + 1e-9)[0]
                hi = min(Fraction(int(r_m[pos_a][q]), int(a_m[pos_a][q])) for q in cand)
            if np.any(neg_a):
                fr = r_m[neg_a] / a_m[neg_a]
                cand = np.nonzero(fr >= fr.max() - np.abs(fr.max()) * 1e-9 - 1e-9)[0]
                lo = max(Fraction(int(r_m[neg_a][q]), int(a_m[neg_a][q])) for q in cand)
            if hi is None or lo is None:
                continue  # unbounded: cannot happen for a periodic set
            if lo < hi:
                if j != i:
                    nbrs.add(j)
        res.append(sorted(nbrs))
    return res


def incircle_int(a, b, c, d) -> int:
    """Sign of the incircle determinant with Python integers."""
    adx, ady = int(a[0]) - int(d[0]), int(a[1]) - int(d[1])
    bdx, bdy = int(b[0]) - int(d[0]), int(b[1]) - int(d[1])
    cdx, cdy = int(c[0]) - int(d[0]), int(c[1]) - int(d[1])
    det = ((adx * adx + ady * ady) * (bdx * cdy - bdy * cdx)
           + (bdx * bdx + bdy * bdy) * (cdx * ady - cdy * adx)
           + (cdx * cdx + cdy * cdy) * (adx * bdy - ady * bdx))
    return (det > 0) - (det < 0)


def orient_int(a, b, c) -> int:
    v = (int(b[0]) - int(a[0])) * (int(c[1]) - int(a[1])) - (int(b[1]) - int(a[1])) * (int(c[0]) - int(a[0]))
    return (v > 0) - (v < 0)
