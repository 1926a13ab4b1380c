"""Seeded triangular meshes (input data only).

``square_mesh``: a jittered ``nx x nx`` grid on the unit square.  Interior points
move by U(-J h, J h) in each coordinate; boundary points move only along their
side; corners stay fixed.  Each cell is split by the in-circle test and Lawson
edge flips then run until every interior edge is locally Delaunay
(``diag="delaunay"``), or every cell is split along the same diagonal
(``diag="fixed"``, an unjittered right-triangle grid when ``jitter=0``).

``star_mesh``: a triangulated unit disk made of concentric point rings
(ring j holds 6j points, jittered by U(-J, J) of the angular spacing and
U(-J/2, J/2) of the ring spacing; the outer ring holds a multiple of 12
unjittered points so it contains the 12 polygon vertex angles), mapped
radially, ``(rho, theta) -> (rho * R(theta), theta)``, onto a star-shaped
12-gon whose vertex radii are U(0.6, 1.0).  ``R(theta)`` is the polygon's
polar boundary.  The mapped rings are then stitched ring to ring
(shorter-diagonal rule among counter-clockwise candidates).

Triangles are returned counter-clockwise, node coordinates as float64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import rng


@dataclass
class Mesh:
    xy: np.ndarray          # (n, 2) float64
    tri: np.ndarray         # (t, 3) int32, counter-clockwise
    n_boundary_ring: int    # number of nodes on the outer boundary (generator knowledge)

    @property
    def n(self) -> int:
        return int(self.xy.shape[0])

    @property
    def t(self) -> int:
        return int(self.tri.shape[0])


def _orient(xy, tri):
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    return (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])


def _incircle(a, b, c, d) -> float:
    """> 0 iff d lies strictly inside the circumcircle of counter-clockwise (a, b, c)."""
    adx, ady = a[0] - d[0], a[1] - d[1]
    bdx, bdy = b[0] - d[0], b[1] - d[1]
    cdx, cdy = c[0] - d[0], c[1] - d[1]
    ad = adx * adx + ady * ady
    bd = bdx * bdx + bdy * bdy
    cd = cdx * cdx + cdy * cdy
    return (adx * (bdy * cd - bd * cdy) - ady * (bdx * cd - bd * cdx) + ad * (bdx * cdy - bdy * cdx))


def _lawson(xy: np.ndarray, tri: list) -> list:
    """Flip interior edges until every one is locally Delaunay."""
    def key(u, v):
        return (u, v) if u < v else (v, u)

    edge_tris = {}
    for t, (a, b, c) in enumerate(tri):
        for u, v in ((a, b), (b, c), (c, a)):
            edge_tris.setdefault(key(u, v), []).append(t)
    stack = [e for e, ts in edge_tris.items() if len(ts) == 2]
    guard = 0
    while stack:
        guard += 1
        if guard > 50 * len(tri) + 1000:
            raise RuntimeError("Lawson flips did not terminate")
        e = stack.pop()
        ts = edge_tris.get(e)
        if ts is None or len(ts) != 2:
            continue
        t1, t2 = ts
        u, v = e
        a1 = [w for w in tri[t1] if w not in (u, v)][0]
        a2 = [w for w in tri[t2] if w not in (u, v)][0]
        tt = tri[t1]
        i = tt.index(a1)
        p, q = tt[(i + 1) % 3], tt[(i + 2) % 3]  # a1 -> p -> q counter-clockwise
        if _incircle(xy[a1], xy[p], xy[q], xy[a2]) <= 0.0:
            continue
        # flip edge (p, q) to (a1, a2): new triangles (a1, p, a2) and (a1, a2, q)
        n1 = [a1, p, a2]
        n2 = [a1, a2, q]
        for t in (t1, t2):
            a, b, c = tri[t]
            for x, y in ((a, b), (b, c), (c, a)):
                lst = edge_tris[key(x, y)]
                lst.remove(t)
                if not lst:
                    del edge_tris[key(x, y)]
        tri[t1], tri[t2] = n1, n2
        for t in (t1, t2):
            a, b, c = tri[t]
            for x, y in ((a, b), (b, c), (c, a)):
                edge_tris.setdefault(key(x, y), []).append(t)
        for x, y in ((a1, p), (p, a2), (a2, q), (q, a1)):
            stack.append(key(x, y))
    return tri


def square_mesh(nx: int, seed: int = 0, jitter: float = 0.3, diag: str = "delaunay") -> Mesh:
    h = 1.0 / (nx - 1)
    jj, ii = np.meshgrid(np.arange(nx), np.arange(nx), indexing="ij")
    x = ii.ravel() * h
    y = jj.ravel() * h
    n = nx * nx
    if jitter > 0.0:
        u = rng.uniform(seed, rng.TAG_MESH_JITTER, 2 * n).reshape(n, 2)
        dx = (-1.0 + 2.0 * u[:, 0]) * jitter * h
        dy = (-1.0 + 2.0 * u[:, 1]) * jitter * h
        ib = ii.ravel()
        jb = jj.ravel()
        on_x_side = (ib == 0) | (ib == nx - 1)      # left/right: move along y only
        on_y_side = (jb == 0) | (jb == nx - 1)      # bottom/top: move along x only
        corner = on_x_side & on_y_side
        dx = np.where(on_x_side, 0.0, dx)
        dy = np.where(on_y_side, 0.0, dy)
        dx[corner] = 0.0
        dy[corner] = 0.0
        x = x + dx
        y = y + dy
    xy = np.stack([x, y], axis=1)
    tri = []
    for j in range(nx - 1):
        for i in range(nx - 1):
            a = j * nx + i
            b = a + 1
            c = a + nx + 1
            d = a + nx
            if diag == "fixed" or _incircle(xy[a], xy[b], xy[c], xy[d]) <= 0.0:
                tri.append([a, b, c])
                tri.append([a, c, d])
            else:
                tri.append([a, b, d])
                tri.append([b, c, d])
    if diag == "delaunay":
        tri = _lawson(xy, tri)
    tri = np.asarray(tri, dtype=np.int32)
    assert np.all(_orient(xy, tri) > 0.0)
    return Mesh(xy, tri, 4 * (nx - 1))


def _stitch(inner_idx, inner_xy, outer_idx, outer_xy):
    """Triangles between two closed rings whose points are sorted by angle.

    Walks both rings once; at each step it adds the candidate triangle that is
    counter-clockwise and has the shorter new edge.
    """
    m, M = len(inner_idx), len(outer_idx)
    a0 = np.arctan2(inner_xy[0, 1], inner_xy[0, 0])
    oa = np.arctan2(outer_xy[:, 1], outer_xy[:, 0])
    s = int(np.argmin(np.abs(np.angle(np.exp(1j * (oa - a0))))))
    outer_idx = np.roll(outer_idx, -s)
    outer_xy = np.roll(outer_xy, -s, axis=0)
    ix, iy = inner_xy[:, 0].tolist(), inner_xy[:, 1].tolist()
    ox, oy = outer_xy[:, 0].tolist(), outer_xy[:, 1].tolist()
    ii, oo = inner_idx.tolist(), outer_idx.tolist()
    out = []
    a = b = 0
    while a < m or b < M:
        pa, pa1 = a % m, (a + 1) % m
        pb, pb1 = b % M, (b + 1) % M
        ok_in = ok_out = False
        d_in = d_out = 0.0
        if a < m:   # triangle (in[a], out[b], in[a+1])
            o1 = (ox[pb] - ix[pa]) * (iy[pa1] - iy[pa]) - (oy[pb] - iy[pa]) * (ix[pa1] - ix[pa])
            ok_in = o1 > 0.0
            d_in = (ix[pa1] - ox[pb]) ** 2 + (iy[pa1] - oy[pb]) ** 2
        if b < M:   # triangle (in[a], out[b], out[b+1])
            o2 = (ox[pb] - ix[pa]) * (oy[pb1] - iy[pa]) - (oy[pb] - iy[pa]) * (ox[pb1] - ix[pa])
            ok_out = o2 > 0.0
            d_out = (ox[pb1] - ix[pa]) ** 2 + (oy[pb1] - iy[pa]) ** 2
        if ok_in and (not ok_out or d_in <= d_out):
            out.append((ii[pa], oo[pb], ii[pa1]))
            a += 1
        elif ok_out:
            out.append((ii[pa], oo[pb], oo[pb1]))
            b += 1
        else:
            raise RuntimeError("ring stitching found no valid triangle")
    return np.asarray(out, dtype=np.int64)


def star_polygon(seed: int, n_vertices: int = 12, rmin: float = 0.6, rmax: float = 1.0) -> np.ndarray:
    u = rng.uniform(seed, rng.TAG_STAR_RADII, n_vertices)
    r = rmin + (rmax - rmin) * u
    ang = 2.0 * np.pi * np.arange(n_vertices) / n_vertices
    return np.stack([r * np.cos(ang), r * np.sin(ang)], axis=1)


def polar_radius(V: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Distance from the origin to the boundary of star polygon V along direction theta."""
    nv = V.shape[0]
    th = np.mod(theta, 2 * np.pi)
    k = np.minimum((th / (2 * np.pi / nv)).astype(np.int64), nv - 1)
    Va = V[k]
    Vb = V[(k + 1) % nv]
    ux, uy = np.cos(th), np.sin(th)
    num = Va[:, 0] * Vb[:, 1] - Va[:, 1] * Vb[:, 0]
    ex, ey = Vb[:, 0] - Va[:, 0], Vb[:, 1] - Va[:, 1]
    den = ux * ey - uy * ex
    return num / den


def star_mesh(n_target: int, seed: int = 0, jitter: float = 0.3, n_vertices: int = 12) -> Mesh:
    R = max(2, int(round(math.sqrt(n_target / 3.0))))
    m_out = n_vertices * int(math.ceil(6 * R / n_vertices))
    counts = [1] + [6 * j for j in range(1, R)] + [m_out]
    n = sum(counts)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    u = rng.uniform(seed, rng.TAG_MESH_JITTER, 2 * n).reshape(n, 2)
    rho = np.zeros(n)
    ang = np.zeros(n)
    for j in range(1, R + 1):
        s, c = starts[j], counts[j]
        k = np.arange(c)
        if j < R:
            off = 0.5 * (j % 2)
            ang[s:s + c] = 2 * np.pi * (k + off + jitter * (-1.0 + 2.0 * u[s:s + c, 0])) / c
            rho[s:s + c] = (j + 0.5 * jitter * (-1.0 + 2.0 * u[s:s + c, 1])) / R
        else:
            ang[s:s + c] = 2 * np.pi * k / c
            rho[s:s + c] = 1.0
    V = star_polygon(seed, n_vertices)
    Rth = polar_radius(V, ang)
    Rth[0] = 1.0
    xy = np.stack([rho * Rth * np.cos(ang), rho * Rth * np.sin(ang)], axis=1)
    xy[0] = 0.0
    tris = []
    # fan around the centre
    r1 = np.arange(starts[1], starts[1] + counts[1])
    tris.append(np.stack([np.zeros(counts[1], np.int64), r1, np.roll(r1, -1)], axis=1))
    for j in range(1, R):
        ii = np.arange(starts[j], starts[j] + counts[j])
        oo = np.arange(starts[j + 1], starts[j + 1] + counts[j + 1])
        tris.append(_stitch(ii, xy[ii], oo, xy[oo]))
    tri = np.concatenate(tris).astype(np.int32)
    o = _orient(xy, tri)
    if not np.all(o > 0.0):
        raise RuntimeError("star mesh: %d inverted triangles" % int(np.sum(o <= 0.0)))
    return Mesh(xy, tri, m_out)
