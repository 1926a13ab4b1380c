"""P1 finite-element assembly of -Lap(u) = f in Omega, u = g on the boundary (Section II, Eqs. 1-2).

Test infrastructure (see the package docstring).  FP64 throughout.

Readings where the paper is silent:
* Dirichlet nodes are the endpoints of boundary edges (edges in exactly one triangle).
* Dirichlet data are eliminated symmetrically: the unknowns are the free nodes,
  ``b_f -= A_fD g_D``, so the free-free matrix is SPD as conjugate gradients needs.
* The load of the paper's quadratic ``f`` (Section IV-A, Eq. 24) is integrated
  exactly through its P2 interpolant; a nodal ``f`` is integrated with the
  consistent P1 mass matrix.
* The sparsity pattern is the mesh edge graph plus the diagonal, exact zeros kept.
* Contributions are summed in ascending triangle order.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


def paper_f(r: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Forcing term of the data set, f = r1 (x-1)^2 + r2 y^2 + r3 (Section IV-A, Eq. 24)."""
    return r[0] * (x - 1.0) ** 2 + r[1] * y ** 2 + r[2]


def paper_g(r: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Dirichlet data of the data set, g = r4 x^2 + r5 y^2 + r6 xy + r7 x + r8 y + r9 (Eq. 25)."""
    return r[3] * x ** 2 + r[4] * y ** 2 + r[5] * x * y + r[6] * x + r[7] * y + r[8]


def mesh_edges(tri: np.ndarray):
    """Unique undirected edges (sorted pairs) and how many triangles hold each."""
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]]).astype(np.int64)
    e.sort(axis=1)
    edges, counts = np.unique(e, axis=0, return_counts=True)
    return edges, counts


def dirichlet_mask(n: int, tri: np.ndarray) -> np.ndarray:
    """Nodes on the domain boundary: endpoints of edges that belong to one triangle only."""
    edges, counts = mesh_edges(tri)
    mask = np.zeros(n, dtype=bool)
    b = edges[counts == 1]
    mask[b[:, 0]] = True
    mask[b[:, 1]] = True
    return mask


def triangle_geometry(xy: np.ndarray, tri: np.ndarray):
    """Per triangle: b_k = y_{k+1} - y_{k+2}, c_k = x_{k+2} - x_{k+1} (k cyclic) and the area |T|."""
    x = xy[tri, 0]
    y = xy[tri, 1]
    bb = np.stack([y[:, 1] - y[:, 2], y[:, 2] - y[:, 0], y[:, 0] - y[:, 1]], axis=1)
    cc = np.stack([x[:, 2] - x[:, 1], x[:, 0] - x[:, 2], x[:, 1] - x[:, 0]], axis=1)
    area = 0.5 * np.abs(bb[:, 0] * cc[:, 1] - bb[:, 1] * cc[:, 0])
    return bb, cc, area


def element_stiffness(xy: np.ndarray, tri: np.ndarray) -> np.ndarray:
    """K_T[i][j] = (b_i b_j + c_i c_j) / (4 |T|): the P1 stiffness of grad(phi_i).grad(phi_j) over T."""
    bb, cc, area = triangle_geometry(xy, tri)
    Ke = (bb[:, :, None] * bb[:, None, :] + cc[:, :, None] * cc[:, None, :]) / (4.0 * area)[:, None, None]
    return Ke


def element_load_quadratic(xy: np.ndarray, tri: np.ndarray, fun) -> np.ndarray:
    """Exact int_T f lambda_i for quadratic f, through f's P2 interpolant.

    With int_T lambda^a lambda^b lambda^c = 2|T| a! b! c! / (a+b+c+2)! the P2
    basis gives int_T f lambda_i = |T| [f_i/30 - (f_j + f_l)/60 + 2 (f_ij + f_il)/15 + f_jl/15],
    vertices i, j, l and edge midpoints ij, il, jl.
    """
    _, _, area = triangle_geometry(xy, tri)
    P = xy[tri]                      # (t, 3, 2)
    fv = fun(P[:, :, 0], P[:, :, 1])  # vertex values
    out = np.empty((tri.shape[0], 3))
    for i in range(3):
        j, l = (i + 1) % 3, (i + 2) % 3
        mij = 0.5 * (P[:, i] + P[:, j])
        mil = 0.5 * (P[:, i] + P[:, l])
        mjl = 0.5 * (P[:, j] + P[:, l])
        fij = fun(mij[:, 0], mij[:, 1])
        fil = fun(mil[:, 0], mil[:, 1])
        fjl = fun(mjl[:, 0], mjl[:, 1])
        out[:, i] = area * (fv[:, i] / 30.0 - (fv[:, j] + fv[:, l]) / 60.0
                            + 2.0 * (fij + fil) / 15.0 + fjl / 15.0)
    return out


def element_load_nodal(xy: np.ndarray, tri: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Consistent P1 mass times nodal f: int_T f_h lambda_i = |T|/12 (2 f_i + f_j + f_l)."""
    _, _, area = triangle_geometry(xy, tri)
    fv = f[tri]
    return (area / 12.0)[:, None] * (fv + fv.sum(axis=1, keepdims=True))


def csr_pattern(n: int, tri: np.ndarray):
    """Row pointers and sorted column indices of the mesh edge graph plus the diagonal."""
    edges, _ = mesh_edges(tri)
    rows = np.concatenate([edges[:, 0], edges[:, 1], np.arange(n)])
    cols = np.concatenate([edges[:, 1], edges[:, 0], np.arange(n)])
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, cols


@dataclass
class Problem:
    n: int
    xy: np.ndarray
    tri: np.ndarray
    dirichlet: np.ndarray       # bool (n,)
    free: np.ndarray            # mesh ids of the free nodes, ascending
    free_id: np.ndarray         # (n,) free id of a mesh node, -1 on Dirichlet nodes
    A_full: sp.csr_matrix       # full stiffness, explicit zeros kept
    b_full: np.ndarray          # full load vector
    g: np.ndarray               # Dirichlet values at every node (0 on free nodes)
    A: sp.csr_matrix            # free-free block A_ff (SPD), explicit zeros kept
    b: np.ndarray               # b_f - A_fD g_D

    @property
    def n_free(self) -> int:
        return int(self.free.shape[0])

    def full_solution(self, x_free: np.ndarray) -> np.ndarray:
        u = self.g.copy()
        u[self.free] = x_free
        return u


def _row_search(rowptr, cols, r, col):
    """Position of column ``col`` inside CSR row ``r`` (columns sorted within rows)."""
    stride = int(cols.max()) + 2
    key = r.astype(np.int64) * stride + col
    allkey = np.repeat(np.arange(rowptr.shape[0] - 1), np.diff(rowptr)) * stride + cols
    idx = np.searchsorted(allkey, key)
    assert np.all(allkey[idx] == key)
    return idx


def assemble(xy: np.ndarray, tri: np.ndarray, coeffs: np.ndarray | None = None,
             f_nodal: np.ndarray | None = None, g_nodal: np.ndarray | None = None,
             dirichlet: np.ndarray | None = None) -> Problem:
    """Galerkin system A u = b of Eq. 2 with first-order Lagrange elements (Section II).

    Either the paper's polynomial family (``coeffs`` = r_1..r_9) or nodal ``f``
    and ``g`` arrays.
    """
    n = xy.shape[0]
    tri = np.asarray(tri, dtype=np.int64)
    if dirichlet is None:
        dirichlet = dirichlet_mask(n, tri)
    dirichlet = np.asarray(dirichlet, dtype=bool)
    rowptr, cols = csr_pattern(n, tri)

    Ke = element_stiffness(xy, tri)
    rows_ij = np.repeat(tri, 3, axis=1).reshape(-1)      # row vertex of entry (a, c)
    cols_ij = np.tile(tri, (1, 3)).reshape(-1)           # column vertex of entry (a, c)
    pos = _row_search(rowptr, cols, rows_ij, cols_ij)
    vals = np.zeros(cols.shape[0])
    np.add.at(vals, pos, Ke.reshape(-1))                 # unbuffered, ascending triangle order
    A_full = sp.csr_matrix((vals, cols, rowptr), shape=(n, n))

    if coeffs is not None:
        Fe = element_load_quadratic(xy, tri, lambda x, y: paper_f(coeffs, x, y))
        g = paper_g(coeffs, xy[:, 0], xy[:, 1])
    else:
        Fe = element_load_nodal(xy, tri, np.asarray(f_nodal, dtype=np.float64))
        g = np.asarray(g_nodal, dtype=np.float64).copy()
    b_full = np.zeros(n)
    np.add.at(b_full, tri.reshape(-1), Fe.reshape(-1))
    g = np.where(dirichlet, g, 0.0)

    free = np.nonzero(~dirichlet)[0]
    free_id = -np.ones(n, dtype=np.int64)
    free_id[free] = np.arange(free.shape[0])
    A, bf = eliminate(A_full, b_full, g, dirichlet, free, free_id)
    return Problem(n, xy, tri, dirichlet, free, free_id, A_full, b_full, g, A, bf)


def eliminate(A_full, b_full, g, dirichlet, free, free_id):
    """Free-free block and lifted right-hand side: A_ff and b_f - A_fD g_D."""
    n = A_full.shape[0]
    rowptr, cols, vals = A_full.indptr, A_full.indices, A_full.data
    row_of = np.repeat(np.arange(n), np.diff(rowptr))
    free_row = ~dirichlet[row_of]
    keep = free_row & ~dirichlet[cols]
    counts = np.zeros(n, dtype=np.int64)
    np.add.at(counts, row_of[keep], 1)
    nf = free.shape[0]
    new_ptr = np.zeros(nf + 1, dtype=np.int64)
    new_ptr[1:] = np.cumsum(counts[free])
    A = sp.csr_matrix((vals[keep], free_id[cols[keep]], new_ptr), shape=(nf, nf))
    # lifting: sum A_ij g_j over the Dirichlet columns of each free row, in column order
    lift_sel = free_row & dirichlet[cols]
    lift = np.zeros(n)
    np.add.at(lift, row_of[lift_sel], vals[lift_sel] * g[cols[lift_sel]])
    return A, b_full[free] - lift[free]
