"""Overlapping decomposition, coarse space and local DSS graphs (Section II-A, Section III-B).

Test infrastructure (see the package docstring).

Readings where the paper is silent or names a tool that is not available here:
* The partitioner (METIS in Section IV-A) is recursive coordinate bisection of
  the free nodes: split along the longer bounding-box side, the lower part takes
  floor(|S| * floor(K/2) / K) nodes in the order (coordinate, other coordinate, id).
* The overlap of Section IV-A counts adjacency layers of the free-free matrix graph.
* The partition of unity that the Nicolaides coarse space needs (Section II-A)
  is w_ij = 1 / (number of subdomains holding node j).
* The local graph of subdomain i (Section III-B) holds its unknowns S_i
  (ascending id) and then its halo: mesh neighbours of S_i outside S_i,
  Dirichlet nodes included, ascending mesh id.  Edges are directed: every
  mesh neighbour s of an unknown t gives the edge s -> t, so the graph is
  undirected among unknowns and halo nodes only point inward.
* Edge features are scaled by the mean mesh edge length h_bar.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import fem


def rcb(xy: np.ndarray, K: int) -> np.ndarray:
    """Recursive coordinate bisection of points ``xy`` (one per free node) into K parts."""
    n = xy.shape[0]
    part = np.empty(n, dtype=np.int64)

    def split(ids: np.ndarray, k: int, base: int) -> None:
        if k == 1:
            part[ids] = base
            return
        x, y = xy[ids, 0], xy[ids, 1]
        if (x.max() - x.min()) >= (y.max() - y.min()):
            order = np.lexsort((ids, y, x))   # by x, then y, then id
        else:
            order = np.lexsort((ids, x, y))   # by y, then x, then id
        k1 = k // 2
        n1 = (ids.shape[0] * k1) // k
        s = ids[order]
        split(s[:n1], k1, base)
        split(s[n1:], k - k1, base + k1)

    split(np.arange(n), K, 0)
    return part


def neighbours(A: sp.csr_matrix, nodes: np.ndarray) -> np.ndarray:
    """Column indices of the given rows: the graph neighbours of ``nodes`` with the nodes themselves."""
    ptr, col = A.indptr, A.indices
    lo, hi = ptr[nodes], ptr[nodes + 1]
    return np.unique(np.concatenate([col[l:h] for l, h in zip(lo, hi)]))


def overlap_sets(A: sp.csr_matrix, part: np.ndarray, K: int, delta: int) -> list:
    """S_i: part i grown by ``delta`` layers of the matrix graph; the index set of R_i (Section II-A)."""
    sets = []
    for i in range(K):
        S = np.nonzero(part == i)[0]
        for _ in range(delta):
            S = np.union1d(S, neighbours(A, S))
        sets.append(S.astype(np.int64))
    return sets


def multiplicity(sets: list, n: int) -> np.ndarray:
    m = np.zeros(n, dtype=np.int64)
    for S in sets:
        m[S] += 1
    return m


def coarse_basis(sets: list, n: int) -> sp.csr_matrix:
    """Z = [z_1 .. z_K], z_i = R_i^T (partition-of-unity weights on S_i): Nicolaides' R_0 = Z^T (Section II-A)."""
    m = multiplicity(sets, n)
    rows = np.concatenate(sets)
    cols = np.concatenate([np.full(S.shape[0], i) for i, S in enumerate(sets)])
    vals = 1.0 / m[rows]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, len(sets)))


def coarse_matrix(A: sp.csr_matrix, Z: sp.csr_matrix) -> np.ndarray:
    """A_0 = R_0 A R_0^T = Z^T A Z, dense K x K (Eq. 7)."""
    return (Z.T @ (A @ Z)).toarray()


def mesh_adjacency(n: int, tri: np.ndarray):
    """Sorted neighbour lists of the full mesh graph (no self loops)."""
    edges, _ = fem.mesh_edges(tri)
    rows = np.concatenate([edges[:, 0], edges[:, 1]])
    cols = np.concatenate([edges[:, 1], edges[:, 0]])
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(ptr, rows + 1, 1)
    return np.cumsum(ptr), cols


def mean_edge_length(xy: np.ndarray, tri: np.ndarray) -> float:
    """h_bar: the mean length of the mesh's edges."""
    edges, _ = fem.mesh_edges(tri)
    d = xy[edges[:, 1]] - xy[edges[:, 0]]
    return float(np.mean(np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2)))


@dataclass
class LocalGraph:
    nodes: np.ndarray   # mesh ids: unknowns first (ascending), then halo (ascending)
    n_int: int          # number of unknowns k_i
    src: np.ndarray     # local ids, edge src -> dst
    dst: np.ndarray
    xy: np.ndarray      # mesh coordinates of the local nodes


def local_graph(problem: fem.Problem, S_free: np.ndarray, adj=None) -> LocalGraph:
    """Graph G_i of Section III-B (Eq. 17) for the subdomain whose unknowns are the free ids ``S_free``."""
    if adj is None:
        adj = mesh_adjacency(problem.n, problem.tri)
    ptr, col = adj
    interior = problem.free[S_free]                       # ascending mesh ids
    nb = np.unique(np.concatenate([col[ptr[v]:ptr[v + 1]] for v in interior]))
    halo = np.setdiff1d(nb, interior)
    nodes = np.concatenate([interior, halo])
    local = {int(v): k for k, v in enumerate(nodes)}
    src, dst = [], []
    for t_loc, v in enumerate(interior):
        for s in col[ptr[v]:ptr[v + 1]]:
            src.append(local[int(s)])
            dst.append(t_loc)
    return LocalGraph(nodes, int(interior.shape[0]), np.asarray(src, np.int64),
                      np.asarray(dst, np.int64), problem.xy[nodes])


@dataclass
class Decomposition:
    K: int
    delta: int
    part: np.ndarray
    sets: list
    mult: np.ndarray
    Z: sp.csr_matrix
    A0: np.ndarray


def decompose(problem: fem.Problem, K: int, delta: int, part: np.ndarray | None = None) -> Decomposition:
    if part is None:
        part = rcb(problem.xy[problem.free], K)
    sets = overlap_sets(problem.A, part, K, delta)
    mult = multiplicity(sets, problem.n_free)
    Z = coarse_basis(sets, problem.n_free)
    A0 = coarse_matrix(problem.A, Z)
    return Decomposition(K, delta, part, sets, mult, Z, A0)
