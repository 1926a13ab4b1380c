"""Pins of the oracle's decomposition (Section II-A, Section III-B): hand-computed splits,
BFS distances, partition of unity and the local graph's halo rules."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import synth
from oracle import fem, partition as pt


def test_rcb_line_hand_example():
    """10 points on a line, K = 3: floor(10/3) = 3 go to part 0, then 7 split 3 | 4."""
    x = np.array([5, 1, 9, 0, 3, 8, 2, 7, 4, 6], dtype=float)
    xy = np.column_stack([x, np.zeros(10)])
    part = pt.rcb(xy, 3)
    expected_by_x = [0, 0, 0, 1, 1, 1, 2, 2, 2, 2]
    assert list(part[np.argsort(x)]) == expected_by_x


def test_rcb_grid_quadrants_and_ties():
    """4x4 unit grid, K = 4: the first cut is along x (equal extents), then along y: quadrants."""
    g = np.array([[i, j] for j in range(4) for i in range(4)], dtype=float)
    part = pt.rcb(g, 4)
    for (i, j), p in zip(g, part):
        assert p == (0 if i < 2 else 2) + (0 if j < 2 else 1)
    # ties in the cut coordinate are broken by the other coordinate, then by id
    xy = np.zeros((5, 2))
    xy[:, 1] = [0.0, 0.0, 1.0, 0.0, 1.0]
    xy[:, 0] = 0.0
    part = pt.rcb(xy, 2)           # extents: x 0, y 1 -> cut along y, n1 = 2
    assert list(part) == [0, 0, 1, 1, 1]


def _workload_problem(name="square2k", seed=0):
    w = synth.workload(name, seed)
    P = fem.assemble(w.mesh.xy, w.mesh.tri, coeffs=w.coeffs)
    return w, P


def test_rcb_cover_and_balance():
    w, P = _workload_problem()
    for K in (1, 3, 4, 7):
        part = pt.rcb(P.xy[P.free], K)
        sizes = np.bincount(part, minlength=K)
        assert sizes.sum() == P.n_free and sizes.min() > 0
        assert sizes.max() - sizes.min() <= int(np.ceil(np.log2(K))) + 1


def test_overlap_equals_bfs_distance():
    w, P = _workload_problem()
    part = pt.rcb(P.xy[P.free], 4)
    G = sp.csr_matrix((np.ones(P.A.nnz), P.A.indices, P.A.indptr), shape=P.A.shape)  # pattern incl. zeros
    for delta in (1, 2, 3):
        sets = pt.overlap_sets(P.A, part, 4, delta)
        for i, S in enumerate(sets):
            dist = csg.shortest_path(G, unweighted=True, indices=np.nonzero(part == i)[0], directed=False).min(axis=0)
            assert np.array_equal(S, np.nonzero(dist <= delta)[0])


def test_partition_of_unity_and_coarse_matrix():
    w, P = _workload_problem()
    D = pt.decompose(P, 4, 2)
    Z = D.Z
    assert np.max(np.abs(np.asarray(Z.sum(axis=1)).ravel() - 1.0)) < 1e-15
    A0 = D.A0
    assert np.allclose(A0, A0.T, rtol=0, atol=1e-13 * np.abs(A0).max())
    assert np.all(np.linalg.eigvalsh(A0) > 0)
    # sum_i z_i = 1, hence A_0 1 = Z^T (A 1)
    assert np.allclose(A0.sum(axis=1), Z.T @ (P.A @ np.ones(P.n_free)), rtol=1e-12, atol=1e-12)


def test_local_graph_halo_and_edge_directions():
    m = synth.square_mesh(9, seed=1)
    P = fem.assemble(m.xy, m.tri, coeffs=synth.poly_coeffs(1))
    D = pt.decompose(P, 3, 1)
    edges, _ = fem.mesh_edges(m.tri)
    nbr = {v: set() for v in range(m.n)}
    for a, b in edges:
        nbr[a].add(int(b))
        nbr[b].add(int(a))
    for S in D.sets:
        g = pt.local_graph(P, S)
        interior = set(int(v) for v in P.free[S])
        halo = set().union(*[nbr[v] for v in interior]) - interior
        assert list(g.nodes[:g.n_int]) == sorted(interior)
        assert list(g.nodes[g.n_int:]) == sorted(halo)
        E = set(zip(g.nodes[g.src].tolist(), g.nodes[g.dst].tolist()))
        expected = {(s, t) for t in interior for s in nbr[t]}
        assert E == expected
        # undirected among unknowns, halo nodes only point inward
        for s, t in E:
            if s in interior:
                assert (t, s) in E
            else:
                assert (t, s) not in E
