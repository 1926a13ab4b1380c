"""GPU setup kernels against the oracle: assembly (Section II), partition, overlap, local graphs, coarse matrix."""
import numpy as np
import pytest

import synth
from oracle import fem, partition as pt
from helpers import csr_from_gpu, gpu_setup, oracle_setup

pytestmark = pytest.mark.gpu

CASES = [("square2k", 0), ("star20000", 1), ("square2k", 3)]


@pytest.fixture(scope="module")
def ddg():
    import paper_2402_08296_b300 as m
    return m


@pytest.fixture(scope="module")
def ctx(ddg):
    c = ddg.ddg_create(0)
    yield c
    ddg.ddg_destroy(c)


@pytest.mark.parametrize("name,seed", CASES)
def test_assembly_matches_oracle(ddg, ctx, name, seed):
    w = synth.workload(name, seed)
    P = fem.assemble(w.mesh.xy, w.mesh.tri, coeffs=w.coeffs)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs)
    try:
        info = ddg.ddg_problem_info(p)
        assert info["n_free"] == P.n_free
        A, b = csr_from_gpu(ddg, p)
        # same pattern, explicit zeros included: bit-exact indices
        assert np.array_equal(A.indptr, P.A.indptr) and np.array_equal(A.indices, P.A.indices)
        scale = np.abs(P.A.data).max()
        assert np.max(np.abs(A.data - P.A.data)) <= 1e-12 * scale
        assert np.max(np.abs(b - P.b)) <= 1e-12 * max(1.0, np.abs(P.b).max())
        assert (A != A.T).nnz == 0
        assert abs(info["hbar"] - pt.mean_edge_length(w.mesh.xy, w.mesh.tri)) < 1e-13
    finally:
        ddg.ddg_problem_destroy(p)


def test_nodal_assembly_and_user_dirichlet(ddg, ctx):
    m = synth.square_mesh(21, seed=5)
    f = np.sin(m.xy[:, 0]) + m.xy[:, 1]
    g = np.cos(m.xy[:, 1])
    dmask = fem.dirichlet_mask(m.n, m.tri)
    dmask[m.n // 2] = True                      # one extra interior Dirichlet node
    P = fem.assemble(m.xy, m.tri, f_nodal=f, g_nodal=g, dirichlet=dmask)
    p = ddg.ddg_mesh_upload(ctx, m.xy, m.tri, dirichlet=dmask.astype(np.uint8))
    try:
        ddg.ddg_assemble_nodal(p, f, g)
        A, b = csr_from_gpu(ddg, p)
        assert np.array_equal(A.indices, P.A.indices)
        assert np.max(np.abs(A.data - P.A.data)) <= 1e-12 * np.abs(P.A.data).max()
        assert np.max(np.abs(b - P.b)) <= 1e-12 * np.abs(P.b).max()
    finally:
        ddg.ddg_problem_destroy(p)


def test_bad_mesh_is_reported(ddg, ctx):
    m = synth.square_mesh(5, seed=0)
    tri = m.tri.copy()
    tri[3] = tri[3][[0, 2, 1]]                 # one clockwise triangle
    with pytest.raises(ddg.DdgError) as e:
        ddg.ddg_mesh_upload(ctx, m.xy, tri)
    assert e.value.status == ddg.DDG_BAD_MESH


@pytest.mark.parametrize("name,seed,K,delta", [("square2k", 0, 4, 1), ("square2k", 2, 7, 2),
                                                ("star20000", 1, 20, 2), ("star20000", 4, 13, 3)])
def test_partition_overlap_bit_exact(ddg, ctx, name, seed, K, delta):
    w = synth.workload(name, seed)
    P, D = oracle_setup(w.mesh, w.coeffs, K, delta)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, K, delta)
    try:
        part, sub_ptr, sub_idx, mult = ddg.ddg_partition_download(p)
        assert np.array_equal(part, D.part)
        assert np.array_equal(mult, D.mult)
        for i, S in enumerate(D.sets):
            assert np.array_equal(sub_idx[sub_ptr[i]:sub_ptr[i + 1]], S)
        A0, A0inv = ddg.ddg_coarse_download(p)
        assert np.max(np.abs(A0 - D.A0)) <= 1e-12 * np.abs(D.A0).max()
        assert np.max(np.abs(A0inv @ D.A0 - np.eye(K))) < 1e-9
    finally:
        ddg.ddg_problem_destroy(p)


def test_user_partition(ddg, ctx):
    w = synth.workload("square2k", 6)
    P = fem.assemble(w.mesh.xy, w.mesh.tri, coeffs=w.coeffs)
    part = (P.xy[P.free, 0] * 3).astype(np.int64).clip(0, 2)      # three vertical strips
    D = pt.decompose(P, 3, 2, part=part)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs)
    try:
        ddg.ddg_partition(p, 3, 2, part=part)
        _, sub_ptr, sub_idx, _ = ddg.ddg_partition_download(p)
        for i, S in enumerate(D.sets):
            assert np.array_equal(sub_idx[sub_ptr[i]:sub_ptr[i + 1]], S)
        with pytest.raises(ddg.DdgError):
            ddg.ddg_partition(p, 2, 1, part=part)                   # value 2 out of range for K = 2
    finally:
        ddg.ddg_problem_destroy(p)


@pytest.mark.parametrize("name,seed,K,delta", [("square2k", 0, 4, 1), ("star20000", 1, 20, 2)])
def test_local_graphs_bit_exact(ddg, ctx, name, seed, K, delta):
    w = synth.workload(name, seed)
    P, D = oracle_setup(w.mesh, w.coeffs, K, delta)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, K, delta)
    try:
        loc_ptr, n_int, loc_node, nbr_ptr, nbr = ddg.ddg_graph_download(p)
        adj = pt.mesh_adjacency(P.n, P.tri)
        eo = 0
        for i, S in enumerate(D.sets):
            g = pt.local_graph(P, S, adj)
            nl = loc_ptr[i + 1] - loc_ptr[i]
            assert n_int[i] == g.n_int and nl == g.nodes.shape[0]
            assert np.array_equal(loc_node[loc_ptr[i]:loc_ptr[i + 1]], g.nodes)
            ptr = nbr_ptr[loc_ptr[i] + i: loc_ptr[i + 1] + i + 1]
            lst = nbr[eo: eo + ptr[-1]]
            eo += ptr[-1]
            for j in range(nl):
                got = np.sort(lst[ptr[j]:ptr[j + 1]])
                if j < g.n_int:
                    want = np.sort(g.src[g.dst == j])        # every in-neighbour of an unknown
                else:
                    want = np.sort(g.dst[g.src == j])        # a halo node's out-neighbours
                assert np.array_equal(got, want)
    finally:
        ddg.ddg_problem_destroy(p)
