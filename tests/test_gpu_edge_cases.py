"""Degenerate cases of the method on the CUDA path: zero residuals and right-hand sides,
a start vector that already solves the system, one subdomain (Section III-A with K = 1),
every free node its own subdomain (K = n_free), and inputs the library must refuse."""
import numpy as np
import pytest

import synth
from oracle import ddm, dss, fem, partition as pt
from helpers import assert_close, gpu_setup, oracle_setup, rel

pytestmark = pytest.mark.gpu

KBAR, D = 30, 10
SCHEDULES = [("0", None), ("1", None), ("2", "128"), ("3", "128"), ("3", "256"), ("4", None), ("6", None)]


@pytest.fixture(scope="module")
def ddg():
    import paper_2402_08296_b300 as m
    return m


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


@pytest.fixture(scope="module")
def ctx(ddg):
    c = ddg.ddg_create(0)
    yield c
    ddg.ddg_destroy(c)


def _dev(torch, a):
    return torch.as_tensor(np.asarray(a, dtype=np.float64)).cuda()


def _corrections(ddg, torch, p, r, sizes):
    rd = _dev(torch, r)
    corr = torch.zeros(int(sum(sizes)), dtype=torch.float64, device="cuda")
    s = torch.zeros(len(sizes), dtype=torch.float64, device="cuda")
    ddg.ddg_local_corrections(p, rd, corr, s)
    torch.cuda.synchronize()
    return corr.cpu().numpy(), s.cpu().numpy()


def _check_against_oracle(P, Dd, W, alpha, r, corr, s):
    """Eq. 15 per subdomain: s_i * GNN(r_i / s_i) with s_i = |r_i|; zero where s_i = 0."""
    adj = pt.mesh_adjacency(P.n, P.tri)
    hbar = pt.mean_edge_length(P.xy, P.tri)
    off = 0
    for i, S in enumerate(Dd.sets):
        got = corr[off:off + len(S)]
        off += len(S)
        si = np.linalg.norm(r[S])
        assert abs(s[i] - si) <= 1e-14 * max(si, 1e-300)
        if si == 0.0:
            assert np.all(got == 0.0), i
            continue
        g = pt.local_graph(P, S, adj)
        ref = si * dss.forward(g.xy, g.n_int, g.src, g.dst, r[S] / si, W, KBAR, D, alpha, hbar)
        assert_close(got, ref, 1e-4, i)


@pytest.mark.parametrize("schedule,chunk_t", SCHEDULES)
def test_zero_local_residual_gives_a_zero_correction(ddg, ctx, torch, schedule, chunk_t, monkeypatch):
    """A subdomain whose restricted residual vanishes (s_i = 0) contributes nothing, although
    the network with biases maps a zero input to a nonzero output; its neighbours, whose
    residuals lose the shared overlap entries, still match the oracle."""
    monkeypatch.setenv("DDG_GNN_SCHEDULE", schedule)
    if chunk_t:
        monkeypatch.setenv("DDG_GNN_CHUNK_T", chunk_t)
    w = synth.workload("star20000", 7)
    P, Dd = oracle_setup(w.mesh, w.coeffs, 20, 2)
    W = synth.dss_weights(KBAR, D, 7, bias_scale=0.1)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, 20, 2)
    m = ddg.ddg_model_create(ctx, KBAR, D, 0.02, W)
    try:
        ddg.ddg_setup_precond(p, ddg.DDG_DDM_GNN, m, ddg.DDG_COARSE)
        r = synth.residual_vector(P.n_free, 71)
        for i in (0, 11):
            r[Dd.sets[i]] = 0.0
        corr, s = _corrections(ddg, torch, p, r, [len(S) for S in Dd.sets])
        assert s[0] == 0.0 and s[11] == 0.0
        _check_against_oracle(P, Dd, W, 0.02, r, corr, s)
    finally:
        ddg.ddg_problem_destroy(p)
        ddg.ddg_model_destroy(m)


@pytest.mark.parametrize("kind", ["lu", "gnn"])
def test_zero_residual_preconditions_to_zero(ddg, ctx, torch, kind):
    """M^-1 0 = 0 exactly for both preconditioners, coarse level included (Eq. 16)."""
    w = synth.workload("square2k", 3)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, 4, 1)
    m = ddg.ddg_model_create(ctx, KBAR, D, 1e-3, synth.dss_weights(KBAR, D, 3, bias_scale=0.1))
    try:
        if kind == "lu":
            ddg.ddg_setup_precond(p, ddg.DDG_DDM_LU, None, ddg.DDG_COARSE)
        else:
            ddg.ddg_setup_precond(p, ddg.DDG_DDM_GNN, m, ddg.DDG_COARSE)
        nf = ddg.ddg_problem_info(p)["n_free"]
        rd = torch.zeros(nf, dtype=torch.float64, device="cuda")
        zd = torch.full_like(rd, 7.0)
        ddg.ddg_precondition(p, rd, zd)
        torch.cuda.synchronize()
        assert torch.count_nonzero(zd).item() == 0
    finally:
        ddg.ddg_problem_destroy(p)
        ddg.ddg_model_destroy(m)


@pytest.mark.parametrize("kind", ["lu", "gnn"])
def test_zero_right_hand_side_has_the_zero_solution(ddg, ctx, kind):
    """f = 0 and g = 0 give b = 0, whose solution is u = 0: the solve returns it with zero
    iterations and status OK, from a zero or from a random start vector."""
    w = synth.workload("square2k", 4)
    p = ddg.ddg_mesh_upload(ctx, w.mesh.xy, w.mesh.tri)
    m = ddg.ddg_model_create(ctx, KBAR, D, 1e-3, synth.dss_weights(KBAR, D, 4))
    try:
        n = ddg.ddg_problem_info(p)["n_nodes"]
        ddg.ddg_assemble_nodal(p, np.zeros(n), np.zeros(n))
        _, _, _, b = ddg.ddg_matrix_download(p)
        assert not np.any(b)
        ddg.ddg_partition(p, 4, 1)
        if kind == "lu":
            ddg.ddg_setup_precond(p, ddg.DDG_DDM_LU, None, ddg.DDG_COARSE)
        else:
            ddg.ddg_setup_precond(p, ddg.DDG_DDM_GNN, m, ddg.DDG_COARSE)
        nf = ddg.ddg_problem_info(p)["n_free"]
        for x0 in (None, synth.residual_vector(nf, 41)):
            rep, x = ddg.ddg_fcg_solve(p, 1e-6, 50, 10, x0=x0)
            assert rep["status"] == ddg.DDG_OK and rep["iterations"] == 0
            assert rep["true_rel_residual"] == 0.0
            assert not np.any(x)
            assert ddg.ddg_fcg_history(p).size == 0
    finally:
        ddg.ddg_problem_destroy(p)
        ddg.ddg_model_destroy(m)


def test_start_vector_that_meets_the_tolerance_needs_no_iteration(ddg, ctx):
    """Restarting from a converged solution ends at once; a start vector that does not meet
    the tolerance still iterates and converges."""
    w = synth.workload("square2k", 5)
    P, _ = oracle_setup(w.mesh, w.coeffs, 4, 1)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, 4, 1)
    try:
        ddg.ddg_setup_precond(p, ddg.DDG_DDM_LU, None, ddg.DDG_COARSE)
        rep, x = ddg.ddg_fcg_solve(p, 1e-10, 200, 10)
        assert rep["status"] == ddg.DDG_OK and rep["iterations"] > 1
        xf = x[P.free]
        rep2, x2 = ddg.ddg_fcg_solve(p, 1e-6, 200, 10, x0=xf)
        assert rep2["status"] == ddg.DDG_OK and rep2["iterations"] == 0
        assert rep2["rel_residual"] < 1e-6
        assert np.array_equal(x2, x)
        rep3, x3 = ddg.ddg_fcg_solve(p, 1e-12, 200, 10, x0=xf)
        assert rep3["status"] == ddg.DDG_OK and rep3["iterations"] >= 1
        assert ddm.true_relative_residual(P.A, P.b, x3[P.free]) < 1e-11
    finally:
        ddg.ddg_problem_destroy(p)


def test_one_subdomain_with_exact_local_solve_is_a_direct_solver(ddg, ctx):
    """K = 1 without overlap or coarse level: M^-1 = A^-1, so FCG ends after one step; with
    the coarse level it takes as many steps as the oracle's two-level method."""
    w = synth.workload("square2k", 6)
    P, Dd = oracle_setup(w.mesh, w.coeffs, 1, 0)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, 1, 0)
    try:
        ddg.ddg_setup_precond(p, ddg.DDG_DDM_LU, None, 0)
        rep, x = ddg.ddg_fcg_solve(p, 1e-10, 20, 10)
        assert rep["status"] == ddg.DDG_OK and rep["iterations"] == 1
        assert ddm.true_relative_residual(P.A, P.b, x[P.free]) < 1e-11
        ddg.ddg_setup_precond(p, ddg.DDG_DDM_LU, None, ddg.DDG_COARSE)
        asm = ddm.TwoLevelASM(P, Dd, coarse=True)
        _, it_ref, _ = ddm.fcg(P.A, P.b, asm.apply_lu, 1e-10, 20, 10)
        rep, x = ddg.ddg_fcg_solve(p, 1e-10, 20, 10)
        assert rep["status"] == ddg.DDG_OK and abs(rep["iterations"] - it_ref) <= 1
    finally:
        ddg.ddg_problem_destroy(p)


def test_one_subdomain_gnn_corrections(ddg, ctx, torch):
    """K = 1: the whole free set is one graph of ~2,000 nodes, halo = Dirichlet ring."""
    w = synth.workload("square2k", 8)
    P, Dd = oracle_setup(w.mesh, w.coeffs, 1, 0)
    W = synth.dss_weights(KBAR, D, 8, bias_scale=0.1)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, 1, 0)
    m = ddg.ddg_model_create(ctx, KBAR, D, 0.02, W)
    try:
        ddg.ddg_setup_precond(p, ddg.DDG_DDM_GNN, m, ddg.DDG_COARSE)
        r = synth.residual_vector(P.n_free, 81)
        corr, s = _corrections(ddg, torch, p, r, [len(S) for S in Dd.sets])
        _check_against_oracle(P, Dd, W, 0.02, r, corr, s)
    finally:
        ddg.ddg_problem_destroy(p)
        ddg.ddg_model_destroy(m)


def _tiny(seed):
    mesh = synth.square_mesh(12, seed=seed, jitter=0.3)
    coeffs = synth.poly_coeffs(seed)
    P = fem.assemble(mesh.xy, mesh.tri, coeffs=coeffs)
    return mesh, coeffs, P


@pytest.mark.parametrize("delta", [0, 1])
def test_every_free_node_its_own_subdomain_lu(ddg, ctx, torch, delta):
    """K = n_free: 1x1 local problems (point Jacobi) without overlap, star patches with one
    layer; the coarse space then spans the whole free set (delta = 0) or nearly so."""
    mesh, coeffs, P = _tiny(9)
    K = P.n_free
    Dd = pt.decompose(P, K, delta)
    asm = ddm.TwoLevelASM(P, Dd, coarse=True)
    p = gpu_setup(ddg, ctx, mesh, coeffs, K, delta)
    try:
        ddg.ddg_setup_precond(p, ddg.DDG_DDM_LU, None, ddg.DDG_COARSE)
        r = synth.residual_vector(P.n_free, 91)
        rd = _dev(torch, r)
        zd = torch.zeros_like(rd)
        ddg.ddg_precondition(p, rd, zd)
        torch.cuda.synchronize()
        assert rel(zd.cpu().numpy(), asm.apply_lu(r)) < 1e-11
        _, it_ref, _ = ddm.fcg(P.A, P.b, asm.apply_lu, 1e-10, 200, 10)
        rep, x = ddg.ddg_fcg_solve(p, 1e-10, 200, 10)
        assert rep["status"] == ddg.DDG_OK and abs(rep["iterations"] - it_ref) <= 1
    finally:
        ddg.ddg_problem_destroy(p)


@pytest.mark.parametrize("schedule,chunk_t", SCHEDULES)
def test_every_free_node_its_own_subdomain_gnn(ddg, ctx, torch, schedule, chunk_t, monkeypatch):
    """K = n_free with one overlap layer: ~100 graphs of 3 to 10 nodes, far fewer nodes than
    one chunk holds, so many graphs share a chunk and most chunks of the grid stay empty."""
    monkeypatch.setenv("DDG_GNN_SCHEDULE", schedule)
    if chunk_t:
        monkeypatch.setenv("DDG_GNN_CHUNK_T", chunk_t)
    mesh, coeffs, P = _tiny(10)
    K = P.n_free
    Dd = pt.decompose(P, K, 1)
    W = synth.dss_weights(KBAR, D, 10, bias_scale=0.1)
    p = gpu_setup(ddg, ctx, mesh, coeffs, K, 1)
    m = ddg.ddg_model_create(ctx, KBAR, D, 0.02, W)
    try:
        ddg.ddg_setup_precond(p, ddg.DDG_DDM_GNN, m, ddg.DDG_COARSE)
        r = synth.residual_vector(P.n_free, 101)
        corr, s = _corrections(ddg, torch, p, r, [len(S) for S in Dd.sets])
        _check_against_oracle(P, Dd, W, 0.02, r, corr, s)
    finally:
        ddg.ddg_problem_destroy(p)
        ddg.ddg_model_destroy(m)


def test_inputs_the_library_refuses(ddg, ctx):
    """Each returns DDG_INVALID_ARG (or DDG_BAD_MESH) and leaves the context usable."""
    # one triangle whose three nodes are all on the boundary: no free node
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2]], np.int32)
    with pytest.raises(ddg.DdgError) as e:
        ddg.ddg_mesh_upload(ctx, xy, tri)
    assert e.value.status == ddg.DDG_INVALID_ARG
    # a node index outside the node list
    with pytest.raises(ddg.DdgError) as e:
        ddg.ddg_mesh_upload(ctx, xy, np.array([[0, 1, 3]], np.int32))
    assert e.value.status in (ddg.DDG_INVALID_ARG, ddg.DDG_BAD_MESH)
    w = synth.workload("square2k", 11)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs)
    try:
        nf = ddg.ddg_problem_info(p)["n_free"]
        for K, delta in ((0, 1), (nf + 1, 1), (4, -1), (4, 17)):
            with pytest.raises(ddg.DdgError) as e:
                ddg.ddg_partition(p, K, delta)
            assert e.value.status == ddg.DDG_INVALID_ARG, (K, delta)
        with pytest.raises(ddg.DdgError) as e:
            ddg.ddg_fcg_solve(p, 0.0, 10, 10)
        assert e.value.status == ddg.DDG_INVALID_ARG
        with pytest.raises(ddg.DdgError) as e:
            ddg.ddg_fcg_solve(p, 1e-6, 10, 17)
        assert e.value.status == ddg.DDG_INVALID_ARG
        # still usable: a plain CG solve on the same problem converges
        rep, _ = ddg.ddg_fcg_solve(p, 1e-6, 2000, 1)
        assert rep["status"] == ddg.DDG_OK
    finally:
        ddg.ddg_problem_destroy(p)
