"""GPU flexible CG against the oracle's Krylov drivers (Algorithm 1; flexible CG)."""
import os

import numpy as np
import pytest

import synth
from oracle import ddm
from helpers import assert_close, gpu_setup, oracle_setup

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2402_08296_b300", "weights", "dss_k30_d10.npy")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ddg():
    import paper_2402_08296_b300 as m
    return m


@pytest.fixture(scope="module")
def ctx(ddg):
    c = ddg.ddg_create(0)
    yield c
    ddg.ddg_destroy(c)


def test_unpreconditioned_cg_matches_oracle(ddg, ctx):
    w = synth.workload("square2k", 0)
    P, _ = oracle_setup(w.mesh, w.coeffs, 1, 0)
    _, it_ref, _ = ddm.pcg(P.A, P.b, lambda r: r, 1e-8, 2000)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs)
    try:
        ddg.ddg_setup_precond(p, ddg.DDG_NONE)
        rep, x = ddg.ddg_fcg_solve(p, 1e-8, 2000, 1)
        assert rep["status"] == 0
        assert abs(rep["iterations"] - it_ref) <= 1
        assert ddm.true_relative_residual(P.A, P.b, x[P.free]) <= 1.01e-8
        assert np.array_equal(x[P.dirichlet], P.g[P.dirichlet])
    finally:
        ddg.ddg_problem_destroy(p)


@pytest.mark.parametrize("m_trunc", [1, 10])
def test_ddm_lu_pcg_small_config(ddg, ctx, m_trunc):
    """4 subdomains, 1-layer overlap, Nicolaides coarse space, PCG to 1e-8 (the small DDM-LU configuration)."""
    w = synth.workload("square2k", 1)
    P, Dd = oracle_setup(w.mesh, w.coeffs, 4, 1)
    asm = ddm.TwoLevelASM(P, Dd)
    _, it_ref, _ = ddm.pcg(P.A, P.b, asm.apply_lu, 1e-8, 500)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, 4, 1)
    try:
        ddg.ddg_setup_precond(p, ddg.DDG_DDM_LU, None, ddg.DDG_COARSE)
        rep, x = ddg.ddg_fcg_solve(p, 1e-8, 500, m_trunc)
        assert rep["status"] == 0
        assert abs(rep["iterations"] - it_ref) <= 1
        tr = ddm.true_relative_residual(P.A, P.b, x[P.free])
        assert tr <= 1.01e-8 and abs(tr - rep["true_rel_residual"]) < 1e-10
        u_ref = P.full_solution(np.linalg.solve(P.A.toarray(), P.b))
        assert np.max(np.abs(x - u_ref)) < 1e-6 * np.abs(u_ref).max()
    finally:
        ddg.ddg_problem_destroy(p)


def test_ddm_lu_fcg_star(ddg, ctx):
    w = synth.workload("star20000", 5)
    P, Dd = oracle_setup(w.mesh, w.coeffs, w.K, 2)
    asm = ddm.TwoLevelASM(P, Dd)
    _, it_ref, _ = ddm.fcg(P.A, P.b, asm.apply_lu, 1e-6, 500, 10)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, w.K, 2)
    try:
        ddg.ddg_setup_precond(p, ddg.DDG_DDM_LU, None, ddg.DDG_COARSE)
        rep, x = ddg.ddg_fcg_solve(p, 1e-6, 500, 10)
        assert rep["status"] == 0 and abs(rep["iterations"] - it_ref) <= 1
        assert ddm.true_relative_residual(P.A, P.b, x[P.free]) <= 1.01e-6
    finally:
        ddg.ddg_problem_destroy(p)


def test_solve_is_deterministic(ddg, ctx):
    w = synth.workload("star20000", 6)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, w.K, 2)
    m = ddg.ddg_model_create(ctx, 30, 10, 1e-3, synth.dss_weights(30, 10, 6))
    try:
        ddg.ddg_setup_precond(p, ddg.DDG_DDM_GNN, m, ddg.DDG_COARSE)
        r1, x1 = ddg.ddg_fcg_solve(p, 1e-6, 40, 10)
        r2, x2 = ddg.ddg_fcg_solve(p, 1e-6, 40, 10)
        assert r1["iterations"] == r2["iterations"]
        assert np.array_equal(x1, x2)
    finally:
        ddg.ddg_problem_destroy(p)
        ddg.ddg_model_destroy(m)


def test_failures_are_status_codes(ddg, ctx):
    """Host-side fault injection: every failure returns a status, none hangs or aborts."""
    w = synth.workload("square2k", 2)
    # HBM budget too small for the problem
    small = ddg.ddg_create(0, 1 << 16)
    try:
        with pytest.raises(ddg.DdgError) as e:
            ddg.ddg_mesh_upload(small, w.mesh.xy, w.mesh.tri)
        assert e.value.status == ddg.DDG_OOM
    finally:
        ddg.ddg_destroy(small)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, 4, 1)
    try:
        # a part left empty by a user partition
        part = np.zeros(ddg.ddg_problem_info(p)["n_free"], np.int32)
        with pytest.raises(ddg.DdgError) as e:
            ddg.ddg_partition(p, 2, 1, part=part)
        assert e.value.status == ddg.DDG_INVALID_ARG
        ddg.ddg_partition(p, 4, 1)
        # calls out of order / bad arguments
        with pytest.raises(ddg.DdgError):
            ddg.ddg_setup_precond(p, ddg.DDG_DDM_GNN, None)
        with pytest.raises(ddg.DdgError):
            ddg.ddg_model_create(ctx, 30, 12, 1e-3, np.zeros(30 * (11 * 144 + 15 * 12 + 1), np.float32))
        # non-finite weights: the Krylov loop reports a breakdown instead of iterating on NaN
        W = synth.dss_weights(30, 10, 0)
        W[5] = np.nan
        m = ddg.ddg_model_create(ctx, 30, 10, 1e-3, W)
        try:
            ddg.ddg_setup_precond(p, ddg.DDG_DDM_GNN, m, ddg.DDG_COARSE)
            rep, _ = ddg.ddg_fcg_solve(p, 1e-6, 50, 10)
            assert rep["status"] == ddg.DDG_BREAKDOWN and rep["iterations"] <= 1
        finally:
            ddg.ddg_setup_precond(p, ddg.DDG_NONE)
            ddg.ddg_model_destroy(m)
        # an iteration cap is reported, not an endless loop
        rep, _ = ddg.ddg_fcg_solve(p, 1e-12, 3, 10)
        assert rep["status"] == ddg.DDG_NOT_CONVERGED and rep["iterations"] == 3
    finally:
        ddg.ddg_problem_destroy(p)


def test_gnn_schedules_agree_and_graph_replay_matches_direct(ddg, ctx, monkeypatch):
    """Every GNN schedule gives the same local corrections as schedule 0 (element-wise), and
    for every schedule the CUDA-graph replay of the FCG period gives the same iterates as
    direct launches."""
    import torch
    w = synth.workload("star20000", 3)
    W = synth.dss_weights(30, 10, 3, bias_scale=0.1)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, w.K, 2)
    m = ddg.ddg_model_create(ctx, 30, 10, 0.02, W)
    ref = None
    try:
        for schedule in ["0", "1", "2", "3", "4", "6"]:
            monkeypatch.setenv("DDG_GNN_SCHEDULE", schedule)
            monkeypatch.delenv("DDG_NO_GRAPH", raising=False)
            ddg.ddg_setup_precond(p, ddg.DDG_DDM_GNN, m, ddg.DDG_COARSE)
            info = ddg.ddg_problem_info(p)
            r = torch.as_tensor(synth.residual_vector(info["n_free"], 5)).cuda()
            corr = torch.zeros(info["sum_k"], dtype=torch.float64, device="cuda")
            s = torch.zeros(info["K"], dtype=torch.float64, device="cuda")
            ddg.ddg_local_corrections(p, r, corr, s)
            torch.cuda.synchronize()
            got = corr.cpu().numpy()
            if ref is None:
                ref = got
            else:
                assert_close(got, ref, 1e-5, schedule)
            r1, x1 = ddg.ddg_fcg_solve(p, 1e-6, 45, 10)
            monkeypatch.setenv("DDG_NO_GRAPH", "1")
            r2, x2 = ddg.ddg_fcg_solve(p, 1e-6, 45, 10)
            assert r1["iterations"] == r2["iterations"] and np.array_equal(x1, x2), schedule
            assert r1["gnn_schedule"] == int(schedule)
    finally:
        ddg.ddg_problem_destroy(p)
        ddg.ddg_model_destroy(m)


@pytest.mark.parametrize("schedule", ["auto", "3", "4", "6"])
def test_ddm_gnn_solve_judged_by_the_oracle(ddg, ctx, schedule, monkeypatch):
    """DDM-GNN FCG(10) with the trained weights to 1e-6 on a ~20k-node star domain: the oracle's
    own assembly gives the true relative residual, and x is within kappa * tol of the oracle's
    1e-12 DDM-LU solve (reading C-19)."""
    if schedule != "auto":
        monkeypatch.setenv("DDG_GNN_SCHEDULE", schedule)
    w = synth.workload("star20000", 7)
    P, Dd = oracle_setup(w.mesh, w.coeffs, w.K, 2)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, w.K, 2)
    m = ddg.ddg_model_create(ctx, 30, 10, 1e-3, np.load(WEIGHTS).astype(np.float32))
    try:
        ddg.ddg_setup_precond(p, ddg.DDG_DDM_GNN, m, ddg.DDG_COARSE)
        rep, x = ddg.ddg_fcg_solve(p, 1e-6, 500, 10)
        assert rep["status"] == ddg.DDG_OK, rep
        tr = ddm.true_relative_residual(P.A, P.b, x[P.free])
        assert tr <= 1.01e-6 and abs(tr - rep["true_rel_residual"]) <= 1e-9
        assert np.array_equal(x[P.dirichlet], P.g[P.dirichlet])
        asm = ddm.TwoLevelASM(P, Dd)
        xs, _, _ = ddm.pcg(P.A, P.b, asm.apply_lu, 1e-12, 1000)
        kappa = ddm.condition_estimate(P.A, lambda v: ddm.pcg(P.A, v, asm.apply_lu, 1e-6, 1000)[0], iters=3)
        assert np.linalg.norm(x[P.free] - xs) <= kappa * (tr + 1e-12) * np.linalg.norm(xs)
    finally:
        ddg.ddg_problem_destroy(p)
        ddg.ddg_model_destroy(m)


def test_a_weight_copy_that_never_arrives_ends_in_a_timeout_status(ddg, ctx, monkeypatch):
    """The persistent GNN kernel waits about one second for each block's weights (bulk copy and
    mbarrier); a test hook withholds the first copy, so every CTA's wait runs out.  The solve
    reports DDG_TIMEOUT, and the context is usable afterwards.  No fault, trap or hang."""
    w = synth.workload("square2k", 4)
    W = synth.dss_weights(30, 10, 4)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, 4, 1)
    m = ddg.ddg_model_create(ctx, 30, 10, 1e-3, W)
    try:
        monkeypatch.setenv("DDG_GNN_SCHEDULE", "0")
        ddg.ddg_setup_precond(p, ddg.DDG_DDM_GNN, m, ddg.DDG_COARSE)
        monkeypatch.setenv("DDG_TEST_WAIT_TIMEOUT", "1")
        with pytest.raises(ddg.DdgError) as e:
            ddg.ddg_fcg_solve(p, 1e-6, 1, 10)
        assert e.value.status == ddg.DDG_TIMEOUT
        monkeypatch.delenv("DDG_TEST_WAIT_TIMEOUT")
        # usable afterwards: the same GNN runs to its iteration cap (untrained weights), and a
        # DDM-LU solve on the same problem converges
        rep, _ = ddg.ddg_fcg_solve(p, 1e-6, 20, 10)
        assert rep["status"] in (ddg.DDG_OK, ddg.DDG_NOT_CONVERGED) and rep["iterations"] >= 1
        ddg.ddg_setup_precond(p, ddg.DDG_DDM_LU, None, ddg.DDG_COARSE)
        rep, _ = ddg.ddg_fcg_solve(p, 1e-6, 300, 10)
        assert rep["status"] == ddg.DDG_OK
    finally:
        ddg.ddg_problem_destroy(p)
        ddg.ddg_model_destroy(m)


def test_residual_history_of_a_solve(ddg, ctx):
    """ddg_fcg_history: one relative residual per iteration, ending at the report's value."""
    w = synth.workload("square2k", 5)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, 4, 1)
    try:
        ddg.ddg_setup_precond(p, ddg.DDG_DDM_LU, None, ddg.DDG_COARSE)
        rep, _ = ddg.ddg_fcg_solve(p, 1e-8, 200, 10)
        h = ddg.ddg_fcg_history(p)
        assert rep["status"] == ddg.DDG_OK and len(h) == rep["iterations"]
        assert h[-1] == rep["rel_residual"] and h[-1] < 1e-8 <= h[-2]
        assert np.all(np.isfinite(h)) and h[0] < 1.0
    finally:
        ddg.ddg_problem_destroy(p)

