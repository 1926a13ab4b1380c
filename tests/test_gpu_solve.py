"""GPU flexible CG against the oracle's Krylov drivers (Algorithm 1; flexible CG)."""
import numpy as np
import pytest

import synth
from oracle import ddm
from helpers import gpu_setup, oracle_setup

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
        assert ddm.true_relative_residual(P.A, P.b, x[P.free]) < 1.2e-8
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
        assert tr < 1.2e-8 and abs(tr - rep["true_rel_residual"]) < 1e-10
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
        assert ddm.true_relative_residual(P.A, P.b, x[P.free]) < 1.2e-6
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
