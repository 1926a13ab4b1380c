"""Serving: requests that arrive while others run are admitted and overlap on the GPU,
every result equals the stand-alone solve of the same problem (bitwise), and the oracle
confirms every served solution (true relative residual of Algorithm 1's stopping test)."""
import os
import time

import numpy as np
import pytest

import synth
from oracle import ddm, fem, partition as pt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2402_08296_b300", "weights", "dss_k30_d10.npy")

pytestmark = pytest.mark.gpu


def _wait(ddg, ctx, tickets, sizes, timeout=300.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t, n in zip(tickets, sizes):
            if t in out:
                continue
            st, rep, x = ddg.ddg_poll(ctx, t, n)
            if st != ddg.DDG_PENDING:
                out[t] = (st, rep, x)
        assert time.time() - t0 < timeout, "requests did not finish"
        time.sleep(0.002)
    return out


@pytest.mark.parametrize("mode", ["fused", "separate"])
def test_results_alone_equal_results_in_the_mix(mode, monkeypatch):
    """fused: the DDM-GNN requests share one GNN launch per block (schedule 3, chunk width 128);
    separate: every request runs its own kernels on its own stream."""
    import paper_2402_08296_b300 as ddg
    # the stand-alone solves use the schedule the request loop's fused steps use
    monkeypatch.setenv("DDG_GNN_SCHEDULE", "3")
    monkeypatch.setenv("DDG_GNN_CHUNK_T", "128")
    ctx = ddg.ddg_create(0)
    # the trained weights, so that the DDM-GNN requests converge and the oracle can judge them
    W = np.load(WEIGHTS).astype(np.float32)
    m = ddg.ddg_model_create(ctx, 30, 10, 1e-3, W)
    try:
        reqs = []
        for i, n in enumerate([6000, 20000, 9000, 40000, 12000, 5000, 15000, 7000]):
            mesh = synth.star_mesh(n, seed=300 + i)
            kind = ddg.DDG_DDM_GNN if i % 2 == 0 else ddg.DDG_DDM_LU
            reqs.append((mesh, synth.poly_coeffs(300 + i), kind))
        # alone: one after the other, each with the blocking solver
        alone = []
        for mesh, r, kind in reqs:
            p = ddg.ddg_mesh_upload(ctx, mesh.xy, mesh.tri)
            ddg.ddg_assemble_poly(p, r)
            K = max(1, int(ddg.ddg_problem_info(p)["n_free"] / 1000 + 0.5))
            ddg.ddg_partition(p, K, 2)
            ddg.ddg_setup_precond(p, kind, m if kind == ddg.DDG_DDM_GNN else None, ddg.DDG_COARSE)
            rep, x = ddg.ddg_fcg_solve(p, 1e-6, 600, 10)
            alone.append((rep, x))
            ddg.ddg_problem_destroy(p)
        # in the mix: all submitted at once, solved concurrently by the scheduler
        ddg.ddg_serve_config(ctx, 6, fuse_gnn=(mode == "fused"))
        tickets = [ddg.ddg_submit(ctx, mesh.xy, mesh.tri, r, kind, m if kind == ddg.DDG_DDM_GNN else None,
                                  max_iter=600) for mesh, r, kind in reqs]
        res = _wait(ddg, ctx, tickets, [mesh.n for mesh, _, _ in reqs])
        for t, (rep_a, x_a), (mesh, r, kind) in zip(tickets, alone, reqs):
            st, rep, x = res[t]
            assert st == rep_a["status"] == ddg.DDG_OK
            assert rep["iterations"] == rep_a["iterations"]
            assert np.array_equal(x, x_a)
            # the oracle's own assembly of the request judges the served solution
            P = fem.assemble(mesh.xy, mesh.tri, coeffs=r)
            tr = ddm.true_relative_residual(P.A, P.b, x[P.free])
            assert tr <= 1.01e-6 and abs(tr - rep["true_rel_residual"]) <= 1e-9, (kind, tr)
            assert np.array_equal(x[P.dirichlet], P.g[P.dirichlet])
            if kind == ddg.DDG_DDM_GNN and mesh.n <= 20000:
                # and the solution itself: within kappa * tol of the oracle's 1e-12 DDM-LU solve (reading C-19)
                K = max(1, int(P.n_free / 1000 + 0.5))
                asm = ddm.TwoLevelASM(P, pt.decompose(P, K, 2))
                xs, _, _ = ddm.pcg(P.A, P.b, asm.apply_lu, 1e-12, 1000)
                kappa = ddm.condition_estimate(P.A, lambda v: ddm.pcg(P.A, v, asm.apply_lu, 1e-6, 1000)[0], iters=3)
                assert np.linalg.norm(x[P.free] - xs) <= kappa * (tr + 1e-12) * np.linalg.norm(xs)
        stats = ddg.ddg_serve_stats(ctx)
        assert stats["completed"] == len(reqs) and stats["pending"] == 0 and stats["active"] == 0
        assert stats["p99_ms"] >= stats["p50_ms"] > 0
        with pytest.raises(ddg.DdgError):
            ddg.ddg_poll(ctx, tickets[0], reqs[0][0].n)       # a ticket is collected once
    finally:
        ddg.ddg_model_destroy(m)
        ddg.ddg_destroy(ctx)


def test_admission_waits_for_the_hbm_budget():
    import paper_2402_08296_b300 as ddg
    budget = 200 << 20
    ctx = ddg.ddg_create(0, budget)
    try:
        meshes = [synth.star_mesh(30000, seed=400 + i) for i in range(5)]
        tickets = [ddg.ddg_submit(ctx, mesh.xy, mesh.tri, synth.poly_coeffs(400 + i), ddg.DDG_DDM_LU, max_iter=400)
                   for i, mesh in enumerate(meshes)]
        peak = 0
        t0 = time.time()
        done = {}
        while len(done) < len(tickets):
            stats = ddg.ddg_serve_stats(ctx)
            peak = max(peak, stats["reserved_bytes"])
            for t, mesh in zip(tickets, meshes):
                if t not in done:
                    st, rep, x = ddg.ddg_poll(ctx, t, mesh.n)
                    if st != ddg.DDG_PENDING:
                        done[t] = st
            assert time.time() - t0 < 300
            time.sleep(0.001)
        assert all(st == ddg.DDG_OK for st in done.values())
        assert peak <= budget
    finally:
        ddg.ddg_destroy(ctx)


def test_a_full_admission_queue_answers_busy():
    import paper_2402_08296_b300 as ddg
    ctx = ddg.ddg_create(0)
    try:
        ddg.ddg_serve_config(ctx, 1, max_pending=2)
        mesh = synth.star_mesh(20000, seed=500)
        r = synth.poly_coeffs(500)
        got, busy = [], 0
        for _ in range(8):   # submitted faster than one slot drains them
            try:
                got.append(ddg.ddg_submit(ctx, mesh.xy, mesh.tri, r, ddg.DDG_DDM_LU, max_iter=400))
            except ddg.DdgError as e:
                assert e.status == ddg.DDG_BUSY
                busy += 1
        assert busy > 0 and len(got) >= 2
        res = _wait(ddg, ctx, got, [mesh.n] * len(got))
        assert all(st == ddg.DDG_OK for st, _, _ in res.values())
    finally:
        ddg.ddg_destroy(ctx)

