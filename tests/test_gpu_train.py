"""Hand-written training kernels (Section III-B, Eq. 23; Section IV-B) against the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import dss, fem, partition as pt
from helpers import gpu_setup

pytestmark = pytest.mark.gpu

D = 10


def oracle_loss(W, kbar, alpha, P, Dd, graphs, r, adj, hbar):
    """mean over graphs of sum_k L_res(r_hat^k) (Eqs. 11, 23), FP64."""
    tot = 0.0
    A = P.A.tocsr()
    for i in graphs:
        S = Dd.sets[i]
        g = pt.local_graph(P, S, adj)
        c = r[S] / np.linalg.norm(r[S])
        _, outs = dss.forward(g.xy, g.n_int, g.src, g.dst, c, W, kbar, D, alpha, hbar, return_all=True)
        Ai = A[S][:, S]
        tot += sum(dss.residual_loss(Ai, u, c) for u in outs)
    return tot / len(graphs)


def test_loss_and_gradient_match_oracle_finite_differences():
    import torch
    import paper_2402_08296_b300 as ddg
    kbar, alpha = 3, 0.2
    w = synth.workload("square2k", 3)
    P = fem.assemble(w.mesh.xy, w.mesh.tri, coeffs=w.coeffs)
    Dd = pt.decompose(P, 4, 1)
    adj = pt.mesh_adjacency(P.n, P.tri)
    hbar = pt.mean_edge_length(P.xy, P.tri)
    W = synth.dss_weights(kbar, D, 8, bias_scale=0.2, gain=2.0).astype(np.float64)
    r = synth.residual_vector(P.n_free, 9)
    graphs = [0, 2, 3]
    ctx = ddg.ddg_create(0)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, 4, 1)
    m = ddg.ddg_model_create(ctx, kbar, D, alpha, W.astype(np.float32))
    try:
        rd = torch.as_tensor(r).cuda()
        loss, grad = ddg.ddg_train_loss_grad(p, m, rd, graphs, W.size)
        Wf = W.astype(np.float32).astype(np.float64)
        ref = oracle_loss(Wf, kbar, alpha, P, Dd, graphs, r, adj, hbar)
        assert abs(loss - ref) <= 1e-4 * abs(ref)
        rng = np.random.default_rng(0)
        # every parameter kind of every block: sample coordinates across the flat vector
        idx = np.unique(np.concatenate([rng.choice(W.size, 40, replace=False),
                                        np.argsort(-np.abs(grad))[:10]]))
        eps = 1e-5
        fd = []
        for q in idx:
            Wp, Wm = Wf.copy(), Wf.copy()
            Wp[q] += eps
            Wm[q] -= eps
            fd.append((oracle_loss(Wp, kbar, alpha, P, Dd, graphs, r, adj, hbar)
                       - oracle_loss(Wm, kbar, alpha, P, Dd, graphs, r, adj, hbar)) / (2 * eps))
        fd = np.array(fd)
        scale = np.abs(fd).max()
        assert scale > 0
        assert np.max(np.abs(grad[idx] - fd)) <= 2e-3 * scale, np.max(np.abs(grad[idx] - fd)) / scale
    finally:
        ddg.ddg_problem_destroy(p)
        ddg.ddg_model_destroy(m)
        ddg.ddg_destroy(ctx)


def test_training_reduces_the_loss():
    import paper_2402_08296_b300 as ddg
    kbar = 30
    w = synth.workload("star20000", 11)
    ctx = ddg.ddg_create(0)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, w.K, 2)
    m = ddg.ddg_model_create(ctx, kbar, D, 1e-3, None, seed=11)
    try:
        n_w = kbar * synth.n_weights_per_block(D)
        w0 = ddg.ddg_model_get_weights(m, n_w)
        rep = ddg.ddg_train_local_model(p, m, steps=150, batch=16, harvest_iters=30, seed=3)
        assert rep["samples"] > 0 and rep["steps"] == 150
        assert rep["loss_last"] < 0.8 * rep["loss_first"], rep
        w1 = ddg.ddg_model_get_weights(m, n_w)
        assert np.all(np.isfinite(w1)) and not np.array_equal(w0, w1)
        # the trained model is usable by the preconditioner right away
        ddg.ddg_setup_precond(p, ddg.DDG_DDM_GNN, m, ddg.DDG_COARSE)
        r2, _ = ddg.ddg_fcg_solve(p, 1e-6, 400, 10)
        assert r2["status"] in (ddg.DDG_OK, ddg.DDG_NOT_CONVERGED)
    finally:
        ddg.ddg_problem_destroy(p)
        ddg.ddg_model_destroy(m)
        ddg.ddg_destroy(ctx)


def test_autograd_function_trains_through_the_hand_written_backward():
    """dss_residual_loss: torch.autograd sees the library's loss and gradient; a few Adam
    steps of torch.optim through it lower the loss, and ddg_model_set_weights round-trips."""
    import torch
    import paper_2402_08296_b300 as ddg
    kbar, alpha = 4, 0.1
    w = synth.workload("square2k", 5)
    P = fem.assemble(w.mesh.xy, w.mesh.tri, coeffs=w.coeffs)
    W0 = synth.dss_weights(kbar, D, 11, bias_scale=0.05)
    r = synth.residual_vector(P.n_free, 12)
    ctx = ddg.ddg_create(0)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs, 4, 1)
    m = ddg.ddg_model_create(ctx, kbar, D, alpha, W0)
    try:
        rd = torch.as_tensor(r).cuda()
        graphs = [0, 1, 2, 3]
        wt = torch.nn.Parameter(torch.as_tensor(W0).cuda())
        loss = ddg.dss_residual_loss(wt, p, m, rd, graphs)
        loss.backward()
        l_ref, g_ref = ddg.ddg_train_loss_grad(p, m, rd, graphs, W0.size)
        assert float(loss) == l_ref
        # weight gradients are summed with float atomics across CTAs: equal up to summation order
        g = wt.grad.cpu().numpy()
        assert np.allclose(g, g_ref, rtol=1e-4, atol=1e-6 * np.abs(g_ref).max())
        assert np.array_equal(ddg.ddg_model_get_weights(m, W0.size), W0)
        opt = torch.optim.Adam([wt], lr=1e-3)
        first = float(loss)
        for _ in range(30):
            opt.zero_grad()
            loss = ddg.dss_residual_loss(wt, p, m, rd, graphs)
            loss.backward()
            opt.step()
        assert float(loss) < first
    finally:
        ddg.ddg_problem_destroy(p)
        ddg.ddg_model_destroy(m)
        ddg.ddg_destroy(ctx)

