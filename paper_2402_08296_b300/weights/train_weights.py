"""Prepare the DSS weights of the benchmark with the library's own training kernels.

Recipe of Section IV-A/IV-B: random star-shaped domains (seeds disjoint from the
benchmark's and the tests'), each decomposed into ~1000-node subdomains with
two overlap layers; ``ddg_train_local_model`` harvests the residuals of
DDM-LU preconditioned CG on the domain and trains the model on the resulting
local problems (Adam, lr 1e-2, gradient-norm clip 1e-2, plateau decay).  The
Adam state lives in the model, so the meshes form one optimisation; the
learning rate drops x0.1 when the mean loss of a pass over all meshes stops
improving.

Usage (needs a GPU): python paper_2402_08296_b300/weights/train_weights.py --minutes 15 [--kbar 30]
    [--init weights.npy --lr 1e-3] [--nodes 50000 --nodes-max 200000] [--patience 4]
Writes dss_k{kbar}_d10.npy (flat float32 weights, layout of include/ddg.h): of the weights after
every pass, those with which DDM-GNN FCG needs the fewest iterations on a held-out domain.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import paper_2402_08296_b300 as ddg  # noqa: E402
import synth  # noqa: E402

D, ALPHA = 10, 1e-3


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--minutes", type=float, default=15.0)
    ap.add_argument("--meshes", type=int, default=8)
    ap.add_argument("--nodes", type=int, default=30000)
    ap.add_argument("--nodes-max", type=int, default=0,
                    help="if given, mesh sizes log-uniform between --nodes and this (seeded)")
    ap.add_argument("--patience", type=int, default=2,
                    help="passes without a 1 %% lower mean loss before the learning rate drops x0.1")
    ap.add_argument("--steps", type=int, default=200, help="optimiser steps per mesh and pass")
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--harvest", type=int, default=60)
    ap.add_argument("--kbar", type=int, default=30, help="message-passing blocks (Section III-B)")
    ap.add_argument("--init", default=None, help="start from these flat weights instead of Xavier")
    ap.add_argument("--lr", type=float, default=1e-2, help="initial learning rate")
    ap.add_argument("--val-nodes", type=int, default=50000,
                    help="held-out star domain on which the weights of every training pass are scored by FCG iterations")
    ap.add_argument("--out", default=None)
    ap.add_argument("--log", default=None)
    a = ap.parse_args()
    KBAR = a.kbar
    if a.out is None:
        a.out = os.path.join(HERE, f"dss_k{KBAR}_d{D}.npy")
    log = open(a.log, "w") if a.log else sys.stdout
    ctx = ddg.ddg_create(0)
    w0 = np.load(a.init).astype(np.float32) if a.init else None
    model = ddg.ddg_model_create(ctx, KBAR, D, ALPHA, w0, seed=2024)
    # held-out problem (seed disjoint from training, tests and benchmark): the kept weights are
    # those whose DDM-GNN FCG reaches 1e-6 in the fewest iterations
    vm = synth.star_mesh(a.val_nodes, seed=7001)
    val = ddg.ddg_mesh_upload(ctx, vm.xy, vm.tri)
    ddg.ddg_assemble_poly(val, synth.poly_coeffs(7001))
    ddg.ddg_partition(val, max(1, int(round((vm.n - vm.n_boundary_ring) / 1000.0))), 2)

    def val_iterations():
        ddg.ddg_setup_precond(val, ddg.DDG_DDM_GNN, model, ddg.DDG_COARSE)
        rep, _ = ddg.ddg_fcg_solve(val, 1e-6, 1000, 10, want_x=False)
        return rep["iterations"] if rep["status"] == ddg.DDG_OK else 10 ** 6
    problems = []
    sizes = [a.nodes] * a.meshes
    if a.nodes_max > a.nodes:
        rng = np.random.default_rng(4999)
        sizes = [int(round(np.exp(rng.uniform(np.log(a.nodes), np.log(a.nodes_max))))) for _ in range(a.meshes)]
    for s in range(a.meshes):
        seed = 5000 + s
        m = synth.star_mesh(sizes[s], seed=seed)
        K = max(1, int(round((m.n - m.n_boundary_ring) / 1000.0)))
        p = ddg.ddg_mesh_upload(ctx, m.xy, m.tri)
        ddg.ddg_assemble_poly(p, synth.poly_coeffs(seed))
        ddg.ddg_partition(p, K, 2)
        problems.append(p)
    lr, best, stale, rnd = a.lr, np.inf, 0, 0
    t0 = time.time()
    n_w = KBAR * synth.n_weights_per_block(D)
    best_it = val_iterations()
    best_w = ddg.ddg_model_get_weights(model, n_w)
    print(f"start: held-out FCG iterations {best_it}", file=log, flush=True)
    while time.time() - t0 < 60.0 * a.minutes:
        losses = []
        for i, p in enumerate(problems):
            rep = ddg.ddg_train_local_model(p, model, steps=a.steps, batch=a.batch, lr=lr, clip=1e-2,
                                            harvest_iters=a.harvest, seed=1000 * rnd + i)
            losses.append(rep["loss_last"])
            print(f"pass {rnd} mesh {i} samples {rep['samples']} loss {rep['loss_first']:.3e} -> "
                  f"{rep['loss_last']:.3e} lr {lr:.1e} {rep['ms'] / 1e3:.1f}s t {time.time() - t0:.0f}s",
                  file=log, flush=True)
            if time.time() - t0 > 60.0 * a.minutes:
                break
        its = val_iterations()
        if its < best_it:
            best_it, best_w = its, ddg.ddg_model_get_weights(model, n_w)
        print(f"pass {rnd} held-out FCG iterations {its} (best {best_it})", file=log, flush=True)
        mean = float(np.mean(losses))
        if mean < 0.99 * best:
            best, stale = mean, 0
        else:
            stale += 1
            if stale >= a.patience:
                lr, stale = lr * 0.1, 0
        rnd += 1
    np.save(a.out, best_w)
    print(f"saved {a.out} after {rnd} passes (held-out FCG iterations {best_it})", file=log, flush=True)
    for p in problems + [val]:
        ddg.ddg_problem_destroy(p)
    ddg.ddg_model_destroy(model)
    ddg.ddg_destroy(ctx)


if __name__ == "__main__":
    main()
