"""Offline preparation of the DSS weights used by the benchmark (Section IV-A/IV-B recipe).

Not part of the solver: it produces ``dss_k30_d10.npy``, the flat weight vector
(layout of include/ddg.h) that ``ddg_model_create`` loads.

Data (Section IV-A): random star-shaped domains; each global problem is solved
by PCG with the two-level DDM-LU preconditioner through the library, and
every iteration's normalised restricted residuals R_i r^n / |R_i r^n| become
local samples G_i = (Omega_{h,i}, c).

Model and loss (Section III-B, Eqs. 18-23): kbar blocks of Phi_out, Phi_in,
Psi and a decoder per block, H^0 = 0, h += alpha Psi(...); the training loss
is the sum over blocks of the local residual loss
L_res(r_hat^k) = mean_i ((R_i A R_i^T r_hat^k - c)_i^2)   (Eq. 11).
Optimiser (Section IV-B): Adam, learning rate 1e-2, gradient-norm clipping
1e-2, learning rate x0.1 on plateaus; Xavier initialisation, zero biases.
The network is evaluated with torch's autograd here; this script is a data
and weight generator and none of its code is on the solver's path.

Usage (needs a GPU): python paper_2402_08296_b300/weights/train_dss.py --minutes 15
"""
from __future__ import annotations

import argparse
import math
import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import paper_2402_08296_b300 as ddg  # noqa: E402
import synth  # noqa: E402

KBAR, D, ALPHA = 30, 10, 1e-3


# ---------------------------------------------------------------- data
def harvest(ctx, mesh, coeffs, K, delta, max_iter=60, tol=1e-6, dev="cuda"):
    """Graphs, local matrices and normalised local residuals of every DDM-LU PCG iteration."""
    p = ddg.ddg_mesh_upload(ctx, mesh.xy, mesh.tri)
    try:
        ddg.ddg_assemble_poly(p, coeffs)
        ddg.ddg_partition(p, K, delta)
        ddg.ddg_setup_precond(p, ddg.DDG_DDM_LU, None, ddg.DDG_COARSE)
        info = ddg.ddg_problem_info(p)
        rowptr, col, val, b = ddg.ddg_matrix_download(p)
        _, sub_ptr, sub_idx, _ = ddg.ddg_partition_download(p)
        loc_ptr, n_int, loc_node, nbr_ptr, nbr = ddg.ddg_graph_download(p)
        hbar = info["hbar"]
        # PCG (Algorithm 1) with the library's DDM-LU preconditioner; vector algebra in torch
        bt = torch.as_tensor(b, device=dev)
        x = torch.zeros_like(bt)
        r = bt.clone()
        z = torch.zeros_like(bt)
        q = torch.zeros_like(bt)
        ddg.ddg_precondition(p, r, z)
        pp = z.clone()
        rho = torch.dot(r, z)
        residuals = [r.clone()]
        for _ in range(max_iter):
            ddg.ddg_apply_A(p, pp, q)
            al = rho / torch.dot(pp, q)
            x += al * pp
            r -= al * q
            if float(torch.linalg.norm(r) / torch.linalg.norm(bt)) < tol:
                break
            residuals.append(r.clone())
            ddg.ddg_precondition(p, r, z)
            rho_new = torch.dot(r, z)
            pp = z + (rho_new / rho) * pp
            rho = rho_new
        R = torch.stack(residuals).cpu().numpy()          # (iters, n_free)
    finally:
        ddg.ddg_problem_destroy(p)
    graphs = []
    eo = 0
    for i in range(K):
        S = sub_idx[sub_ptr[i]:sub_ptr[i + 1]]
        k = int(n_int[i])
        nl = int(loc_ptr[i + 1] - loc_ptr[i])
        nodes = loc_node[loc_ptr[i]:loc_ptr[i + 1]]
        ptr = nbr_ptr[loc_ptr[i] + i: loc_ptr[i + 1] + i + 1]
        lst = nbr[eo: eo + ptr[-1]]
        eo += ptr[-1]
        src, dst = [], []
        for t in range(k):                                 # every neighbour s of an unknown t: s -> t
            for s in lst[ptr[t]:ptr[t + 1]]:
                src.append(int(s))
                dst.append(t)
        xy = mesh.xy[nodes]
        xy = (xy - xy[:k].mean(axis=0)) / hbar
        # local matrix R_i A R_i^T (COO over the unknowns)
        pos = {int(f): a for a, f in enumerate(S)}
        li, lj, lv = [], [], []
        for a, f in enumerate(S):
            for e in range(rowptr[f], rowptr[f + 1]):
                c_ = pos.get(int(col[e]))
                if c_ is not None:
                    li.append(a); lj.append(c_); lv.append(val[e])
        cs = R[:, S]
        nrm = np.linalg.norm(cs, axis=1)
        cs = cs[nrm > 0] / nrm[nrm > 0, None]
        graphs.append(dict(k=k, n=nl, xy=xy.astype(np.float32), src=np.array(src), dst=np.array(dst),
                           ai=np.array(li), aj=np.array(lj), av=np.array(lv, np.float32), c=cs.astype(np.float32)))
    return graphs


# ---------------------------------------------------------------- model
class DSS(torch.nn.Module):
    def __init__(self, kbar, d, alpha):
        super().__init__()
        self.kbar, self.d, self.alpha = kbar, d, alpha
        L = torch.nn.Linear
        mk = lambda i, o: torch.nn.Sequential(L(i, d), torch.nn.ReLU(), L(d, o))
        self.phi_out = torch.nn.ModuleList([mk(2 * d + 3, d) for _ in range(kbar)])
        self.phi_in = torch.nn.ModuleList([mk(2 * d + 3, d) for _ in range(kbar)])
        self.psi = torch.nn.ModuleList([mk(3 * d + 1, d) for _ in range(kbar)])
        self.dec = torch.nn.ModuleList([mk(d, 1) for _ in range(kbar)])
        for m in self.modules():
            if isinstance(m, torch.nn.Linear):
                torch.nn.init.xavier_uniform_(m.weight)
                torch.nn.init.zeros_(m.bias)

    def forward(self, xy, c, src, dst, n):
        H = xy.new_zeros(n, self.d)
        dv = xy[dst] - xy[src]
        e = torch.cat([dv, dv.norm(dim=1, keepdim=True)], dim=1)
        outs = []
        for k in range(self.kbar):
            m_out = self.phi_out[k](torch.cat([H[src], H[dst], e], 1))
            m_in = self.phi_in[k](torch.cat([H[dst], H[src], e], 1))
            po = H.new_zeros(n, self.d).index_add_(0, src, m_out)
            pi = H.new_zeros(n, self.d).index_add_(0, dst, m_in)
            H = H + self.alpha * self.psi[k](torch.cat([H, c[:, None], po, pi], 1))
            outs.append(self.dec[k](H)[:, 0])
        return outs

    def flat(self) -> np.ndarray:
        parts = []
        for k in range(self.kbar):
            for m in (self.phi_out[k], self.phi_in[k], self.psi[k], self.dec[k]):
                for lin in (m[0], m[2]):
                    parts += [lin.weight.detach().cpu().numpy().ravel(), lin.bias.detach().cpu().numpy().ravel()]
        return np.concatenate(parts).astype(np.float32)


def make_batch(graphs, picks, rng, dev):
    xs, cs, srcs, dsts, ai, aj, av, interior, gid = [], [], [], [], [], [], [], [], []
    off = 0
    ioff = 0
    for b, g in enumerate(picks):
        G = graphs[g]
        row = G["c"][rng.integers(G["c"].shape[0])]
        c = np.zeros(G["n"], np.float32)
        c[:G["k"]] = row
        xs.append(G["xy"]); cs.append(c)
        srcs.append(G["src"] + off); dsts.append(G["dst"] + off)
        ai.append(G["ai"] + ioff); aj.append(G["aj"] + off); av.append(G["av"])
        interior.append(np.arange(G["k"]) + off)
        gid.append(np.full(G["k"], b))
        off += G["n"]
        ioff += G["k"]
    T = lambda a, dt=torch.float32: torch.as_tensor(np.concatenate(a), dtype=dt, device=dev)
    return dict(xy=T(xs), c=T(cs), src=T(srcs, torch.long), dst=T(dsts, torch.long), ai=T(ai, torch.long),
                aj=T(aj, torch.long), av=T(av), interior=T(interior, torch.long), gid=T(gid, torch.long),
                n=off, ni=ioff, nb=len(picks))


def loss_fn(outs, B):
    """sum over blocks of the mean over graphs of L_res (Eqs. 11, 23)."""
    cint = B["c"][B["interior"]]
    counts = torch.bincount(B["gid"], minlength=B["nb"]).float()
    total = 0.0
    for r_hat in outs:
        Au = torch.zeros(B["ni"], device=cint.device).index_add_(0, B["ai"], B["av"] * r_hat[B["aj"]])
        res2 = (Au - cint) ** 2
        per = torch.zeros(B["nb"], device=cint.device).index_add_(0, B["gid"], res2) / counts
        total = total + per.mean()
    return total


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--minutes", type=float, default=15.0)
    ap.add_argument("--meshes", type=int, default=24)
    ap.add_argument("--nodes", type=int, default=7000)
    ap.add_argument("--batch", type=int, default=48)
    ap.add_argument("--out", default=os.path.join(HERE, "dss_k30_d10.npy"))
    ap.add_argument("--log", default=None)
    a = ap.parse_args()
    dev = "cuda"
    torch.manual_seed(0)
    ctx = ddg.ddg_create(0)
    t0 = time.time()
    graphs = []
    for s in range(a.meshes):
        seed = 1000 + s
        n = a.nodes if s % 3 else 3 * a.nodes
        m = synth.star_mesh(n, seed=seed)
        K = max(1, int(round((m.n - m.n_boundary_ring) / 1000.0)))
        graphs += harvest(ctx, m, synth.poly_coeffs(seed), K, 2, dev=dev)
    nval = max(4, len(graphs) // 10)
    val, train = graphs[:nval], graphs[nval:]
    log = open(a.log, "w") if a.log else sys.stdout
    print(f"harvested {len(graphs)} graphs, {sum(g['c'].shape[0] for g in graphs)} samples in "
          f"{time.time() - t0:.1f}s", file=log, flush=True)
    model = DSS(KBAR, D, ALPHA).to(dev)
    opt = torch.optim.Adam(model.parameters(), lr=1e-2)
    sched = torch.optim.lr_scheduler.ReduceLROnPlateau(opt, factor=0.1, patience=8)
    rng = np.random.default_rng(0)
    vb = make_batch(val, list(range(len(val))), np.random.default_rng(1), dev)
    step, t_start = 0, time.time()
    best = (math.inf, model.flat())
    while time.time() - t_start < 60.0 * a.minutes:
        B = make_batch(train, rng.integers(len(train), size=a.batch), rng, dev)
        outs = model(B["xy"], B["c"], B["src"], B["dst"], B["n"])
        loss = loss_fn(outs, B)
        opt.zero_grad()
        loss.backward()
        torch.nn.utils.clip_grad_norm_(model.parameters(), 1e-2)
        opt.step()
        step += 1
        if step % 100 == 0:
            with torch.no_grad():
                vo = model(vb["xy"], vb["c"], vb["src"], vb["dst"], vb["n"])
                vl = float(loss_fn(vo[-1:], vb))
            sched.step(vl)
            if vl < best[0]:
                best = (vl, model.flat())
            print(f"step {step} train {float(loss):.4e} val_last {vl:.4e} lr {opt.param_groups[0]['lr']:.1e} "
                  f"t {time.time() - t_start:.0f}s", file=log, flush=True)
    np.save(a.out, best[1])
    print(f"saved {a.out} (val {best[0]:.4e}, {step} steps)", file=log, flush=True)
    ddg.ddg_destroy(ctx)


if __name__ == "__main__":
    main()
