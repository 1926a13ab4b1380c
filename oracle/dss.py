"""Deep Statistical Solver forward pass, FP64, literal per-edge form (Section III-B, Eqs. 18-22).

Test infrastructure (see the package docstring).

One inference on a local graph G_i = (Omega_{h,i}, c) (Eq. 17):
* H^0 = 0, one d-vector per node (Initialization).
* For k = 1..kbar, block M^k (Eq. 21):
    phi_out_j = sum over edges j -> l of Phi_out^k(h_j, h_l, d_jl, |d_jl|)      (Eq. 18)
    phi_in_j  = sum over edges l -> j of Phi_in^k(h_j, h_l, d_lj, |d_lj|)       (Eq. 19)
    h_j      += alpha * Psi^k(h_j, c_j, phi_out_j, phi_in_j)                    (Eq. 20)
  for every node, halo included.
* Output r_hat = D^kbar(H^kbar) on the unknowns (Eq. 22; the other decoders
  only enter the training loss, Eq. 23).

Readings: every MLP is Linear -> ReLU -> Linear with hidden width d
(Section IV-B), which reproduces the weight counts of Table 2 exactly;
d_jl = (x_l - x_j) / h_bar, so d_lj = -d_jl; c is zero on halo nodes.

Weight layout per block, row-major W[out][in]:
Phi_out W1[d][2d+3] b1[d] W2[d][d] b2[d]; Phi_in the same; Psi W1[d][3d+1]
b1[d] W2[d][d] b2[d]; D W1[d][d] b1[d] W2[1][d] b2[1].
Input orders: Phi [h_j, h_l, d_x, d_y, |d|]; Psi [h_j, c_j, phi_out_j, phi_in_j].
"""
from __future__ import annotations

import numpy as np


def block_shapes(d: int):
    """(name, shape) of every tensor of one block, in storage order."""
    s = []
    for mlp_name in ("phi_out", "phi_in"):
        s += [(mlp_name + ".W1", (d, 2 * d + 3)), (mlp_name + ".b1", (d,)),
              (mlp_name + ".W2", (d, d)), (mlp_name + ".b2", (d,))]
    s += [("psi.W1", (d, 3 * d + 1)), ("psi.b1", (d,)), ("psi.W2", (d, d)), ("psi.b2", (d,))]
    s += [("dec.W1", (d, d)), ("dec.b1", (d,)), ("dec.W2", (1, d)), ("dec.b2", (1,))]
    return s


def n_weights(kbar: int, d: int) -> int:
    return kbar * sum(int(np.prod(shape)) for _, shape in block_shapes(d))


def unpack(w: np.ndarray, kbar: int, d: int) -> list:
    """Split the flat weight vector into per-block dictionaries of FP64 arrays."""
    w = np.asarray(w, dtype=np.float64)
    assert w.shape[0] == n_weights(kbar, d)
    blocks, pos = [], 0
    for _ in range(kbar):
        blk = {}
        for name, shape in block_shapes(d):
            cnt = int(np.prod(shape))
            blk[name] = w[pos:pos + cnt].reshape(shape)
            pos += cnt
        blocks.append(blk)
    return blocks


def mlp(x: np.ndarray, W1, b1, W2, b2) -> np.ndarray:
    """Linear -> ReLU -> Linear on the rows of x (Section IV-B)."""
    return np.maximum(x @ W1.T + b1, 0.0) @ W2.T + b2


def forward(xy: np.ndarray, n_int: int, src: np.ndarray, dst: np.ndarray, c: np.ndarray,
            w: np.ndarray, kbar: int, d: int, alpha: float, hbar: float,
            return_all: bool = False):
    """r_hat^kbar on the n_int unknowns of one local graph (node coordinates ``xy``, edges src -> dst).

    ``c`` holds the normalised local residual on the unknowns.  With
    ``return_all`` the decoded states after every block are returned too.
    """
    blocks = unpack(w, kbar, d)
    n = xy.shape[0]
    cc = np.zeros(n)
    cc[:n_int] = c
    H = np.zeros((n, d))
    dvec = (xy[dst] - xy[src]) / hbar          # x_dst - x_src
    dnorm = np.sqrt(dvec[:, 0] ** 2 + dvec[:, 1] ** 2)[:, None]
    decoded = []
    for blk in blocks:
        # Eq. 18: edge j -> l seen from its source j = src, l = dst; d_jl = x_l - x_j
        x_out = np.concatenate([H[src], H[dst], dvec, dnorm], axis=1)
        m_out = mlp(x_out, blk["phi_out.W1"], blk["phi_out.b1"], blk["phi_out.W2"], blk["phi_out.b2"])
        phi_out = np.zeros((n, d))
        np.add.at(phi_out, src, m_out)
        # Eq. 19: edge l -> j seen from its target j = dst, l = src; d_lj = x_j - x_l
        x_in = np.concatenate([H[dst], H[src], dvec, dnorm], axis=1)
        m_in = mlp(x_in, blk["phi_in.W1"], blk["phi_in.b1"], blk["phi_in.W2"], blk["phi_in.b2"])
        phi_in = np.zeros((n, d))
        np.add.at(phi_in, dst, m_in)
        # Eq. 20
        x_psi = np.concatenate([H, cc[:, None], phi_out, phi_in], axis=1)
        H = H + alpha * mlp(x_psi, blk["psi.W1"], blk["psi.b1"], blk["psi.W2"], blk["psi.b2"])
        if return_all:
            decoded.append(mlp(H, blk["dec.W1"], blk["dec.b1"], blk["dec.W2"], blk["dec.b2"])[:n_int, 0])
    last = blocks[-1]
    r_hat = mlp(H, last["dec.W1"], last["dec.b1"], last["dec.W2"], last["dec.b2"])[:n_int, 0]
    if return_all:
        return r_hat, decoded
    return r_hat


def forward_factorised(xy, n_int, src, dst, c, w, kbar, d, alpha, hbar):
    """The same map with the edge MLPs split algebraically (the form the CUDA path evaluates).

    W1 [h_j, h_l, e] = Wa h_j + Wb h_l + We e, so the two d x d products are
    taken once per node, and sum_l (W2 relu(z_jl) + b2) = W2 sum_l relu(z_jl) + deg_j b2.
    Equal to ``forward`` in exact arithmetic.
    """
    blocks = unpack(w, kbar, d)
    n = xy.shape[0]
    cc = np.zeros(n)
    cc[:n_int] = c
    H = np.zeros((n, d))
    e = (xy[dst] - xy[src]) / hbar
    e = np.concatenate([e, np.sqrt(e[:, 0] ** 2 + e[:, 1] ** 2)[:, None]], axis=1)
    deg_out = np.bincount(src, minlength=n).astype(np.float64)[:, None]
    deg_in = np.bincount(dst, minlength=n).astype(np.float64)[:, None]
    for blk in blocks:
        sums = []
        for name, own, other, deg in (("phi_out", src, dst, deg_out), ("phi_in", dst, src, deg_in)):
            W1 = blk[name + ".W1"]
            Wa, Wb, We = W1[:, :d], W1[:, d:2 * d], W1[:, 2 * d:]
            Pa = H @ Wa.T + blk[name + ".b1"]
            Pb = H @ Wb.T
            z = np.maximum(Pa[own] + Pb[other] + e @ We.T, 0.0)
            S = np.zeros((n, d))
            np.add.at(S, own, z)
            sums.append(S @ blk[name + ".W2"].T + deg * blk[name + ".b2"])
        x_psi = np.concatenate([H, cc[:, None], sums[0], sums[1]], axis=1)
        H = H + alpha * mlp(x_psi, blk["psi.W1"], blk["psi.b1"], blk["psi.W2"], blk["psi.b2"])
    last = blocks[-1]
    return mlp(H, last["dec.W1"], last["dec.b1"], last["dec.W2"], last["dec.b2"])[:n_int, 0]


def residual_loss(A_loc, u: np.ndarray, b: np.ndarray) -> float:
    """L_res(u, G) = (1/N) sum_i (-b_i + sum_j a_ij u_j)^2 (Eq. 11)."""
    r = A_loc @ u - b
    return float(np.mean(r * r))
