"""Two-level additive Schwarz preconditioners and the Krylov drivers (Sections II-A, III-A; Algorithm 1).

Test infrastructure (see the package docstring).  FP64 throughout.

* DDM-LU: M^-1 r = R_0^T (R_0 A R_0^T)^-1 R_0 r + sum_i R_i^T (R_i A R_i^T)^-1 R_i r (Eq. 7),
  local matrices factorised by sparse LU (scipy's SuperLU), the coarse matrix by Cholesky.
* DDM-GNN (Section III-A): coarse term r_c (Eq. 13); each local solve is one
  DSS inference on G_i = (Omega_{h,i}, R_i r / |R_i r|) (Eqs. 14, 17); the
  gluing is z = r_c + sum_i R_i^T |R_i r| r~_i (Eq. 16).
* PCG: Algorithm 1.  FCG(m): flexible CG (Notay, SIAM J. Sci. Comput. 22, 2000),
  each new direction A-orthogonalised against the last m ones; needed because
  the DDM-GNN preconditioner is not linear.

Readings: the stopping test is |r_k| / |b| < tol with x_0 = 0 (the paper
calls the tolerance a relative residual); a subdomain whose restricted
residual is zero contributes no correction; the gluing uses the boolean
extension R_i^T, or the partition-of-unity weights when ``pou`` is set.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from . import dss, fem, partition


class TwoLevelASM:
    def __init__(self, problem: fem.Problem, dec: partition.Decomposition, coarse: bool = True):
        self.problem = problem
        self.dec = dec
        self.coarse = coarse
        A = problem.A.tocsc()
        self.local_lu = [spla.splu(A[S][:, S].tocsc()) for S in dec.sets]
        self.A0_chol = sla.cho_factor(dec.A0, lower=True) if coarse else None

    def coarse_term(self, r: np.ndarray) -> np.ndarray:
        """r_c = R_0^T (R_0 A R_0^T)^-1 R_0 r (Eq. 13)."""
        if not self.coarse:
            return np.zeros_like(r)
        y = self.dec.Z.T @ r
        return self.dec.Z @ sla.cho_solve(self.A0_chol, y)

    def local_lu_solve(self, i: int, r: np.ndarray) -> np.ndarray:
        """(R_i A R_i^T)^-1 R_i r."""
        return self.local_lu[i].solve(r[self.dec.sets[i]])

    def apply_lu(self, r: np.ndarray) -> np.ndarray:
        """DDM-LU, Eq. 7 (Eq. 6 without the coarse term)."""
        z = self.coarse_term(r)
        for i, S in enumerate(self.dec.sets):
            z[S] += self.local_lu_solve(i, r)
        return z


class DDMGNN:
    """DDM-GNN preconditioner (Section III-A) with an FP64 DSS model."""

    def __init__(self, asm: TwoLevelASM, w: np.ndarray, kbar: int, d: int, alpha: float,
                 pou: bool = False, local_solver=None):
        self.asm = asm
        self.w, self.kbar, self.d, self.alpha = w, kbar, d, alpha
        self.pou = pou
        p = asm.problem
        adj = partition.mesh_adjacency(p.n, p.tri)
        self.graphs = [partition.local_graph(p, S, adj) for S in asm.dec.sets]
        self.hbar = partition.mean_edge_length(p.xy, p.tri)
        # local_solver(i, c) may replace the DSS inference (used to check the gluing)
        self.local_solver = local_solver

    def local_correction(self, i: int, r: np.ndarray):
        """(|R_i r|, r~_i) for subdomain i (Eqs. 14-15)."""
        S = self.asm.dec.sets[i]
        ri = r[S]
        s = float(np.sqrt(np.sum(ri * ri)))
        if s == 0.0:
            return 0.0, np.zeros(S.shape[0])
        c = ri / s
        if self.local_solver is not None:
            return s, self.local_solver(i, c)
        g = self.graphs[i]
        return s, dss.forward(g.xy, g.n_int, g.src, g.dst, c, self.w, self.kbar, self.d, self.alpha, self.hbar)

    def apply(self, r: np.ndarray) -> np.ndarray:
        z = self.asm.coarse_term(r)                 # step 1, Eq. 13
        mult = self.asm.dec.mult
        for i, S in enumerate(self.asm.dec.sets):   # step 2, one subdomain at a time
            s, rt = self.local_correction(i, r)
            if self.pou:
                z[S] += s * rt / mult[S]            # step 3 with partition-of-unity weights
            else:
                z[S] += s * rt                      # step 3, Eq. 16
        return z


def pcg(A, b: np.ndarray, M, tol: float, max_iter: int):
    """Algorithm 1 with u_0 = 0; returns (u, iterations, history of |r|/|b|).
    b = 0 returns u = 0 after zero iterations (reading C-21: |r|/|b| is undefined there)."""
    u = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return u, 0, []
    z = M(r)
    p = z.copy()
    rho = r @ z
    hist = []
    for it in range(1, max_iter + 1):
        q = A @ p
        alpha = rho / (p @ q)
        u = u + alpha * p
        r = r - alpha * q
        rel = np.linalg.norm(r) / bn
        hist.append(rel)
        if rel < tol:
            return u, it, hist
        z = M(r)
        rho_new = r @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
    return u, max_iter, hist


def fcg(A, b: np.ndarray, M, tol: float, max_iter: int, m: int):
    """Flexible CG with truncation m and u_0 = 0; returns (u, iterations, history of |r|/|b|).
    b = 0 returns u = 0 after zero iterations (reading C-21)."""
    u = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return u, 0, []
    P, Q, PQ = [], [], []
    hist = []
    for it in range(1, max_iter + 1):
        z = M(r)
        p = z.copy()
        for pj, qj, pqj in zip(P, Q, PQ):
            p = p - ((z @ qj) / pqj) * pj
        q = A @ p
        pq = p @ q
        alpha = (p @ r) / pq
        u = u + alpha * p
        r = r - alpha * q
        P.append(p)
        Q.append(q)
        PQ.append(pq)
        if len(P) > m:
            P.pop(0)
            Q.pop(0)
            PQ.pop(0)
        rel = np.linalg.norm(r) / bn
        hist.append(rel)
        if rel < tol:
            return u, it, hist
    return u, max_iter, hist


def true_relative_residual(A, b, u) -> float:
    return float(np.linalg.norm(b - A @ u) / np.linalg.norm(b))


def condition_estimate(A, solve=None, iters: int = 8) -> float:
    """Estimate of the 2-norm condition number of the SPD matrix A, for the solution check of
    reading C-19 (|x - x*| / |x*| <= kappa |b - A x| / |b|): the Gershgorin bound on the
    largest eigenvalue (max absolute row sum, never below it) over the smallest eigenvalue,
    taken as the Rayleigh quotient of `iters` steps of inverse iteration from the constant
    vector.  `solve(v)` returns A^-1 v (default: scipy's sparse LU, for small A)."""
    lam_max = float(abs(A).sum(axis=1).max())
    if solve is None:
        solve = spla.splu(A.tocsc()).solve
    v = np.ones(A.shape[0])
    for _ in range(iters):
        v = solve(v)
        v /= np.linalg.norm(v)
    lam_min = float(v @ (A @ v))
    return lam_max / lam_min
