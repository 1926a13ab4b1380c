"""Shared set-up for the GPU parity tests: the same seeded inputs built on the CUDA path and in the oracle."""
import numpy as np

import synth
from oracle import fem, partition as pt


def oracle_setup(mesh, coeffs, K, delta):
    P = fem.assemble(mesh.xy, mesh.tri, coeffs=coeffs)
    D = pt.decompose(P, K, delta)
    return P, D


def gpu_setup(ddg, ctx, mesh, coeffs, K=None, delta=None):
    p = ddg.ddg_mesh_upload(ctx, mesh.xy, mesh.tri)
    ddg.ddg_assemble_poly(p, coeffs)
    if K is not None:
        ddg.ddg_partition(p, K, delta)
    return p


def csr_from_gpu(ddg, p):
    import scipy.sparse as sp
    rowptr, col, val, b = ddg.ddg_matrix_download(p)
    n = rowptr.shape[0] - 1
    return sp.csr_matrix((val, col, rowptr), shape=(n, n)), b


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def max_rel(a, b):
    """max_j |a_j - b_j| / max_j |b_j|: the element-wise error against the reference's scale."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def assert_close(got, ref, tol, what=None):
    """Both the norm-wise and the element-wise relative error within `tol`: a single wrong
    entry of a large vector (a halo, chunk-border or masking slip) fails the element-wise bound
    even where it hides in the norm."""
    n, e = rel(got, ref), max_rel(got, ref)
    assert n < tol and e <= tol, (what, n, e)
