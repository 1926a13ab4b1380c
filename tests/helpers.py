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
