"""The allocation-free SpMV-and-dot entry point agrees with ddg_apply_A.

Some callers cannot allocate device memory (a capture they do not own, an
allocator closed after start-up, a loop that cannot wait on cudaMalloc).
ddg_apply_A_dot_noalloc serves them with scratch compiled into the library.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import synth
from helpers import gpu_setup

pytestmark = pytest.mark.gpu


def test_noalloc_spmv_dot_matches_apply_A_twice():
    import torch
    import paper_2402_08296_b300 as ddg
    from oracle import fem

    w = synth.workload("star20000", 7)
    P = fem.assemble(w.mesh.xy, w.mesh.tri, coeffs=w.coeffs)
    ctx = ddg.ddg_create(0)
    p = gpu_setup(ddg, ctx, w.mesh, w.coeffs)
    try:
        for call in range(2):
            x = torch.as_tensor(synth.residual_vector(P.n_free, 100 + call)).cuda()
            y_ref = torch.zeros_like(x)
            ddg.ddg_apply_A(p, x, y_ref)
            y = torch.full_like(x, float("nan"))
            xy = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            ddg.ddg_apply_A_dot_noalloc(p, x, y, xy)
            torch.cuda.synchronize()
            ref = y_ref.cpu().numpy()
            got = y.cpu().numpy()
            assert np.max(np.abs(got - ref)) <= 1e-13 * np.abs(ref).max()
            # and against the oracle's own matrix: y = A_ff x and x.y
            xh = x.cpu().numpy()
            y_or = P.A @ xh
            assert np.max(np.abs(got - y_or)) <= 1e-12 * np.abs(y_or).max()
            dot_ref = float(np.dot(xh, y_or))
            assert abs(float(xy.item()) - dot_ref) <= 1e-12 * abs(dot_ref)
    finally:
        ddg.ddg_problem_destroy(p)
        ddg.ddg_destroy(ctx)
