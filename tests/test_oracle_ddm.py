"""Pins of the oracle's Schwarz preconditioners and Krylov drivers (Eqs. 6-7, 13-16; Algorithm 1)."""
import numpy as np
import pytest

import synth
from oracle import ddm, fem, partition as pt


@pytest.fixture(scope="module")
def small():
    m = synth.square_mesh(17, seed=3)
    P = fem.assemble(m.xy, m.tri, coeffs=synth.poly_coeffs(3))
    return P


def test_single_subdomain_one_level_is_a_direct_solve(small):
    P = small
    D = pt.decompose(P, 1, 1)
    asm = ddm.TwoLevelASM(P, D, coarse=False)
    u, it, _ = ddm.pcg(P.A, P.b, asm.apply_lu, 1e-10, 50)
    assert it == 1
    assert ddm.true_relative_residual(P.A, P.b, u) < 1e-12


def test_single_subdomain_two_level_converges_in_two(small):
    P = small
    D = pt.decompose(P, 1, 1)
    asm = ddm.TwoLevelASM(P, D, coarse=True)
    _, it, _ = ddm.pcg(P.A, P.b, asm.apply_lu, 1e-10, 50)
    assert it <= 2


def test_ddm_lu_is_symmetric_positive_and_local_solves_exact(small):
    P = small
    D = pt.decompose(P, 4, 2)
    asm = ddm.TwoLevelASM(P, D)
    x = synth.residual_vector(P.n_free, 1)
    y = synth.residual_vector(P.n_free, 2)
    Mx, My = asm.apply_lu(x), asm.apply_lu(y)
    assert abs(y @ Mx - x @ My) < 1e-12 * abs(y @ Mx)
    assert x @ Mx > 0 and y @ My > 0
    A = P.A.tocsr()
    for i, S in enumerate(D.sets):
        v = asm.local_lu_solve(i, x)
        Ai = A[S][:, S]
        assert np.linalg.norm(Ai @ v - x[S]) < 1e-12 * np.linalg.norm(x[S])


def test_pcg_solution_matches_dense_solve(small):
    P = small
    D = pt.decompose(P, 4, 1)
    asm = ddm.TwoLevelASM(P, D)
    u, _, _ = ddm.pcg(P.A, P.b, asm.apply_lu, 1e-13, 200)
    exact = np.linalg.solve(P.A.toarray(), P.b)
    assert np.max(np.abs(u - exact)) < 1e-9 * np.max(np.abs(exact))


def test_fcg_with_fixed_spd_preconditioner_matches_pcg(small):
    P = small
    D = pt.decompose(P, 4, 1)
    asm = ddm.TwoLevelASM(P, D)
    _, it_p, hp = ddm.pcg(P.A, P.b, asm.apply_lu, 1e-10, 200)
    for m in (1, 3, 10):
        _, it_f, hf = ddm.fcg(P.A, P.b, asm.apply_lu, 1e-10, 200, m)
        assert abs(it_f - it_p) <= 1
        k = min(len(hp), len(hf))
        assert np.allclose(hp[:k - 1], hf[:k - 1], rtol=1e-4)


def test_zero_right_hand_side_has_the_zero_solution(small):
    """A is SPD, so A u = 0 only for u = 0; both drivers return it without iterating (reading C-21)."""
    P = small
    D = pt.decompose(P, 4, 1)
    asm = ddm.TwoLevelASM(P, D)
    z = np.zeros(P.n_free)
    for u, it, h in (ddm.pcg(P.A, z, asm.apply_lu, 1e-6, 50), ddm.fcg(P.A, z, asm.apply_lu, 1e-6, 50, 10)):
        assert it == 0 and h == [] and not np.any(u)


def test_unpreconditioned_cg_finite_termination():
    m = synth.square_mesh(5, seed=0)
    P = fem.assemble(m.xy, m.tri, coeffs=synth.poly_coeffs(0))
    u, it, _ = ddm.pcg(P.A, P.b, lambda r: r, 1e-12, 100)
    assert it <= P.n_free
    assert ddm.true_relative_residual(P.A, P.b, u) < 1e-11


def test_gnn_gluing_with_exact_local_solver_equals_ddm_lu(small):
    """With r~_i = (R_i A R_i^T)^-1 c_i, Eq. 16's |R_i r| r~_i is the exact local solve, so DDM-GNN = DDM-LU."""
    P = small
    D = pt.decompose(P, 4, 2)
    asm = ddm.TwoLevelASM(P, D)
    lus = asm.local_lu
    gnn = ddm.DDMGNN(asm, synth.dss_weights(2, 4, 0), 2, 4, 1e-3, local_solver=lambda i, c: lus[i].solve(c))
    r = synth.residual_vector(P.n_free, 5)
    assert np.allclose(gnn.apply(r), asm.apply_lu(r), rtol=1e-12, atol=1e-13)
    # a zero local residual gives no correction, only the coarse term
    r2 = np.zeros(P.n_free)
    assert np.allclose(gnn.apply(r2), 0.0)


def test_overlap_and_coarse_space_reduce_iterations():
    """Sanity trends of Table 1 (Section IV-C): more overlap, fewer iterations; the coarse space helps."""
    m = synth.square_mesh(33, seed=8)
    P = fem.assemble(m.xy, m.tri, coeffs=synth.poly_coeffs(8))
    its = {}
    for delta in (1, 2, 4):
        D = pt.decompose(P, 8, delta)
        its[delta] = ddm.pcg(P.A, P.b, ddm.TwoLevelASM(P, D).apply_lu, 1e-6, 500)[1]
    assert its[1] >= its[2] >= its[4]
    m = synth.square_mesh(49, seed=8)
    P = fem.assemble(m.xy, m.tri, coeffs=synth.poly_coeffs(8))
    D = pt.decompose(P, 32, 2)
    one = ddm.pcg(P.A, P.b, ddm.TwoLevelASM(P, D, coarse=False).apply_lu, 1e-6, 500)[1]
    two = ddm.pcg(P.A, P.b, ddm.TwoLevelASM(P, D).apply_lu, 1e-6, 500)[1]
    assert two < one


def test_condition_estimate_bounds_the_dense_condition_number():
    """The estimate against the dense eigenvalues of a small A_ff: at least the true condition
    number up to the inverse iteration's error (1e-6 here: the two smallest eigenvalues of
    the Dirichlet Laplacian are well apart), and within the factor the Gershgorin bound allows
    (at most 2 for these meshes, whose largest eigenvalue is at least half the largest row sum)."""
    w = synth.workload("square2k", 3)
    P = fem.assemble(w.mesh.xy, w.mesh.tri, coeffs=w.coeffs)
    ev = np.linalg.eigvalsh(P.A.toarray())
    kappa = ev[-1] / ev[0]
    est = ddm.condition_estimate(P.A)
    assert kappa * (1 - 1e-6) <= est <= 2.0 * kappa, (kappa, est)
