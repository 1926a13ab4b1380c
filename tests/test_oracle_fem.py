"""Pins of the oracle's P1 assembly (Section II, Eqs. 1-2) against closed forms and exact integration."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla
import sympy

import synth
from oracle import fem


def solve(P):
    return P.full_solution(spla.spsolve(P.A.tocsc(), P.b))


@pytest.mark.parametrize("seed", [0, 1])
def test_affine_solution_reproduced(seed):
    """f = 0 and affine g: the P1 solution is the affine function itself, at every node."""
    m = synth.square_mesh(21, seed=seed)
    r = np.zeros(9)
    r[6], r[7], r[8] = 1.5, -2.0, 0.25          # g = 1.5 x - 2 y + 0.25
    P = fem.assemble(m.xy, m.tri, coeffs=r)
    u = solve(P)
    exact = 1.5 * m.xy[:, 0] - 2.0 * m.xy[:, 1] + 0.25
    assert np.max(np.abs(u - exact)) < 1e-13


def test_affine_solution_star_mesh():
    m = synth.star_mesh(3000, seed=2)
    exact = 0.5 - m.xy[:, 0] + 3.0 * m.xy[:, 1]
    P = fem.assemble(m.xy, m.tri, f_nodal=np.zeros(m.n), g_nodal=exact)
    assert np.max(np.abs(solve(P) - exact)) < 1e-12


def test_quadratic_nodally_exact_on_right_triangle_grid():
    """u = x^2 + y^2 + xy, f = -4: on an unjittered grid with one diagonal the P1
    matrix is the 5-point stencil, which is exact for quadratics."""
    m = synth.square_mesh(17, jitter=0.0, diag="fixed")
    r = np.zeros(9)
    r[2] = -4.0                                  # f = r3
    r[3], r[4], r[5] = 1.0, 1.0, 1.0             # g = x^2 + y^2 + xy
    P = fem.assemble(m.xy, m.tri, coeffs=r)
    x, y = m.xy[:, 0], m.xy[:, 1]
    assert np.max(np.abs(solve(P) - (x * x + y * y + x * y))) < 1e-12
    # the hypotenuse couplings are exact zeros that stay in the pattern
    A = P.A_full
    assert A.nnz == fem.csr_pattern(m.n, m.tri)[1].shape[0]
    assert np.sum(A.data == 0.0) > 0


def test_smooth_solution_converges_at_second_order():
    """u = sin(pi x) sinh(pi y) / sinh(pi) is harmonic; the max nodal error falls like h^2."""
    for jitter, sizes, lo, hi in ((0.0, (17, 33, 65), 3.9, 4.1), (0.3, (33, 65, 129), 3.0, 5.5)):
        errs = []
        for nx in sizes:
            m = synth.square_mesh(nx, seed=3, jitter=jitter)
            x, y = m.xy[:, 0], m.xy[:, 1]
            u = np.sin(np.pi * x) * np.sinh(np.pi * y) / np.sinh(np.pi)
            P = fem.assemble(m.xy, m.tri, f_nodal=np.zeros(m.n), g_nodal=u)
            errs.append(np.max(np.abs(solve(P) - u)))
        ratios = [errs[0] / errs[1], errs[1] / errs[2]]
        assert all(lo < q < hi for q in ratios), (jitter, errs, ratios)


def test_stiffness_row_sums_vanish_and_free_block_is_spd():
    m = synth.square_mesh(25, seed=4)
    P = fem.assemble(m.xy, m.tri, coeffs=synth.poly_coeffs(4))
    rows = np.asarray(P.A_full.sum(axis=1)).ravel()
    assert np.max(np.abs(rows)) < 1e-13 * np.max(np.abs(P.A_full.data))
    A = P.A
    assert (A != A.T).nnz == 0                     # bitwise symmetric
    sla.cholesky(A.toarray())                      # SPD


def test_load_sums_to_integral_of_f():
    """sum_i b_i = int_Omega f; on the unit square int (r1 (x-1)^2 + r2 y^2 + r3) = r1/3 + r2/3 + r3."""
    m = synth.square_mesh(31, seed=5)
    r = synth.poly_coeffs(5)
    P = fem.assemble(m.xy, m.tri, coeffs=r)
    assert abs(P.b_full.sum() - (r[0] / 3 + r[1] / 3 + r[2])) < 1e-12 * (abs(r).sum())


def test_element_load_matches_exact_symbolic_integral():
    """int_T f lambda_i for the paper's quadratic f (Eq. 24), integrated symbolically."""
    X, Y, s, t = sympy.symbols("X Y s t")
    r = [sympy.Rational(k, 7) for k in (3, -5, 2, 1, 1, 1, 1, 1, 1)]
    f = r[0] * (X - 1) ** 2 + r[1] * Y ** 2 + r[2]
    verts = [(sympy.Rational(1, 10), sympy.Rational(2, 10)), (sympy.Rational(9, 10), sympy.Rational(3, 10)),
             (sympy.Rational(4, 10), sympy.Rational(8, 10))]
    (x0, y0), (x1, y1), (x2, y2) = verts
    xs = x0 + s * (x1 - x0) + t * (x2 - x0)
    ys = y0 + s * (y1 - y0) + t * (y2 - y0)
    jac = abs((x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0))
    lam = [1 - s - t, s, t]
    fs = f.subs({X: xs, Y: ys})
    exact = [float(sympy.integrate(sympy.integrate(fs * lam[i] * jac, (t, 0, 1 - s)), (s, 0, 1))) for i in range(3)]
    xy = np.array([[float(a), float(b)] for a, b in verts])
    tri = np.array([[0, 1, 2]])
    rr = np.array([float(v) for v in r])
    got = fem.element_load_quadratic(xy, tri, lambda x, y: fem.paper_f(rr, x, y))[0]
    assert np.allclose(got, exact, rtol=1e-14, atol=1e-15)


def test_element_stiffness_matches_gradient_products():
    """K_T[i][j] = |T| grad(lambda_i) . grad(lambda_j), gradients from solving the affine interpolation."""
    xy = np.array([[0.1, 0.2], [0.9, 0.3], [0.4, 0.8]])
    tri = np.array([[0, 1, 2]])
    V = np.column_stack([np.ones(3), xy])
    G = np.linalg.inv(V)[1:, :]                  # column i = grad(lambda_i)
    area = 0.5 * abs(np.linalg.det(np.column_stack([xy[1] - xy[0], xy[2] - xy[0]])))
    expected = area * G.T @ G
    assert np.allclose(fem.element_stiffness(xy, tri)[0], expected, rtol=1e-13, atol=1e-14)


def test_dirichlet_lifting_matches_full_system():
    """Solving the free block with lifting equals solving the full system with g imposed by row replacement."""
    m = synth.square_mesh(9, seed=6)
    r = synth.poly_coeffs(6)
    P = fem.assemble(m.xy, m.tri, coeffs=r)
    A = P.A_full.toarray()
    b = P.b_full.copy()
    D = np.nonzero(P.dirichlet)[0]
    A[D, :] = 0.0
    A[D, D] = 1.0
    b[D] = P.g[D]
    u_full = np.linalg.solve(A, b)
    assert np.max(np.abs(u_full - solve(P))) < 1e-10


def test_element_load_nodal_matches_symbolic_integral_of_the_interpolant():
    """int_T f_h lambda_i with f_h the P1 interpolant of arbitrary nodal values, integrated
    symbolically; a wrong mass weight (e.g. f_i + f_j + f_l in place of 2 f_i + f_j + f_l) fails."""
    s, t = sympy.symbols("s t")
    verts = [(sympy.Rational(1, 10), sympy.Rational(2, 10)), (sympy.Rational(9, 10), sympy.Rational(3, 10)),
             (sympy.Rational(4, 10), sympy.Rational(8, 10))]
    fv = [sympy.Rational(3, 2), sympy.Rational(-7, 3), sympy.Rational(5, 4)]
    (x0, y0), (x1, y1), (x2, y2) = verts
    jac = abs((x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0))
    lam = [1 - s - t, s, t]
    fh = sum(fv[k] * lam[k] for k in range(3))
    exact = [float(sympy.integrate(sympy.integrate(fh * lam[i] * jac, (t, 0, 1 - s)), (s, 0, 1))) for i in range(3)]
    xy = np.array([[float(a), float(b)] for a, b in verts])
    got = fem.element_load_nodal(xy, np.array([[0, 1, 2]]), np.array([float(v) for v in fv]))[0]
    assert np.allclose(got, exact, rtol=1e-14, atol=1e-15)


def test_nodal_load_of_affine_f_is_exact_and_sums_to_the_integral():
    """For affine f the P1 interpolant is f itself, so the consistent-mass load equals the exact
    element integral (the quadratic rule, itself pinned symbolically above), and its total is
    sum_T |T| (f_a + f_b + f_c) / 3 (the exact integral of an affine function over a triangle)."""
    m = synth.star_mesh(2000, seed=8)
    fun = lambda x, y: 2.5 - 1.25 * x + 0.75 * y
    f = fun(m.xy[:, 0], m.xy[:, 1])
    got = fem.element_load_nodal(m.xy, m.tri, f)
    ref = fem.element_load_quadratic(m.xy, m.tri, fun)
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))
    _, _, area = fem.triangle_geometry(m.xy, m.tri)
    total = float(np.sum(area * f[m.tri].sum(axis=1) / 3.0))
    assert abs(got.sum() - total) <= 1e-13 * abs(total)


def test_quadratic_solution_with_nodal_forcing():
    """The nodal-f path with f != 0: u = x^2 + y^2 + xy has -Lap(u) = -4, a constant, whose
    consistent-mass load is exact; on the right-triangle grid the P1 solution is nodally exact."""
    m = synth.square_mesh(17, jitter=0.0, diag="fixed")
    x, y = m.xy[:, 0], m.xy[:, 1]
    u = x * x + y * y + x * y
    P = fem.assemble(m.xy, m.tri, f_nodal=np.full(m.n, -4.0), g_nodal=u)
    assert np.max(np.abs(solve(P) - u)) < 1e-12
