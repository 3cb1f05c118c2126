"""Pins of the oracle's solves (no GPU): closed-form fixed points, the
literal Algorithm 1 against the converged answer, second-order accuracy and
the degenerate cases."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2311_16935_gb300 import inputs


def _rel(a, b, valid):
    a = np.asarray(a)[valid]
    b = np.asarray(b)[valid]
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _quadratic(shape, spacing, seed):
    p, g = inputs.quadratic_field(shape, spacing, seed=seed)
    return p.numpy(), g.numpy()


@pytest.mark.parametrize("spacing", [(0.1, 0.13), (1.0, 1.0)])
def test_quadratic_is_exact_fixed_point_2d(spacing):
    """For a quadratic pressure with its exact gradient the trapezoidal face
    average is exact, so every path step of Eq. PressureIntegrator1 holds
    exactly and the true pressure is the fixed point of Algorithm 1 (up to a
    constant) for any mask and spacing."""
    shape = (13, 17)
    p, g = _quadratic(shape, spacing, seed=1)
    rng = np.random.default_rng(2)
    valid = rng.random(shape) > 0.15
    grid = oracle.Grid(valid, spacing)
    want = oracle.gauge(grid, p)
    P_lu = oracle.solve_direct(grid, g)
    assert _rel(P_lu, want, valid) < 1e-12
    P_cg, it, res = oracle.solve_cg(grid, g, tol=1e-14)
    assert _rel(P_cg, want, valid) < 1e-11
    P_lit, n, er, ep = oracle.solve_literal(grid, g, tol=1e-12)
    assert _rel(P_lit, want, valid) < 1e-9
    assert oracle.residual(grid, g, p) < 1e-12


@pytest.mark.parametrize("spacing", [(1.0, 1.0, 1.0), (1.0, 1.3, 0.7)])
def test_quadratic_is_exact_fixed_point_3d(spacing):
    shape = (6, 7, 8)
    p, g = _quadratic(shape, spacing, seed=3)
    z, y, x = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    valid = (x - 4) ** 2 + (y - 3) ** 2 + (z - 3) ** 2 >= 2.5 ** 2
    grid = oracle.Grid(valid, spacing)
    want = oracle.gauge(grid, p)
    assert _rel(oracle.solve_direct(grid, g), want, valid) < 1e-12
    P_cg, it, res = oracle.solve_cg(grid, g, tol=1e-14)
    assert _rel(P_cg, want, valid) < 1e-11


def test_literal_limit_equals_definition():
    """Algorithm 1 iterated to convergence (exact inner solves) reaches the
    same answer as the direct solve of (I - T) P = S, on a noisy
    non-integrable field with a mask; eps_R falls below the threshold."""
    rng = np.random.default_rng(4)
    shape = (10, 12)
    valid = rng.random(shape) > 0.2
    grid = oracle.Grid(valid, (0.1, 0.13))
    f = rng.normal(size=(2,) + shape)
    P_def = oracle.solve_direct(grid, f)
    P_lit, n, er, ep = oracle.solve_literal(grid, f, tol=1e-12)
    assert er[-1] <= 1e-12
    assert er[-1] < er[0]
    assert _rel(P_lit, P_def, valid) < 1e-9
    # the residual of the definition's answer, measured by the oracle's
    # independent per-cell evaluation
    assert oracle.residual(grid, f, P_def) < 1e-12


def test_cg_matches_direct_3d_noisy():
    rng = np.random.default_rng(5)
    shape = (6, 7, 9)
    valid = rng.random(shape) > 0.2
    grid = oracle.Grid(valid, (1.0, 1.0, 1.0))
    f = rng.normal(size=(3,) + shape)
    P_def = oracle.solve_direct(grid, f)
    P_cg, it, res = oracle.solve_cg(grid, f, tol=1e-14)
    assert res <= 1e-13
    assert _rel(P_cg, P_def, valid) < 1e-11


def test_outer_map_commutes_with_constant_shift():
    """One outer iteration P -> M^{-1}(W^n P + S) maps P + c to F(P) + c
    (rows of W^{n+1}_off + W^n sum to one), so a resumed solve from a
    gauge-shifted pressure follows the same path."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    rng = np.random.default_rng(6)
    shape = (7, 8)
    valid = np.ones(shape, bool)
    grid = oracle.Grid(valid, (1.0, 1.0))
    f = rng.normal(size=(2,) + shape)
    W1, Wn = oracle.operators(grid)
    S = oracle.source(grid, f).reshape(-1)
    M = (sp.identity(grid.n) - W1).tocsc()
    P = rng.normal(size=grid.n)
    F1 = spla.spsolve(M, Wn @ P + S)
    F2 = spla.spsolve(M, Wn @ (P + 3.7) + S)
    np.testing.assert_allclose(F2 - F1, 3.7, atol=1e-11)


def test_second_order_accuracy_taylor_vortex():
    """The face-averaged gradient is second-order accurate (Section 2.1), so
    the error of the converged answer against the analytic pressure of the
    decaying Taylor vortex (Section 3.1) falls ~4x per halving of the
    spacing."""
    errs = []
    for n in (17, 33, 65):
        L = 4.0
        h = 2 * L / (n - 1)
        x = -L + np.arange(n) * h
        X, Y = np.meshgrid(x, x)
        r2 = X * X + Y * Y
        # nondimensional Taylor vortex with H = nu = rho = 1 at t = 1:
        # P = -1/(64 pi^2) exp(-r^2/2)
        P = -1.0 / (64 * math.pi**2) * np.exp(-r2 / 2)
        dPdr_over_r = 1.0 / (64 * math.pi**2) * np.exp(-r2 / 2)
        g = np.stack([dPdr_over_r * X, dPdr_over_r * Y])
        grid = oracle.Grid(np.ones((n, n), bool), (h, h))
        Pc, it, res = oracle.solve_cg(grid, g, tol=1e-14)
        want = oracle.gauge(grid, P)
        errs.append(np.sqrt(np.mean((Pc - want) ** 2)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.2 < r1 < 4.8 and 3.2 < r2 < 4.8, errs


def test_degenerate_cases():
    """An isolated valid cell has an empty row (its pressure is just the
    component constant, 0 after the gauge); disconnected components each get
    zero mean; a grid with no valid cell returns all NaN; S = 0 gives P = 0."""
    valid = np.zeros((5, 7), bool)
    valid[0, 0] = True  # isolated
    valid[2:5, 2:4] = True  # component 1
    valid[1:4, 5:7] = True  # component 2
    grid = oracle.Grid(valid, (1.0, 1.0))
    lab, nc = oracle.labels(grid)
    assert nc == 3
    f = np.random.default_rng(0).normal(size=(2, 5, 7))
    P = oracle.solve_direct(grid, f)
    assert P[0, 0] == 0.0
    for c in range(nc):
        assert abs(P[lab == c].mean()) < 1e-14
    assert np.isnan(P[~valid]).all()
    P2, it, res = oracle.solve_cg(grid, f, tol=1e-14)
    assert _rel(P2, P, valid) < 1e-11
    empty = oracle.Grid(np.zeros((3, 3), bool), (1.0, 1.0))
    assert np.isnan(oracle.solve_direct(empty, np.zeros((2, 3, 3)))).all()
    one = oracle.Grid(np.ones((4, 4), bool), (1.0, 1.0))
    P0, it, res = oracle.solve_cg(one, np.zeros((2, 4, 4)))
    assert (P0 == 0).all() and res == 0.0
    # a 1 x N strip is a valid 2D grid
    strip = oracle.Grid(np.ones((1, 9), bool), (1.0, 1.0))
    fs = np.zeros((2, 1, 9))
    fs[0] = 2.0  # dP/dx = 2 -> P = 2x + const
    Ps = oracle.solve_direct(strip, fs)
    np.testing.assert_allclose(np.diff(Ps[0]), 2.0, atol=1e-12)


def test_noise_lowers_attainable_accuracy_but_converges():
    """Sanity of the workload generator with the oracle: the 64^2 Lamb-Oseen
    field converges to eps_R <= 1e-10 from P^0 = 0 (Algorithm 1 with exact
    inner solves), matching the direct answer."""
    prob = inputs.lamb_oseen_2d()
    f = prob.grad.numpy()
    grid = oracle.Grid(prob.mask.numpy().astype(bool), prob.spacing)
    P_def = oracle.solve_direct(grid, f)
    P_cg, it, res = oracle.solve_cg(grid, f, tol=1e-14)
    assert _rel(P_cg, P_def, grid.valid) < 1e-11


def _masked_problem(shape, spacing, seed, drop=0.15):
    rng = np.random.default_rng(seed)
    valid = rng.random(shape) > drop
    f = rng.normal(size=(len(shape),) + shape)
    return oracle.Grid(valid, spacing), f


def test_anderson_depth_zero_is_algorithm_1():
    """Depth 0 is Algorithm 1 step for step: the same eps_R history and the
    same answer as the literal oracle."""
    grid, f = _masked_problem((11, 13), (0.1, 0.13), 21)
    P_lit, n_lit, er_lit, _ = oracle.solve_literal(grid, f, tol=1e-9)
    P_aa, n_aa, er_aa = oracle.solve_outer_anderson(grid, f, 0, tol=1e-9)
    assert n_aa == n_lit
    np.testing.assert_allclose(er_aa, er_lit, rtol=1e-12, atol=0)
    assert _rel(P_aa, P_lit, grid.valid) < 1e-13


@pytest.mark.parametrize("depth", [1, 3, 8])
def test_anderson_reaches_the_fixed_point_faster(depth):
    grid, f = _masked_problem((14, 19), (0.1, 0.13), 3)
    want = oracle.solve_direct(grid, f)
    _, n_lit, _, _ = oracle.solve_literal(grid, f, tol=1e-11)
    P, n, er = oracle.solve_outer_anderson(grid, f, depth, tol=1e-11)
    assert er[-1] <= 1e-11
    assert _rel(P, want, grid.valid) < 1e-9
    assert n < n_lit / 2


def _gmres_brute_force(A, b, k):
    """The k-th GMRES iterate from x0 = 0 by definition: the minimiser of
    ||b - A x|| over the Krylov space span{b, A b, ..., A^(k-1) b}, from an
    explicit (twice orthogonalised) basis and a dense least-squares solve."""
    Q = np.zeros((b.size, k))
    v = b / np.linalg.norm(b)
    for j in range(k):
        for _ in range(2):
            v = v - Q[:, :j] @ (Q[:, :j].T @ v)
        Q[:, j] = v / np.linalg.norm(v)
        v = A @ Q[:, j]
    y = np.linalg.lstsq(A @ Q, b, rcond=None)[0]
    return Q @ y


def test_anderson_is_gmres_on_the_outer_map():
    """For the affine outer map G(x) = M^-1 W^n x + M^-1 S, Anderson mixing
    without truncation satisfies x_{k+1} = G(x_k^GMRES), with x_k^GMRES the
    k-th GMRES iterate of (I - M^-1 W^n) x = M^-1 S (Walker & Ni 2011,
    Theorem 2.2).  GMRES is computed here by its definition, independently of
    the mixing formula, so a wrong sign, index or difference in the mixing
    fails this."""
    grid, f = _masked_problem((5, 6), (0.1, 0.13), 8, drop=0.1)
    lu, Wnv, K, Sv, vidx = oracle._outer_parts(grid, f)
    n = vidx.size
    Glin = lu.solve(Wnv.toarray())
    b = lu.solve(Sv)
    A = np.eye(n) - Glin
    its = {}
    oracle.solve_outer_anderson(grid, f, depth=50, tol=0.0, max_outer=8, callback=lambda k, x: its.__setitem__(k, x))
    for k in range(1, 7):
        xg = _gmres_brute_force(A, b, k)
        want = Glin @ xg + b
        assert np.linalg.norm(its[k + 1] - want) <= 1e-8 * np.linalg.norm(want), k
