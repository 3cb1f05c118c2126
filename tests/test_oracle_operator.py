"""Pins of the oracle's source vector and operators (no GPU)."""
import math

import numpy as np
import pytest

import oracle


def _paper_cell(c):
    return (c - 1) % 3, 2 - (c - 1) // 3


@pytest.mark.parametrize("D", [1.0, 0.25])
def test_appendix_source_examples(D):
    """Appendix: S_1 = -D/8 [f_x(2) + f_x(1) - f_y(4) - f_y(1)] and
    S_5 = -D/8 [f_x(6) - f_x(4) + f_y(2) - f_y(8)] on the 3x3 example
    (the paper's f_y(4) enters with a minus sign because cell 4 is south of
    cell 1)."""
    rng = np.random.default_rng(0)
    f = rng.normal(size=(2, 3, 3))
    grid = oracle.Grid(np.ones((3, 3), bool), (D, D))
    S = oracle.source(grid, f)

    def fx(c):
        i, j = _paper_cell(c)
        return f[0, j, i]

    def fy(c):
        i, j = _paper_cell(c)
        return f[1, j, i]

    i1, j1 = _paper_cell(1)
    i5, j5 = _paper_cell(5)
    assert S[j1, i1] == pytest.approx(-D / 8 * (fx(2) + fx(1) - fy(4) - fy(1)), rel=1e-13)
    assert S[j5, i5] == pytest.approx(-D / 8 * (fx(6) - fx(4) + fy(2) - fy(8)), rel=1e-13)


@pytest.mark.parametrize("ndim,spacing", [(2, (0.1, 0.13)), (3, (1.0, 1.0, 1.0)), (3, (1.0, 1.3, 0.7))])
def test_source_sums_to_zero_per_component(ndim, spacing):
    """Each face's contribution to S appears in its two cells with opposite
    signs (symmetric face totals), so S sums to zero over every connected
    component: the singular system is consistent."""
    rng = np.random.default_rng(1)
    shape = (9, 11) if ndim == 2 else (6, 5, 7)
    valid = rng.random(shape) > 0.3
    grid = oracle.Grid(valid, spacing)
    f = rng.normal(size=(ndim,) + shape)
    f[:, ~valid] = np.nan  # missing data must never be read
    S = oracle.source(grid, f)
    assert np.isfinite(S).all()
    lab, nc = oracle.labels(grid)
    for c in range(nc):
        m = lab == c
        assert abs(S[m].sum()) <= 1e-13 * (np.abs(S).sum() + 1)


def _random_grid(ndim, spacing, seed=2, p=0.3):
    rng = np.random.default_rng(seed)
    shape = (8, 9) if ndim == 2 else (5, 6, 4)
    return oracle.Grid(rng.random(shape) > p, spacing)


@pytest.mark.parametrize("ndim,spacing", [(2, (0.1, 0.13)), (2, (1.0, 1.0)), (3, (1.0, 1.3, 0.7))])
def test_T_is_row_stochastic_and_symmetric(ndim, spacing):
    """T = W^{n+1}_off + W^n has unit row sums on valid rows (counts sum to
    A_tot); its off-diagonal entries are b~_j F_j / A_tot, so I - T is
    symmetric, positive semidefinite, with the constants of each connected
    component as its null space."""
    grid = _random_grid(ndim, spacing)
    W1, Wn = oracle.operators(grid)
    T = (W1 + Wn).toarray()
    v = grid.valid.reshape(-1)
    np.testing.assert_allclose(T[v].sum(axis=1), 1.0, rtol=0, atol=1e-14)
    K = (np.eye(grid.n) - T)[np.ix_(v, v)]
    np.testing.assert_allclose(K, K.T, rtol=0, atol=1e-15)
    # off-diagonal entries are the face totals over A_tot
    A = oracle.ray_counts(grid)
    nx, ny = int(grid.dims[0]), int(grid.dims[1])
    idx = np.flatnonzero(v)
    for q in idx[:20]:
        i, j, k = q % nx, (q // nx) % ny, q // (nx * ny)
        for f in range(2 * ndim):
            a = f // 2
            d = [0, 0, 0]
            d[a] = 1 if f % 2 == 0 else -1
            ni, nj, nk = i + d[0], j + d[1], k + d[2]
            if 0 <= ni < nx and 0 <= nj < ny and 0 <= nk < int(grid.dims[2]):
                nq = (nk * ny + nj) * nx + ni
                if v[nq]:
                    assert T[q, nq] == pytest.approx(grid.F[a] / grid.a_tot, rel=1e-13)
    ev = np.linalg.eigvalsh(K)
    assert ev.min() > -1e-13
    lab, nc = oracle.labels(grid)
    assert int((np.abs(ev) < 1e-11).sum()) == nc
    np.testing.assert_allclose(K @ np.ones(K.shape[0]), 0.0, atol=1e-14)


def test_M_is_not_symmetric():
    """The paper's system matrix M = I - W^{n+1}_off is not symmetric: on the
    3x3 example w_E of cell 1 is (c_xy + c_xx)/(8D) = 0.1768 while w_W of
    cell 2 is c_xy/(8D) = 0.0732 (Table tab:Coeffs)."""
    grid = oracle.Grid(np.ones((3, 3), bool), (1.0, 1.0))
    W1, _ = oracle.operators(grid)
    W1 = W1.toarray()
    i1, j1 = _paper_cell(1)
    i2, j2 = _paper_cell(2)
    q1, q2 = j1 * 3 + i1, j2 * 3 + i2
    assert W1[q1, q2] == pytest.approx(0.1768, abs=5e-5)
    assert W1[q2, q1] == pytest.approx(0.0732, abs=5e-5)
    M = np.eye(9) - W1
    assert np.abs(M - M.T).max() > 0.1


@pytest.mark.parametrize("ndim,spacing", [(2, (0.1, 0.13)), (3, (1.0, 1.0, 1.0))])
def test_apply_matches_sparse(ndim, spacing):
    grid = _random_grid(ndim, spacing, seed=4)
    A = oracle.ray_counts(grid)
    W1, Wn = oracle.operators(grid, A)
    x = np.random.default_rng(0).normal(size=grid.n)
    x[~grid.valid.reshape(-1)] = 0
    v = grid.valid.reshape(-1)
    np.testing.assert_allclose(oracle.apply(grid, A, 0, x).reshape(-1)[v], (W1 @ x)[v], atol=1e-14)
    np.testing.assert_allclose(oracle.apply(grid, A, 1, x).reshape(-1)[v], (Wn @ x)[v], atol=1e-14)
    np.testing.assert_allclose(oracle.apply(grid, A, 2, x).reshape(-1)[v], (x - W1 @ x - Wn @ x)[v], atol=1e-14)


def test_brute_force_ray_average_matches_matrix_form():
    """Brute force averaging of all straight-line path steps through every
    cell (Section 2.1) equals the matrix form of Eq. ExplicitEqn,
    W^{n+1}_off P^{n+1} + W^n P^n + S, for arbitrary P^n, P^{n+1}, f and a
    random mask -- within the quadrature error of the ray average."""
    rng = np.random.default_rng(8)
    valid = rng.random((5, 6)) > 0.3
    spacing = (0.1, 0.13)
    grid = oracle.Grid(valid, spacing)
    f = rng.normal(size=(2, 5, 6))
    Pn = rng.normal(size=(5, 6))
    Pn1 = rng.normal(size=(5, 6))
    W1, Wn = oracle.operators(grid)
    S = oracle.source(grid, f).reshape(-1)
    rhs = (W1 @ Pn1.reshape(-1) + Wn @ Pn.reshape(-1) + S).reshape(5, 6)
    brute = oracle.brute_force_update_2d(grid, f, Pn, Pn1, n_t=200, n_theta=2000)
    np.testing.assert_allclose(brute[valid], rhs[valid], atol=5e-5)
    # a sign error in the path step is caught
    flipped = oracle.source(grid, -f).reshape(-1)
    rhs_bad = (W1 @ Pn1.reshape(-1) + Wn @ Pn.reshape(-1) + flipped).reshape(5, 6)
    assert np.abs(brute[valid] - rhs_bad[valid]).max() > 1e-2
