"""Pins of the oracle's ray counts and constants against what the paper
prints and what geometry fixes (no GPU)."""
import math
import os
import re

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "appendix_3x3_coeffs.txt")
ROWS = ["AC_n", "AC_np1", "AE_n", "AE_np1", "AW_n", "AW_np1", "AN_n", "AN_np1", "AS_n", "AS_np1"]


def _eval_symbol(expr, D, cxx, cyy, cxy):
    total = 0.0
    for term in expr.split("+"):
        m = re.fullmatch(r"(\d*)(D|cxx|cyy|cxy)?", term.strip())
        assert m, term
        k = float(m.group(1)) if m.group(1) else 1.0
        sym = m.group(2)
        if sym is None:
            total += k  # plain number (only "0" occurs)
        else:
            total += k * {"D": D, "cxx": cxx, "cyy": cyy, "cxy": cxy}[sym]
    return total


def _paper_cell_to_ij(c):
    # paper numbers cells row by row from the top-left; its south neighbour is
    # the next row.  Physical y grows northwards, so row r of the paper is j = 2 - r.
    return (c - 1) % 3, 2 - (c - 1) // 3


def _golden_table():
    table = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            table[parts[0]] = parts[1:]
    return table


@pytest.mark.parametrize("D", [1.0, 0.37])
def test_appendix_table(D):
    """Table tab:Coeffs (appendix): 88 of the 90 printed ray counts are
    reproduced exactly.  The remaining two -- cell 4's A_N^n and A_N^{n+1} --
    are printed swapped: Eqs. ANnp1/ANn give A_N^{n+1} = c_xy and
    A_N^n = c_xy + c_yy for cell 4 (its north neighbour, cell 1, has a valid
    east neighbour only), which is also what the mirror-image cell 6 shows in
    the same table."""
    table = _golden_table()
    grid = oracle.Grid(np.ones((3, 3), bool), (D, D))
    A = oracle.ray_counts(grid)
    c = grid.c.reshape(3, 3)
    cxx, cyy, cxy = c[0, 0], c[1, 1], c[0, 1]
    assert grid.a_tot == pytest.approx(8 * D, rel=1e-15)  # appendix: A_tot = 8 Delta
    mismatches = []
    for r, name in enumerate(ROWS):
        for cell in range(1, 10):
            want = _eval_symbol(table[name][cell - 1], D, cxx, cyy, cxy)
            i, j = _paper_cell_to_ij(cell)
            got = A[j * 3 + i, r]
            if abs(got - want) > 1e-14 * D:
                mismatches.append((name, cell, got, want))
    assert sorted((m[0], m[1]) for m in mismatches) == [("AN_n", 4), ("AN_np1", 4)]
    i4, j4 = _paper_cell_to_ij(4)
    i6, j6 = _paper_cell_to_ij(6)
    a4 = A[j4 * 3 + i4]
    a6 = A[j6 * 3 + i6]
    assert a4[6] == pytest.approx(cxy + cyy) and a4[7] == pytest.approx(cxy)
    assert a4[6] == pytest.approx(a6[6]) and a4[7] == pytest.approx(a6[7])
    # and the printed pair is exactly the swap
    assert _eval_symbol(table["AN_n"][3], D, cxx, cyy, cxy) == pytest.approx(a4[7])
    assert _eval_symbol(table["AN_np1"][3], D, cxx, cyy, cxy) == pytest.approx(a4[6])


def test_appendix_constants():
    """Appendix: with dx = dy = D, c_xx = c_yy = D(2 sqrt2 - 2), c_xy = D(2 - sqrt2)."""
    c, F, a_tot = oracle.constants_2d(0.5, 0.5)
    assert c[0, 0] == pytest.approx(0.5 * (2 * math.sqrt(2) - 2), rel=1e-14)
    assert c[1, 1] == pytest.approx(0.5 * (2 * math.sqrt(2) - 2), rel=1e-14)
    assert c[0, 1] == pytest.approx(0.5 * (2 - math.sqrt(2)), rel=1e-14)


@pytest.mark.parametrize("dx,dy", [(1.0, 1.0), (0.1, 0.13), (2.0, 0.7)])
def test_boundary_example(dx, dy):
    """Eqs. AE_Boundary_example / AE_Boundary_example2: when the east cell's
    north neighbour is missing (rays at 0 < theta < pi/2 then start at E),
    A_E^n = dx + dy - sqrt(dx^2 + dy^2) and A_E^{n+1} = 2 dy - A_E^n."""
    valid = np.ones((3, 4), bool)
    # cell C = (i=1, j=1); E = (2, 1); EN = (2, 2) missing
    valid[2, 2] = False
    grid = oracle.Grid(valid, (dx, dy))
    A = oracle.ray_counts(grid)
    rec = A[1 * 4 + 1]
    dd = math.sqrt(dx * dx + dy * dy)
    assert rec[2] == pytest.approx(dx + dy - dd, rel=1e-13)
    assert rec[3] == pytest.approx(dy - dx + dd, rel=1e-13)
    assert rec[2] + rec[3] == pytest.approx(2 * dy, rel=1e-14)


@pytest.mark.parametrize("dx,dy", [(1.0, 1.0), (0.1, 0.13), (3.0, 0.2)])
def test_face_totals_2d(dx, dy):
    """Eq. AE_Interior: the rays through an interior x-face total 2 dy, so
    c_xx + 2 c_xy = 2 dy; likewise c_yy + 2 c_xy = 2 dx.  Eq. Atot2D."""
    c, F, a_tot = oracle.constants_2d(dx, dy)
    assert c[0, 0] + 2 * c[0, 1] == pytest.approx(2 * dy, rel=1e-14)
    assert c[1, 1] + 2 * c[0, 1] == pytest.approx(2 * dx, rel=1e-14)
    assert a_tot == pytest.approx(4 * (dx + dy))
    assert (c >= 0).all()


@pytest.mark.parametrize("ndim,spacing", [(2, (0.1, 0.13)), (2, (1.0, 1.0)), (3, (1.0, 1.0, 1.0)),
                                          (3, (1.0, 1.3, 0.7))])
def test_counts_sum_to_atot(ndim, spacing):
    """Appendix: all ray counts of a cell sum to A_tot ("always required"),
    for any mask."""
    rng = np.random.default_rng(5)
    shape = (7, 9) if ndim == 2 else (5, 6, 7)
    valid = rng.random(shape) > 0.3
    grid = oracle.Grid(valid, spacing)
    A = oracle.ray_counts(grid)
    sums = A.sum(axis=1)[valid.reshape(-1)]
    np.testing.assert_allclose(sums, grid.a_tot, rtol=1e-13)
    assert (A >= -1e-15).all()
    assert np.all(A[:, 1] == 0.0)  # A_C^{n+1} = 0 (Eq. wcnp1)


def test_isotropic_3d_printed_values():
    """Section 2.2.3 prints c_jj = 0.6277684243304 D^2 and
    c_jk = 0.6284560573148 D^2 for isotropic grids."""
    far, near = oracle.isotropic_3d_factors()
    assert far == pytest.approx(0.6277684243304, abs=6e-14)
    assert near == pytest.approx(0.6284560573148, abs=6e-14)


def test_quadrature_reproduces_isotropic_closed_form():
    """Eq. FarFaceEquation and Eqs. IAc-ICc at dx = dy = dz reproduce the
    closed forms of Eqs. ConstantFarFace/ConstantNearFaces, and scale as D^2."""
    far, near = oracle.isotropic_3d_factors()
    for D in (1.0, 0.3):
        c, F, a_tot = oracle.constants_3d(D, D, D)
        for a in range(3):
            for b in range(3):
                want = (far if a == b else near) * D * D
                assert c[a, b] == pytest.approx(want, rel=1e-11)
        assert a_tot == pytest.approx(6 * math.pi * D * D)


@pytest.mark.parametrize("h", [(1.0, 1.3, 0.7), (0.5, 2.0, 1.0), (1.0, 1.0, 3.0)])
def test_3d_face_totals_anisotropic(h):
    """Every ray through the face normal to a lands in exactly one of the far
    face or the four side faces of the neighbour, so c_aa + 2 sum_b c_ab must
    equal the face total pi h_b h_c (Section 2.2.2); and c_jk = c_kj."""
    c, F, a_tot = oracle.constants_3d(*h)
    for a in range(3):
        o = [b for b in range(3) if b != a]
        assert c[a, a] + 2 * c[a, o[0]] + 2 * c[a, o[1]] == pytest.approx(F[a], rel=1e-10)
        assert F[a] == pytest.approx(math.pi * h[o[0]] * h[o[1]])
    np.testing.assert_allclose(c, c.T, rtol=1e-10)
    assert a_tot == pytest.approx(F.sum() * 2)


@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (1.0, 1.3, 0.7)])
def test_3d_constants_monte_carlo(h):
    """Brute force: Monte-Carlo ray tracing reproduces the quadrature
    constants to within 5 standard errors."""
    c, _, _ = oracle.constants_3d(*h)
    mc, err = oracle.monte_carlo_constants_3d(*h, samples=400_000, seed=11)
    assert (np.abs(mc - c) <= 5 * err + 1e-12).all(), (mc, c, err)


@pytest.mark.parametrize("spacing", [(1.0, 1.0), (0.1, 0.13), (1.0, 2.5)])
def test_brute_force_ray_counts_2d(spacing):
    """Brute force: direct quadrature of the ray integral over (s, theta) with
    one-cell ray tracing reproduces the ray counts of every cell of a random
    masked grid."""
    rng = np.random.default_rng(3)
    valid = rng.random((5, 6)) > 0.35
    grid = oracle.Grid(valid, spacing)
    A = oracle.ray_counts(grid)
    B = oracle.brute_force_counts_2d(grid, n_t=200, n_theta=2000)
    scale = grid.a_tot
    np.testing.assert_allclose(B, A, atol=2e-5 * scale, rtol=0)


def test_brute_force_detects_swapped_constants():
    """The brute-force check is sharp enough to catch c_xx and c_yy swapped on
    an anisotropic grid (a plausible transcription error)."""
    valid = np.ones((4, 4), bool)
    valid[0, 0] = False
    spacing = (0.1, 0.13)
    c, F, a_tot = oracle.constants_2d(*spacing)
    bad = c.copy()
    bad[0, 0], bad[1, 1] = c[1, 1], c[0, 0]
    g_bad = oracle.Grid(valid, spacing, constants=(bad, F, a_tot))
    g_ok = oracle.Grid(valid, spacing)
    B = oracle.brute_force_counts_2d(g_ok, n_t=100, n_theta=1000)
    assert np.abs(oracle.ray_counts(g_bad) - B).max() > 1e-3 * a_tot
