"""FP64 CPU oracle for matrix-based omnidirectional pressure integration
(Zigunov & Charonko, arXiv 2311.16935).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports, links or calls anything here, and this package imports nothing
from the product package.

What it computes, each piece written from the paper:

* ``constants_2d``          Eq. cxx2D (c_xx, c_yy, c_xy), Eq. Atot2D, Eq. AE_Interior
* ``constants_3d_isotropic`` Eqs. ConstantFarFace / ConstantNearFaces (closed form)
* ``constants_3d``          Eq. FarFaceEquation and Eqs. IAc, IB1c, IB2c, ICc by
                            quadrature (arbitrary dx, dy, dz)
* ``ray_counts``            Eqs. Acn, AEnp1, AEn, ANnp1, ANn and the 3D pattern
                            (Section 2.2) for every cell of a masked grid
* ``source``                last sum of Eq. ExplicitEqn
* ``operators``             W^{n+1} (off-diagonal) and W^n of Eq. MatrixEquation
* ``residual``              Eq. ResidualMomentum (and Eq. ResidualPressure)
* ``solve_direct``          the converged answer (fixed point of Algorithm 1) by
                            sparse LU of the bordered singular system (tiny grids)
* ``solve_cg``              the same answer by plain FP64 CG (medium grids)
* ``solve_literal``         Algorithm 1 as written: each outer iteration solves
                            Eq. MatrixEquation exactly (sparse LU, the analogue of
                            the paper's Matlab backslash)
* ``solve_outer_anderson``  Algorithm 1's outer map P -> M^-1 (W^n P + S), boundary
                            term refreshed every iteration, accelerated by Anderson
                            mixing of depth m (Anderson 1965, in the difference form
                            of Walker & Ni 2011); m = 0 is Algorithm 1 itself
* ``brute_force_counts_2d`` the ray counts of every cell by direct quadrature of
                            the ray integral (Eq. AE_Interior's (s, theta) integral,
                            classifying each ray by tracing it back one cell)
* ``monte_carlo_constants_3d`` the 3D c_jk by Monte-Carlo ray tracing
* ``rotating_ray_solve_2d``  whole straight rays at finite ray density (the
                            rotating-parallel-ray integration whose limit of
                            infinitely many rays the method takes), iterated;
                            a trend check against the fixed point, not parity
* ``pressure_update``       Eq. ResidualPressure

Pressure is defined up to a constant (Eq. 1); every solve here returns the
answer with zero mean on each connected component of valid cells and NaN on
missing cells.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (plain gcc, OpenMP) next to its source."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        I = ctypes.c_int
        lib.orc_ray_counts.argtypes = [I, P, P, P, P, D, P, P]
        lib.orc_source.argtypes = [I, P, P, P, P, D, P, P, P]
        lib.orc_labels.argtypes = [I, P, P, P]
        lib.orc_labels.restype = I64
        lib.orc_apply.argtypes = [I, P, P, P, D, I, P, P]
        lib.orc_solve_cg.argtypes = [I, P, P, P, D, P, P, D, I64, P]
        lib.orc_residual_norms.argtypes = [I, P, P, P, P, D, P, P, P, P]
        lib.orc_residual_at.argtypes = [I, P, P, P, P, D, P, P, P, P, I64, P]
        lib.orc_num_threads.restype = I
        lib.orc_set_num_threads.argtypes = [I]
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(t: int) -> None:
    _load().orc_set_num_threads(int(t))


# --------------------------------------------------------------------------
# Grid description
# --------------------------------------------------------------------------

class Grid:
    """A uniform grid with a validity mask.

    ``valid`` is a boolean array of shape (ny, nx) in 2D or (nz, ny, nx) in
    3D (x fastest); ``spacing`` is (dx, dy) or (dx, dy, dz).  Cells outside
    the array are missing (b = 1), as in the appendix's example domain.
    """

    def __init__(self, valid, spacing, constants=None):
        valid = np.ascontiguousarray(np.asarray(valid, dtype=bool))
        self.ndim = valid.ndim
        if self.ndim not in (2, 3):
            raise ValueError("grid must be 2D or 3D")
        if len(spacing) != self.ndim:
            raise ValueError("spacing must have one entry per axis")
        self.valid = valid
        self.valid_u8 = valid.astype(np.uint8)
        self.h = np.zeros(3)
        self.h[: self.ndim] = spacing
        shape = valid.shape[::-1]  # (nx, ny[, nz])
        self.dims = np.array(list(shape) + [1] * (3 - self.ndim), dtype=np.int64)
        if constants is None:
            constants = constants_2d(*spacing) if self.ndim == 2 else constants_3d(*spacing)
        self.c, self.F, self.a_tot = constants
        self.c = np.ascontiguousarray(self.c, dtype=np.float64).reshape(9)
        self.F = np.ascontiguousarray(self.F, dtype=np.float64)
        self.n = int(valid.size)
        self.rec = 2 + 4 * self.ndim

    def _ptrs(self):
        return (self.dims.ctypes.data, self.valid_u8.ctypes.data, self.c.ctypes.data, self.F.ctypes.data)


# --------------------------------------------------------------------------
# Constants
# --------------------------------------------------------------------------

def constants_2d(dx: float, dy: float):
    """Eq. cxx2D: c_xx = 2(dd - dx), c_yy = 2(dd - dy), c_xy = dx + dy - dd,
    dd = sqrt(dx^2 + dy^2).  Face totals (Eq. AE_Interior): x-faces 2 dy,
    y-faces 2 dx.  A_tot = 4 (dx + dy) (Eq. Atot2D)."""
    dd = math.sqrt(dx * dx + dy * dy)
    c = np.zeros((3, 3))
    c[0, 0] = 2.0 * (dd - dx)
    c[1, 1] = 2.0 * (dd - dy)
    c[0, 1] = c[1, 0] = dx + dy - dd
    F = np.array([2.0 * dy, 2.0 * dx, 0.0])
    return c, F, 4.0 * (dx + dy)


def isotropic_3d_factors():
    """The dimensionless closed forms of Eqs. ConstantFarFace (j = k) and
    ConstantNearFaces (j != k)."""
    s2 = math.sqrt(2.0)
    far = math.log(4.0 / 3.0) - s2 * math.atan(s2) + s2 / 2.0 * math.atan(10.0 * s2 / 23.0) + math.pi * (s2 - 1.0)
    near = math.pi / 2.0 - 0.25 * math.log(4.0 / 3.0) - s2 / 4.0 * math.atan(10.0 * s2 / 23.0) - s2 / 2.0 * math.atan(s2)
    return far, near


def _face_totals_3d(dx, dy, dz):
    # Section 2.2.2: a face normal to y has total projection pi*dx*dz; likewise
    # for the others.  A_tot = 2 pi (dx dy + dx dz + dy dz).
    F = np.array([math.pi * dy * dz, math.pi * dx * dz, math.pi * dx * dy])
    return F, 2.0 * math.pi * (dx * dy + dx * dz + dy * dz)


def constants_3d_isotropic(delta: float):
    far, near = isotropic_3d_factors()
    c = np.full((3, 3), near * delta * delta)
    np.fill_diagonal(c, far * delta * delta)
    F, a_tot = _face_totals_3d(delta, delta, delta)
    return c, F, a_tot


def far_face_integral(dj: float, dl1: float, dl2: float) -> float:
    """Eq. FarFaceEquation: the far-face constant c_jj for a cell with spacing
    dj along the face normal and dl1, dl2 along the other two axes."""
    from scipy.integrate import quad

    def g(phi):
        l1c, l1s = dl1 * math.cos(phi), dl1 * math.sin(phi)
        at = math.atan(dj / l1s)
        return math.pi * (dl2 * l1s - dj * l1c) + 2.0 * (dj * l1c * at - dl2 * l1s * at)

    return quad(g, math.atan(dj / dl2), math.pi / 2, epsabs=1e-15, epsrel=1e-13, limit=400)[0]


def dihedral_integral(dj: float, dk: float, dl: float) -> float:
    """c_jk (j != k) = I_A + I_B1 + I_B2 + I_C  (Eqs. IAc, IB1c, IB2c, ICc);
    dl is the spacing along the third axis."""
    from scipy.integrate import quad

    ia = dl * dl / 2.0 * math.atanh(
        dj * dj * dk * dk / (2 * dl**4 + 2 * dl * dl * dj * dj + 2 * dl * dl * dk * dk + dj * dj * dk * dk))
    a = math.atan(dj / dl)

    def b1(phi):
        kc, ks = dk * math.cos(phi), dk * math.sin(phi)
        return (dl * ks * (math.atan(dl / kc) - dl * kc / (dl * dl + kc * kc))
                + kc * ks * (math.log(kc / math.sqrt(kc * kc + dl * dl)) + dl * dl / (2 * (dl * dl + kc * kc))))

    def b2(phi):
        kc, ks = dk * math.cos(phi), dk * math.sin(phi)
        return (dl * ks * (math.atan(dj / ks) - dj * ks / (dj * dj + ks * ks))
                + kc * ks * (math.log(ks / math.sqrt(ks * ks + dj * dj)) + dj * dj / (2 * (dj * dj + ks * ks))))

    def ic(phi):
        s, c = math.sin(phi), math.cos(phi)
        return 0.5 * dj * dk * dk * s * (2 * dl * s - dj * c) / (dj * dj + dk * dk * s * s)

    opts = dict(epsabs=1e-15, epsrel=1e-13, limit=400)
    return ia + quad(b1, 0.0, a, **opts)[0] + quad(b2, a, math.pi / 2, **opts)[0] + quad(ic, a, math.pi / 2, **opts)[0]


def constants_3d(dx: float, dy: float, dz: float):
    """All six c_jk for arbitrary spacing by quadrature (Section 2.2.2)."""
    h = (dx, dy, dz)
    c = np.zeros((3, 3))
    for a in range(3):
        o = [b for b in range(3) if b != a]
        c[a, a] = far_face_integral(h[a], h[o[0]], h[o[1]])
        for b in o:
            l = [q for q in range(3) if q not in (a, b)][0]
            c[a, b] = dihedral_integral(h[a], h[b], h[l])
    F, a_tot = _face_totals_3d(dx, dy, dz)
    return c, F, a_tot


# --------------------------------------------------------------------------
# Ray counts, source, operators
# --------------------------------------------------------------------------

def ray_counts(grid: Grid) -> np.ndarray:
    """Per-cell ray counts, shape (n, 2 + 4*ndim): A_C^n, A_C^{n+1}, then
    (A_f^n, A_f^{n+1}) for faces E, W, N, S[, F, B]."""
    lib = _load()
    A = np.zeros((grid.n, grid.rec))
    dims, val, c, F = grid._ptrs()
    lib.orc_ray_counts(grid.ndim, dims, val, c, F, grid.a_tot, grid.h.ctypes.data, A.ctypes.data)
    return A


def source(grid: Grid, f) -> np.ndarray:
    """Source vector S (last sum of Eq. ExplicitEqn).  ``f`` has shape
    (ndim,) + valid.shape; component a is the gradient along axis a (x first).
    Returns S with the grid's shape (0 on missing cells)."""
    lib = _load()
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
    if f.shape != (grid.ndim,) + grid.valid.shape:
        raise ValueError("f must have shape (ndim,) + grid shape")
    S = np.zeros(grid.n)
    dims, val, c, F = grid._ptrs()
    lib.orc_source(grid.ndim, dims, val, c, F, grid.a_tot, grid.h.ctypes.data, f.ctypes.data, S.ctypes.data)
    return S.reshape(grid.valid.shape)


def labels(grid: Grid):
    """Connected components of the valid cells (face adjacency)."""
    lib = _load()
    lab = np.zeros(grid.n, dtype=np.int32)
    nc = lib.orc_labels(grid.ndim, grid.dims.ctypes.data, grid.valid_u8.ctypes.data, lab.ctypes.data)
    return lab.reshape(grid.valid.shape), int(nc)


def operators(grid: Grid, A: np.ndarray | None = None):
    """Sparse W^{n+1}_off and W^n (Eq. MatrixEquation, Eq. weights) over all
    cells of the box (rows and columns of missing cells are empty)."""
    import scipy.sparse as sp

    if A is None:
        A = ray_counts(grid)
    nx, ny, nz = (int(v) for v in grid.dims)
    offs = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    rows1, cols1, vals1 = [], [], []
    rowsn, colsn, valsn = [], [], []
    flat_valid = grid.valid.reshape(-1)
    idx_all = np.arange(grid.n)
    i = idx_all % nx
    j = (idx_all // nx) % ny
    k = idx_all // (nx * ny)
    vi = flat_valid
    rowsn.append(idx_all[vi]); colsn.append(idx_all[vi]); valsn.append(A[vi, 0] / grid.a_tot)
    for f in range(2 * grid.ndim):
        di, dj, dk = offs[f]
        ni, nj, nk = i + di, j + dj, k + dk
        inside = (ni >= 0) & (ni < nx) & (nj >= 0) & (nj < ny) & (nk >= 0) & (nk < nz)
        nidx = np.where(inside, (nk * ny + nj) * nx + ni, 0)
        ok = vi & inside & flat_valid[nidx]
        rows1.append(idx_all[ok]); cols1.append(nidx[ok]); vals1.append(A[ok, 3 + 2 * f] / grid.a_tot)
        rowsn.append(idx_all[ok]); colsn.append(nidx[ok]); valsn.append(A[ok, 2 + 2 * f] / grid.a_tot)
    W1 = sp.csr_matrix((np.concatenate(vals1), (np.concatenate(rows1), np.concatenate(cols1))), shape=(grid.n, grid.n))
    Wn = sp.csr_matrix((np.concatenate(valsn), (np.concatenate(rowsn), np.concatenate(colsn))), shape=(grid.n, grid.n))
    return W1, Wn


def apply(grid: Grid, A: np.ndarray, which: int, x) -> np.ndarray:
    """which = 0: W^{n+1}_off x; 1: W^n x; 2: (I - W^{n+1}_off - W^n) x."""
    lib = _load()
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))
    y = np.zeros(grid.n)
    lib.orc_apply(grid.ndim, grid.dims.ctypes.data, grid.valid_u8.ctypes.data, A.ctypes.data, grid.a_tot, which,
                  x.ctypes.data, y.ctypes.data)
    return y.reshape(grid.valid.shape)


def residual(grid: Grid, f, P) -> float:
    """eps_R of Eq. ResidualMomentum: ||(I - W^{n+1}_off - W^n) P - S|| / ||S||,
    L2 norms over valid cells; 0 when S = 0."""
    num, den = residual_norms(grid, f, P)
    return 0.0 if den == 0.0 else math.sqrt(num / den)


def residual_norms(grid: Grid, f, P):
    lib = _load()
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
    P = np.ascontiguousarray(np.asarray(P, dtype=np.float64).reshape(-1))
    out = np.zeros(2)
    dims, val, c, F = grid._ptrs()
    lib.orc_residual_norms(grid.ndim, dims, val, c, F, grid.a_tot, grid.h.ctypes.data, f.ctypes.data, P.ctypes.data,
                           out.ctypes.data)
    return float(out[0]), float(out[1])


def residual_at(grid: Grid, f, P, flat_idx) -> np.ndarray:
    """Per-cell residual ((I - T) P - S) at the given flat indices."""
    lib = _load()
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
    P = np.ascontiguousarray(np.asarray(P, dtype=np.float64).reshape(-1))
    idx = np.ascontiguousarray(np.asarray(flat_idx, dtype=np.int64))
    out = np.zeros(idx.size)
    dims, val, c, F = grid._ptrs()
    lib.orc_residual_at(grid.ndim, dims, val, c, F, grid.a_tot, grid.h.ctypes.data, f.ctypes.data, P.ctypes.data,
                        idx.ctypes.data, idx.size, out.ctypes.data)
    return out


def pressure_update(P_new, P_old, valid) -> float:
    """eps_P of Eq. ResidualPressure: ||P^{n+1} - P^n||_2 / ||P^{n+1}||_2, the
    L2 norms over the valid cells; 0 when P^{n+1} = 0 there."""
    v = np.asarray(valid, dtype=bool)
    a = np.asarray(P_new)[v]
    b = np.asarray(P_old)[v]
    den = np.linalg.norm(a)
    return 0.0 if den == 0.0 else float(np.linalg.norm(a - b) / den)


def gauge(grid: Grid, P) -> np.ndarray:
    """Remove the mean on each connected component; NaN on missing cells."""
    lab, nc = labels(grid)
    out = np.array(P, dtype=np.float64, copy=True).reshape(grid.valid.shape)
    for cidx in range(nc):
        m = lab == cidx
        out[m] -= out[m].mean()
    out[~grid.valid] = np.nan
    return out


# --------------------------------------------------------------------------
# Solves
# --------------------------------------------------------------------------

def solve_direct(grid: Grid, f) -> np.ndarray:
    """Fixed point of Algorithm 1 on a tiny grid: (I - T) P = S with one
    zero-mean constraint per component, by sparse LU of the bordered system
    [[I - T, B], [B^T, 0]] (B = component indicator columns)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    S = source(grid, f).reshape(-1)
    W1, Wn = operators(grid)
    vidx = np.flatnonzero(grid.valid.reshape(-1))
    nv = vidx.size
    if nv == 0:
        return np.full(grid.valid.shape, np.nan)
    K = (sp.identity(grid.n, format="csr") - W1 - Wn)[vidx][:, vidx]
    lab, nc = labels(grid)
    labv = lab.reshape(-1)[vidx]
    B = sp.csr_matrix((np.ones(nv), (np.arange(nv), labv)), shape=(nv, nc))
    big = sp.bmat([[K, B], [B.T, None]], format="csc")
    rhs = np.concatenate([S[vidx], np.zeros(nc)])
    sol = spla.splu(big).solve(rhs)
    P = np.full(grid.n, np.nan)
    P[vidx] = sol[:nv]
    return gauge(grid, P.reshape(grid.valid.shape))


def solve_cg(grid: Grid, f, tol: float = 1e-14, maxit: int = 1_000_000, P0=None):
    """Fixed point of Algorithm 1 by plain FP64 CG (C code, OpenMP loops).
    Returns (P, iterations, final eps_R)."""
    lib = _load()
    A = ray_counts(grid)
    S = source(grid, f).reshape(-1)
    P = np.zeros(grid.n) if P0 is None else np.array(P0, dtype=np.float64).reshape(-1).copy()
    info = np.zeros(2)
    lib.orc_solve_cg(grid.ndim, grid.dims.ctypes.data, grid.valid_u8.ctypes.data, A.ctypes.data, grid.a_tot,
                     S.ctypes.data, P.ctypes.data, float(tol), int(maxit), info.ctypes.data)
    return P.reshape(grid.valid.shape), int(info[0]), float(info[1])


def solve_literal(grid: Grid, f, tol: float = 1e-10, max_outer: int = 100000, P0=None, history: bool = True):
    """Algorithm 1 as written.  P^0 = 0 (or P0); each outer iteration solves
    Eq. MatrixEquation, (I - W^{n+1}_off) P^{n+1} = W^n P^n + S, exactly by
    sparse LU; eps_R (Eq. ResidualMomentum) and eps_P (Eq. ResidualPressure)
    are recorded after every iteration; stops when eps_R <= tol.
    Returns (P gauged, n_outer, eps_R history, eps_P history)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    S = source(grid, f).reshape(-1)
    W1, Wn = operators(grid)
    vidx = np.flatnonzero(grid.valid.reshape(-1))
    I = sp.identity(grid.n, format="csr")
    M = (I - W1)[vidx][:, vidx].tocsc()
    Wnv = Wn[vidx][:, vidx]
    K = (I - W1 - Wn)[vidx][:, vidx]
    Sv = S[vidx]
    snorm = np.linalg.norm(Sv)
    lu = spla.splu(M)
    P = np.zeros(vidx.size) if P0 is None else np.array(P0, dtype=np.float64).reshape(-1)[vidx].copy()
    eps_r, eps_p = [], []
    n = 0
    while n < max_outer:
        Pn1 = lu.solve(Wnv @ P + Sv)
        n += 1
        er = 0.0 if snorm == 0 else float(np.linalg.norm(K @ Pn1 - Sv) / snorm)
        ep = pressure_update(Pn1, P, np.ones(Pn1.size, dtype=bool))
        if history:
            eps_r.append(er)
            eps_p.append(ep)
        P = Pn1
        if er <= tol:
            break
    out = np.full(grid.n, np.nan)
    out[vidx] = P
    return gauge(grid, out.reshape(grid.valid.shape)), n, eps_r, eps_p


def _outer_parts(grid: Grid, f):
    """The pieces of Algorithm 1 on the valid cells: LU of M = I - W^{n+1}_off,
    W^n, the fixed-point operator I - W^{n+1}_off - W^n and S."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    S = source(grid, f).reshape(-1)
    W1, Wn = operators(grid)
    vidx = np.flatnonzero(grid.valid.reshape(-1))
    I = sp.identity(grid.n, format="csr")
    M = (I - W1)[vidx][:, vidx].tocsc()
    return spla.splu(M), Wn[vidx][:, vidx], (I - W1 - Wn)[vidx][:, vidx], S[vidx], vidx


def solve_outer_anderson(grid: Grid, f, depth: int, tol: float = 1e-10, max_outer: int = 100000, P0=None,
                         callback=None):
    """Anderson acceleration of Algorithm 1.

    The outer map is Algorithm 1's step, G(P) = M^-1 (W^n P + S) with M =
    I - W^{n+1}_off (Eq. MatrixEquation, solved exactly by sparse LU): the
    boundary term W^n P is refreshed from the current iterate every time.
    With f_k = G(x_k) - x_k and the last min(k, depth) differences
    dF_i = f_{i+1} - f_i, dG_i = G(x_{i+1}) - G(x_i), each step takes
    gamma = argmin || f_k - dF gamma ||_2 (a least-squares solve) and
    x_{k+1} = G(x_k) - dG gamma.  depth = 0 gives x_{k+1} = G(x_k), i.e.
    Algorithm 1 unchanged.  Every fixed point of G is Algorithm 1's fixed
    point.  eps_R (Eq. ResidualMomentum) of each new iterate is recorded;
    callback(n, x) (optional) sees every new iterate on the valid cells.
    Returns (P gauged, n_outer, eps_R history)."""
    lu, Wnv, K, Sv, vidx = _outer_parts(grid, f)
    snorm = np.linalg.norm(Sv)
    x = np.zeros(vidx.size) if P0 is None else np.array(P0, dtype=np.float64).reshape(-1)[vidx].copy()
    dF, dG = [], []
    f_prev = g_prev = None
    eps_r = []
    n = 0
    while n < max_outer:
        g = lu.solve(Wnv @ x + Sv)
        fk = g - x
        if f_prev is not None and depth > 0:
            dF.append(fk - f_prev)
            dG.append(g - g_prev)
            if len(dF) > depth:
                dF.pop(0)
                dG.pop(0)
        f_prev, g_prev = fk, g
        if dF:
            DF = np.stack(dF, axis=1)
            gamma = np.linalg.lstsq(DF, fk, rcond=None)[0]
            x = g - np.stack(dG, axis=1) @ gamma
        else:
            x = g
        n += 1
        if callback is not None:
            callback(n, x.copy())
        er = 0.0 if snorm == 0 else float(np.linalg.norm(K @ x - Sv) / snorm)
        eps_r.append(er)
        if er <= tol:
            break
    out = np.full(grid.n, np.nan)
    out[vidx] = x
    return gauge(grid, out.reshape(grid.valid.shape)), n, eps_r


# --------------------------------------------------------------------------
# Brute force: rays
# --------------------------------------------------------------------------

def _trace_class_2d(ha, hb, t, theta):
    """Trace a ray backwards from the point t (0 < t < hb) of the face it
    crossed, into the neighbour cell, at angle theta from the face normal
    (-pi/2 < theta < pi/2).  Returns 0 if it entered the neighbour through
    its far face, +1 / -1 through its side face at +b / -b."""
    ct, st = np.cos(theta), np.sin(theta)
    t_far = ha / ct
    with np.errstate(divide="ignore", invalid="ignore"):
        t_side = np.where(st > 0, (hb - t) / st, np.where(st < 0, t / (-st), np.inf))
    return np.where(t_far <= t_side, 0, np.where(st > 0, 1, -1))


def brute_force_counts_2d(grid: Grid, n_t: int = 400, n_theta: int = 4000) -> np.ndarray:
    """Ray counts of every cell by brute-force quadrature of the ray integral
    A = int int R(s, theta) ds dtheta (Eq. AE_Interior and Section 2.2.1).

    For each face of each valid cell, rays cross the face at n_t midpoints t
    and n_theta midpoint angles, each carrying the projected measure
    h_b cos(theta) dt dtheta / h_b.  Each ray is traced back one cell through
    the face neighbour j: if j is missing the ray starts at C (A_C^n); else if
    the cell it came from before j is missing it starts at j (A_j^n), and
    otherwise it continues from the same iteration (A_j^{n+1}).  No closed
    form or constant of the paper is used."""
    if grid.ndim != 2:
        raise ValueError("2D only")
    nx, ny = int(grid.dims[0]), int(grid.dims[1])
    h = grid.h
    valid = grid.valid

    def isv(i, j):
        return 0 <= i < nx and 0 <= j < ny and bool(valid[j, i])

    # per axis: the measure of rays by predecessor class (far, +side, -side)
    cls_measure = {}
    for a in range(2):
        b = 1 - a
        ha, hb = h[a], h[b]
        t = (np.arange(n_t) + 0.5) / n_t * hb
        th = (np.arange(n_theta) + 0.5) / n_theta * np.pi - np.pi / 2
        T, TH = np.meshgrid(t, th, indexing="ij")
        w = np.cos(TH) * (hb / n_t) * (np.pi / n_theta)
        cl = _trace_class_2d(ha, hb, T, TH)
        cls_measure[a] = {q: float(w[cl == q].sum()) for q in (0, 1, -1)}
    offs = [(1, 0), (-1, 0), (0, 1), (0, -1)]
    out = np.zeros((grid.n, grid.rec))
    for j in range(ny):
        for i in range(nx):
            if not valid[j, i]:
                continue
            rec = out[j * nx + i]
            for f in range(4):
                a = f // 2
                di, dj = offs[f]
                ni, nj = i + di, j + dj
                tot = sum(cls_measure[a].values())
                if not isv(ni, nj):
                    rec[0] += tot
                    continue
                for q, m in cls_measure[a].items():
                    if q == 0:
                        pi_, pj_ = ni + di, nj + dj
                    elif a == 0:
                        pi_, pj_ = ni, nj + q
                    else:
                        pi_, pj_ = ni + q, nj
                    if isv(pi_, pj_):
                        rec[3 + 2 * f] += m
                    else:
                        rec[2 + 2 * f] += m
    return out


def monte_carlo_constants_3d(dx: float, dy: float, dz: float, samples: int = 1_000_000, seed: int = 0):
    """Monte-Carlo estimate of the 3D constants by ray tracing (Section 2.2.2):
    for the face normal to each axis a, rays cross the face at a uniform point
    with directions drawn from the projected (cosine-weighted) hemisphere,
    whose total measure is the face total pi * h_b * h_c.  Each ray is traced
    back through the neighbour cell and tallied by the face it entered that
    cell through: the far face gives c_aa, the two side faces normal to b give
    2 c_ab.  Returns (c estimate 3x3, standard error 3x3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = np.array([dx, dy, dz])
    c = np.zeros((3, 3))
    err = np.zeros((3, 3))
    for a in range(3):
        o = [b for b in range(3) if b != a]
        u1, u2 = rng.random(samples), rng.random(samples)
        r = np.sqrt(u1)
        phi = 2 * np.pi * u2
        d = np.zeros((samples, 3))
        d[:, a] = np.sqrt(1.0 - u1)
        d[:, o[0]] = r * np.cos(phi)
        d[:, o[1]] = r * np.sin(phi)
        p = np.zeros((samples, 3))
        p[:, o[0]] = rng.random(samples) * h[o[0]]
        p[:, o[1]] = rng.random(samples) * h[o[1]]
        tfar = h[a] / d[:, a]
        tb = []
        for b in o:
            with np.errstate(divide="ignore", invalid="ignore"):
                tb.append(np.where(d[:, b] > 0, (h[b] - p[:, b]) / d[:, b],
                                   np.where(d[:, b] < 0, p[:, b] / -d[:, b], np.inf)))
        allt = np.stack([tfar] + tb, axis=1)
        which = np.argmin(allt, axis=1)
        total = np.pi * h[o[0]] * h[o[1]]
        for q, ax in enumerate([a] + o):
            frac = np.mean(which == q)
            se = math.sqrt(frac * (1 - frac) / samples)
            scale = total if ax == a else total / 2.0  # two side faces per other axis
            c[a, ax] = frac * scale
            err[a, ax] = se * scale
    return c, err


def brute_force_update_2d(grid: Grid, f, P_n, P_np1, n_t: int = 200, n_theta: int = 2000) -> np.ndarray:
    """Right-hand side of one outer iteration by brute-force averaging over
    rays (Section 2.1): every ray (s, theta) through a valid cell C enters it
    through one face, from face neighbour j.  If j is missing the ray starts
    at C and carries P_C^n.  Otherwise it carries P_j^i plus the one-cell path
    integral of Eq. PressureIntegrator1 with the face-averaged gradient,
    P_j - dj (f(j) + f(C))/2, where i = n+1 if the ray reached j from a valid
    cell and i = n if it started at j.  The average over all rays, weighted by
    their measure, is returned (per cell; NaN on missing cells).

    Uses only ray tracing and the path rule: neither the ray-count formulas,
    the constants nor the assembled source vector."""
    if grid.ndim != 2:
        raise ValueError("2D only")
    nx, ny = int(grid.dims[0]), int(grid.dims[1])
    h = grid.h
    valid = grid.valid
    f = np.asarray(f, dtype=np.float64)
    Pn = np.asarray(P_n, dtype=np.float64).reshape(ny, nx)
    Pn1 = np.asarray(P_np1, dtype=np.float64).reshape(ny, nx)

    def isv(i, j):
        return 0 <= i < nx and 0 <= j < ny and bool(valid[j, i])

    cls_measure = {}
    for a in range(2):
        b = 1 - a
        ha, hb = h[a], h[b]
        t = (np.arange(n_t) + 0.5) / n_t * hb
        th = (np.arange(n_theta) + 0.5) / n_theta * np.pi - np.pi / 2
        T, TH = np.meshgrid(t, th, indexing="ij")
        w = np.cos(TH) * (hb / n_t) * (np.pi / n_theta)
        cl = _trace_class_2d(ha, hb, T, TH)
        cls_measure[a] = {q: float(w[cl == q].sum()) for q in (0, 1, -1)}
    offs = [(1, 0), (-1, 0), (0, 1), (0, -1)]
    out = np.full((ny, nx), np.nan)
    for j in range(ny):
        for i in range(nx):
            if not valid[j, i]:
                continue
            num = 0.0
            den = 0.0
            for fc in range(4):
                a = fc // 2
                di, dj = offs[fc]
                ni, nj = i + di, j + dj
                for q, m in cls_measure[a].items():
                    den += m
                    if not isv(ni, nj):
                        num += m * Pn[j, i]
                        continue
                    step = -(di * h[0] + dj * h[1]) * 0.5 * (f[a, nj, ni] + f[a, j, i])
                    if q == 0:
                        pi_, pj_ = ni + di, nj + dj
                    elif a == 0:
                        pi_, pj_ = ni, nj + q
                    else:
                        pi_, pj_ = ni + q, nj
                    src = Pn1[nj, ni] if isv(pi_, pj_) else Pn[nj, ni]
                    num += m * (src + step)
            out[j, i] = num / den
    return out


# --------------------------------------------------------------------------
# Whole straight rays (the rotating-parallel-ray integration the method takes
# to the limit of infinitely many rays, Section "Limit of Infinite Rays")
# --------------------------------------------------------------------------

def _line_cells_2d(x0, y0, ux, uy, nx, ny, hx, hy):
    """Cells crossed, in order, by the line (x0, y0) + t (ux, uy), t over all
    reals.  Cell (i, j) is the rectangle of half-widths hx/2, hy/2 about the
    node (i hx, j hy).  Each piece of the line between two consecutive grid
    lines lies in one cell, found from the piece's midpoint."""
    lo = (-0.5 * hx, -0.5 * hy)
    hi = ((nx - 0.5) * hx, (ny - 0.5) * hy)
    t0, t1 = -np.inf, np.inf
    for p, u, a, b in ((x0, ux, lo[0], hi[0]), (y0, uy, lo[1], hi[1])):
        if u == 0.0:
            if not a < p < b:
                return []
            continue
        ta, tb = (a - p) / u, (b - p) / u
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    if not t1 > t0:
        return []
    ts = [t0, t1]
    if ux != 0.0:
        ts += [t for t in (((k - 0.5) * hx - x0) / ux for k in range(nx + 1)) if t0 < t < t1]
    if uy != 0.0:
        ts += [t for t in (((k - 0.5) * hy - y0) / uy for k in range(ny + 1)) if t0 < t < t1]
    ts.sort()
    cells = []
    for a, b in zip(ts[:-1], ts[1:]):
        if b - a <= 1e-12 * (t1 - t0):
            continue
        tm = 0.5 * (a + b)
        i = min(max(int(math.floor((x0 + tm * ux) / hx + 0.5)), 0), nx - 1)
        j = min(max(int(math.floor((y0 + tm * uy) / hy + 0.5)), 0), ny - 1)
        if not cells or cells[-1] != (i, j):
            cells.append((i, j))
    return cells


def rotating_ray_map_2d(grid: Grid, f, n_theta: int, ds: float):
    """The averaging map of whole straight rays: P^{n+1} = R P^n + c.

    Lines at n_theta midpoint angles theta in [0, 2 pi) (each line traversed
    in the direction theta, so every line is also run backwards by theta +
    pi) and parallel offsets s spaced ds apart cover the grid.  Along a line,
    a ray starts at its first valid cell after a missing one (or after
    entering the array) with that cell's previous iterate P^n, and crossing
    the face from cell A into cell B adds the path step of Eq.
    PressureIntegrator1, (x_B - x_A)_a (f_a(A) + f_a(B)) / 2 along the face's
    axis a.  Each cell's new value is the mean, over every ray through it
    (each the same measure ds dtheta), of the ray's value there.
    Returns (R, c, vidx): R (valid x valid) and c on the valid cells vidx.
    Lines through a cell corner exactly (measure zero) are skipped."""
    if grid.ndim != 2:
        raise ValueError("2D only")
    nx, ny = int(grid.dims[0]), int(grid.dims[1])
    hx, hy = float(grid.h[0]), float(grid.h[1])
    valid = grid.valid
    f = np.asarray(f, dtype=np.float64)
    vidx = np.flatnonzero(valid.reshape(-1))
    pos = -np.ones(grid.n, dtype=np.int64)
    pos[vidx] = np.arange(vidx.size)
    R = np.zeros((vidx.size, vidx.size))
    c = np.zeros(vidx.size)
    cnt = np.zeros(vidx.size)
    xc, yc = 0.5 * (nx - 1) * hx, 0.5 * (ny - 1) * hy
    rad = 0.5 * math.hypot(nx * hx, ny * hy) + max(hx, hy)
    n_s = int(math.ceil(2 * rad / ds))
    for it in range(n_theta):
        th = (it + 0.5) * 2 * math.pi / n_theta
        ux, uy = math.cos(th), math.sin(th)
        for ks in range(n_s):
            s = -rad + (ks + 0.5) * ds
            cells = _line_cells_2d(xc - s * uy, yc + s * ux, ux, uy, nx, ny, hx, hy)
            if any(abs(a[0] - b[0]) + abs(a[1] - b[1]) != 1 for a, b in zip(cells[:-1], cells[1:])):
                continue  # passes through a corner
            start, acc, prev = -1, 0.0, None
            for i, j in cells:
                if not valid[j, i]:
                    start, prev = -1, None
                    continue
                q = pos[j * nx + i]
                if start < 0:
                    start, acc = q, 0.0
                else:
                    pi_, pj_ = prev
                    if pi_ != i:
                        acc += (i - pi_) * hx * 0.5 * (f[0, pj_, pi_] + f[0, j, i])
                    else:
                        acc += (j - pj_) * hy * 0.5 * (f[1, pj_, pi_] + f[1, j, i])
                R[q, start] += 1.0
                c[q] += acc
                cnt[q] += 1.0
                prev = (i, j)
    seen = cnt > 0
    R[seen] /= cnt[seen, None]
    c[seen] /= cnt[seen]
    return R, c, vidx


def rotating_ray_solve_2d(grid: Grid, f, n_theta: int, ds: float, tol: float = 1e-13, max_iter: int = 100000):
    """Iterate the whole-ray average P^{n+1} = R P^n + c (rotating_ray_map_2d)
    from P^0 = 0 until the gauged iterate stops changing.  The map moves the
    per-component constant by a fixed amount per iteration when c has a
    component along R's stationary distribution, so each iterate is gauged
    (per-component mean removed); the gauged iterates converge.
    Returns (P gauged with NaN on missing cells, iterations)."""
    R, c, vidx = rotating_ray_map_2d(grid, f, n_theta, ds)
    lab, nc = labels(grid)
    labv = lab.reshape(-1)[vidx]
    members = [labv == k for k in range(nc)]

    def gauge_v(x):
        for m in members:
            x[m] -= x[m].mean()
        return x

    P = np.zeros(vidx.size)
    n = 0
    for n in range(1, max_iter + 1):
        Pn = gauge_v(R @ P + c)
        done = np.linalg.norm(Pn - P) <= tol * max(np.linalg.norm(Pn), 1e-300)
        P = Pn
        if done:
            break
    out = np.full(grid.n, np.nan)
    out[vidx] = P
    return out.reshape(grid.valid.shape), n
