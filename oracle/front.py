"""FP64 CPU oracle of the source-term front ends: the pressure gradient f that
the integration consumes, computed from velocity data.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the product library
never imports or calls it, and it imports nothing from the product package.

The paper lumps the right-hand side of the momentum balance into a "source
term" f(u) and integrates it; it uses three forms:

* ``incompressible``  Eq. 1 (Section 1): f = -rho (du/dt + (u . grad) u)
                      + mu lap u, from time-resolved snapshots;
* ``rans``            Eq. RANS_f (Section 3.3): f_i = -rho (U_j dU_i/dx_j
                      + d<u_i' u_j'>/dx_j), from the mean velocity and the
                      Reynolds stresses, viscous terms dropped;
* ``compressible``    Eq. compressible-pressure (Section 3.4): the 3 x 3 (or
                      2 x 2) system (delta_ij + <u_i u_j>/(R T)) g_j =
                      -(1/(R T)) (d<u_i u_j>/dx_j - <u_i u_j>/T dT/dx_j) for
                      g = grad ln(P / P_inf), with <u_i u_j> = U_i U_j +
                      <u_i' u_j'> and T from the adiabatic relation
                      T / T_inf = 1 + (gamma - 1)/2 M_inf^2 (1 - |U|^2 / V_inf^2).

The paper does not state its finite-difference scheme.  The reading used on
both sides: on a valid cell, the derivative along an axis is the centred
difference when both neighbours on that axis are valid; otherwise the
second-order one-sided three-point difference towards the valid side when the
next cell on that side is valid too, else the two-point difference, else 0.
The second derivative is the centred three-point formula, else the
three-point one-sided formula, else 0.  Derivatives of products (the
conservative terms) difference the product field.  Missing cells get f = 0
(the integration never reads them).

Arrays are (ny, nx) in 2D and (nz, ny, nx) in 3D; vector and tensor fields
carry a leading component axis (x, y[, z]; stresses xx, yy, [zz,] xy[, xz,
yz]).
"""
from __future__ import annotations

import numpy as np


def _shift(a, axis, k, fill):
    """out[i] = a[i + k] along ``axis`` (numpy axis), ``fill`` outside."""
    out = np.full_like(a, fill)
    n = a.shape[axis]
    if abs(k) >= n:
        return out
    src = [slice(None)] * a.ndim
    dst = [slice(None)] * a.ndim
    if k > 0:
        src[axis], dst[axis] = slice(k, None), slice(0, n - k)
    else:
        src[axis], dst[axis] = slice(0, n + k), slice(-k, None)
    out[tuple(dst)] = a[tuple(src)]
    return out


def _naxis(valid, a):
    """numpy axis of spatial axis a (0 = x, 1 = y, 2 = z)."""
    return valid.ndim - 1 - a


def d1(q, valid, a, h):
    """dq/dx_a by the rule in the module docstring."""
    ax = _naxis(valid, a)
    q = np.asarray(q, dtype=np.float64)
    vp, vm = _shift(valid, ax, 1, False), _shift(valid, ax, -1, False)
    vpp, vmm = _shift(valid, ax, 2, False), _shift(valid, ax, -2, False)
    qp, qm = _shift(q, ax, 1, 0.0), _shift(q, ax, -1, 0.0)
    qpp, qmm = _shift(q, ax, 2, 0.0), _shift(q, ax, -2, 0.0)
    out = np.zeros_like(q)
    central = vp & vm
    plus3 = ~central & vp & vpp
    plus2 = ~central & vp & ~vpp
    minus3 = ~central & ~vp & vm & vmm
    minus2 = ~central & ~vp & vm & ~vmm
    out[central] = (qp - qm)[central] / (2 * h)
    out[plus3] = (-3 * q + 4 * qp - qpp)[plus3] / (2 * h)
    out[plus2] = (qp - q)[plus2] / h
    out[minus3] = (3 * q - 4 * qm + qmm)[minus3] / (2 * h)
    out[minus2] = (q - qm)[minus2] / h
    out[~valid] = 0.0
    return out


def d2(q, valid, a, h):
    """d^2 q / dx_a^2 by the rule in the module docstring."""
    ax = _naxis(valid, a)
    q = np.asarray(q, dtype=np.float64)
    vp, vm = _shift(valid, ax, 1, False), _shift(valid, ax, -1, False)
    vpp, vmm = _shift(valid, ax, 2, False), _shift(valid, ax, -2, False)
    qp, qm = _shift(q, ax, 1, 0.0), _shift(q, ax, -1, 0.0)
    qpp, qmm = _shift(q, ax, 2, 0.0), _shift(q, ax, -2, 0.0)
    out = np.zeros_like(q)
    central = vp & vm
    plus = ~central & vp & vpp
    minus = ~central & ~plus & vm & vmm
    out[central] = (qp - 2 * q + qm)[central] / (h * h)
    out[plus] = (q - 2 * qp + qpp)[plus] / (h * h)
    out[minus] = (q - 2 * qm + qmm)[minus] / (h * h)
    out[~valid] = 0.0
    return out


def stress_index(ndim):
    """(i, j) -> plane of the symmetric stress input."""
    if ndim == 2:
        pairs = [(0, 0), (1, 1), (0, 1)]
    else:
        pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    idx = {}
    for k, (i, j) in enumerate(pairs):
        idx[(i, j)] = idx[(j, i)] = k
    return idx


def incompressible(valid, spacing, u, u_prev=None, u_next=None, dt=1.0, rho=1.0, mu=0.0):
    """Eq. 1: f = -rho (du/dt + (u . grad) u) + mu lap u.  du/dt is the
    centred difference of the neighbouring snapshots when both are given,
    the one-sided difference with the one given, else 0 (steady)."""
    valid = np.asarray(valid, bool)
    nd = valid.ndim
    u = np.asarray(u, dtype=np.float64)
    f = np.zeros_like(u)
    for i in range(nd):
        if u_prev is not None and u_next is not None:
            dudt = (np.asarray(u_next[i], np.float64) - np.asarray(u_prev[i], np.float64)) / (2 * dt)
        elif u_next is not None:
            dudt = (np.asarray(u_next[i], np.float64) - u[i]) / dt
        elif u_prev is not None:
            dudt = (u[i] - np.asarray(u_prev[i], np.float64)) / dt
        else:
            dudt = np.zeros_like(u[i])
        conv = sum(u[j] * d1(u[i], valid, j, spacing[j]) for j in range(nd))
        lap = sum(d2(u[i], valid, j, spacing[j]) for j in range(nd))
        f[i] = -rho * (dudt + conv) + mu * lap
        f[i][~valid] = 0.0
    return f


def rans(valid, spacing, U, stress, rho=1.0):
    """Eq. RANS_f: f_i = -rho (U_j dU_i/dx_j + d<u_i' u_j'>/dx_j)."""
    valid = np.asarray(valid, bool)
    nd = valid.ndim
    U = np.asarray(U, dtype=np.float64)
    R = np.asarray(stress, dtype=np.float64)
    si = stress_index(nd)
    f = np.zeros_like(U)
    for i in range(nd):
        conv = sum(U[j] * d1(U[i], valid, j, spacing[j]) for j in range(nd))
        div = sum(d1(R[si[(i, j)]], valid, j, spacing[j]) for j in range(nd))
        f[i] = -rho * (conv + div)
        f[i][~valid] = 0.0
    return f


def temperature(U, gamma, mach_inf, v_inf, t_inf):
    """T = T_inf (1 + (gamma - 1)/2 M_inf^2 (1 - |U|^2 / V_inf^2))."""
    U = np.asarray(U, dtype=np.float64)
    v2 = np.sum(U * U, axis=0)
    return t_inf * (1.0 + 0.5 * (gamma - 1.0) * mach_inf ** 2 * (1.0 - v2 / v_inf ** 2))


def compressible(valid, spacing, U, stress, gamma, mach_inf, v_inf, t_inf, r_gas):
    """Eq. compressible-pressure solved per cell for g = grad ln(P / P_inf).
    Returns (g, T)."""
    valid = np.asarray(valid, bool)
    nd = valid.ndim
    U = np.asarray(U, dtype=np.float64)
    R = np.asarray(stress, dtype=np.float64)
    si = stress_index(nd)
    T = temperature(U, gamma, mach_inf, v_inf, t_inf)
    uu = {}
    for i in range(nd):
        for j in range(nd):
            uu[(i, j)] = U[i] * U[j] + R[si[(i, j)]]
    dT = [d1(T, valid, j, spacing[j]) for j in range(nd)]
    rhs = np.zeros_like(U)
    for i in range(nd):
        div = sum(d1(uu[(i, j)], valid, j, spacing[j]) for j in range(nd))
        corr = sum(uu[(i, j)] * dT[j] for j in range(nd)) / T
        rhs[i] = -(div - corr) / (r_gas * T)
    g = np.zeros_like(U)
    vidx = np.argwhere(valid)
    for c in map(tuple, vidx):
        A = np.eye(nd)
        for i in range(nd):
            for j in range(nd):
                A[i, j] += uu[(i, j)][c] / (r_gas * T[c])
        g[(slice(None),) + c] = np.linalg.solve(A, rhs[(slice(None),) + c])
    return g, T
