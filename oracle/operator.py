"""Staggered C-grid linear rotating shallow-water operator (FP64, scipy.sparse).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 4 of arXiv 2008.11607 states the operator A for f = (eta, u, v):
eta_t = -(u_x + v_y), u_t = -eta_x + v, v_t = -eta_y - u on the doubly
periodic unit square.  This module discretises the dimensional form
eta_t = -H(x, y) (u_x + v_y), u_t = -g eta_x + f v, v_t = -g eta_y - f u on a
staggered (Arakawa C) grid with second-order centred differences:

* eta_{i,j} at ((i + 1/2) dx, (j + 1/2) dy), u_{i,j} at ((i + 1) dx, (j + 1/2) dy),
  v_{i,j} at ((i + 1/2) dx, (j + 1) dy); H is sampled at eta points.
* divergence at eta points uses backward differences of u and v;
  the gradient at u / v points uses forward differences of eta;
* Coriolis: v averaged over the four v points around a u point, and u over
  the four u points around a v point (the transpose of the first average), so
  that the discrete operator conserves the energy
  sum (g/H) eta^2 + u^2 + v^2.
The unknown vector is [eta.ravel(), u.ravel(), v.ravel()] with arrays shaped
(ny, nx), x (index i) fastest.  This module is "parity unpinned" on its own; the
tests pin it against the closed-form Fourier symbol, dense expm and the energy
invariant.
"""
import math

import numpy as np
import scipy.sparse as sp


def cgrid_operator(nx, ny, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0):
    """Return A as a scipy.sparse CSR matrix of size 3 nx ny (real FP64).

    ``H`` is a scalar or an (ny, nx) array of depths at eta points.
    """
    n = nx * ny
    dx = Lx / nx
    dy = Ly / ny
    Hf = np.broadcast_to(np.asarray(H, dtype=np.float64), (ny, nx))
    rows, cols, vals = [], [], []

    def idx(field, i, j):
        return field * n + (j % ny) * nx + (i % nx)

    def put(r, c, v):
        rows.append(r)
        cols.append(c)
        vals.append(v)

    for j in range(ny):
        for i in range(nx):
            # eta row: -H (  (u_{i,j} - u_{i-1,j}) / dx + (v_{i,j} - v_{i,j-1}) / dy )
            r = idx(0, i, j)
            h_ij = Hf[j, i]
            put(r, idx(1, i, j), -h_ij / dx)
            put(r, idx(1, i - 1, j), h_ij / dx)
            put(r, idx(2, i, j), -h_ij / dy)
            put(r, idx(2, i, j - 1), h_ij / dy)
            # u row: -g (eta_{i+1,j} - eta_{i,j}) / dx + f * avg4(v)
            r = idx(1, i, j)
            put(r, idx(0, i + 1, j), -g / dx)
            put(r, idx(0, i, j), g / dx)
            for (di, dj) in ((0, 0), (1, 0), (0, -1), (1, -1)):
                put(r, idx(2, i + di, j + dj), 0.25 * f)
            # v row: -g (eta_{i,j+1} - eta_{i,j}) / dy - f * avg4(u)
            r = idx(2, i, j)
            put(r, idx(0, i, j + 1), -g / dy)
            put(r, idx(0, i, j), g / dy)
            for (di, dj) in ((0, 0), (-1, 0), (0, 1), (-1, 1)):
                put(r, idx(1, i + di, j + dj), -0.25 * f)
    A = sp.coo_matrix((vals, (rows, cols)), shape=(3 * n, 3 * n)).tocsr()
    A.sum_duplicates()
    return A


def energy_weight(nx, ny, g=1.0, H=1.0):
    """Diagonal of the weight W = diag(g/H, 1, 1) in which A is skew."""
    Hf = np.broadcast_to(np.asarray(H, dtype=np.float64), (ny, nx)).ravel()
    return np.concatenate([g / Hf, np.ones(nx * ny), np.ones(nx * ny)])


def symbol(kx, ky, nx, ny, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0):
    """Fourier symbol B(k) (3x3 complex) of the constant-depth C-grid operator.

    With the DFT convention fhat_k = sum_j f_j e^{-2 pi i k j / n}, a shift by
    +1 multiplies by e^{i theta}.  Forward difference (e^{i theta} - 1)/dx,
    backward difference (1 - e^{-i theta})/dx, four-point average
    P = (1 + e^{i theta_x})(1 + e^{-i theta_y}) / 4 (v to u) and conj(P) (u to v).
    """
    dx = Lx / nx
    dy = Ly / ny
    tx = 2.0 * math.pi * kx / nx
    ty = 2.0 * math.pi * ky / ny
    ex, ey = np.exp(1j * tx), np.exp(1j * ty)
    dxf = (ex - 1.0) / dx
    dyf = (ey - 1.0) / dy
    dxb = (1.0 - 1.0 / ex) / dx
    dyb = (1.0 - 1.0 / ey) / dy
    P = (1.0 + ex) * (1.0 + 1.0 / ey) / 4.0
    Pu = (1.0 + 1.0 / ex) * (1.0 + ey) / 4.0
    return np.array([[0.0, -H * dxb, -H * dyb],
                     [-g * dxf, 0.0, f * P],
                     [-g * dyf, -f * Pu, 0.0]], dtype=np.complex128)


def spectral_radius_constant(nx, ny, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0):
    """rho(A) for constant H: the largest |eigenvalue| of B(k) over the k grid.

    Computed by brute force with numpy eigenvalues on every wavenumber (slow,
    plain); meant for small grids in tests.
    """
    best = 0.0
    for ky in range(ny):
        for kx in range(nx):
            ev = np.linalg.eigvals(symbol(kx, ky, nx, ny, Lx, Ly, g, f, H))
            best = max(best, float(np.max(np.abs(ev))))
    return best


def spectral_radius_bound(nx, ny, Lx=1.0, Ly=1.0, g=1.0, f=1.0, Hmax=1.0):
    """Upper bound rho(A) <= sqrt(g Hmax (4/dx^2 + 4/dy^2)) + |f| for variable depth.

    In the variables (sqrt(g/H) eta, u, v) the wave part is skew with norm at
    most sqrt(g Hmax) times the norm of the discrete gradient (<= sqrt(4/dx^2 +
    4/dy^2)), and the Coriolis part has norm at most |f|.
    """
    dx = Lx / nx
    dy = Ly / ny
    return math.sqrt(g * Hmax * (4.0 / dx ** 2 + 4.0 / dy ** 2)) + abs(f)


def symbol_grid(nx, ny, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0):
    """B(k) at every wavenumber at once: a (3, 3, ny, nx) complex array whose
    [:, :, ky, kx] slice equals ``symbol(kx, ky, ...)``.  The same entries as
    ``symbol`` (Section 4 operator on the C grid: forward/backward differences
    and the four-point Coriolis average), written with numpy broadcasting so
    that large grids can be checked field-wide."""
    dx = Lx / nx
    dy = Ly / ny
    tx = 2.0 * np.pi * np.arange(nx) / nx
    ty = 2.0 * np.pi * np.arange(ny) / ny
    ex = np.exp(1j * tx)[None, :]
    ey = np.exp(1j * ty)[:, None]
    one = np.ones((ny, nx))
    dxf = (ex - 1.0) / dx * one
    dyf = (ey - 1.0) / dy * one
    dxb = (1.0 - 1.0 / ex) / dx * one
    dyb = (1.0 - 1.0 / ey) / dy * one
    P = (1.0 + ex) * (1.0 + 1.0 / ey) / 4.0
    Pu = (1.0 + 1.0 / ex) * (1.0 + ey) / 4.0
    B = np.zeros((3, 3, ny, nx), dtype=np.complex128)
    B[0, 1] = -H * dxb
    B[0, 2] = -H * dyb
    B[1, 0] = -g * dxf
    B[1, 2] = f * P
    B[2, 0] = -g * dyf
    B[2, 1] = -f * Pu
    return B


def schrodinger_operator(nx, ny, Lx=1.0, Ly=1.0):
    """A = i (d_xx + d_yy) by second-order centred differences with periodic
    boundaries on an nx x ny grid (x fastest), as a complex scipy.sparse CSR
    matrix of size nx ny.  With ny = 1 this is the paper's A_2 of Section 3.2
    (the free Schroedinger operator; on [-1, 1] with step 1/35, nx = 70, its
    eigenvalues lie in i[-4900, 0])."""
    n = nx * ny
    dx = Lx / nx
    dy = Ly / ny
    rows, cols, vals = [], [], []
    for j in range(ny):
        for i in range(nx):
            r = j * nx + i
            for di, dj, w in ((1, 0, 1.0 / dx ** 2), (-1, 0, 1.0 / dx ** 2), (0, 1, 1.0 / dy ** 2),
                              (0, -1, 1.0 / dy ** 2), (0, 0, -2.0 / dx ** 2 - 2.0 / dy ** 2)):
                if ny == 1 and dj != 0:
                    continue
                if ny == 1 and di == 0 and dj == 0:
                    w = -2.0 / dx ** 2
                rows.append(r)
                cols.append(((j + dj) % ny) * nx + (i + di) % nx)
                vals.append(1j * w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n), dtype=np.complex128)
