"""Adjoint of the REXII step and its gradient with respect to the depth field
(FP64, scipy).  TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

With the single-shift form r(tau A) = sum_j beta_j (tau A - z_j)^{-1}
(partial fractions of the terms of eq. REXI_Modified_matrix; for real input
the reduced set of eq. modifiedRexiMatrixReducedSum and a real part), a real
loss L of out = r(tau A) f with G = dL/d out (G = dL/dRe + i dL/dIm) has
  dL/d f  = r(tau A)^H G,
  dL/d H_k = tau Re sum_j beta_j conj(y_{j, eta, k}) (div x_j)_k,
with x_j = (tau A - z_j)^{-1} f and y_j = (tau A - z_j)^{-H} G, because the
depth enters A only through the eta row, (A v)_eta = -H (div v).  Every solve
is a sparse LU, one pole at a time.  Pinned in the tests against central
finite differences of the oracle's forward step.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import coeffs
from . import operator as op


def divergence(v, nx, ny, Lx=1.0, Ly=1.0):
    """(u_{i,j} - u_{i-1,j}) / dx + (v_{i,j} - v_{i,j-1}) / dy at eta points; v is
    the stacked (eta, u, v) vector."""
    n = nx * ny
    u = v[n:2 * n].reshape(ny, nx)
    w = v[2 * n:].reshape(ny, nx)
    return ((u - np.roll(u, 1, axis=1)) * (nx / Lx) + (w - np.roll(w, 1, axis=0)) * (ny / Ly)).ravel()


def rexii_adjoint_sparse(A, G, tau, h, M, real_input=True):
    """r(tau A)^H G by one sparse LU per pole of the conjugate-transposed shifts."""
    poles, weights = coeffs.single_shift_poles(h, M, real_input)
    n_unk = A.shape[0]
    Id = sp.identity(n_unk, dtype=np.complex128, format="csc")
    AH = sp.csc_matrix(A.T, dtype=np.complex128)
    acc = np.zeros(n_unk, dtype=np.complex128)
    for z, w in zip(poles, weights):
        acc += np.conj(w) * spla.splu((tau * AH - np.conj(z) * Id).tocsc()).solve(np.asarray(G, np.complex128))
    return acc.real.astype(np.complex128) if real_input else acc


def grad_depth_sparse(nx, ny, H, f0, G, tau, h, M, Lx=1.0, Ly=1.0, g=1.0, f=1.0, real_input=True):
    """dL/dH at eta points for one step out = r(tau A(H)) f0 with dL/d out = G."""
    A = op.cgrid_operator(nx, ny, Lx, Ly, g, f, H)
    poles, weights = coeffs.single_shift_poles(h, M, real_input)
    n_unk = A.shape[0]
    n = nx * ny
    Id = sp.identity(n_unk, dtype=np.complex128, format="csc")
    Ac = sp.csc_matrix(A, dtype=np.complex128)
    grad = np.zeros(n)
    f0 = np.asarray(f0, np.complex128)
    G = np.asarray(G, np.complex128)
    for z, w in zip(poles, weights):
        lu = spla.splu((tau * Ac - z * Id).tocsc())
        x = lu.solve(f0)
        y = lu.solve(G, trans="H")
        grad += tau * np.real(w * np.conj(y[:n]) * divergence(x, nx, ny, Lx, Ly))
    return grad.reshape(ny, nx)
