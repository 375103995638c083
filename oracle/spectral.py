"""Spectral-derivative LRSW operator on a collocated periodic grid (the
discretisation behind eq. lswRoh of Section 4), for the paper-reproduction
checks.  TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

d/dx acts on each Fourier mode as multiplication by i k', k' = 2 pi k / Lx with
the signed wavenumber k in (-n/2, n/2] (the Nyquist mode taken as +n/2, the
convention of the library's spectral symbol).  The operator is
A = [[0, -H d/dx, -H d/dy], [-g d/dx, 0, f], [-g d/dy, -f, 0]].
"""
import math

import numpy as np
import scipy.sparse as sp


def signed_wavenumbers(n, L):
    k = np.arange(n)
    ks = np.where(2 * k <= n, k, k - n)
    return 2.0 * math.pi * ks / L


def derivative_matrix(n, L):
    """Dense n x n matrix of the spectral derivative (F^{-1} diag(i k') F)."""
    F = np.fft.fft(np.eye(n), axis=0)
    Finv = np.fft.ifft(np.eye(n), axis=0)
    return Finv @ np.diag(1j * signed_wavenumbers(n, L)) @ F


def spectral_operator(nx, ny, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0):
    """A as a (complex) scipy.sparse CSR matrix of size 3 nx ny, state order
    [eta, u, v], each (ny, nx) with x fastest."""
    Dx = np.kron(np.eye(ny), derivative_matrix(nx, Lx))
    Dy = np.kron(derivative_matrix(ny, Ly), np.eye(nx))
    n = nx * ny
    I = np.eye(n)
    Z = np.zeros((n, n))
    A = np.block([[Z, -H * Dx, -H * Dy], [-g * Dx, Z, f * I], [-g * Dy, -f * I, Z]])
    return sp.csr_matrix(A)


def symbol(kx, ky, nx, ny, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0):
    """3x3 symbol of the spectral operator at wavenumber index (kx, ky)."""
    a = signed_wavenumbers(nx, Lx)[kx]
    b = signed_wavenumbers(ny, Ly)[ky]
    return np.array([[0.0, -H * 1j * a, -H * 1j * b],
                     [-g * 1j * a, 0.0, f],
                     [-g * 1j * b, -f, 0.0]], dtype=np.complex128)


def spectral_radius(nx, ny, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0):
    """max over the discrete wavenumbers of omega = sqrt(gH |k'|^2 + f^2)."""
    a = np.max(np.abs(signed_wavenumbers(nx, Lx)))
    b = np.max(np.abs(signed_wavenumbers(ny, Ly)))
    return math.sqrt(g * H * (a * a + b * b) + f * f)
