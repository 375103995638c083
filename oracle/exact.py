"""Reference exponentials e^{tau A} f0 (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``expm_dense``: scipy.linalg.expm of the dense operator (Pade; the routine
  the paper compares against in Section 3.2), for tiny grids.
* ``exp_closed_form``: constant depth only.  Each Fourier mode evolves by the
  3x3 symbol B(k), whose characteristic polynomial is lambda^3 + omega^2 lambda
  with omega^2 = gH(|dx|^2 + |dy|^2) + f^2 |P|^2, so
  e^{tau B} = I + (sin(tau omega)/omega) B + ((1 - cos(tau omega))/omega^2) B^2
  (the omega -> 0 limit is I + tau B + tau^2 B^2 / 2).
* ``exp_closed_form_grid``: the same formula evaluated at every wavenumber at
  once with numpy arrays (for checking whole 2048 x 2048 fields), with
  1 - cos(t) written as 2 sin^2(t / 2), which is the same number without the
  cancellation at small t.
"""
import math

import numpy as np
import scipy.linalg

from . import operator as op


def expm_dense(A, f0, tau):
    """e^{tau A} f0 with scipy.linalg.expm on the dense matrix."""
    E = scipy.linalg.expm(tau * A.toarray())
    return E @ np.asarray(f0)


def omega2_of(B):
    """omega^2 = sum of the principal 2x2 minors of B (char. poly. coefficient)."""
    return float((-(B[0, 1] * B[1, 0]) - (B[0, 2] * B[2, 0]) - (B[1, 2] * B[2, 1])).real)


def exp_closed_form(state, tau, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0, symbol_fn=None):
    """e^{tau A} state for constant H; ``state`` is (3, ny, nx).  ``symbol_fn``
    (default: the C-grid symbol) maps (kx, ky, nx, ny, Lx, Ly, g, f, H) to B(k)."""
    state = np.asarray(state, dtype=np.complex128)
    _, ny, nx = state.shape
    fh = np.fft.fft2(state, axes=(1, 2))
    out = np.zeros_like(fh)
    I3 = np.eye(3)
    for ky in range(ny):
        for kx in range(nx):
            B = (symbol_fn or op.symbol)(kx, ky, nx, ny, Lx, Ly, g, f, H)
            w2 = omega2_of(B)
            w = math.sqrt(max(w2, 0.0))
            if w * tau < 1e-8:
                E = I3 + tau * B + 0.5 * tau * tau * (B @ B)
            else:
                E = I3 + (math.sin(tau * w) / w) * B + ((1.0 - math.cos(tau * w)) / w2) * (B @ B)
            out[:, ky, kx] = E @ fh[:, ky, kx]
    return np.fft.ifft2(out, axes=(1, 2))


def exp_closed_form_grid(state, tau, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0, spectrum=False):
    """e^{tau A} state for constant H at every wavenumber at once (C grid).

    Per wavenumber e^{tau B} fhat = fhat + (sin(tau w)/w) B fhat
    + (2 sin^2(tau w / 2)/w^2) B^2 fhat with w^2 the sum of the principal 2x2
    minors of B (characteristic polynomial lambda^3 + w^2 lambda); where
    tau w < 1e-8 the Taylor limit fhat + tau B fhat + tau^2/2 B^2 fhat.
    ``spectrum=True`` returns the result's 2-D DFT (3, ny, nx) instead of the
    field.  Pinned against ``exp_closed_form`` (one wavenumber at a time) and
    dense expm in tests/test_oracle_exact.py."""
    state = np.asarray(state, dtype=np.complex128)
    _, ny, nx = state.shape
    fh = np.fft.fft2(state, axes=(1, 2))
    B = op.symbol_grid(nx, ny, Lx, Ly, g, f, H)
    w2 = (-(B[0, 1] * B[1, 0]) - (B[0, 2] * B[2, 0]) - (B[1, 2] * B[2, 1])).real
    w = np.sqrt(np.maximum(w2, 0.0))
    Bf = np.einsum("ijyx,jyx->iyx", B, fh)
    BBf = np.einsum("ijyx,jyx->iyx", B, Bf)
    t = tau * w
    small = t < 1e-8
    ws = np.where(small, 1.0, w)
    s1 = np.where(small, tau, np.sin(t) / ws)
    s2 = np.where(small, 0.5 * tau * tau, 2.0 * np.sin(0.5 * t) ** 2 / (ws * ws))
    out = fh + s1[None] * Bf + s2[None] * BBf
    if spectrum:
        return out
    return np.fft.ifft2(out, axes=(1, 2))
