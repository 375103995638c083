"""Reference exponentials e^{tau A} f0 (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``expm_dense``: scipy.linalg.expm of the dense operator (Pade; the routine
  the paper compares against in Section 3.2), for tiny grids.
* ``exp_closed_form``: constant depth only.  Each Fourier mode evolves by the
  3x3 symbol B(k), whose characteristic polynomial is lambda^3 + omega^2 lambda
  with omega^2 = gH(|dx|^2 + |dy|^2) + f^2 |P|^2, so
  e^{tau B} = I + (sin(tau omega)/omega) B + ((1 - cos(tau omega))/omega^2) B^2
  (the omega -> 0 limit is I + tau B + tau^2 B^2 / 2).
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
