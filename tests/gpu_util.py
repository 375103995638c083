"""Helpers shared by the GPU parity tests (oracle calls + device plumbing)."""
import math

import numpy as np
import pytest

from oracle import coeffs as C
from oracle import operator as O
from oracle import rexi as R


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11607_gb300 import build as B

    B.build()
    return torch


def to_dev(torch, arr):
    return torch.from_numpy(np.ascontiguousarray(arr, dtype=np.complex128)).cuda()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def oracle_step(state, dt, M, real_input=True, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0, h=0.5, terms=None):
    _, ny, nx = state.shape
    A = O.cgrid_operator(nx, ny, Lx, Ly, g, f, H)
    out = R.rexii_apply_sparse(A, state.ravel(), dt, h, M, real_input=real_input, terms=terms)
    return out.reshape(state.shape)


TOL = {"fp64": 1e-10, "plain": 1e-10, "mixed": 1e-8}


# ---------------------------------------------------------------------------
# Error model of the Fourier path (used for the tolerances of the full-size
# and paper-reproduction tests).
#
# The step applies r(tau B(k)) per wavenumber, r(ix) = sum_n T_n(x) with the
# REXII terms T_n(x) = (c1_n h mu + c2_n (x + h n)) / ((h mu)^2 + (x + h n)^2)
# (eq. modifiedRexi).  B(k) is normal for H = g (skew-Hermitian), so by
# Theorem 1 with cond = 1 the per-wavenumber error is at most
#   eps_r + delta_pole  (relative to |fhat(k)|)  plus  delta_fft max_k |fhat(k)|,
# * eps_r = max_{|x| <= tau rho} |r(ix) - e^{ix}|: the approximation error,
#   evaluated by the oracle on a 0.02-spaced grid (r varies on the scale of the
#   pole distance h|mu| ~ 2.6), times 1.25;
# * delta_pole: rounding of the term sum.  Each term carries a relative error
#   of at most kt u and each accumulation step one of at most ks u of the
#   running partial sum S_k.  Treating these as independent zero-mean errors
#   (probabilistic rounding analysis, Higham and Mary 2019), the sum's error
#   exceeds lam u (kt sqrt(sum |T_n|^2) + ks sqrt(sum |S_k|^2)) with
#   probability at most 2 exp(-lam^2 / 2); lam = 8 (< 3e-14 per evaluation).
#   FP64 form: u = 2^-53, kt = 4 (rcp seed, two-term correction, two fma),
#   ks = 1.  Double-float form: u = 2^-48 (the pair's unit roundoff u32^2),
#   kt = 20: the quotient's low word is the remainder (n - T_h d) times the
#   FP32 reciprocal seed r0, so r0's error (<= 2 u32) times the remainder
#   (<= 1.5 u32 |T|) gives 6u, the remainder's three FP32 roundings 9u, and
#   the low words of numerator and denominator about 4u; ks = 20: the
#   accumulator's low word takes two FP32 roundings per term and grows by at
#   most u32 max|S| per term between renormalisations (every 16 terms), so the
#   k-th term after one adds at most (2k + 1) u max|S|, whose root mean square
#   over a block of 16 is 18.5.  The partial sums run over contiguous term
#   ranges, so sqrt(sum |S_k|^2) is bounded by 2 sqrt(n) max_k |cumulative
#   sum|.
# * delta_fft: the forward and inverse transforms (the library's and the
#   check's), lam kf u log2(nx ny) of the LARGEST wavenumber amplitude, kf = 8:
#   the butterflies spread the rounding of the large modes over every output,
#   so on a spectrum concentrated in a few modes (|k|^-3) the floor follows the
#   largest amplitude, not the rms (numpy's own transform of the |k|^-3 input
#   is Hermitian only to 1.2e-13 of the rms, 1.3e-16 of the largest mode).
# ---------------------------------------------------------------------------

_FORM_ROUNDING = {"fp64": (2.0 ** -53, 4.0, 1.0, 8.0), "mixed": (2.0 ** -48, 20.0, 20.0, 8.0),
                  "plain": (2.0 ** -53, 8.0, 1.0, 8.0)}
_LAM = 8.0


def scalar_error_max(tau_rho, h, M, step=0.02):
    """max_{0 <= x <= tau_rho} |r(ix) - e^{ix}| on a grid of spacing `step`
    (r(-ix) = conj r(ix), so the negative half adds nothing)."""
    x = np.arange(0.0, tau_rho + step, step)
    return float(np.max(np.abs(C.rexii_scalar(x, h, M) - np.exp(1j * x))))


def pole_rounding_bound(form, tau_rho, h, M):
    """delta_pole of the error model above, at the worse of x = 0 and x = tau_rho."""
    u, kt, ks, _ = _FORM_ROUNDING[form]
    mu, a = C.table_a()
    ns, c1, c2 = C.c_coeffs_sliced(h, M, mu, a)
    worst = 0.0
    for x in (0.0, float(tau_rho)):
        T = (c1 * h * mu + c2 * (x + h * ns)) / ((C.alpha(-ns, h, mu) - 1j * x) * (C.alpha(ns, h, mu) + 1j * x))
        sT = math.sqrt(float(np.sum(np.abs(T) ** 2)))
        sS = 2.0 * math.sqrt(len(T)) * float(np.max(np.abs(np.cumsum(T))))
        worst = max(worst, _LAM * u * (kt * sT + ks * sS))
    return worst


def fft_rounding_bound(form, nx, ny):
    """delta_fft of the error model above (relative to the largest amplitude)."""
    u, _, _, kf = _FORM_ROUNDING[form]
    return _LAM * kf * u * math.log2(nx * ny)
