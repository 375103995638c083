"""Re-fit of the rational approximation of the Gaussian (Section 2.1, Step 2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

R(x) = a0 mu / (x^2 + mu^2) + sum_{l=1}^{L} [2 mu Re(a_l)(mu^2 + l^2 + x^2)
       + 2 l Im(a_l)(mu^2 + l^2 - x^2)] / [x^4 + 2(mu^2 - l^2) x^2 + (mu^2 + l^2)^2]
(eq. A(x,mu)) is linear in y = [a0, Re a_1..a_L, Im a_1..a_L]; the paper fits
it to psi_1(x) = exp(-x^2/4)/sqrt(4 pi) in least squares (eq. minl2approx) on
points chosen one at a time like Leja points, starting at x_1 = 0.  The paper
gives neither the number of points nor the candidate interval; this module
takes them as parameters ("parity unpinned" beyond the error level: the test
checks that the refit reaches the paper's accuracy, not that it reproduces
Table tab:coef_al digit by digit).
"""
import math

import numpy as np

from . import coeffs


def design_row(x, mu, L):
    x = np.asarray(x, dtype=np.float64)
    x2 = x * x
    cols = [mu / (x2 + mu * mu)]
    den = [x2 * x2 + 2.0 * (mu * mu - l * l) * x2 + (mu * mu + l * l) ** 2 for l in range(1, L + 1)]
    for l in range(1, L + 1):
        cols.append(2.0 * mu * (mu * mu + l * l + x2) / den[l - 1])
    for l in range(1, L + 1):
        cols.append(2.0 * l * (mu * mu + l * l - x2) / den[l - 1])
    return np.stack(cols, axis=-1)


def leja_points(K, xmax, n_candidates=20001):
    """Greedy Leja sequence on [0, xmax] (R is even), starting at 0: each new
    point maximises the product of distances to the points chosen so far."""
    cand = np.linspace(0.0, xmax, n_candidates)
    pts = [0.0]
    logd = np.log(np.abs(cand - 0.0) + 1e-300)
    for _ in range(K - 1):
        i = int(np.argmax(logd))
        pts.append(cand[i])
        logd += np.log(np.abs(cand - cand[i]) + 1e-300)
    return np.array(pts)


def refit(mu=None, L=coeffs.L, K=200, xmax=40.0):
    """Least-squares coefficients on K Leja points of [0, xmax]; returns a[-L..L]."""
    if mu is None:
        mu, _ = coeffs.table_a()
    x = leja_points(K, xmax)
    G = design_row(x, mu, L)
    rhs = np.exp(-x * x / 4.0) / math.sqrt(4.0 * math.pi)
    scale = np.max(np.abs(G), axis=0)
    y, *_ = np.linalg.lstsq(G / scale, rhs, rcond=None)
    y = y / scale
    a = np.zeros(2 * L + 1, dtype=np.complex128)
    a[L] = y[0]
    for l in range(1, L + 1):
        a[L + l] = complex(y[l], y[L + l])
        a[L - l] = np.conj(a[L + l])
    return mu, a
