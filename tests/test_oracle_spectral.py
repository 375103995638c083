"""Pins for the spectral-derivative operator used to reproduce Section 4."""
import math

import numpy as np

from oracle import exact as E
from oracle import spectral as S


def test_derivative_exact_on_resolved_modes():
    n = 16
    x = np.arange(n) / n
    D = S.derivative_matrix(n, 1.0)
    for m in (1, 3, 7):
        assert np.max(np.abs(D @ np.sin(2 * math.pi * m * x) - 2 * math.pi * m * np.cos(2 * math.pi * m * x))) < 1e-11


def test_spectral_radius_matches_lswRoh():
    """eq. lswRoh: rho = sqrt(2 pi^2 D^2 + 1) on the unit square, H = g = f = 1."""
    for D in (6, 8):
        A = S.spectral_operator(D, D)
        rho = np.max(np.abs(np.linalg.eigvals(A.toarray())))
        assert abs(rho - math.sqrt(2 * math.pi ** 2 * D * D + 1)) < 1e-9
        assert abs(S.spectral_radius(D, D) - rho) < 1e-9


def test_closed_form_matches_expm_spectral():
    nx, ny = 6, 5
    A = S.spectral_operator(nx, ny, 1.1, 0.9, 1.3, 0.7, 0.8)
    st = np.random.default_rng(0).standard_normal((3, ny, nx)) + 0j
    ref = E.expm_dense(A, st.ravel(), 0.07)
    cf = E.exp_closed_form(st, 0.07, 1.1, 0.9, 1.3, 0.7, 0.8, symbol_fn=S.symbol).ravel()
    assert np.linalg.norm(cf - ref) / np.linalg.norm(ref) < 1e-12
