"""Pins for the oracle's operator and matrix REXII (CPU only).

The references are independent of the oracle's REXII arithmetic: dense
scipy.linalg.expm (Pade), the closed-form exponential of the 3x3 Fourier
symbol, exact invariants of the continuous problem (energy, semigroup,
linearity) and Theorem 1 of the paper.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import coeffs as C
from oracle import exact as E
from oracle import operator as O
from oracle import rexi as R
from paper_2008_11607_gb300 import inputs


def _wnorm(v, w):
    return math.sqrt(float(np.sum(w * np.abs(v) ** 2)))


def test_operator_is_skew_in_energy_weight():
    """W A is skew-symmetric for W = diag(g/H, 1, 1): the discrete energy is conserved."""
    H = inputs.variable_depth(10, 8, seed=3)
    A = O.cgrid_operator(10, 8, Lx=1.3, Ly=0.9, g=2.0, f=0.7, H=H)
    W = sp.diags(O.energy_weight(10, 8, g=2.0, H=H))
    S = (W @ A).toarray()
    assert np.max(np.abs(S + S.T)) < 1e-12 * np.max(np.abs(S))


def test_spectral_radius_closed_form():
    """H = g = f = 1 on the unit square: rho(A) = 2 sqrt(2) D for even D, and the
    dense eigenvalues are imaginary (sigma(A) in iR, Section 1)."""
    for D in (8, 12):
        A = O.cgrid_operator(D, D)
        ev = np.linalg.eigvals(A.toarray())
        assert np.max(np.abs(ev.real)) < 1e-10
        assert abs(np.max(np.abs(ev)) - 2 * math.sqrt(2) * D) < 1e-9
        assert abs(O.spectral_radius_constant(D, D) - 2 * math.sqrt(2) * D) < 1e-9


def test_spectral_radius_bound_variable_depth():
    H = inputs.variable_depth(12, 12, seed=0)
    A = O.cgrid_operator(12, 12, H=H)
    ev = np.linalg.eigvals(A.toarray())
    rho = np.max(np.abs(ev))
    assert np.max(np.abs(ev.real)) < 1e-9
    assert rho <= O.spectral_radius_bound(12, 12, Hmax=H.max()) + 1e-9


def test_symbol_matches_operator_on_fourier_modes():
    """A applied to a single Fourier mode equals B(k) times the mode."""
    nx, ny, Lx, Ly, g, f, H = 6, 5, 1.2, 0.8, 1.5, 0.6, 2.0
    A = O.cgrid_operator(nx, ny, Lx, Ly, g, f, H)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for kx, ky in ((0, 0), (1, 2), (5, 4), (3, 0)):
        mode = np.exp(2j * math.pi * (kx * ii / nx + ky * jj / ny))
        B = O.symbol(kx, ky, nx, ny, Lx, Ly, g, f, H)
        for c in range(3):
            vec = np.zeros((3, ny, nx), dtype=np.complex128)
            vec[c] = mode
            out = (A @ vec.ravel()).reshape(3, ny, nx)
            for r in range(3):
                assert np.max(np.abs(out[r] - B[r, c] * mode)) < 1e-11


def test_closed_form_exponential_matches_expm():
    nx, ny = 8, 6
    A = O.cgrid_operator(nx, ny, 1.0, 0.75, 1.3, 0.8, 0.9)
    f0 = inputs.complex_random_state(nx, ny, seed=1)
    tau = 0.05
    ref = E.expm_dense(A, f0.ravel(), tau)
    cf = E.exp_closed_form(f0, tau, 1.0, 0.75, 1.3, 0.8, 0.9).ravel()
    assert np.linalg.norm(cf - ref) / np.linalg.norm(ref) < 1e-13


@pytest.mark.parametrize("real_input", [True, False])
def test_rexii_chain_matches_expm_constant_depth(real_input):
    """eq. matrixAccuracyBound: with tau rho <= (M - 11) h the matrix REXII is at
    the scalar accuracy (Theorem 1; cond = 1 for a normal operator)."""
    D = 8
    A = O.cgrid_operator(D, D)
    rho = 2 * math.sqrt(2) * D
    tau = 20.0 / rho
    M = C.pole_count_M(tau * rho, 0.5, 1e-16)
    f0 = inputs.gaussian_bump(D, D, width=0.15) if real_input else inputs.complex_random_state(D, D, 2)
    ref = E.expm_dense(A, f0.ravel(), tau)
    out = R.rexii_apply_sparse(A, f0.ravel(), tau, 0.5, M, real_input=real_input)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-12


def test_rexii_chain_matches_expm_variable_depth():
    nx, ny = 8, 8
    H = inputs.variable_depth(nx, ny, seed=5)
    A = O.cgrid_operator(nx, ny, H=H, f=1.0)
    ev = np.linalg.eigvals(A.toarray())
    rho = float(np.max(np.abs(ev)))
    tau = 30.0 / rho
    M = C.pole_count_M(tau * rho, 0.5, 1e-16)
    f0 = inputs.kminus3_field(nx, ny, seed=0)
    ref = E.expm_dense(A, f0.ravel(), tau)
    out = R.rexii_apply_sparse(A, f0.ravel(), tau, 0.5, M)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-12


def test_theorem1_bound_in_energy_norm():
    """Theorem 1 with cond(V) = 1 (skew in the W inner product): the W-norm error
    is at most max_j |REXII(i tau lambda_j) - e^{i tau lambda_j}| ||f0||_W."""
    nx = ny = 6
    H = inputs.variable_depth(nx, ny, seed=7)
    A = O.cgrid_operator(nx, ny, H=H)
    w = O.energy_weight(nx, ny, H=H)
    lam = np.linalg.eigvals(A.toarray()).imag
    tau = 0.9
    h = 0.5
    M = 25  # deliberately short so the scalar error is large and the bound is tight
    scalar_err = np.max(np.abs(C.rexii_scalar(tau * lam, h, M) - np.exp(1j * tau * lam)))
    f0 = inputs.complex_random_state(nx, ny, 4).ravel()
    err = E.expm_dense(A, f0, tau) - R.rexii_apply_sparse(A, f0, tau, h, M, real_input=False)
    assert scalar_err > 1e-6
    assert _wnorm(err, w) <= scalar_err * _wnorm(f0, w) * (1 + 1e-9)


def test_partial_fraction_poles_equal_chain():
    D = 6
    A = O.cgrid_operator(D, D, f=0.5)
    tau, M = 0.4, 20
    f0 = inputs.kminus3_field(D, D, seed=3).ravel()
    a = R.rexii_apply_sparse(A, f0, tau, 0.5, M)
    b = R.rexii_apply_poles(A, f0, tau, 0.5, M)
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-12


def test_energy_semigroup_linearity():
    nx = ny = 8
    H = inputs.variable_depth(nx, ny, seed=1)
    A = O.cgrid_operator(nx, ny, H=H)
    w = O.energy_weight(nx, ny, H=H)
    rho = O.spectral_radius_bound(nx, ny, Hmax=H.max())
    t1, t2 = 10.0 / rho, 14.0 / rho
    M = lambda t: C.pole_count_M(t * rho, 0.5, 1e-16)
    f0 = inputs.kminus3_field(nx, ny, seed=9).ravel()
    g0 = inputs.gaussian_bump(nx, ny, width=0.2).ravel()
    r1 = R.rexii_apply_sparse(A, f0, t1, 0.5, M(t1))
    assert abs(_wnorm(r1, w) - _wnorm(f0, w)) < 1e-12 * _wnorm(f0, w)
    r12 = R.rexii_apply_sparse(A, r1, t2, 0.5, M(t2))
    r3 = R.rexii_apply_sparse(A, f0, t1 + t2, 0.5, M(t1 + t2))
    assert np.linalg.norm(r12 - r3) / np.linalg.norm(r3) < 1e-12
    lin = R.rexii_apply_sparse(A, 2.0 * f0 - 3.0 * g0, t1, 0.5, M(t1))
    sep = 2.0 * r1 - 3.0 * R.rexii_apply_sparse(A, g0, t1, 0.5, M(t1))
    assert np.linalg.norm(lin - sep) / np.linalg.norm(sep) < 1e-13


def test_mean_height_mode_scaled_by_r0():
    """At k = 0 the eta row and column of B vanish, so the mean of eta is
    multiplied by REXII(0) (= 1 to the scalar accuracy)."""
    D = 8
    A = O.cgrid_operator(D, D)
    f0 = inputs.kminus3_field(D, D, seed=2)
    f0[0] += 0.3
    tau = 5.0
    M = C.pole_count_M(tau * 2 * math.sqrt(2) * D, 0.5, 1e-16)
    out = R.rexii_apply_sparse(A, f0.ravel(), tau, 0.5, M).reshape(3, D, D)
    r0 = complex(C.rexii_scalar(np.array([0.0]), 0.5, M)[0])
    assert abs(out[0].mean() - r0.real * f0[0].mean()) < 1e-13
    assert abs(r0 - 1.0) < 1e-13


def test_first_matrix_example_A1():
    """Section 3.2, matrix A_1: second-order periodic FD of d/dx on [0, 1] with
    step 1/70, f0 = 1/(2 + cos 2 pi x); REXII (reduced sum) against expm reaches
    ~1e-13 once rho(A_1) <= (M - 11) h (Fig. 2a as described in the text)."""
    n = 70
    dx = 1.0 / n
    x = np.arange(n) * dx
    A1 = sp.diags([np.full(n - 1, 0.5 / dx), np.full(n - 1, -0.5 / dx)], [1, -1]).tolil()
    A1[0, n - 1] = -0.5 / dx
    A1[n - 1, 0] = 0.5 / dx
    A1 = A1.tocsr()
    ev = np.linalg.eigvals(A1.toarray())
    rho = float(np.max(np.abs(ev)))
    # eigenvalues i sin(2 pi k / 70) / dx lie in i[-70, 70]; the largest is 69.93
    assert np.max(np.abs(ev.real)) < 1e-10 and 69.9 < rho <= 70.0
    f0 = 1.0 / (2.0 + np.cos(2 * math.pi * x))
    ref = E.expm_dense(A1, f0, 1.0)
    h = 0.5
    M_ok = C.pole_count_M(rho, h, 1e-16)
    good = R.rexii_apply_sparse(A1, f0, 1.0, h, M_ok)
    assert np.linalg.norm(good - ref) / np.linalg.norm(ref) < 1e-12
    bad = R.rexii_apply_sparse(A1, f0, 1.0, h, M_ok - 40)
    # f0 is smooth, so the modes near rho carry little weight; 40 terms short of
    # the rule the error is still ~7e-7, far above the converged level
    assert np.linalg.norm(bad - ref) / np.linalg.norm(ref) > 1e-8


def test_single_mode_chain_matches_closed_form():
    """The per-term chain on one 3x3 Fourier symbol (used for sampled checks of
    large grids) against the closed-form exponential of that symbol."""
    D = 2048
    tau = 1000.0 / (2 * math.sqrt(2) * D)
    M = C.pole_count_M(1000.0, 0.5, 1e-10)
    rng = np.random.default_rng(0)
    for kx, ky in ((0, 0), (1, 0), (1024, 1024), (700, 3), (2047, 1500)):
        B = O.symbol(kx, ky, D, D)
        fh = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        w2 = E.omega2_of(B)
        w = math.sqrt(w2)
        Eexp = np.eye(3) + (math.sin(tau * w) / w) * B + ((1 - math.cos(tau * w)) / w2) * (B @ B)
        out = R.rexii_apply_dense_mode(B, fh, tau, 0.5, M, real_input=False)
        assert np.linalg.norm(out - Eexp @ fh) / np.linalg.norm(fh) < 1e-10
