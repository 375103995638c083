"""Pins for the oracle's original REXI (eq. originalRexi, eq. originalREXImatrix)
and REXI Extended (eq. REXIE) with the spectral shift of the remark in
Section 2.2 (CPU only).

References independent of the functions under test: the printed REXI errors
of Tables 2-7 (tests/golden/paper_rexi_errors.txt), e^{ix}, dense
scipy.linalg.expm of the A_1 and A_2 matrices of Section 3.2, the algebraic
identity that makes REXI and REXII equal for real x (Section 2.1 Step 3), and
two independent evaluations of the matrix form (sparse LU per term against a
per-wavenumber resolvent sum).
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import coeffs as C
from oracle import exact as E
from oracle import operator as O
from oracle import rexi as R
from oracle import spectral as S
from paper_2008_11607_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rexi_rows():
    with open(os.path.join(GOLDEN, "paper_rexi_errors.txt")) as fh:
        for ln in fh:
            if ln.strip() and not ln.startswith("#"):
                p = ln.split()
                yield p[0], float(p[1]), float(p[2]), int(p[3]), float(p[4]), float(p[5])


@pytest.mark.parametrize("h,M", [(0.2, 3), (0.5, 30), (1.0, 12)])
def test_beta_sliced_equals_loop_form(h, M):
    _, b1, b2 = C.beta_coeffs(h, M)
    _, s1, s2 = C.beta_coeffs_sliced(h, M)
    scale = max(np.max(np.abs(b1)), np.max(np.abs(b2)))
    assert np.max(np.abs(b1 - s1)) < 1e-14 * scale and np.max(np.abs(b2 - s2)) < 1e-14 * scale


def test_beta_and_c_are_the_same_numbers_rearranged():
    """beta^{Re} = Re c1 + i Re c2 and beta^{Im} = Im c1 + i Im c2 (both are
    h sum a_k b_{n-k} split by real and imaginary parts of a_k and b): the
    reason REXI and REXII agree for real x (Section 2.1 Step 3)."""
    _, c1, c2 = C.c_coeffs(0.5, 25)
    _, br, bi = C.beta_coeffs(0.5, 25)
    assert np.max(np.abs(br - (c1.real + 1j * c2.real))) < 1e-13
    assert np.max(np.abs(bi - (c1.imag + 1j * c2.imag))) < 1e-13


@pytest.mark.parametrize("rho", [30.0, 200.0])
def test_original_rexi_scalar_equals_rexii_and_eix(rho):
    h = 0.5
    M = C.pole_count_M(rho, h, 1e-16)
    x = np.linspace(-rho, rho, 2001)
    a = C.rexi_original_scalar(x, h, M)
    b = C.rexii_scalar(x, h, M)
    assert np.max(np.abs(a - b)) < 1e-13
    assert np.max(np.abs(a - np.exp(1j * x))) < 1e-13


def test_original_rexi_matrix_two_evaluations_agree():
    """Sparse LU per term on the C-grid operator against the per-wavenumber
    resolvent sum with the C-grid symbol."""
    nx, ny = 8, 6
    st = inputs.kminus3_field(nx, ny, seed=2)
    st[2] = inputs.kminus3_field(nx, ny, seed=3)[0]
    A = O.cgrid_operator(nx, ny, g=1.3, f=0.7, H=0.8)
    tau, h, M = 0.05, 0.2, 60
    a = R.rexi_original_apply_sparse(A, st.ravel(), tau, h, M).reshape(st.shape)
    b = R.rexi_original_apply_modes(st, tau, h, M, O.symbol, g=1.3, f=0.7, H=0.8)
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-12


def test_original_rexi_less_accurate_than_rexii_on_A1():
    """Section 3.2 (Fig. 2b as described): A_1 has complex eigenvectors, so the
    real part cannot be pulled through V and the original REXI is far less
    accurate than REXII at the M of eq. matrixAccuracyBound."""
    n = 70
    dx = 1.0 / n
    x = np.arange(n) * dx
    A1 = sp.diags([np.full(n - 1, 0.5 / dx), np.full(n - 1, -0.5 / dx)], [1, -1]).tolil()
    A1[0, n - 1] = -0.5 / dx
    A1[n - 1, 0] = 0.5 / dx
    A1 = A1.tocsr()
    f0 = 1.0 / (2.0 + np.cos(2 * math.pi * x))
    ref = E.expm_dense(A1, f0, 1.0)
    M = C.pole_count_M(70.0, 0.5, 1e-16)
    e2 = np.linalg.norm(R.rexii_apply_sparse(A1, f0, 1.0, 0.5, M) - ref) / np.linalg.norm(ref)
    e1 = np.linalg.norm(R.rexi_original_apply_sparse(A1, f0, 1.0, 0.5, M) - ref) / np.linalg.norm(ref)
    assert e2 < 1e-12 and e1 > 1e3 * e2, (e1, e2)


@pytest.mark.parametrize("row", [r for r in rexi_rows() if r[3] <= 20000])
def test_paper_rexi_rows_reproduced(row):
    """The REXI rows of Tables 2-7 that the oracle evaluates in seconds: the
    max-norm error against the exact exponential of the spectral operator
    matches the printed CPU column to 2 % (the printed values have three
    digits)."""
    scen, tau, h, M, cpu, _ = row
    D = 128
    st = inputs.paper_scenario(scen, D, D)
    ref = E.exp_closed_form(st, tau, symbol_fn=S.symbol).real
    out = R.rexi_original_apply_modes(st, tau, h, M, S.symbol).real
    err = float(np.max(np.abs(out - ref)))
    assert abs(err - cpu) <= 0.02 * cpu, (scen, tau, M, err, cpu)


def test_schrodinger_operator_spectrum():
    """A = i(d_xx + d_yy): eigenvalues i(-4/dx^2 sin^2(pi kx/nx) - 4/dy^2 sin^2(pi ky/ny))."""
    nx, ny, Lx, Ly = 6, 5, 1.3, 0.7
    A = O.schrodinger_operator(nx, ny, Lx, Ly).toarray()
    ev = np.sort(np.linalg.eigvals(A).imag)
    kx, ky = np.meshgrid(np.arange(nx), np.arange(ny))
    lam = -(4 / (Lx / nx) ** 2) * np.sin(np.pi * kx / nx) ** 2 - (4 / (Ly / ny) ** 2) * np.sin(np.pi * ky / ny) ** 2
    assert np.max(np.abs(ev - np.sort(lam.ravel()))) < 1e-10
    assert np.max(np.abs(A + A.conj().T)) < 1e-12  # skew-Hermitian


def test_rexie_A2_with_and_without_shift():
    """Section 3.2, matrix A_2 (i d_xx on [-1, 1], step 1/35, eigenvalues in
    i[-4900, 0]) with f0 = 1/(2 + cos(2 pi x)): with the shift nu = -2450 i
    the pole count for rho(A') = 2450 reaches the dense expm to 1e-12; the
    same M without the shift covers only half the spectrum and fails."""
    A2 = O.schrodinger_operator(70, 1, Lx=2.0)
    ev = np.linalg.eigvals(A2.toarray())
    assert abs(ev.imag.min() + 4900.0) < 1e-8 and abs(ev.imag.max()) < 1e-8
    x = -1.0 + np.arange(70) * (2.0 / 70)
    f0 = 1.0 / (2.0 + np.cos(2 * math.pi * x))
    ref = E.expm_dense(A2, f0, 1.0)
    M = C.pole_count_M(2450.0, 0.5, 1e-16)
    shifted = R.rexie_apply(A2, f0, 1.0, 0.5, M, sigma=-2450.0)
    plain = R.rexie_apply(A2, f0, 1.0, 0.5, M, sigma=0.0)
    assert np.linalg.norm(shifted - ref) / np.linalg.norm(ref) < 1e-12
    assert np.linalg.norm(plain - ref) / np.linalg.norm(ref) > 1e-7


def test_rexie_equals_rexii_on_skew_hermitian_A2():
    """A_2 is skew-Hermitian with real eigenvectors: REXIE (one solve per term)
    and REXII (two solves per term, complex mode) give the same vector."""
    A2 = O.schrodinger_operator(40, 1, Lx=2.0)
    x = -1.0 + np.arange(40) * (2.0 / 40)
    f0 = 1.0 / (2.0 + np.cos(2 * math.pi * x))
    rho = 4.0 / (2.0 / 40) ** 2
    M = C.pole_count_M(rho * 0.01, 0.5, 1e-16)
    a = R.rexie_apply(A2, f0, 0.01, 0.5, M)
    b = R.rexii_apply_sparse(A2, f0, 0.01, 0.5, M, real_input=False)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-12
