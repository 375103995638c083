"""Planted mistakes: each plausible error in the oracle must fail a pin.

The mistakes are planted in the oracle (monkeypatched, CPU only); the pins
are the same checks as in test_oracle_coeffs / test_oracle_matrix, here in a
compact form that returns the measured error.
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


def scalar_pin():
    rho, h = 60.0, 0.5
    M = C.pole_count_M(rho, h, 1e-16)
    x = np.linspace(-rho, rho, 301)
    return np.max(np.abs(C.rexii_scalar(x, h, M) - np.exp(1j * x)))


def double_sum_pin():
    x = np.linspace(-20, 20, 41)
    return np.max(np.abs(C.rexi_double_sum(x, 0.5, 25) - C.rexii_scalar(x, 0.5, 25)))


def gaussian_pin():
    h, M = 0.5, 40
    x = np.linspace(-(M - 11) * h, (M - 11) * h, 201)
    return np.max(np.abs(C.gaussian_sum(x, h, M) - np.exp(1j * x)))


def skew_pin():
    H = inputs.variable_depth(6, 6, seed=0)
    A = O.cgrid_operator(6, 6, H=H)
    S = (sp.diags(O.energy_weight(6, 6, H=H)) @ A).toarray()
    return np.max(np.abs(S + S.T))


def symbol_pin():
    nx, ny = 6, 5
    A = O.cgrid_operator(nx, ny, f=0.7, g=1.3, H=0.8)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    worst = 0.0
    for kx, ky in ((1, 2), (5, 4)):
        mode = np.exp(2j * math.pi * (kx * ii / nx + ky * jj / ny))
        B = O.symbol(kx, ky, nx, ny, g=1.3, f=0.7, H=0.8)
        for c in range(3):
            vec = np.zeros((3, ny, nx), dtype=np.complex128)
            vec[c] = mode
            out = (A @ vec.ravel()).reshape(3, ny, nx)
            for r in range(3):
                worst = max(worst, np.max(np.abs(out[r] - B[r, c] * mode)))
    return worst


def expm_pin():
    D = 6
    A = O.cgrid_operator(D, D)
    rho = 2 * math.sqrt(2) * D
    tau = 12.0 / rho
    M = C.pole_count_M(12.0, 0.5, 1e-16)
    f0 = inputs.kminus3_field(D, D, seed=1).ravel()
    ref = E.expm_dense(A, f0, tau)
    out = R.rexii_apply_sparse(A, f0, tau, 0.5, M)
    return np.linalg.norm(out - ref) / np.linalg.norm(ref)


def test_pins_pass_unmodified():
    assert scalar_pin() < 1e-13
    assert double_sum_pin() < 1e-13
    assert gaussian_pin() < 1e-13
    assert skew_pin() < 1e-12
    assert symbol_pin() < 1e-11
    assert expm_pin() < 1e-12


def test_mutation_b_sign(monkeypatch):
    monkeypatch.setattr(C, "b_coeff", lambda m, h: np.exp(1j * np.asarray(m, float) * h) * math.exp(h * h))
    assert gaussian_pin() > 1e-3 and scalar_pin() > 1e-3


def test_mutation_swapped_c1_c2(monkeypatch):
    orig = C.c_coeffs

    def swapped(h, M, mu=None, a=None):
        ns, c1, c2 = orig(h, M, mu, a)
        return ns, c2, c1

    monkeypatch.setattr(C, "c_coeffs", swapped)
    assert scalar_pin() > 1e-3


def test_mutation_index_range(monkeypatch):
    """L1(n) off by one: the single sum no longer equals the double sum."""
    mu, a = C.table_a()

    def bad(h, M, mu_=None, a_=None):
        N = M + C.L
        ns = np.arange(-N, N + 1)
        c1 = np.zeros(2 * N + 1, complex)
        c2 = np.zeros(2 * N + 1, complex)
        for idx, n in enumerate(ns):
            for k in range(max(-C.L, n - M + 1), min(C.L, n + M) + 1):
                c1[idx] += h * a[C.L + k].real * C.b_coeff(n - k, h)
                c2[idx] += h * a[C.L + k].imag * C.b_coeff(n - k, h)
        return ns, c1, c2

    monkeypatch.setattr(C, "c_coeffs", bad)
    assert double_sum_pin() > 1e-10


def test_mutation_table_entry(monkeypatch):
    """A mistyped digit in Table A shows in the fit error."""
    rows = list(C.TABLE_A)
    s, re_t, im_t = rows[5]
    rows[5] = (s, re_t.replace("218558", "228558"), im_t)
    assert rows[5][1] != re_t
    monkeypatch.setattr(C, "TABLE_A", rows)
    mu, a = C.table_a()
    x = np.linspace(-60, 60, 2001)
    assert np.max(np.abs(C.psi(x, 1.0) - C.rational_gaussian(x, mu, a))) > 1e-6


def test_mutation_coriolis_not_transposed(monkeypatch):
    orig = O.cgrid_operator

    def bad(nx, ny, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0):
        A = orig(nx, ny, Lx, Ly, g, f, H).tolil()
        n = nx * ny
        # v row uses the u->v average at the wrong offsets (same as v->u)
        for j in range(ny):
            for i in range(nx):
                r = 2 * n + j * nx + i
                for (di, dj) in ((0, 0), (-1, 0), (0, 1), (-1, 1)):
                    A[r, n + ((j + dj) % ny) * nx + (i + di) % nx] = 0.0
                for (di, dj) in ((0, 0), (1, 0), (0, -1), (1, -1)):
                    A[r, n + ((j + dj) % ny) * nx + (i + di) % nx] = -0.25 * f
        return A.tocsr()

    monkeypatch.setattr(O, "cgrid_operator", bad)
    assert skew_pin() > 1e-3


def test_mutation_divergence_sign(monkeypatch):
    orig = O.cgrid_operator

    def bad(nx, ny, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0):
        A = orig(nx, ny, Lx, Ly, g, f, H).tolil()
        n = nx * ny
        A[:n, :] = -A[:n, :]
        return A.tocsr()

    monkeypatch.setattr(O, "cgrid_operator", bad)
    assert skew_pin() > 1e-3


def test_mutation_symbol_conjugated_average(monkeypatch):
    orig = O.symbol

    def bad(*args, **kw):
        B = orig(*args, **kw)
        # use conj(P) for the v->u average and P for the u->v average
        B[1, 2], B[2, 1] = np.conj(B[1, 2]), np.conj(B[2, 1])
        return B

    monkeypatch.setattr(O, "symbol", bad)
    assert symbol_pin() > 1e-3


@pytest.mark.parametrize("which", ["alpha_swap", "gamma_one", "c2_sign"])
def test_mutation_chain(monkeypatch, which):
    orig = C.matrix_term_weights

    def bad(h, M, real_input=True, mu=None, a=None):
        out = []
        for n, an, amn, C1, C2, gam in orig(h, M, real_input, mu, a):
            if which == "alpha_swap":
                an, amn = amn, an
            elif which == "gamma_one":
                gam = 1.0
            elif which == "c2_sign":
                C2 = -C2
            out.append((n, an, amn, C1, C2, gam))
        return out

    monkeypatch.setattr(C, "matrix_term_weights", bad)
    assert expm_pin() > 1e-3


# ---------------------------------------------------------------------------
# The original REXI, REXIE, the shift and the field-wide exponential.

def rexi_row_pin():
    """WS1, tau = 1, h = 0.2, M = 150 at D = 128: the printed 6.98e-2 (Table tab:w11)."""
    from oracle import spectral as S

    st = inputs.paper_scenario("ws1", 128, 128)
    ref = E.exp_closed_form(st, 1.0, symbol_fn=S.symbol).real
    out = R.rexi_original_apply_modes(st, 1.0, 0.2, 150, S.symbol).real
    return abs(float(np.max(np.abs(out - ref))) - 6.98e-2) / 6.98e-2


def a2_pin():
    """A_2 with the shift nu = -2450 i against dense expm (Section 3.2)."""
    A2 = O.schrodinger_operator(70, 1, Lx=2.0)
    x = -1.0 + np.arange(70) * (2.0 / 70)
    f0 = 1.0 / (2.0 + np.cos(2 * math.pi * x))
    ref = E.expm_dense(A2, f0, 1.0)
    got = R.rexie_apply(A2, f0, 1.0, 0.5, C.pole_count_M(2450.0, 0.5, 1e-16), sigma=-2450.0)
    return np.linalg.norm(got - ref) / np.linalg.norm(ref)


def grid_exp_pin():
    st = inputs.complex_random_state(6, 5, seed=2)
    A = O.cgrid_operator(6, 5, 1.1, 0.9, 1.5, 0.6, 2.0)
    ref = E.expm_dense(A, st.ravel(), 0.7).reshape(st.shape)
    got = E.exp_closed_form_grid(st, 0.7, 1.1, 0.9, 1.5, 0.6, 2.0)
    return np.linalg.norm(got - ref) / np.linalg.norm(ref)


def test_new_pins_pass_unmodified():
    assert rexi_row_pin() < 0.02
    assert a2_pin() < 1e-12
    assert grid_exp_pin() < 1e-12


def test_mutation_beta_uses_the_wrong_part_of_b(monkeypatch):
    """beta^Re built from Im(b_m) instead of Re(b_m): the REXI row no longer
    reproduces the printed error."""
    orig = C.beta_coeffs_sliced

    def bad(h, M, mu=None, a=None):
        ns, br, bi = orig(h, M, mu, a)
        return ns, bi, br

    monkeypatch.setattr(C, "beta_coeffs_sliced", bad)
    assert rexi_row_pin() > 0.5


def test_mutation_rexie_shift_phase_sign(monkeypatch):
    """e^{-i tau sigma} instead of e^{+i tau sigma} when undoing the shift."""
    orig = R.rexie_apply

    def bad(A, f0, tau, h, M, sigma=0.0):
        return orig(A, f0, tau, h, M, sigma) * np.exp(-2j * tau * sigma)

    monkeypatch.setattr(R, "rexie_apply", bad)
    assert a2_pin() > 1e-3


def test_mutation_rexie_drops_the_imaginary_part(monkeypatch):
    """REXIE without its i Re(beta^Im ...) half is the original REXI, which
    approximates only cos on an operator i B."""
    monkeypatch.setattr(C, "beta_coeffs", lambda h, M, mu=None, a=None: (
        C.beta_coeffs_sliced(h, M, mu, a)[0], C.beta_coeffs_sliced(h, M, mu, a)[1],
        np.zeros_like(C.beta_coeffs_sliced(h, M, mu, a)[2])))
    assert a2_pin() > 1e-3


@pytest.mark.parametrize("which", ["sin_sign", "missing_B2"])
def test_mutation_grid_exponential(monkeypatch, which):
    orig = O.symbol_grid

    def bad(*args, **kw):
        B = orig(*args, **kw)
        if which == "sin_sign":
            return -B  # e^{-tau B}: the sin term changes sign, the B^2 term does not
        B2 = B.copy()
        B2[1, 0] = B2[2, 0] = 0.0  # a dropped gradient column
        return B2

    monkeypatch.setattr(O, "symbol_grid", bad)
    assert grid_exp_pin() > 1e-3
