"""Pins for the oracle's coefficient arithmetic (CPU only).

Each test checks the oracle against something other than itself: values the
paper prints, closed forms (e^{ix}, the Gaussian), or a brute-force double sum.
"""
import math
import os

import numpy as np
import pytest

from oracle import coeffs as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def test_table_a_fit_error_below_paper_bound():
    """Section 2.1 Step 2: max |psi_1 - R| < 8e-15 (tested at 1e-14 on [-60, 60])."""
    mu, a = C.table_a()
    x = np.linspace(-60.0, 60.0, 48001)
    err = np.max(np.abs(C.psi(x, 1.0) - C.rational_gaussian(x, mu, a)))
    assert err < 1e-14


def test_table_a_other_sign_reading_breaks_fit():
    """The rejected reading of the sign column gives an O(1) error."""
    mu, a = C.table_a("whole")
    x = np.linspace(-60.0, 60.0, 4001)
    assert np.max(np.abs(C.psi(x, 1.0) - C.rational_gaussian(x, mu, a))) > 1.0


def test_real_closed_form_matches_complex_sum():
    """eq. A(x,mu) is the real form of eq. ratapproxgaush1 for a_{-l} = conj(a_l)."""
    mu, a = C.table_a()
    x = np.linspace(-40.0, 40.0, 8001)
    assert np.max(np.abs(C.rational_gaussian_real_form(x, mu, a) - C.rational_gaussian(x, mu, a))) < 2e-14
    assert np.max(np.abs(C.rational_gaussian_real_form(x, mu, a) - C.psi(x, 1.0))) < 1e-14


def test_conjugate_symmetry_of_a():
    mu, a = C.table_a()
    for l in range(1, C.L + 1):
        assert a[C.L - l] == np.conj(a[C.L + l])
    assert a[C.L].imag == 0.0


@pytest.mark.parametrize("h,bound", [(0.3, 1e-13), (0.5, 1e-13), (1.0, 1e-11)])
def test_gaussian_sum_reproduces_eix(h, bound):
    """Step 1, eq. eixsumM: sum b_m psi_h(x + m h) = e^{ix} for |x| <= (M - 11) h.
    For h = 1 the aliasing term of the Poisson sum (Appendix B) is ~2e-12, the
    level of the h = 1.0 rows of Tables tab:w11 and tab:G1001 (~3e-12)."""
    M = 60
    x = np.linspace(-(M - 11) * h, (M - 11) * h, 2001)
    err = np.max(np.abs(C.gaussian_sum(x, h, M) - np.exp(1j * x)))
    assert err < bound


def test_b_m_closed_form_values():
    """eq. bm: |b_m| = e^{h^2}, arg b_m = -m h."""
    h = 0.5
    for m in (-7, 0, 3, 11):
        b = complex(C.b_coeff(m, h))
        assert abs(abs(b) - math.exp(h * h)) < 1e-15
        assert abs(b - math.exp(h * h) * complex(math.cos(m * h), -math.sin(m * h))) < 1e-15


@pytest.mark.parametrize("h", [0.5, 0.3])
def test_single_sum_equals_double_sum(h):
    """eq. modifiedRexi (with the L1/L2 index ranges) equals eq. RexiNotSimplified."""
    M = 30
    x = np.linspace(-25.0, 25.0, 301)
    d = C.rexi_double_sum(x, h, M)
    s = C.rexii_scalar(x, h, M)
    assert np.max(np.abs(d - s)) < 2e-14


@pytest.mark.parametrize("rho", [50.0, 100.0, 1000.0])
def test_rexii_scalar_accuracy_rule_plus_11(rho):
    """eq. Mformula: with M = ceil(rho/h) + 11, |REXII(ix) - e^{ix}| is near machine
    precision on [-rho, rho] (the paper's Section 3.1 observation)."""
    h = 0.5
    M = C.pole_count_M(rho, h, 1e-16)
    assert M == math.ceil(rho / h) + 11
    x = np.linspace(-rho, rho, 1501)
    assert np.max(np.abs(C.rexii_scalar(x, h, M) - np.exp(1j * x))) < 1e-13


@pytest.mark.parametrize("rho", [50.0, 400.0])
def test_rexii_scalar_accuracy_tol_rule(rho):
    """Appendix B tolerance form of the rule: error <= tol-level for tol = 1e-10."""
    h = 0.5
    M = C.pole_count_M(rho, h, 1e-10)
    x = np.linspace(-rho, rho, 1201)
    assert np.max(np.abs(C.rexii_scalar(x, h, M) - np.exp(1j * x))) < 1e-10


def test_rexii_conjugate_symmetry():
    """Remark before eq. modifiedRexiMatrixReducedSum: conj(c1_n) = c1_{-n},
    conj(c2_n) = -c2_{-n}; hence REXII(-ix) = conj(REXII(ix))."""
    h, M = 0.5, 40
    ns, c1, c2 = C.c_coeffs(h, M)
    # equal up to the rounding of two different summation orders
    assert np.max(np.abs(np.conj(c1) - c1[::-1])) < 1e-14 * np.max(np.abs(c1))
    assert np.max(np.abs(np.conj(c2) + c2[::-1])) < 1e-14 * np.max(np.abs(c2))
    x = np.linspace(0.0, 25.0, 51)
    assert np.max(np.abs(C.rexii_scalar(-x, h, M) - np.conj(C.rexii_scalar(x, h, M)))) < 1e-14


def test_paper_M_values():
    """M printed in Tables tab:w11, tab:w150, tab:w850, tab:G1001, tab:G10050."""
    for row in _rows("paper_M_values.txt"):
        _, _, kind, D, tau, h, Mp, exact = row[:8]
        D, tau, h, Mp, exact = int(D), float(tau), float(h), int(Mp), int(exact)
        rho = math.sqrt(2.0) * math.pi * D if kind == "sqrt2piD" else math.sqrt(2 * math.pi ** 2 * D * D + 1)
        Mr = C.pole_count_M(rho * tau, h, 1e-16)
        if exact:
            assert Mr == Mp, row
        else:
            assert Mp > Mr and Mp - Mr <= 15, row
        assert (Mp - 11) * h >= rho * tau, row


@pytest.mark.slow
def test_table5_onset_of_convergence():
    """Table tab:W8_M: M = 20400 fails, M = 20800 converges (scalar check at the
    largest active eigenvalue, D = 46)."""
    x = 50.0 * math.sqrt(2 * math.pi ** 2 * 46 ** 2 + 1)
    rows = _rows("table5_threshold.txt")
    for M, printed, verdict in [(int(r[0]), float(r[1]), r[2]) for r in rows]:
        err = abs(complex(C.rexii_scalar(np.array([x]), 0.5, M)[0]) - complex(math.cos(x), math.sin(x)))
        if verdict.startswith("fails"):
            assert err > 0.1, (M, err, printed)
        else:
            assert err < 1e-12, (M, err, printed)


def test_appendix_b_constants():
    vals = {r[0]: (float(r[1]), float(r[2])) for r in _rows("appendix_b.txt")}
    v, t = vals["tail_sum_bound"]
    assert abs(C.appendix_b_tail_bound() - v) <= t
    v, t = vals["c_at_1e-16"]
    assert abs(C.c_tol(1e-16) - v) <= t
    assert C.m0_tol(1e-16) == int(vals["m0_at_1e-16"][0])
    # the psi_h(z) <= tol property that defines c
    for tol in (1e-16, 1e-10, 1e-6):
        z = C.c_tol(tol) * 0.7
        assert abs(C.psi(z, 0.7) - tol) / tol < 1e-9


def test_single_shift_poles_equal_term_form():
    """Partial fractions of each REXII term reproduce REXII(ix)."""
    h, M = 0.5, 40
    poles, w = C.single_shift_poles(h, M, real_input=False)
    assert len(poles) == 2 * (2 * (M + C.L) + 1)
    x = np.linspace(-30.0, 30.0, 121)
    z = 1j * x[:, None]
    pf = np.sum(w[None, :] / (z - poles[None, :]), axis=1)
    assert np.max(np.abs(pf - C.rexii_scalar(x, h, M))) < 1e-12
    pr, wr = C.single_shift_poles(h, M, real_input=True)
    assert len(pr) == 2 * (M + C.L + 1)
    # real-reduced set: Re of the sum reproduces the real part for real-valued
    # evaluation through a real matrix; at scalar level check 2x2 rotation block
    # exp([[0, x], [-x, 0]]) via the eigenvalues +-ix.
    pfr = np.sum(wr[None, :] / (z - pr[None, :]), axis=1)
    pfr_m = np.sum(wr[None, :] / (-z - pr[None, :]), axis=1)
    # for a real matrix with eigenvalues +-ix the reduced sum gives Re over the pair
    assert np.max(np.abs(0.5 * (pfr + np.conj(pfr_m)) - C.rexii_scalar(x, h, M))) < 1e-12


@pytest.mark.parametrize("h,M", [(0.5, 3), (0.5, 40), (1.0, 25), (0.1, 60), (0.3, 1)])
def test_sliced_coefficients_equal_loop_form(h, M):
    """c_coeffs_sliced adds the same terms in the same order as the explicit
    loops of c_coeffs; only b_m is evaluated as an array, so the two agree to
    a few ulps of the largest coefficient."""
    ns, c1, c2 = C.c_coeffs(h, M)
    ns2, d1, d2 = C.c_coeffs_sliced(h, M)
    assert np.array_equal(ns, ns2)
    scale = max(np.max(np.abs(c1)), np.max(np.abs(c2)))
    assert np.max(np.abs(c1 - d1)) < 1e-14 * scale
    assert np.max(np.abs(c2 - d2)) < 1e-14 * scale
