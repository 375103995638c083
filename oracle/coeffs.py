"""REXII coefficients, written out from the paper's definitions (FP64, numpy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Citations are to arXiv 2008.11607: Section 2.1 (Steps 1-3), eq. bm,
eq. ratapproxgaush1, eq. A(x,mu), eq. RexiNotSimplified, eq. modifiedRexi,
eq. REXI_Modified_matrix, eq. matrixAccuracyBound, Appendix A (Table
tab:coef_al) and Appendix B.
"""
import math

import numpy as np

L = 24  # number of conjugate pairs in the rational fit, Section 2.1 Step 2

# Appendix A, Table tab:coef_al, transcribed as printed: a separate sign
# column, then the real part and (for l >= 1) the imaginary part.  Reading:
# the sign column is the sign of the REAL part only (an Octave-style print);
# the sign printed inside the complex number belongs to the imaginary part.
# The other reading (negating the whole number) gives a fit error of O(1)
# instead of < 8e-15 (Section 2.1 Step 2), which the tests check.
MU_ROW = ("-", "5.133333333333333")
TABLE_A = [
    ("-", "6.520430828919864e+01", None),
    ("", "4.261818064131437e+01", "+2.761406741120911e+01"),
    ("-", "9.801650304425239e+00", "-2.189295463610722e+01"),
    ("-", "1.054225194693395e+00", "+6.791786454153551e+00"),
    ("", "7.950505668209775e-01", "-8.904997258367445e-01"),
    ("-", "1.218558380859130e-01", "+3.321241563407446e-02"),
    ("", "7.365401806949337e-03", "+2.212802103193251e-03"),
    ("-", "2.801087265991056e-04", "-5.566945197754387e-04"),
    ("", "1.254835436432561e-04", "-2.467200513365371e-04"),
    ("", "2.295472292491263e-04", "-8.494118951459107e-05"),
    ("", "1.858484460459430e-04", "+9.242889460185034e-05"),
    ("", "4.068056518449676e-05", "+1.653479957565515e-04"),
    ("-", "8.341508001647741e-05", "+1.045331460447588e-04"),
    ("-", "9.970528169841103e-05", "-5.856228484297677e-06"),
    ("-", "3.499639858693093e-05", "-6.129059473910835e-05"),
    ("", "2.295021920298455e-05", "-4.099832469456381e-05"),
    ("", "2.931048772724314e-05", "+1.708815129697846e-07"),
    ("", "7.502088478301169e-06", "+1.525082051744077e-05"),
    ("-", "5.815291167450100e-06", "+6.919604247338349e-06"),
    ("-", "4.069948458364005e-06", "-1.440010113050771e-06"),
    ("", "7.932524475429588e-08", "-1.794169428574330e-06"),
    ("", "6.120984882186265e-07", "-1.131894636585849e-07"),
    ("", "5.531365159161319e-08", "+1.585749903175946e-07"),
    ("-", "2.867805871375946e-08", "+1.239499740327838e-08"),
    ("-", "1.143081277095316e-09", "-2.763239274253499e-09"),
]


def _signed(sign, text):
    v = float(text)
    return -v if sign == "-" else v


def table_a(sign_reading="real"):
    """Return (mu, a) with a[l + L] = a_l for l = -L..L (Appendix A).

    ``sign_reading="real"`` applies the sign column to the real part only;
    ``"whole"`` negates the whole complex number (the rejected reading, kept
    only so a test can show that it breaks the fit).  a_{-l} = conj(a_l) as the
    caption of Table tab:coef_al states.
    """
    mu = _signed(*MU_ROW)
    pos = []
    for sign, re_txt, im_txt in TABLE_A:
        im = 0.0 if im_txt is None else float(im_txt)
        if sign_reading == "real":
            pos.append(complex(_signed(sign, re_txt), im))
        elif sign_reading == "whole":
            z = complex(float(re_txt), im)
            pos.append(-z if sign == "-" else z)
        else:
            raise ValueError(sign_reading)
    a = np.zeros(2 * L + 1, dtype=np.complex128)
    for l in range(L + 1):
        a[L + l] = pos[l]
        a[L - l] = np.conj(pos[l])
    return mu, a


def psi(x, h):
    """Gaussian kernel psi_h(x) = (4 pi)^(-1/2) exp(-x^2 / (4 h^2)), eq. psi."""
    x = np.asarray(x, dtype=np.float64)
    return np.exp(-x * x / (4.0 * h * h)) / math.sqrt(4.0 * math.pi)


def rational_gaussian(x, mu, a):
    """R(x) = Re sum_{l=-L}^{L} a_l / (i x + mu + i l), eq. ratapproxgaush1 (h = 1)."""
    x = np.asarray(x, dtype=np.float64)
    acc = np.zeros(x.shape, dtype=np.complex128)
    for l in range(-L, L + 1):
        acc += a[L + l] / (1j * x + mu + 1j * l)
    return acc.real


def rational_gaussian_real_form(x, mu, a):
    """The same R(x) in the real closed form of eq. A(x,mu)."""
    x = np.asarray(x, dtype=np.float64)
    x2 = x * x
    out = a[L].real * mu / (x2 + mu * mu)
    for l in range(1, L + 1):
        al = a[L + l]
        num = 2.0 * mu * al.real * (mu * mu + l * l + x2) + 2.0 * l * al.imag * (mu * mu + l * l - x2)
        den = x2 * x2 + 2.0 * (mu * mu - l * l) * x2 + (mu * mu + l * l) ** 2
        out = out + num / den
    return out


def b_coeff(m, h):
    """b_m = e^{-i m h} e^{h^2}, eq. bm."""
    m = np.asarray(m, dtype=np.float64)
    return np.exp(-1j * m * h) * math.exp(h * h)


def gaussian_sum(x, h, M):
    """Step 1 truncated sum  sum_{m=-M}^{M} b_m psi_h(x + m h),  eq. eixsumM."""
    x = np.asarray(x, dtype=np.float64)
    acc = np.zeros(x.shape, dtype=np.complex128)
    for m in range(-M, M + 1):
        acc += b_coeff(m, h) * psi(x + m * h, h)
    return acc


def c_coeffs(h, M, mu=None, a=None):
    """c_{1,n}, c_{2,n} for n = -N..N (N = M + L), Section 2.1 Step 3.

    c_{1,n} = h sum_{k=L1(n)}^{L2(n)} Re(a_k) b_{n-k},
    c_{2,n} = h sum_{k=L1(n)}^{L2(n)} Im(a_k) b_{n-k},
    L1(n) = max(-L, n - M), L2(n) = min(L, n + M).
    Written with explicit loops so the index ranges can be read off.
    Returns (n, c1, c2) with n = -N..N.
    """
    if mu is None or a is None:
        mu, a = table_a()
    N = M + L
    ns = np.arange(-N, N + 1)
    c1 = np.zeros(2 * N + 1, dtype=np.complex128)
    c2 = np.zeros(2 * N + 1, dtype=np.complex128)
    for idx, n in enumerate(ns):
        L1 = max(-L, n - M)
        L2 = min(L, n + M)
        s1 = 0.0 + 0.0j
        s2 = 0.0 + 0.0j
        for k in range(L1, L2 + 1):
            bnk = b_coeff(n - k, h)
            s1 += a[L + k].real * bnk
            s2 += a[L + k].imag * bnk
        c1[idx] = h * s1
        c2[idx] = h * s2
    return ns, c1, c2


def c_coeffs_sliced(h, M, mu=None, a=None):
    """The same c_{1,n}, c_{2,n} as ``c_coeffs``, accumulated for all n at once:
    for each k = -L..L in increasing order, Re(a_k) b_m and Im(a_k) b_m are
    added to index n = m + k for every m = -M..M.  Every n therefore receives
    the terms of its sum in the same order as in ``c_coeffs`` (k from L1(n)
    to L2(n)), so the two agree to rounding of b_m (pinned in
    tests/test_oracle_coeffs.py); this form is for large M (hundreds of
    thousands of terms), where the loops of ``c_coeffs`` take minutes."""
    if mu is None or a is None:
        mu, a = table_a()
    N = M + L
    ns = np.arange(-N, N + 1)
    b = b_coeff(np.arange(-M, M + 1), h)
    c1 = np.zeros(2 * N + 1, dtype=np.complex128)
    c2 = np.zeros(2 * N + 1, dtype=np.complex128)
    for k in range(-L, L + 1):
        lo = k + L  # index of n = -M + k
        c1[lo:lo + 2 * M + 1] += a[L + k].real * b
        c2[lo:lo + 2 * M + 1] += a[L + k].imag * b
    return ns, h * c1, h * c2


def beta_coeffs(h, M, mu=None, a=None):
    """beta^{Re}_n, beta^{Im}_n for n = -N..N, Section 2.1 Step 3 (the
    coefficients of the original REXI, eq. originalRexi):
    beta^{Re}_n = h sum_{k=L1(n)}^{L2(n)} a_k Re(b_{n-k}),
    beta^{Im}_n = h sum_{k=L1(n)}^{L2(n)} a_k Im(b_{n-k}),
    L1(n) = max(-L, n - M), L2(n) = min(L, n + M).  Explicit loops.
    Returns (n, beta_re, beta_im)."""
    if mu is None or a is None:
        mu, a = table_a()
    N = M + L
    ns = np.arange(-N, N + 1)
    br = np.zeros(2 * N + 1, dtype=np.complex128)
    bi = np.zeros(2 * N + 1, dtype=np.complex128)
    for idx, n in enumerate(ns):
        s1 = 0.0 + 0.0j
        s2 = 0.0 + 0.0j
        for k in range(max(-L, n - M), min(L, n + M) + 1):
            bnk = complex(b_coeff(n - k, h))
            s1 += a[L + k] * bnk.real
            s2 += a[L + k] * bnk.imag
        br[idx] = h * s1
        bi[idx] = h * s2
    return ns, br, bi


def beta_coeffs_sliced(h, M, mu=None, a=None):
    """``beta_coeffs`` accumulated for all n at once (k outer, in increasing
    order, as ``c_coeffs_sliced``); pinned against the loop form."""
    if mu is None or a is None:
        mu, a = table_a()
    N = M + L
    ns = np.arange(-N, N + 1)
    b = b_coeff(np.arange(-M, M + 1), h)
    br = np.zeros(2 * N + 1, dtype=np.complex128)
    bi = np.zeros(2 * N + 1, dtype=np.complex128)
    for k in range(-L, L + 1):
        lo = k + L
        br[lo:lo + 2 * M + 1] += a[L + k] * b.real
        bi[lo:lo + 2 * M + 1] += a[L + k] * b.imag
    return ns, h * br, h * bi


def rexi_original_scalar(x, h, M, mu=None, a=None):
    """REXI(ix) = sum_{n=-N}^{N} Re(beta^{Re}_n / (ix + alpha_n))
    + i Re(beta^{Im}_n / (ix + alpha_n)), eq. originalRexi (x real)."""
    if mu is None or a is None:
        mu, a = table_a()
    x = np.asarray(x, dtype=np.float64)
    ns, br, bi = beta_coeffs_sliced(h, M, mu, a)
    acc = np.zeros(x.shape, dtype=np.complex128)
    for idx, n in enumerate(ns):
        den = 1j * x + alpha(n, h, mu)
        acc += (br[idx] / den).real + 1j * (bi[idx] / den).real
    return acc


def alpha(n, h, mu):
    """alpha_n = h (mu + i n), Section 2.1 Step 3."""
    return h * (mu + 1j * np.asarray(n, dtype=np.float64))


def rexii_scalar(x, h, M, mu=None, a=None):
    """REXII(ix) = sum_{n=-N}^{N} (c1_n h mu + c2_n (x + h n)) / ((alpha_{-n} - i x)(alpha_n + i x)),
    eq. modifiedRexi.  x real (array)."""
    if mu is None or a is None:
        mu, a = table_a()
    x = np.asarray(x, dtype=np.float64)
    ns, c1, c2 = c_coeffs(h, M, mu, a)
    acc = np.zeros(x.shape, dtype=np.complex128)
    for idx, n in enumerate(ns):
        num = c1[idx] * h * mu + c2[idx] * (x + h * n)
        den = (alpha(-n, h, mu) - 1j * x) * (alpha(n, h, mu) + 1j * x)
        acc += num / den
    return acc


def rexi_double_sum(x, h, M, mu=None, a=None):
    """Brute-force double sum of eq. RexiNotSimplified:
    sum_{m=-M}^{M} b_m sum_{l=-L}^{L} Re( h a_l / (i x + h (mu + i (m + l))) )."""
    if mu is None or a is None:
        mu, a = table_a()
    x = np.asarray(x, dtype=np.float64)
    acc = np.zeros(x.shape, dtype=np.complex128)
    for m in range(-M, M + 1):
        inner = np.zeros(x.shape, dtype=np.float64)
        for l in range(-L, L + 1):
            inner += (h * a[L + l] / (1j * x + h * (mu + 1j * (m + l)))).real
        acc += b_coeff(m, h) * inner
    return acc


def c_tol(tol):
    """c = 2 sqrt(-log(sqrt(4 pi) tol)): psi_h(z) <= tol for |z| >= c h, Appendix B."""
    return 2.0 * math.sqrt(-math.log(math.sqrt(4.0 * math.pi) * tol))


def m0_tol(tol):
    """m_0 = c - 1 rounded up to an integer (Appendix B; m_0 = 11 at tol = 1e-16)."""
    return int(math.ceil(c_tol(tol) - 1.0))


def pole_count_M(tau_rho, h, tol):
    """Smallest M with tau rho(A) <= (M - m_0) h, eq. matrixAccuracyBound with the
    m_0 of Appendix B.  For tol = 1e-16 this is the paper's M = ceil(rho/h) + 11."""
    if not (0.0 < h < math.pi):
        raise ValueError("h must lie in (0, pi) (Section 2.1 Step 1)")
    return int(math.ceil(tau_rho / h)) + m0_tol(tol)


def appendix_b_tail_bound():
    """sum_{k>=1} e^{-4 pi^2 k} = 1/(1 - e^{-4 pi^2}) - 1, Appendix B (~7.15e-18)."""
    q = math.exp(-4.0 * math.pi ** 2)
    return q / (1.0 - q)


def matrix_term_weights(h, M, real_input=True, mu=None, a=None):
    """Per-term data of eq. REXI_Modified_matrix / modifiedRexiMatrixReducedSum.

    Returns a list of (n, alpha_n, alpha_{-n}, C1_n, C2_n, Gamma_n) with
    C1_n = c1_n h mu + c2_n h n and C2_n = i c2_n.  Real input: n = 0..N with
    Gamma_0 = 1, Gamma_n = 2; complex input: n = -N..N with Gamma_n = 1.
    """
    if mu is None or a is None:
        mu, a = table_a()
    ns, c1, c2 = c_coeffs(h, M, mu, a)
    N = M + L
    out = []
    for idx, n in enumerate(ns):
        if real_input and n < 0:
            continue
        gamma = 1.0 if (not real_input or n == 0) else 2.0
        C1 = c1[idx] * h * mu + c2[idx] * h * n
        C2 = 1j * c2[idx]
        out.append((int(n), alpha(n, h, mu), alpha(-n, h, mu), C1, C2, gamma))
    assert len(out) == (N + 1 if real_input else 2 * N + 1)
    return out


def single_shift_poles(h, M, real_input=True, mu=None, a=None):
    """Partial-fraction form of each REXII term: with z = tau * eigenvalue,
    (C1 - C2 z) / ((alpha_{-n} - z)(alpha_n + z))
        = P_n / (alpha_{-n} - z) + Q_n / (alpha_n + z),
    P_n = (C1 - C2 alpha_{-n}) / (alpha_n + alpha_{-n}),
    Q_n = (C1 + C2 alpha_n) / (alpha_n + alpha_{-n}).
    Returned as poles z_j and weights beta_j of  sum_j beta_j / (z - z_j)
    (Gamma_n folded into beta_j): z = alpha_{-n}, beta = -Gamma P_n and
    z = -alpha_n, beta = Gamma Q_n.  J = 2(N+1) (real) or 2(2N+1) (complex).
    """
    poles, weights = [], []
    for n, an, amn, C1, C2, gam in matrix_term_weights(h, M, real_input, mu, a):
        P = (C1 - C2 * amn) / (an + amn)
        Q = (C1 + C2 * an) / (an + amn)
        poles.append(amn)
        weights.append(-gam * P)
        poles.append(-an)
        weights.append(gam * Q)
    return np.array(poles), np.array(weights)
