"""Matrix REXII by sparse direct solves, one pair per term (FP64, scipy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

For each summation index n, Section 4 of arXiv 2008.11607 solves
    (alpha_n I + tau A) g1 = f0,
    (alpha_{-n} I - tau A) g2 = g1,
    g3 = Gamma_n C2_n (g1 + (C1_n / C2_n - alpha_{-n}) g2),
and returns Re sum_{n=0}^{N} g3 (eq. modifiedRexiMatrixReducedSum).  The paper
writes A where the time step tau multiplies it; here tau A is used throughout
(eq. REXI_Modified_matrix).  The factor C2_n is multiplied through,
g3 = Gamma_n (C2_n g1 + (C1_n - C2_n alpha_{-n}) g2), which is the same
algebra without dividing by a C2_n that may be tiny.  Complex input sums
n = -N..N with Gamma_n = 1 and takes no real part.
"""
import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import coeffs


def rexii_apply_sparse(A, f0, tau, h, M, real_input=True, terms=None, mu=None, a=None):
    """r(tau A) f0 with one sparse LU pair per term.

    ``A`` scipy.sparse (real), ``f0`` 1-D vector.  ``terms`` optionally
    restricts the sum to a subset of term indices n (for pole-partition
    tests).  ``mu``, ``a``: another fit of Step 2 than Table tab:coef_al.
    Returns a complex vector (real part taken when real_input).
    """
    f0 = np.asarray(f0)
    n_unk = A.shape[0]
    Id = sp.identity(n_unk, dtype=np.complex128, format="csc")
    Ac = sp.csc_matrix(A, dtype=np.complex128)
    acc = np.zeros(n_unk, dtype=np.complex128)
    for n, an, amn, C1, C2, gam in coeffs.matrix_term_weights(h, M, real_input, mu, a):
        if terms is not None and n not in terms:
            continue
        lu1 = spla.splu((an * Id + tau * Ac).tocsc())
        g1 = lu1.solve(f0.astype(np.complex128))
        lu2 = spla.splu((amn * Id - tau * Ac).tocsc())
        g2 = lu2.solve(g1)
        g3 = gam * (C2 * g1 + (C1 - C2 * amn) * g2)
        acc += g3
    return acc.real.astype(np.complex128) if real_input else acc


def rexii_apply_dense_mode(B, fhat, tau, h, M, real_input=True, term_weights=None):
    """The same per-term chain on one Fourier mode: B is the 3x3 symbol, fhat
    the 3 Fourier coefficients.  Dense numpy solves.  No real part is taken
    (a single mode of a real field is complex); with real_input the sum runs
    over n = 0..N with Gamma_n and the partner mode -k must be handled by the
    caller through conj symmetry, so for single-mode checks use
    real_input=False, which sums n = -N..N and equals r(tau B) fhat.
    """
    I3 = np.eye(3, dtype=np.complex128)
    acc = np.zeros(3, dtype=np.complex128)
    # term_weights: the list matrix_term_weights(h, M, real_input) returns,
    # passed in by callers that evaluate many modes with the same coefficients
    tw = term_weights if term_weights is not None else coeffs.matrix_term_weights(h, M, real_input)
    for n, an, amn, C1, C2, gam in tw:
        g1 = np.linalg.solve(an * I3 + tau * B, fhat)
        g2 = np.linalg.solve(amn * I3 - tau * B, g1)
        acc += gam * (C2 * g1 + (C1 - C2 * amn) * g2)
    return acc


def rexii_apply_poles(A, f0, tau, h, M, real_input=True):
    """r(tau A) f0 via the single-shift partial-fraction poles:
    sum_j beta_j (tau A - z_j I)^{-1} f0 (real part for real input).
    Used only to cross-check the partial-fraction form against the term chain.
    """
    poles, weights = coeffs.single_shift_poles(h, M, real_input)
    n_unk = A.shape[0]
    Id = sp.identity(n_unk, dtype=np.complex128, format="csc")
    Ac = sp.csc_matrix(A, dtype=np.complex128)
    acc = np.zeros(n_unk, dtype=np.complex128)
    for z, w in zip(poles, weights):
        acc += w * spla.splu((tau * Ac - z * Id).tocsc()).solve(np.asarray(f0, dtype=np.complex128))
    return acc.real.astype(np.complex128) if real_input else acc


def rexi_original_apply_sparse(A, f0, tau, h, M):
    """The original REXI for a real matrix A and a real vector f0,
    eq. originalREXImatrix: sum_{n=-N}^{N} Re(beta^{Re}_n (tau A + alpha_n I)^{-1} f0),
    one sparse LU per term (Section 2.3).  Returns a complex vector with zero
    imaginary part."""
    mu, a = coeffs.table_a()
    ns, br, _ = coeffs.beta_coeffs(h, M, mu, a)
    f0 = np.asarray(f0, dtype=np.complex128)
    Id = sp.identity(A.shape[0], dtype=np.complex128, format="csc")
    Ac = sp.csc_matrix(A, dtype=np.complex128)
    acc = np.zeros(A.shape[0])
    for idx, n in enumerate(ns):
        g = spla.splu((tau * Ac + coeffs.alpha(n, h, mu) * Id).tocsc()).solve(f0)
        acc += (br[idx] * g).real
    return acc.astype(np.complex128)


def rexi_original_apply_modes(state, tau, h, M, symbol_fn, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0):
    """eq. originalREXImatrix for a constant-coefficient operator given by its
    per-wavenumber 3x3 symbol (``symbol_fn(kx, ky, nx, ny, Lx, Ly, g, f, H)``):
    the solves (tau A + alpha_n I)^{-1} act mode by mode, so
    sum_n beta^{Re}_n (tau B(k) + alpha_n I)^{-1} fhat(k) is formed for each
    wavenumber with a non-zero coefficient (through the eigen-decomposition of
    tau B(k), numpy.linalg.eig, where the sum of resolvents is diagonal),
    transformed back, and its real part taken in physical space (the Re of
    eq. originalREXImatrix acts on the vector, not mode by mode).  For the
    paper's D = 128 scenarios (Section 4)."""
    state = np.asarray(state, dtype=np.complex128)
    _, ny, nx = state.shape
    mu, a = coeffs.table_a()
    ns, br, _ = coeffs.beta_coeffs_sliced(h, M, mu, a)
    al = coeffs.alpha(ns, h, mu)
    fh = np.fft.fft2(state, axes=(1, 2))
    amp = np.sum(np.abs(fh), axis=0)
    acc = np.zeros_like(fh)
    for ky, kx in np.argwhere(amp > 1e-12 * amp.max()):
        B = symbol_fn(kx, ky, nx, ny, Lx, Ly, g, f, H)
        ev, V = np.linalg.eig(tau * B)
        c = np.linalg.solve(V, fh[:, ky, kx])
        s = np.array([np.sum(br / (e + al)) for e in ev])
        acc[:, ky, kx] = V @ (s * c)
    return np.fft.ifft2(acc, axes=(1, 2)).real.astype(np.complex128)


def rexie_apply(A, f0, tau, h, M, sigma=0.0):
    """REXI Extended, eq. REXIE, for A = iB with B real and f0 real, with the
    shift of the remark in Section 2.2: nu = i sigma, A' = A - nu I,
    e^{tau A} f0 = e^{tau nu} e^{tau A'} f0 and
    e^{tau A'} f0 ~ sum_{n=-N}^{N} Re(beta^{Re}_n g_n) + i Re(beta^{Im}_n g_n),
    g_n = (tau A' + alpha_n I)^{-1} f0: one solve per term (dense LU; A a
    small dense or sparse matrix)."""
    mu, a = coeffs.table_a()
    ns, br, bi = coeffs.beta_coeffs(h, M, mu, a)
    Ad = A.toarray() if sp.issparse(A) else np.asarray(A)
    n_unk = Ad.shape[0]
    Ap = Ad - 1j * sigma * np.eye(n_unk)
    f0 = np.asarray(f0, dtype=np.complex128)
    acc = np.zeros(n_unk, dtype=np.complex128)
    for idx, n in enumerate(ns):
        # LAPACK LU through scipy (numpy.linalg.solve left relative residuals
        # near 1e-11 on some of these shifted systems)
        g = scipy.linalg.lu_solve(scipy.linalg.lu_factor(tau * Ap + coeffs.alpha(n, h, mu) * np.eye(n_unk)), f0)
        acc += (br[idx] * g).real + 1j * (bi[idx] * g).real
    return np.exp(1j * tau * sigma) * acc
