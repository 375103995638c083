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
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import coeffs


def rexii_apply_sparse(A, f0, tau, h, M, real_input=True, terms=None):
    """r(tau A) f0 with one sparse LU pair per term.

    ``A`` scipy.sparse (real), ``f0`` 1-D vector.  ``terms`` optionally
    restricts the sum to a subset of term indices n (for pole-partition
    tests).  Returns a complex vector (real part taken when real_input).
    """
    f0 = np.asarray(f0)
    n_unk = A.shape[0]
    Id = sp.identity(n_unk, dtype=np.complex128, format="csc")
    Ac = sp.csc_matrix(A, dtype=np.complex128)
    acc = np.zeros(n_unk, dtype=np.complex128)
    for n, an, amn, C1, C2, gam in coeffs.matrix_term_weights(h, M, real_input):
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
    for n, an, amn, C1, C2, gam in coeffs.matrix_term_weights(h, M, real_input):
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
