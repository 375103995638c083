"""CPU baseline after Algorithm 1 of Section 4.1 (the paper's CPU
implementation), for the constant-depth C-grid step, on all host cores.

Structure (as in Algorithm 1): transform the initial data; compute all
C_{1,n}, C_{2,n}; then sequentially over the REXII terms n = 0..N solve the
first shifted system (alpha_n I + tau A) g1 = f0 for every wavenumber, apply
the operator to g1 to prepare the second system, solve
(alpha_{-n} I - tau A) g2 = g1, and reduce
acc += Gamma_n (C_{2,n} g1 + (C_{1,n} - C_{2,n} alpha_{-n}) g2)
(the reduce line read as in eq. modifiedRexiMatrixReducedSum); finally the
inverse transform and the real part.  Per wavenumber the shifted solve with
the 3x3 C-grid symbol B (B^3 = -w^2 B) is the closed form
(a I + t B)^{-1} v = v/a - t Bv/(a^2 + t^2 w^2) + t^2 B^2 v/(a (a^2 + t^2 w^2)),
the analogue of the paper's Helmholtz solve plus velocity update.

Real input, as in Algorithm 1: complex transforms of the full spectrum, the
reduced sum n = 0..N of eq. modifiedRexiMatrixReducedSum, and the real part
after the inverse transform (on the half spectrum alone the reduced sum would
lose its real part's Hermitian half).  The wavenumber rows are split into blocks processed by a pool of
threads (NumPy releases the interpreter lock inside its array operations), one
block per task, every term applied to a block before the next block, as the
paper's OpenMP loop parallelises each term over space.

Coefficients come from the oracle's transcription of Table A and Section 2.1
(``oracle.coeffs``); everything timed per term is this module's own code.
Test infrastructure / measurement only: nothing in the library imports it.
"""
import concurrent.futures as cf
import math
import os
import time

import numpy as np

from oracle import coeffs as C


def symbol_entries(nx, ny, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0):
    """The six non-zero symbol entries at every wavenumber (ny, nx):
    (B01, B02, B10, B12, B20, B21), and w^2 (sum of the principal 2x2 minors)."""
    kx = np.arange(nx)
    ky = np.arange(ny)
    ex = np.exp(2j * np.pi * kx / nx)[None, :]
    ey = np.exp(2j * np.pi * ky / ny)[:, None]
    dx, dy = Lx / nx, Ly / ny
    shape = (ny, nx)
    b01 = np.broadcast_to(-H * (1.0 - 1.0 / ex) / dx, shape)
    b02 = np.broadcast_to(-H * (1.0 - 1.0 / ey) / dy, shape)
    b10 = np.broadcast_to(-g * (ex - 1.0) / dx, shape)
    b20 = np.broadcast_to(-g * (ey - 1.0) / dy, shape)
    b12 = f * (1.0 + ex) * (1.0 + 1.0 / ey) / 4.0
    b21 = -f * (1.0 + 1.0 / ex) * (1.0 + ey) / 4.0
    w2 = (-(b01 * b10) - (b02 * b20) - (b12 * b21)).real
    return [np.ascontiguousarray(b) for b in (b01, b02, b10, b12, b20, b21)], np.ascontiguousarray(w2)


def _apply(B, v):
    b01, b02, b10, b12, b20, b21 = B
    return (b01 * v[1] + b02 * v[2], b10 * v[0] + b12 * v[2], b20 * v[0] + b21 * v[1])


def _solve(B, w2, a, t, v):
    """(a I + t B)^{-1} v per wavenumber (closed form above)."""
    Bv = _apply(B, v)
    BBv = _apply(B, Bv)
    d = a * a + (t * t) * w2
    c1 = t / d
    c2 = (t * t) / (a * d)
    return tuple(v[i] / a - c1 * Bv[i] + c2 * BBv[i] for i in range(3))


def term_list(h, M):
    """(alpha_n, alpha_{-n}, Gamma_n C_{2,n}, Gamma_n (C_{1,n} - C_{2,n} alpha_{-n})) for n = 0..N."""
    mu, a = C.table_a()
    ns, c1, c2 = C.c_coeffs_sliced(h, M, mu, a)
    N = M + C.L
    out = []
    for n in range(0, N + 1):
        i = n + N
        gam = 1.0 if n == 0 else 2.0
        an = h * (mu + 1j * n)
        amn = h * (mu - 1j * n)
        C1 = c1[i] * h * mu + c2[i] * h * n
        C2 = 1j * c2[i]
        out.append((an, amn, gam * C2, gam * (C1 - C2 * amn)))
    return out


class Alg1:
    """One REXII step of the constant-depth C-grid operator after Algorithm 1."""

    def __init__(self, nx, ny, tau, h, M, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0, threads=None, block_rows=32):
        self.nx, self.ny, self.tau = nx, ny, tau
        self.threads = threads or os.cpu_count() or 1
        self.B, self.w2 = symbol_entries(nx, ny, Lx, Ly, g, f, H)
        self.terms = term_list(h, M)
        self.blocks = [(r, min(r + block_rows, ny)) for r in range(0, ny, block_rows)]

    def forward(self, state):
        return np.fft.fft2(np.asarray(state, dtype=np.complex128), axes=(1, 2))

    def inverse(self, acc):
        return np.fft.ifft2(acc, axes=(1, 2)).real.astype(np.complex128)

    def _block(self, fh, acc, r0, r1, terms):
        B = [b[r0:r1] for b in self.B]
        w2 = self.w2[r0:r1]
        v = (fh[0, r0:r1], fh[1, r0:r1], fh[2, r0:r1])
        a = [np.zeros_like(v[0]) for _ in range(3)]
        t = self.tau
        for an, amn, gC2, gP in terms:
            g1 = _solve(B, w2, an, t, v)       # (alpha_n I + tau B) g1 = f
            g2 = _solve(B, w2, amn, -t, g1)    # (alpha_{-n} I - tau B) g2 = g1
            for i in range(3):
                a[i] += gC2 * g1[i] + gP * g2[i]
        for i in range(3):
            acc[i, r0:r1] = a[i]

    def sum_terms(self, fh, terms=None):
        terms = self.terms if terms is None else terms
        acc = np.zeros_like(fh)
        with cf.ThreadPoolExecutor(max_workers=self.threads) as ex:
            list(ex.map(lambda b: self._block(fh, acc, b[0], b[1], terms), self.blocks))
        return acc

    def step(self, state):
        return self.inverse(self.sum_terms(self.forward(state)))


def time_sample(nx, ny, tau, h, M, state, n_terms_sample, threads=None):
    """Times the transforms once and `n_terms_sample` evenly spaced terms over
    the whole spectrum; returns (seconds per full step estimated as
    transforms + (N + 1) / n_sample x sampled-term time, details)."""
    t0 = time.perf_counter()
    alg = Alg1(nx, ny, tau, h, M, threads=threads)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    fh = alg.forward(state)
    t_fwd = time.perf_counter() - t0
    idx = np.unique(np.linspace(0, len(alg.terms) - 1, n_terms_sample).round().astype(int))
    sample = [alg.terms[i] for i in idx]
    t0 = time.perf_counter()
    acc = alg.sum_terms(fh, sample)
    t_terms = time.perf_counter() - t0
    t0 = time.perf_counter()
    alg.inverse(acc)
    t_inv = time.perf_counter() - t0
    n_all = len(alg.terms)
    est = t_fwd + t_inv + t_setup + t_terms * n_all / len(sample)
    return est, {"setup_s": t_setup, "forward_fft_s": t_fwd, "inverse_fft_s": t_inv, "terms_sampled": len(sample),
                 "terms_total": n_all, "sampled_terms_s": t_terms, "threads": alg.threads}


def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                low = ln.lower()
                if low.startswith("model name") or low.startswith("cpu part") or low.startswith("hardware"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.processor() or platform.machine()
