"""Pins for the oracle's adjoint and depth gradient: the dot-product identity
and central finite differences of the (expm-pinned) forward step."""
import math

import numpy as np

from oracle import adjoint as AD
from oracle import coeffs as C
from oracle import operator as O
from oracle import rexi as R
from paper_2008_11607_gb300 import inputs


def test_adjoint_dot_product():
    nx, ny = 6, 5
    H = inputs.variable_depth(nx, ny, seed=1)
    A = O.cgrid_operator(nx, ny, H=H)
    tau, M = 0.2, 30
    x = inputs.complex_random_state(nx, ny, seed=2).ravel()
    y = inputs.complex_random_state(nx, ny, seed=3).ravel()
    Rx = R.rexii_apply_sparse(A, x, tau, 0.5, M, real_input=False)
    RHy = AD.rexii_adjoint_sparse(A, y, tau, 0.5, M, real_input=False)
    assert abs(np.vdot(y, Rx) - np.vdot(RHy, x)) < 1e-12 * abs(np.vdot(y, Rx))


def test_divergence_matches_operator_row():
    nx, ny = 7, 4
    H = inputs.variable_depth(nx, ny, seed=4)
    A = O.cgrid_operator(nx, ny, Lx=1.2, Ly=0.7, H=H)
    v = inputs.complex_random_state(nx, ny, seed=5).ravel()
    assert np.max(np.abs((A @ v)[:nx * ny] + H.ravel() * AD.divergence(v, nx, ny, 1.2, 0.7))) < 1e-12


def test_grad_depth_central_differences():
    """L = 1/2 ||eta(out) - target||^2 for one step; directional derivative
    along random depth perturbations against central differences (eps 1e-6)."""
    nx, ny = 6, 6
    H = inputs.variable_depth(nx, ny, seed=6)
    f0 = inputs.kminus3_field(nx, ny, seed=7).ravel()
    target = inputs.kminus3_field(nx, ny, seed=8)[0].real.ravel()
    rho = O.spectral_radius_bound(nx, ny, Hmax=H.max() * 1.01)
    tau = 12.0 / rho
    M = C.pole_count_M(12.0, 0.5, 1e-16)
    n = nx * ny

    def loss(Hd):
        out = R.rexii_apply_sparse(O.cgrid_operator(nx, ny, H=Hd), f0, tau, 0.5, M).real
        return 0.5 * np.sum((out[:n] - target) ** 2), out

    L0, out = loss(H)
    G = np.zeros(3 * n, dtype=np.complex128)
    G[:n] = out[:n] - target
    grad = AD.grad_depth_sparse(nx, ny, H, f0, G, tau, 0.5, M)
    rng = np.random.default_rng(0)
    eps = 1e-6
    for _ in range(3):
        d = rng.standard_normal((ny, nx))
        fd = (loss(H + eps * d)[0] - loss(H - eps * d)[0]) / (2 * eps)
        an = float(np.sum(grad * d))
        assert abs(fd - an) < 1e-7 * max(abs(an), 1e-12) + 1e-12, (fd, an)


def test_grad_depth_complex_input():
    nx, ny = 5, 4
    H = inputs.variable_depth(nx, ny, seed=9)
    f0 = inputs.complex_random_state(nx, ny, seed=10).ravel()
    Gt = inputs.complex_random_state(nx, ny, seed=11).ravel()
    tau = 0.15
    M = 30

    def lin(Hd):  # L = Re <Gt, out>
        out = R.rexii_apply_sparse(O.cgrid_operator(nx, ny, H=Hd), f0, tau, 0.5, M, real_input=False)
        return float(np.real(np.vdot(Gt, out)))

    grad = AD.grad_depth_sparse(nx, ny, H, f0, Gt, tau, 0.5, M, real_input=False)
    d = np.random.default_rng(1).standard_normal((ny, nx))
    eps = 1e-6
    fd = (lin(H + eps * d) - lin(H - eps * d)) / (2 * eps)
    assert abs(fd - np.sum(grad * d)) < 1e-7 * abs(fd)
