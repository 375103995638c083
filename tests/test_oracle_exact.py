"""Pins for the field-wide closed-form exponential of the oracle (CPU only).

``exp_closed_form_grid`` evaluates e^{tau B(k)} at every wavenumber at once so
that whole 2048 x 2048 outputs can be checked.  It is pinned here against
things other than itself: the one-wavenumber-at-a-time loop
``exp_closed_form`` (which builds each 3x3 symbol by ``operator.symbol``),
dense scipy.linalg.expm of the sparse C-grid operator (Section 3.2's
reference routine), and exact properties of the exponential of a
skew-Hermitian generator (energy conservation, the semigroup property).
"""
import math

import numpy as np
import pytest

from oracle import exact as E
from oracle import operator as O
from paper_2008_11607_gb300 import inputs


@pytest.mark.parametrize("nx,ny,Lx,Ly,g,f,H", [(6, 5, 1.2, 0.8, 1.5, 0.6, 2.0), (8, 8, 1.0, 1.0, 1.0, 1.0, 1.0),
                                             (7, 10, 0.9, 1.4, 2.0, 0.0, 0.5)])
def test_symbol_grid_equals_symbol(nx, ny, Lx, Ly, g, f, H):
    B = O.symbol_grid(nx, ny, Lx, Ly, g, f, H)
    for ky in range(ny):
        for kx in range(nx):
            assert np.max(np.abs(B[:, :, ky, kx] - O.symbol(kx, ky, nx, ny, Lx, Ly, g, f, H))) < 1e-12


@pytest.mark.parametrize("nx,ny,Lx,Ly,g,f,H,tau", [(12, 10, 1.3, 0.8, 2.0, 0.6, 0.7, 0.9),
                                                 (16, 16, 1.0, 1.0, 1.0, 1.0, 1.0, 3.0),
                                                 (9, 7, 1.0, 1.0, 1.0, 0.0, 1.0, 0.2)])
def test_grid_form_equals_per_wavenumber_loop(nx, ny, Lx, Ly, g, f, H, tau):
    st = inputs.complex_random_state(nx, ny, seed=5)
    ref = E.exp_closed_form(st, tau, Lx, Ly, g, f, H)
    got = E.exp_closed_form_grid(st, tau, Lx, Ly, g, f, H)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13


@pytest.mark.parametrize("nx,ny,g,f,H", [(6, 5, 1.5, 0.6, 2.0), (4, 8, 1.0, 1.0, 1.0), (5, 5, 1.0, 0.0, 1.0)])
def test_grid_form_equals_dense_expm(nx, ny, g, f, H):
    """Against scipy.linalg.expm of the sparse operator (f = 0 includes the
    omega = 0 wavenumber k = 0, where the Taylor limit is taken)."""
    A = O.cgrid_operator(nx, ny, 1.1, 0.9, g, f, H)
    st = inputs.complex_random_state(nx, ny, seed=2)
    tau = 0.7
    ref = E.expm_dense(A, st.ravel(), tau).reshape(st.shape)
    got = E.exp_closed_form_grid(st, tau, 1.1, 0.9, g, f, H)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12


def test_grid_form_conserves_energy_and_composes():
    """H = g = 1: B(k) is skew-Hermitian, so e^{tau B} is unitary per
    wavenumber (energy conserved) and e^{2 tau A} = e^{tau A} e^{tau A}."""
    st = inputs.kminus3_field(64, 48, seed=3)
    a = E.exp_closed_form_grid(st, 0.37)
    assert abs(np.linalg.norm(a) / np.linalg.norm(st) - 1.0) < 1e-13
    b = E.exp_closed_form_grid(a, 0.37)
    c = E.exp_closed_form_grid(st, 0.74)
    assert np.linalg.norm(b - c) / np.linalg.norm(c) < 1e-13


def test_grid_form_spectrum_option_is_the_dft_of_the_field():
    st = inputs.complex_random_state(10, 6, seed=9)
    out = E.exp_closed_form_grid(st, 0.5, g=1.2, f=0.4, H=0.8)
    spec = E.exp_closed_form_grid(st, 0.5, g=1.2, f=0.4, H=0.8, spectrum=True)
    assert np.max(np.abs(np.fft.fft2(out, axes=(1, 2)) - spec)) < 1e-12 * np.max(np.abs(spec))
