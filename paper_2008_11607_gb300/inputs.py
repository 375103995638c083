"""Seeded synthetic workloads (no REXI arithmetic in here).

Shared by the tests, the oracle checks and the benchmark so that both sides of
every comparison see the same arrays.  States are complex128 arrays shaped
(3, ny, nx) = (eta, u, v) on the staggered grid (eta at cell centres), x fastest.
"""
import math

import numpy as np


def cell_centres(nx, ny, Lx=1.0, Ly=1.0):
    """Coordinates of the eta points ((i + 1/2) dx, (j + 1/2) dy), shaped (ny, nx)."""
    x = (np.arange(nx) + 0.5) * (Lx / nx)
    y = (np.arange(ny) + 0.5) * (Ly / ny)
    return np.meshgrid(x, y, indexing="xy")


def gaussian_bump(nx, ny, amp=0.1, width=0.05, Lx=1.0, Ly=1.0, centre=(0.5, 0.5)):
    """eta = amp exp(-r^2 / (2 width^2)), r from ``centre`` by the periodic
    minimum image; u = v = 0."""
    X, Y = cell_centres(nx, ny, Lx, Ly)
    ddx = X - centre[0]
    ddy = Y - centre[1]
    ddx -= Lx * np.round(ddx / Lx)
    ddy -= Ly * np.round(ddy / Ly)
    state = np.zeros((3, ny, nx), dtype=np.complex128)
    state[0] = amp * np.exp(-(ddx ** 2 + ddy ** 2) / (2.0 * width ** 2))
    return state


def kminus3_field(nx, ny, seed, max_abs=0.1):
    """Random smooth height field: Fourier amplitude |k|^-3 on integer wave
    vectors k != 0 (0 at k = 0), phases uniform from default_rng(seed); the
    real part of the inverse transform (i.e. the Hermitian-symmetrised
    spectrum) scaled to max|eta| = max_abs; u = v = 0."""
    rng = np.random.default_rng(seed)
    kx = np.fft.fftfreq(nx) * nx
    ky = np.fft.fftfreq(ny) * ny
    KX, KY = np.meshgrid(kx, ky, indexing="xy")
    kk = np.sqrt(KX ** 2 + KY ** 2)
    amp = np.zeros_like(kk)
    nz = kk > 0
    amp[nz] = kk[nz] ** -3.0
    phase = rng.uniform(0.0, 2.0 * math.pi, size=(ny, nx))
    eta = np.fft.ifft2(amp * np.exp(1j * phase)).real
    eta *= max_abs / np.max(np.abs(eta))
    state = np.zeros((3, ny, nx), dtype=np.complex128)
    state[0] = eta
    return state


def complex_random_state(nx, ny, seed, scale=1.0):
    """A genuinely complex state (all three fields), for the complex-input mode."""
    rng = np.random.default_rng(seed)
    return scale * (rng.standard_normal((3, ny, nx)) + 1j * rng.standard_normal((3, ny, nx)))


def white_real_state(nx, ny, seed):
    """Real white-noise state: eta, u and v independent standard normal values
    from default_rng(seed), stored as complex128.  Its spectrum has the same
    expected amplitude at every wavenumber, so a per-wavenumber check of a
    step weighs every wavenumber alike."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((3, ny, nx)).astype(np.complex128)


def variable_depth(nx, ny, seed, n_bumps=8, sigma=0.05, amp=0.1, Lx=1.0, Ly=1.0):
    """H = 1 + 0.4 sin(2 pi x) cos(4 pi y) + n_bumps Gaussian bumps (amplitude
    ``amp``, width ``sigma``, centres uniform from default_rng(seed), periodic
    minimum image), sampled at eta points.  Returns float64 (ny, nx)."""
    rng = np.random.default_rng(seed)
    X, Y = cell_centres(nx, ny, Lx, Ly)
    H = 1.0 + 0.4 * np.sin(2.0 * math.pi * X / Lx) * np.cos(4.0 * math.pi * Y / Ly)
    centres = rng.uniform(0.0, 1.0, size=(n_bumps, 2))
    for cx, cy in centres:
        ddx = X - cx * Lx
        ddy = Y - cy * Ly
        ddx -= Lx * np.round(ddx / Lx)
        ddy -= Ly * np.round(ddy / Ly)
        H += amp * np.exp(-(ddx ** 2 + ddy ** 2) / (2.0 * sigma ** 2))
    return H


def batched_instances(count=96, seed=0, sizes=(128, 192, 256, 384, 512), rho_range=(20.0, 800.0)):
    """Serving-style batch: grid sizes uniform from ``sizes``, tau*rho
    log-uniform in ``rho_range``, |k|^-3 field seeds 0..count-1."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        D = int(rng.choice(sizes))
        tr = float(math.exp(rng.uniform(math.log(rho_range[0]), math.log(rho_range[1]))))
        out.append({"nx": D, "ny": D, "tau_rho": tr, "seed": i})
    return out


def grid_points(nx, ny, Lx=1.0, Ly=1.0):
    """Collocated points (i dx, j dy), shaped (ny, nx) (the spectral grid)."""
    x = np.arange(nx) * (Lx / nx)
    y = np.arange(ny) * (Ly / ny)
    return np.meshgrid(x, y, indexing="xy")


def paper_scenario(name, nx, ny):
    """Initial states of Section 4 on the collocated grid: "ws1" (eq.
    WAVESCENARIO1), "ws2" (eq. WAVESCENARIO2), "gaussian" (eq. GAUSSIANSCENARIO)."""
    X, Y = grid_points(nx, ny)
    pi = math.pi
    s = np.zeros((3, ny, nx), dtype=np.complex128)
    if name == "ws1":
        s[0] = np.sin(4 * pi * X) * np.cos(2 * pi * Y) - 0.2 * np.cos(4 * pi * X) * np.sin(4 * pi * Y)
        s[1] = np.cos(8 * pi * X) * np.cos(2 * pi * Y)
        s[2] = np.cos(4 * pi * X) * np.cos(4 * pi * Y)
    elif name == "ws2":
        s[0] = np.sin(32 * pi * X) * np.cos(16 * pi * Y) - 0.2 * np.cos(32 * pi * X) * np.sin(32 * pi * Y)
        s[1] = np.cos(64 * pi * X) * np.cos(16 * pi * Y)
        s[2] = np.cos(32 * pi * X) * np.cos(32 * pi * Y)
    elif name == "gaussian":
        s[0] = np.exp(-100.0 * ((X - 0.5) ** 2 + (Y - 0.5) ** 2))
        s[1] = 0.1 * np.sin(64 * pi * X) * np.sin(16 * pi * Y)
        s[2] = 0.1 * np.sin(32 * pi * X) * np.sin(32 * pi * Y)
    else:
        raise ValueError(name)
    return s
