"""Seeded synthetic workloads: shapes, determinism and the stated recipes."""
import math

import numpy as np

from paper_2008_11607_gb300 import inputs


def test_gaussian_bump():
    s = inputs.gaussian_bump(64, 64)
    assert s.shape == (3, 64, 64) and s.dtype == np.complex128
    # nearest eta points sit (1/128, 1/128) from the centre
    assert abs(s[0].real.max() - 0.1 * math.exp(-2 * (1 / 128) ** 2 / (2 * 0.05 ** 2))) < 1e-15
    assert np.all(s[1:] == 0) and np.all(s.imag == 0)


def test_kminus3_field():
    a = inputs.kminus3_field(128, 96, seed=3)
    b = inputs.kminus3_field(128, 96, seed=3)
    c = inputs.kminus3_field(128, 96, seed=4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert abs(np.max(np.abs(a[0])) - 0.1) < 1e-15
    assert np.all(a.imag == 0) and np.all(a[1:] == 0)
    spec = np.fft.fft2(a[0].real)
    assert abs(spec[0, 0]) < 1e-12  # no mean
    # rebuild from the stated recipe: |k|^-3 amplitudes, phases from default_rng(seed)
    rng = np.random.default_rng(3)
    phase = rng.uniform(0.0, 2 * math.pi, size=(96, 128))
    KX, KY = np.meshgrid(np.fft.fftfreq(128) * 128, np.fft.fftfreq(96) * 96)
    kk = np.hypot(KX, KY)
    amp = np.where(kk > 0, np.where(kk > 0, kk, 1.0) ** -3.0, 0.0)
    eta = np.fft.ifft2(amp * np.exp(1j * phase)).real
    assert np.max(np.abs(a[0].real - 0.1 * eta / np.max(np.abs(eta)))) < 1e-15


def test_variable_depth():
    H = inputs.variable_depth(256, 256, seed=0)
    assert H.shape == (256, 256)
    assert 0.55 < H.min() and H.max() < 1.9
    assert np.array_equal(H, inputs.variable_depth(256, 256, seed=0))


def test_batched_instances():
    b = inputs.batched_instances()
    assert len(b) == 96
    assert {x["nx"] for x in b} <= {128, 192, 256, 384, 512}
    tr = [x["tau_rho"] for x in b]
    assert 20.0 <= min(tr) and max(tr) <= 800.0
