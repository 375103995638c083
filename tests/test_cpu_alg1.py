"""The Algorithm 1 CPU baseline (baseline/alg1_cpu.py) computes the same REXII
step as the oracle's sparse solve chain (CPU only)."""
import numpy as np

from baseline import alg1_cpu as A1
from oracle import coeffs as C
from oracle import operator as O
from oracle import rexi as R
from paper_2008_11607_gb300 import inputs


def test_alg1_matches_sparse_oracle():
    nx, ny = 16, 12
    st = inputs.kminus3_field(nx, ny, seed=4)
    st[1] = inputs.kminus3_field(nx, ny, seed=5)[0]
    rho = O.spectral_radius_constant(nx, ny)
    dt = 25.0 / rho
    M = C.pole_count_M(25.0, 0.5, 1e-10)
    got = A1.Alg1(nx, ny, dt, 0.5, M, threads=2, block_rows=5).step(st)
    ref = R.rexii_apply_sparse(O.cgrid_operator(nx, ny), st.ravel(), dt, 0.5, M).reshape(st.shape)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12


def test_alg1_sample_timing_runs():
    st = inputs.kminus3_field(32, 32, seed=0)
    est, det = A1.time_sample(32, 32, 0.1, 0.5, 40, st, 8, threads=2)
    assert est > 0 and det["terms_sampled"] == 8 and det["terms_total"] == 65
