"""Helpers shared by the GPU parity tests (oracle calls + device plumbing)."""
import math

import numpy as np
import pytest

from oracle import coeffs as C
from oracle import operator as O
from oracle import rexi as R


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11607_gb300 import build as B

    B.build()
    return torch


def to_dev(torch, arr):
    return torch.from_numpy(np.ascontiguousarray(arr, dtype=np.complex128)).cuda()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def oracle_step(state, dt, M, real_input=True, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0, h=0.5, terms=None):
    _, ny, nx = state.shape
    A = O.cgrid_operator(nx, ny, Lx, Ly, g, f, H)
    out = R.rexii_apply_sparse(A, state.ravel(), dt, h, M, real_input=real_input, terms=terms)
    return out.reshape(state.shape)


TOL = {"fp64": 1e-10, "plain": 1e-10, "mixed": 1e-8}
