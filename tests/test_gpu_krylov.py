"""Parity of the variable-depth (Krylov) path against the FP64 oracle.

The Krylov path solves each REXII term's pair system with CG to a relative
residual rtol (energy norm).  The error that rtol leaves in the step is
bounded, term by term, by (|c2_n| + |c1_n + i c2_n|) / |h mu| * rtol * ||f||_W
(the CG error in the pair norm is at most ||r|| / |h mu| and the term applies
C1 - C2 tau A = -i c2 (alpha_n + tau A) + (c1 + i c2) h mu); the tests use that
bound, converted to the Euclidean norm, when it exceeds 1e-10.
"""
import math

import numpy as np
import pytest

from oracle import coeffs as C
from oracle import operator as O
from oracle import rexi as R
from paper_2008_11607_gb300 import inputs
from tests.gpu_util import rel_l2, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def error_bound(M, rtol, H, g=1.0, real_input=True, h=0.5):
    mu, a = C.table_a()
    ns, c1, c2 = C.c_coeffs(h, M, mu, a)
    gam = np.where(ns == 0, 1.0, 2.0) if real_input else np.ones(len(ns))
    sel = ns >= 0 if real_input else np.ones(len(ns), bool)
    per = (np.abs(c2) + np.abs(c1 + 1j * c2)) / abs(h * mu)
    w = np.concatenate([g / np.ravel(H), np.ones(2)])
    cond = math.sqrt(w.max() / w.min())  # energy norm vs Euclidean norm
    return float(np.sum(gam[sel] * per[sel])) * rtol * cond


def krylov_plan(torch, nx, ny, depth, rtol=1e-13, max_iters=20000, batch=32, form="fp64", **phys):
    from paper_2008_11607_gb300 import rexi

    Hd = torch.from_numpy(np.ascontiguousarray(depth, dtype=np.float64)).cuda()
    plan = rexi.Plan(nx, ny, depth=Hd, form=form, **phys)
    plan.set_krylov(rtol=rtol, max_iters=max_iters, term_batch=batch)
    return plan


@pytest.mark.parametrize("form", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["12x10_real", "16x16_complex", "9x14_phys"])
def test_variable_depth_against_sparse_oracle(case, form):
    torch = torch_cuda()
    phys = {}
    if case == "12x10_real":
        nx, ny, real = 12, 10, True
        st = inputs.kminus3_field(nx, ny, seed=0)
    elif case == "16x16_complex":
        nx, ny, real = 16, 16, False
        st = inputs.complex_random_state(nx, ny, seed=1)
    else:
        nx, ny, real = 9, 14, True
        st = inputs.gaussian_bump(nx, ny, width=0.2)
        phys = dict(Lx=1.4, Ly=0.9, g=1.7, f=0.5)
    H = inputs.variable_depth(nx, ny, seed=3)
    rtol = 1e-13
    plan = krylov_plan(torch, nx, ny, H, rtol=rtol, form=form, **phys)
    dt = 20.0 / plan.rho
    out, info = plan.step(to_dev(torch, st), dt, real_input=real, want_info=True)
    out = out.cpu().numpy()
    assert info.krylov_unconverged == 0 and info.krylov_max_rel_res <= rtol
    A = O.cgrid_operator(nx, ny, H=H, **phys)
    ref = R.rexii_apply_sparse(A, st.ravel(), dt, 0.5, info.M, real_input=real).reshape(st.shape)
    tol = max(1e-10, error_bound(info.M, rtol, H, phys.get("g", 1.0), real))
    assert rel_l2(out, ref) < tol, (rel_l2(out, ref), tol)
    if real:
        assert np.all(out.imag == 0)


def test_constant_depth_krylov_matches_fourier_path():
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    nx, ny = 24, 20
    st = inputs.kminus3_field(nx, ny, seed=4)
    plan_k = krylov_plan(torch, nx, ny, np.full((ny, nx), 1.3), rtol=1e-13)
    plan_f = rexi.Plan(nx, ny, H=1.3)
    # the Krylov plan uses the rigorous bound for rho; use the same dt for both
    dt = 25.0 / plan_k.rho
    a = plan_k.step(to_dev(torch, st), dt).cpu().numpy()
    b = plan_f.step(to_dev(torch, st), dt).cpu().numpy()
    assert rel_l2(a, b) < 1e-10


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_krylov_adjoint_dot_product(form):
    torch = torch_cuda()
    nx, ny = 14, 12
    H = inputs.variable_depth(nx, ny, seed=6)
    plan = krylov_plan(torch, nx, ny, H, rtol=1e-13, form=form)
    dt = 15.0 / plan.rho
    x = inputs.complex_random_state(nx, ny, seed=7)
    y = inputs.complex_random_state(nx, ny, seed=8)
    Rx = plan.step(to_dev(torch, x), dt, real_input=False).cpu().numpy()
    RHy = plan.step_adjoint(to_dev(torch, y), dt, real_input=False).cpu().numpy()
    lhs, rhs = np.vdot(y, Rx), np.vdot(RHy, x)
    assert abs(lhs - rhs) < 1e-9 * abs(lhs)
    A = O.cgrid_operator(nx, ny, H=H)
    M = C.pole_count_M(15.0, 0.5, 1e-10)
    ref = np.conj(R.rexii_apply_sparse(A.T.tocsr(), np.conj(y).ravel(), dt, 0.5, M, real_input=False))
    assert rel_l2(RHy.ravel(), ref) < max(1e-10, error_bound(M, 1e-13, H, real_input=False))


def test_krylov_term_slices_and_iteration_cap():
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    nx, ny = 16, 12
    H = inputs.variable_depth(nx, ny, seed=9)
    st = inputs.kminus3_field(nx, ny, seed=9)
    plan = krylov_plan(torch, nx, ny, H, rtol=1e-13, batch=8)
    dt = 18.0 / plan.rho
    x = to_dev(torch, st)
    full, info = plan.step(x, dt, want_info=True)
    N = info.N
    parts = plan.step(x, dt, terms=(0, 7)) + plan.step(x, dt, terms=(7, N + 1))
    assert rel_l2(parts.cpu().numpy(), full.cpu().numpy()) < 1e-12
    A = O.cgrid_operator(nx, ny, H=H)
    ref = R.rexii_apply_sparse(A, st.ravel(), dt, 0.5, info.M, terms=set(range(7, N + 1))).reshape(st.shape)
    got = plan.step(x, dt, terms=(7, N + 1)).cpu().numpy()
    assert rel_l2(got, ref) < max(1e-10, error_bound(info.M, 1e-13, H))
    # iteration cap: the device stops every term at max_iters and the host gets ENOCONV
    plan.set_krylov(rtol=1e-13, max_iters=3, term_batch=8)
    with pytest.raises(rexi.RexiError) as e:
        plan.step(x, dt)
    assert e.value.status == rexi.REXI_ENOCONV
    # overlapping input and output are rejected
    plan.set_krylov(rtol=1e-10)
    with pytest.raises(rexi.RexiError) as e:
        plan.step(x, dt, out=x)
    assert e.value.status == rexi.REXI_EINVAL


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_downscaled_config3_against_oracle(form):
    """The variable-depth workload (H = 1 + 0.4 sin(2 pi x) cos(4 pi y) + 8 bumps,
    |k|^-3 height) on a 48 x 48 replica with tau rho = 100 and all terms."""
    torch = torch_cuda()
    n = 48
    H = inputs.variable_depth(n, n, seed=0)
    st = inputs.kminus3_field(n, n, seed=0)
    rtol = 1e-12
    plan = krylov_plan(torch, n, n, H, rtol=rtol, batch=64, form=form)
    dt = 100.0 / plan.rho
    out, info = plan.step(to_dev(torch, st), dt, want_info=True)
    assert info.krylov_unconverged == 0
    A = O.cgrid_operator(n, n, H=H)
    ref = R.rexii_apply_sparse(A, st.ravel(), dt, 0.5, info.M).reshape(st.shape)
    assert rel_l2(out.cpu().numpy(), ref) < max(1e-10, error_bound(info.M, rtol, H))


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_full_size_1024_constant_depth_slice_matches_fourier(form):
    """1024 x 1024, tau rho = 400 (the variable-depth workload's size and pole
    count) with constant depth, hardest terms |n| < 6 (near resonance), against
    the Fourier path on the same slice."""
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    n = 1024
    st = inputs.kminus3_field(n, n, seed=0)
    plan_k = krylov_plan(torch, n, n, np.ones((n, n)), rtol=1e-12, batch=6, form=form)
    plan_f = rexi.Plan(n, n)
    dt = 400.0 / plan_k.rho
    x = to_dev(torch, st)
    a, info = plan_k.step(x, dt, terms=(0, 6), want_info=True)
    b = plan_f.step(x, dt, terms=(0, 6))
    assert info.M == C.pole_count_M(400.0, 0.5, 1e-10)
    assert info.krylov_unconverged == 0
    assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 1e-9
