"""Gradients through the REXII step (variable depth): the depth gradient
against the oracle's per-pole formula, the autograd wrappers, and an
8-step checkpointed rollout against central finite differences (step 1e-6,
32 random directions) and the oracle's adjoint rollout."""
import math

import numpy as np
import pytest

from oracle import adjoint as AD
from oracle import coeffs as C
from oracle import operator as O
from oracle import rexi as R
from paper_2008_11607_gb300 import inputs
from tests.gpu_util import rel_l2, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def plan_for(torch, H, form="fp64", rtol=1e-13, method="cg"):
    from paper_2008_11607_gb300 import rexi

    ny, nx = H.shape
    Hd = torch.from_numpy(np.ascontiguousarray(H, dtype=np.float64)).cuda()
    p = rexi.Plan(nx, ny, depth=Hd, form=form)
    p.set_krylov(rtol=rtol, max_iters=20000, term_batch=64)
    p.set_krylov_method(method)
    return p, Hd


@pytest.mark.parametrize("form", ["fp64", "mixed"])
@pytest.mark.parametrize("real", [True, False])
def test_grad_depth_against_oracle(form, real):
    torch = torch_cuda()
    nx, ny = 10, 8
    H = inputs.variable_depth(nx, ny, seed=2)
    plan, _ = plan_for(torch, H, form)
    dt = 15.3 / plan.rho
    f0 = inputs.kminus3_field(nx, ny, seed=3) if real else inputs.complex_random_state(nx, ny, seed=3)
    G = inputs.complex_random_state(nx, ny, seed=4)
    if real:
        G = G.real.astype(np.complex128)
    got, info = plan.grad_depth(to_dev(torch, f0), to_dev(torch, G), dt, real_input=real, want_info=True)
    ref = AD.grad_depth_sparse(nx, ny, H, f0.ravel(), G.ravel(), dt, 0.5, info.M, real_input=real)
    assert info.krylov_unconverged == 0
    assert rel_l2(got.cpu().numpy(), ref) < 1e-9


def test_autograd_step_against_oracle():
    torch = torch_cuda()
    from paper_2008_11607_gb300.autograd import rexi_step

    nx, ny = 12, 10
    H = inputs.variable_depth(nx, ny, seed=5)
    plan, Hd = plan_for(torch, H)
    Hd.requires_grad_(True)
    dt = 12.3 / plan.rho
    f0 = inputs.kminus3_field(nx, ny, seed=6)
    x = to_dev(torch, f0).requires_grad_(True)
    target = to_dev(torch, inputs.kminus3_field(nx, ny, seed=7))
    out = rexi_step(x, plan, dt, depth=Hd)
    loss = 0.5 * torch.sum(torch.abs(out[0] - target[0]) ** 2)
    gx, gH = torch.autograd.grad(loss, [x, Hd])
    G = np.zeros((3, ny, nx), dtype=np.complex128)
    G[0] = (out[0] - target[0]).detach().cpu().numpy()
    M = C.pole_count_M(12.3, 0.5, 1e-10)
    A = O.cgrid_operator(nx, ny, H=H)
    ref_x = AD.rexii_adjoint_sparse(A, G.ravel(), dt, 0.5, M).reshape(G.shape)
    ref_H = AD.grad_depth_sparse(nx, ny, H, f0.ravel(), G.ravel(), dt, 0.5, M)
    assert rel_l2(gx.cpu().numpy(), ref_x) < 1e-9
    assert rel_l2(gH.cpu().numpy(), ref_H) < 1e-9


def _rollout_setup(torch, n=16, seed=0):
    H = inputs.variable_depth(n, n, seed=seed)
    f0 = inputs.kminus3_field(n, n, seed=seed + 1)
    target = inputs.kminus3_field(n, n, seed=1000)[0].real
    return H, f0, target


@pytest.mark.parametrize("method", ["cg", "shared"])
def test_rollout_gradients_central_differences(method):
    """8 steps of tau rho = 20.3, checkpoints every 2 steps, loss
    1/2 ||eta(T) - eta_target||^2; 16 random state directions and 16 random
    depth directions, central differences with step 1e-6, agreement to 1e-6
    relative.  Per-term CG and the shared-Krylov method."""
    torch = torch_cuda()
    from paper_2008_11607_gb300.autograd import rexi_rollout

    n, steps = 16, 8
    H, f0, target = _rollout_setup(torch, n)
    plan, Hd = plan_for(torch, H, method=method)
    dt = 20.3 / plan.rho
    tgt = torch.from_numpy(target).cuda()

    def loss_of(plan_, x):
        s = x
        for _ in range(steps):
            s = plan_.step(s, dt)
        return 0.5 * float(torch.sum((s[0].real - tgt) ** 2))

    x = to_dev(torch, f0).requires_grad_(True)
    Hd.requires_grad_(True)
    sT = rexi_rollout(x, plan, dt, steps, every=2, depth=Hd)
    loss = 0.5 * torch.sum((sT[0].real - tgt) ** 2)
    gx, gH = torch.autograd.grad(loss, [x, Hd])
    rng = np.random.default_rng(42)
    eps = 1e-6
    base = to_dev(torch, f0)
    for _ in range(16):  # state directions (real perturbations of eta, u, v)
        d = rng.standard_normal((3, n, n))
        dd = to_dev(torch, d)
        fd = (loss_of(plan, base + eps * dd) - loss_of(plan, base - eps * dd)) / (2 * eps)
        an = float(torch.sum(gx.real * dd.real))
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-12, (fd, an)
    for _ in range(16):  # depth directions
        d = rng.standard_normal((n, n))
        pp, _ = plan_for(torch, H + eps * d, method=method)
        pm, _ = plan_for(torch, H - eps * d, method=method)
        fd = (loss_of(pp, base) - loss_of(pm, base)) / (2 * eps)
        an = float(torch.sum(gH * torch.from_numpy(d).cuda()))
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-12, (fd, an)


@pytest.mark.parametrize("n,steps,every", [(8, 4, 2), (32, 4, 2), (64, 2, 1)])
def test_rollout_against_oracle_adjoint(n, steps, every):
    """The checkpointed rollout's gradients against the oracle's adjoint
    rollout (one sparse LU per pole for the forward states, the adjoint steps
    and the depth gradients), at 8^2 and at the 32^2 - 64^2 sizes the oracle
    handles in under a minute."""
    torch = torch_cuda()
    from paper_2008_11607_gb300.autograd import rexi_rollout

    H, f0, target = _rollout_setup(torch, n, seed=3)
    plan, Hd = plan_for(torch, H)
    dt = 10.3 / plan.rho
    M = C.pole_count_M(10.3, 0.5, 1e-10)
    x = to_dev(torch, f0).requires_grad_(True)
    Hd.requires_grad_(True)
    sT = rexi_rollout(x, plan, dt, steps, every=every, depth=Hd)
    loss = 0.5 * torch.sum((sT[0].real - torch.from_numpy(target).cuda()) ** 2)
    gx, gH = torch.autograd.grad(loss, [x, Hd])
    # oracle: forward states, then adjoint steps and depth gradients backwards
    A = O.cgrid_operator(n, n, H=H)
    states = [f0.ravel()]
    for _ in range(steps):
        states.append(R.rexii_apply_sparse(A, states[-1], dt, 0.5, M))
    G = np.zeros(3 * n * n, dtype=np.complex128)
    G[: n * n] = states[-1][: n * n].real - target.ravel()
    gH_ref = np.zeros((n, n))
    for j in reversed(range(steps)):
        gH_ref += AD.grad_depth_sparse(n, n, H, states[j], G, dt, 0.5, M)
        G = AD.rexii_adjoint_sparse(A, G, dt, 0.5, M)
    assert rel_l2(gx.cpu().numpy().ravel(), G) < 1e-9
    assert rel_l2(gH.cpu().numpy(), gH_ref) < 1e-9


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_config5_full_size_central_differences(form):
    """The differentiation workload at its stated size: 512^2, depth
    H = 1 + 0.4 sin(2 pi x) cos(4 pi y) + 8 bumps, |k|^-3 initial state,
    8 REXII steps of tau rho = 200.3 (M = 410), checkpoints every 2 steps, loss
    1/2 ||eta(T) - eta_target||^2 (|k|^-3 target, seed 1000), shared-Krylov
    method with error bound 1e-13.  32 random state directions and 32 random
    depth directions by central differences with step 1e-6.  "Agree to 1e-6
    relative error" is read as the relative error of the gradient sampled on
    those directions: for each set of 32 the l2 norm of (fd - adjoint) over
    the directions is within 1e-6 of the l2 norm of the adjoint's directional
    derivatives, and each direction is within 1e-6 of the larger of its own
    derivative and their root mean square.  A direction nearly orthogonal to
    the gradient cannot be held to 1e-6 of its own small derivative: each
    loss evaluation carries FP64 rounding noise of about 1e-12 of |L| = 588
    that the + and - problems do not share (measured: the differences scatter
    by 3e-7 at step 1e-6 and agree to 3e-8 at step 1e-5), which is 1.5e-6 of a
    derivative of 0.33 while the depth derivatives' rms is 4.7.  The loss of a perturbed problem is only
    as smooth as the Krylov stopping rule (its step count can change between
    the + and - evaluations), which adds about rtol |L| / (2 eps) to a
    difference quotient: the bound 1e-13 keeps that below 1e-7 of it.  The
    difference L(+) - L(-) is formed point by point as
    1/2 sum (s+ - s-)(s+ + s- - 2 target) before the sum over the grid:
    the same central difference, without the rounding of two sums of
    262,144 terms (about 1e-12 of |L| = 588 each, which divided by 2 eps
    alone would be 1e-6 of a depth derivative of 0.3)."""
    torch = torch_cuda()
    from paper_2008_11607_gb300.autograd import rexi_rollout

    n, steps, every = 512, 8, 2
    H = inputs.variable_depth(n, n, seed=0)
    f0 = inputs.kminus3_field(n, n, seed=0)
    target = inputs.kminus3_field(n, n, seed=1000)[0].real
    plan, Hd = plan_for(torch, H, form=form, rtol=1e-13, method="shared")
    dt = 200.3 / plan.rho
    tgt = torch.from_numpy(target).cuda()

    def eta_of(plan_, x):
        s = x
        for _ in range(steps):
            s = plan_.step(s, dt)
        return s[0].real

    def loss_diff(ep, em):  # L(+) - L(-) for the final heights ep, em
        return 0.5 * float(torch.sum((ep - em) * (ep + em - 2.0 * tgt)))

    x = to_dev(torch, f0).requires_grad_(True)
    Hd.requires_grad_(True)
    sT = rexi_rollout(x, plan, dt, steps, every=every, depth=Hd)
    loss = 0.5 * torch.sum((sT[0].real - tgt) ** 2)
    gx, gH = torch.autograd.grad(loss, [x, Hd])
    rng = np.random.default_rng(512)
    eps = 1e-6
    base = to_dev(torch, f0)
    def check(kind, fds, ans):
        fds, ans = np.array(fds), np.array(ans)
        rel = np.linalg.norm(fds - ans) / np.linalg.norm(ans)
        scale = np.maximum(np.abs(ans), np.sqrt(np.mean(ans ** 2)))
        worst = float(np.max(np.abs(fds - ans) / scale))
        print("config 5, %s, %s: relative l2 error over 32 directions %.2e, worst scaled %.2e"
              % (form, kind, rel, worst))
        assert rel <= 1e-6, (kind, rel)
        assert worst <= 1e-6, (kind, worst, list(zip(fds, ans)))

    fds, ans = [], []
    for _ in range(32):
        d = to_dev(torch, rng.standard_normal((3, n, n)))
        fds.append(loss_diff(eta_of(plan, base + eps * d), eta_of(plan, base - eps * d)) / (2 * eps))
        ans.append(float(torch.sum(gx.real * d.real)))
    check("state", fds, ans)
    fds, ans = [], []
    for _ in range(32):
        d = rng.standard_normal((n, n))
        pp, _ = plan_for(torch, H + eps * d, form=form, rtol=1e-13, method="shared")
        pm, _ = plan_for(torch, H - eps * d, form=form, rtol=1e-13, method="shared")
        fds.append(loss_diff(eta_of(pp, base), eta_of(pm, base)) / (2 * eps))
        ans.append(float(torch.sum(gH * torch.from_numpy(d).cuda())))
    check("depth", fds, ans)
