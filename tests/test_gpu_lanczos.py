"""Parity of the shared-Krylov (multi-shift Lanczos) method of the
variable-depth path against the FP64 oracle, the per-term CG method and the
Fourier path.

The method stops when its error bound for the whole step, b_k max |phi| on
[-tau rho, tau rho] (relative, energy norm), is below rtol; the tests convert
that to the Euclidean norm with sqrt(max w / min w), w = (g/H, 1, 1).
"""
import math

import numpy as np
import pytest

from oracle import coeffs as C
from oracle import operator as O
from oracle import rexi as R
from paper_2008_11607_gb300 import inputs
from tests.gpu_util import TOL, rel_l2, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def shared_plan(torch, nx, ny, depth, rtol=1e-12, max_iters=20000, form="fp64", **phys):
    from paper_2008_11607_gb300 import rexi

    Hd = torch.from_numpy(np.ascontiguousarray(depth, dtype=np.float64)).cuda()
    plan = rexi.Plan(nx, ny, depth=Hd, form=form, **phys)
    plan.set_krylov(rtol=rtol, max_iters=max_iters, term_batch=64)
    plan.set_krylov_method("shared")
    return plan, Hd


def energy_cond(H, g=1.0):
    w = np.concatenate([g / np.ravel(H), np.ones(1)])
    return math.sqrt(w.max() / w.min())


def energy_norm(x, H, g=1.0):
    e = x[0]
    return math.sqrt(float(np.sum(g / H * np.abs(e) ** 2) + np.sum(np.abs(x[1:]) ** 2)))


@pytest.mark.parametrize("form", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["12x10_real", "16x16_complex", "9x14_phys", "40x36_real", "70x50_complex"])
def test_shared_against_sparse_oracle(case, form):
    torch = torch_cuda()
    phys = {}
    taurho = 20.0
    if case == "12x10_real":
        nx, ny, real = 12, 10, True
        st = inputs.kminus3_field(nx, ny, seed=0)
    elif case == "16x16_complex":
        nx, ny, real = 16, 16, False
        st = inputs.complex_random_state(nx, ny, seed=1)
    elif case == "9x14_phys":
        nx, ny, real = 9, 14, True
        st = inputs.gaussian_bump(nx, ny, width=0.2)
        phys = dict(Lx=1.4, Ly=0.9, g=1.7, f=0.5)
    elif case == "40x36_real":  # two tiles in x, three in y, ragged edges
        nx, ny, real = 40, 36, True
        st = inputs.kminus3_field(nx, ny, seed=2)
        taurho = 60.0
    else:
        nx, ny, real = 70, 50, False
        st = inputs.complex_random_state(nx, ny, seed=3)
        taurho = 45.0
    H = inputs.variable_depth(nx, ny, seed=3)
    rtol = 1e-12
    plan, _ = shared_plan(torch, nx, ny, H, rtol=rtol, form=form, **phys)
    dt = taurho / plan.rho
    out, info = plan.step(to_dev(torch, st), dt, real_input=real, want_info=True)
    out = out.cpu().numpy()
    assert info.krylov_unconverged == 0 and info.krylov_max_rel_res <= rtol
    assert 0 < info.krylov_iters < 20000
    A = O.cgrid_operator(nx, ny, H=H, **phys)
    ref = R.rexii_apply_sparse(A, st.ravel(), dt, 0.5, info.M, real_input=real).reshape(st.shape)
    # the mixed form is double-float for real input (FP64 for complex input)
    tol = max(TOL[form] if real else 1e-10, 10 * rtol * energy_cond(H, phys.get("g", 1.0)))
    assert rel_l2(out, ref) < tol, (rel_l2(out, ref), tol)
    if real:
        assert np.all(out.imag == 0)


def test_shared_matches_per_term_cg():
    """48 x 48 replica of the variable-depth workload, tau rho = 100, all terms:
    shared Lanczos vs one CG per term (both FP64)."""
    torch = torch_cuda()
    n = 48
    H = inputs.variable_depth(n, n, seed=0)
    st = inputs.kminus3_field(n, n, seed=0)
    plan, _ = shared_plan(torch, n, n, H, rtol=1e-12)
    dt = 100.0 / plan.rho
    x = to_dev(torch, st)
    a, info = plan.step(x, dt, want_info=True)
    plan.set_krylov_method("cg")
    plan.set_krylov(rtol=1e-13, term_batch=64)
    b = plan.step(x, dt)
    assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 1e-10
    A = O.cgrid_operator(n, n, H=H)
    ref = R.rexii_apply_sparse(A, st.ravel(), dt, 0.5, info.M).reshape(st.shape)
    assert rel_l2(a.cpu().numpy(), ref) < 1e-10
    # Lanczos steps stay within a small multiple of tau rho
    assert info.krylov_iters < 4 * 100 + 64


def test_shared_adjoint_against_oracle():
    torch = torch_cuda()
    nx, ny = 14, 12
    H = inputs.variable_depth(nx, ny, seed=6)
    plan, _ = shared_plan(torch, nx, ny, H, rtol=1e-13)
    dt = 15.0 / plan.rho
    x = inputs.complex_random_state(nx, ny, seed=7)
    y = inputs.complex_random_state(nx, ny, seed=8)
    Rx = plan.step(to_dev(torch, x), dt, real_input=False).cpu().numpy()
    RHy = plan.step_adjoint(to_dev(torch, y), dt, real_input=False).cpu().numpy()
    lhs, rhs = np.vdot(y, Rx), np.vdot(RHy, x)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    A = O.cgrid_operator(nx, ny, H=H)
    M = C.pole_count_M(15.0, 0.5, 1e-10)
    ref = np.conj(R.rexii_apply_sparse(A.T.tocsr(), np.conj(y).ravel(), dt, 0.5, M, real_input=False))
    assert rel_l2(RHy.ravel(), ref) < 1e-10
    # real-input adjoint: real output
    g = inputs.kminus3_field(nx, ny, seed=9)
    gr = plan.step_adjoint(to_dev(torch, g), dt, real_input=True).cpu().numpy()
    refr = R.rexii_apply_sparse(A.T.tocsr(), g.ravel(), dt, 0.5, M, real_input=True).reshape(g.shape)
    assert np.all(gr.imag == 0) and rel_l2(gr, refr) < 1e-10


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_shared_kept_basis_is_bitwise_identical(form):
    """Vectors kept from the first pass and vectors regenerated in the second
    are the same bits, so the output does not depend on the workspace size."""
    torch = torch_cuda()
    nx, ny = 40, 36
    H = inputs.variable_depth(nx, ny, seed=4)
    st = inputs.kminus3_field(nx, ny, seed=4)
    plan, _ = shared_plan(torch, nx, ny, H, rtol=1e-12, form=form)
    dt = 50.0 / plan.rho
    x = to_dev(torch, st)
    base = plan.workspace_size(dt)
    vec = (3 * nx * ny * 16 + 255) // 256 * 256
    outs = []
    for extra in (0, 1, 2, 7, 10000):
        ws = torch.empty(base + extra * vec, dtype=torch.uint8, device="cuda")
        out, info = plan.step(x, dt, workspace=ws, want_info=True)
        outs.append(out)
    assert info.krylov_iters < 10000
    for o in outs[1:]:
        assert torch.equal(o, outs[0])


@pytest.mark.parametrize("form,real", [("fp64", True), ("mixed", True), ("fp64", False)])
def test_shared_stop_flag_after_convergence(form, real):
    """The host tests a chunk of Lanczos steps while the next chunk runs; the
    device repeats the test and stops that next chunk at once.  A converged
    step reports as run exactly the steps it converged at; its output agrees
    to rounding with that of a plan whose step cap equals that count (there
    the converged chunk is the last one and nothing is enqueued behind it;
    the cap sizes the workspace, and with it how the coefficient sums group
    the poles), and a second call on the same plan gives the same bits."""
    torch = torch_cuda()
    nx, ny = 40, 36
    H = inputs.variable_depth(nx, ny, seed=6)
    st = inputs.kminus3_field(nx, ny, seed=6) if real else inputs.complex_random_state(nx, ny, seed=6)
    plan, _ = shared_plan(torch, nx, ny, H, rtol=1e-11, form=form)
    dt = 120.0 / plan.rho
    x = to_dev(torch, st)
    out, info = plan.step(x, dt, real_input=real, want_info=True)
    kk = int(info.krylov_iters)
    assert int(info.krylov_term_iters) == kk
    assert kk < 20000
    capped, _ = shared_plan(torch, nx, ny, H, rtol=1e-11, max_iters=kk, form=form)
    out2, info2 = capped.step(x, dt, real_input=real, want_info=True)
    assert int(info2.krylov_iters) == kk
    assert rel_l2(out.cpu().numpy(), out2.cpu().numpy()) < 1e-13
    # a second call on the same plan starts with a cleared flag
    out3, info3 = plan.step(x, dt, real_input=real, want_info=True)
    assert int(info3.krylov_iters) == kk
    assert torch.equal(out, out3)


def test_shared_edges():
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    nx, ny = 16, 12
    H = inputs.variable_depth(nx, ny, seed=9)
    st = inputs.kminus3_field(nx, ny, seed=9)
    plan, _ = shared_plan(torch, nx, ny, H, rtol=1e-12)
    dt = 18.0 / plan.rho
    x = to_dev(torch, st)
    full, info = plan.step(x, dt, want_info=True)
    N = info.N
    # zero input: zero output
    z = plan.step(torch.zeros_like(x), dt)
    assert torch.count_nonzero(z).item() == 0
    # a uniform height with zero velocity is in the kernel of A: out = r(0) f
    const = np.zeros_like(st)
    const[0] = 0.7
    y = plan.step(to_dev(torch, const), dt).cpu().numpy()
    r0 = complex(C.rexii_scalar(np.array([0.0]), 0.5, info.M)[0]).real
    assert np.max(np.abs(y - r0 * const)) < 1e-12
    # term slices sum to the full step (each slice to its own bound)
    parts = plan.step(x, dt, terms=(0, 7)) + plan.step(x, dt, terms=(7, N + 1))
    assert rel_l2(parts.cpu().numpy(), full.cpu().numpy()) < 1e-10
    A = O.cgrid_operator(nx, ny, H=H)
    ref = R.rexii_apply_sparse(A, st.ravel(), dt, 0.5, info.M, terms=set(range(7, N + 1))).reshape(st.shape)
    got = plan.step(x, dt, terms=(7, N + 1)).cpu().numpy()
    assert rel_l2(got, ref) < 1e-10
    # empty slice: zeros
    e = plan.step(x, dt, terms=(3, 3))
    assert torch.count_nonzero(e).item() == 0
    # step cap: ENOCONV
    plan.set_krylov(rtol=1e-12, max_iters=16)
    with pytest.raises(rexi.RexiError) as err:
        plan.step(x, dt)
    assert err.value.status == rexi.REXI_ENOCONV
    # overlapping input and output
    plan.set_krylov(rtol=1e-12)
    with pytest.raises(rexi.RexiError) as err:
        plan.step(x, dt, out=x)
    assert err.value.status == rexi.REXI_EINVAL
    # the depth gradient keeps per-term CG and sizes its own workspace
    g = plan.grad_depth(x, x, dt)
    assert torch.isfinite(g).all()
    # constant-depth plans have no Krylov method
    pf = rexi.Plan(nx, ny)
    with pytest.raises(rexi.RexiError) as err:
        pf.set_krylov_method("shared")
    assert err.value.status == rexi.REXI_EUNSUPPORTED


def test_shared_full_size_constant_depth_all_terms_matches_fourier():
    """1024 x 1024, tau rho = 400, every REXII term: shared Lanczos with H = 1
    against the Fourier path (the same rational function, solved exactly per
    wavenumber)."""
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    n = 1024
    st = inputs.kminus3_field(n, n, seed=0)
    plan_k, _ = shared_plan(torch, n, n, np.ones((n, n)), rtol=1e-11)
    plan_f = rexi.Plan(n, n)
    dt = 400.0 / plan_k.rho
    x = to_dev(torch, st)
    a, info = plan_k.step(x, dt, want_info=True)
    b = plan_f.step(x, dt)
    assert info.M == C.pole_count_M(400.0, 0.5, 1e-10)
    assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 1e-10


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_shared_full_size_variable_depth(form):
    """The variable-depth workload at full size (1024 x 1024, H = 1 + 0.4 sin cos
    + bumps, |k|^-3 height, tau rho = 400, every term).  No oracle solve fits
    this size, so: (a) the REXII step preserves the energy norm to the rational
    approximation's accuracy (exp(tau A) is W-unitary, |r(ix)| = 1 + O(tol));
    (b) the lowest terms |n| < 6 agree with per-term CG."""
    torch = torch_cuda()
    n = 1024
    H = inputs.variable_depth(n, n, seed=0)
    st = inputs.kminus3_field(n, n, seed=0)
    plan, _ = shared_plan(torch, n, n, H, rtol=1e-11, form=form)
    dt = 400.0 / plan.rho
    x = to_dev(torch, st)
    out, info = plan.step(x, dt, want_info=True)
    o = out.cpu().numpy()
    assert info.krylov_unconverged == 0
    assert abs(energy_norm(o, H) / energy_norm(st, H) - 1.0) < 1e-9
    a = plan.step(x, dt, terms=(0, 6))
    plan.set_krylov_method("cg")
    plan.set_krylov(rtol=1e-12, term_batch=6)
    b = plan.step(x, dt, terms=(0, 6))
    assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < (1e-9 if form == "fp64" else TOL[form])
    if form == "mixed":  # double-float against FP64 Lanczos on the full step
        plan.set_krylov_method("shared")
        plan.set_krylov(rtol=1e-11)
        plan_f, _ = shared_plan(torch, n, n, H, rtol=1e-11, form="fp64")
        ref = plan_f.step(x, dt)
        assert rel_l2(o, ref.cpu().numpy()) < TOL[form]


@pytest.mark.parametrize("case", ["10x8", "40x36", "70x50"])
def test_shared_grad_depth_against_oracle(case):
    """Depth gradient from the two kept Lanczos bases (real input) against the
    oracle's per-pole formula and against per-term CG."""
    from oracle import adjoint as AD

    torch = torch_cuda()
    nx, ny = {"10x8": (10, 8), "40x36": (40, 36), "70x50": (70, 50)}[case]
    taurho = {"10x8": 15.3, "40x36": 30.0, "70x50": 25.0}[case]
    H = inputs.variable_depth(nx, ny, seed=2)
    plan, _ = shared_plan(torch, nx, ny, H, rtol=1e-13)
    dt = taurho / plan.rho
    f0 = inputs.kminus3_field(nx, ny, seed=3)
    G = inputs.complex_random_state(nx, ny, seed=4).real.astype(np.complex128)
    got, info = plan.grad_depth(to_dev(torch, f0), to_dev(torch, G), dt, want_info=True)
    assert 0 < info.krylov_iters < 20000
    ref = AD.grad_depth_sparse(nx, ny, H, f0.ravel(), G.ravel(), dt, 0.5, info.M)
    assert rel_l2(got.cpu().numpy(), ref) < 1e-9, rel_l2(got.cpu().numpy(), ref)
    plan.set_krylov_method("cg")
    cg = plan.grad_depth(to_dev(torch, f0), to_dev(torch, G), dt)
    assert rel_l2(got.cpu().numpy(), cg.cpu().numpy()) < 1e-9


def test_shared_autograd_rollout_matches_cg():
    """A checkpointed 4-step rollout with the shared method gives the same state
    and depth gradients as per-term CG."""
    from paper_2008_11607_gb300.autograd import rexi_rollout

    torch = torch_cuda()
    n = 24
    H = inputs.variable_depth(n, n, seed=0)
    f0 = inputs.kminus3_field(n, n, seed=1)
    target = torch.from_numpy(inputs.kminus3_field(n, n, seed=1000)[0].real.copy()).cuda()
    grads = {}
    for method in ("shared", "cg"):
        plan, Hd = shared_plan(torch, n, n, H, rtol=1e-13)
        plan.set_krylov_method(method)
        Hd.requires_grad_(True)
        x = to_dev(torch, f0).requires_grad_(True)
        dt = 20.0 / plan.rho
        out = rexi_rollout(x, plan, dt, 4, every=2, depth=Hd)
        loss = 0.5 * torch.sum((out[0].real - target) ** 2)
        grads[method] = [g.cpu().numpy() for g in torch.autograd.grad(loss, [x, Hd])]
    for a, b in zip(grads["shared"], grads["cg"]):
        assert rel_l2(a, b) < 1e-8
