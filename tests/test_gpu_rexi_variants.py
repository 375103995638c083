"""The other rational approximations of Section 2 on the GPU: the original
REXI in its matrix form (eq. originalREXImatrix) on the shallow-water
operator, and REXI Extended (eq. REXIE) with the spectral shift of the remark
in Section 2.2 on the scalar operator i (d_xx + d_yy), whose one-dimensional
case is the A_2 of Section 3.2.  Checked against the oracle's one-solve-per-term
matrix forms, dense expm, and the REXI rows printed in Tables 2-7."""
import math
import os

import numpy as np
import pytest

from oracle import exact as E
from oracle import operator as O
from oracle import rexi as R
from oracle import spectral as S
from paper_2008_11607_gb300 import inputs
from tests.gpu_util import rel_l2, to_dev, torch_cuda

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = {"fp64": 1e-10, "mixed": 1e-8}


def _rexi_rows():
    with open(os.path.join(GOLDEN, "paper_rexi_errors.txt")) as fh:
        for ln in fh:
            if ln.strip() and not ln.startswith("#"):
                p = ln.split()
                yield p[0], float(p[1]), float(p[2]), int(p[3]), float(p[4]), float(p[5])


@pytest.mark.parametrize("form", ["fp64", "mixed"])
@pytest.mark.parametrize("nx,ny", [(12, 10), (9, 8)])
def test_original_rexi_cgrid_against_oracle(form, nx, ny):
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    phys = dict(Lx=1.2, Ly=0.9, g=1.3, f=0.7, H=0.8)
    st = inputs.kminus3_field(nx, ny, seed=3)
    st[1] = inputs.kminus3_field(nx, ny, seed=4)[0]
    plan = rexi.Plan(nx, ny, form=form, h=0.2, **phys)
    plan.set_coefficients("rexi")
    dt = 6.0 / plan.rho
    out, info = plan.step(to_dev(torch, st), dt, want_info=True)
    A = O.cgrid_operator(nx, ny, **phys)
    ref = R.rexi_original_apply_sparse(A, st.ravel(), dt, 0.2, info.M).reshape(st.shape)
    assert rel_l2(out.cpu().numpy(), ref) < TOL[form]


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_paper_rexi_rows_on_gpu(form):
    """Every REXI row of Tables 2-7 (h = 0.2, M up to 5,000,171) with the
    spectral symbol at D = 128: the max-norm error against the exact
    exponential matches the printed CPU column to 2 %."""
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    D = 128
    refs = {}
    for scen, tau, h, M, cpu, _ in _rexi_rows():
        plan = rexi.Plan(D, D, form=form, h=h)
        plan.set_symbol("spectral")
        plan.set_coefficients("rexi")
        plan.set_rho(((M - 11) - 0.5) * h / tau)
        st = inputs.paper_scenario(scen, D, D)
        out, info = plan.step(to_dev(torch, st), tau, tol=1e-16, want_info=True)
        assert info.M == M
        if (scen, tau) not in refs:
            refs[(scen, tau)] = E.exp_closed_form(st, tau, symbol_fn=S.symbol).real
        err = float(np.max(np.abs(out.cpu().numpy().real - refs[(scen, tau)])))
        assert abs(err - cpu) <= 0.02 * cpu, (form, scen, tau, M, err, cpu)


def _a2_state(nx, ny):
    x = -1.0 + np.arange(nx) * (2.0 / nx)
    f0 = 1.0 / (2.0 + np.cos(2 * math.pi * x))
    st = np.zeros((3, ny, nx), dtype=np.complex128)
    st[0] = f0[None, :]
    return st, f0


@pytest.mark.parametrize("form", ["fp64", "mixed"])
@pytest.mark.parametrize("coefs", ["rexie", "rexii"])
def test_A2_with_shift_against_expm(form, coefs):
    """Section 3.2, A_2 = i d_xx on [-1, 1] with step 1/35 (nx = 70; ny = 2
    with data constant in y), f0 = 1/(2 + cos(2 pi x)), tau = 1, shift
    nu = -2450 i: against dense expm of the 70 x 70 matrix and the oracle's
    REXIE with the same M."""
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    nx, ny = 70, 2
    plan = rexi.Plan(nx, ny, Lx=2.0, Ly=1.0, form=form)
    plan.set_symbol("schrodinger")
    plan.set_coefficients(coefs)
    plan.set_shift("value", -2450.0)
    assert abs(plan.shift + 2450.0) < 1e-12
    st, f0 = _a2_state(nx, ny)
    out, info = plan.step(to_dev(torch, st), 1.0, tol=1e-16, real_input=False, want_info=True)
    got = out.cpu().numpy()
    A2 = O.schrodinger_operator(nx, 1, Lx=2.0)
    ref = E.expm_dense(A2, f0, 1.0)
    for j in range(ny):
        assert rel_l2(got[0, j], ref) < (1e-11 if form == "fp64" else 1e-8)
    assert np.max(np.abs(got[1:])) == 0.0
    orc = R.rexie_apply(A2, f0, 1.0, 0.5, info.M, sigma=-2450.0)
    assert rel_l2(got[0, 0], orc) < (1e-11 if form == "fp64" else 1e-8)


@pytest.mark.parametrize("form", ["fp64", "mixed"])
@pytest.mark.parametrize("nx,ny,Lx,Ly", [(12, 10, 1.3, 0.7), (16, 16, 1.0, 1.0), (9, 6, 1.0, 2.0)])
def test_scalar_operator_midpoint_shift_against_oracle(form, nx, ny, Lx, Ly):
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    plan = rexi.Plan(nx, ny, Lx=Lx, Ly=Ly, form=form)
    plan.set_symbol("schrodinger")
    plan.set_shift("midpoint")
    lmin = -(4.0 / (Lx / nx) ** 2) * math.sin(math.pi * (nx // 2) / nx) ** 2 \
           - (4.0 / (Ly / ny) ** 2) * math.sin(math.pi * (ny // 2) / ny) ** 2
    assert abs(plan.shift - 0.5 * lmin) < 1e-9 * abs(lmin)
    assert abs(plan.rho + 0.5 * lmin) < 1e-9 * abs(lmin)
    dt = 30.0 / plan.rho
    A = O.schrodinger_operator(nx, ny, Lx, Ly)
    # REXIE needs real data (its Re parts); REXII takes any complex state
    real = inputs.kminus3_field(nx, ny, seed=5)
    real[1] = inputs.kminus3_field(nx, ny, seed=6)[0]
    plan.set_coefficients("rexie")
    out, info = plan.step(to_dev(torch, real), dt, real_input=False, want_info=True)
    for c in range(2):
        ref = R.rexie_apply(A, real[c].ravel(), dt, 0.5, info.M, sigma=plan.shift).reshape(ny, nx)
        assert rel_l2(out.cpu().numpy()[c], ref) < TOL[form]
    cplx = inputs.complex_random_state(nx, ny, seed=7)
    plan.set_coefficients("rexii")
    out = plan.step(to_dev(torch, cplx), dt, real_input=False).cpu().numpy()
    for c in range(3):
        ref = E.expm_dense(A, cplx[c].ravel(), dt).reshape(ny, nx)
        assert rel_l2(out[c], ref) < max(TOL[form], 1e-10)


def test_scalar_operator_adjoint_is_the_adjoint():
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    nx, ny = 16, 12
    plan = rexi.Plan(nx, ny, form="fp64")
    plan.set_symbol("schrodinger")
    plan.set_shift("midpoint")
    dt = 25.0 / plan.rho
    x = to_dev(torch, inputs.complex_random_state(nx, ny, seed=1))
    y = to_dev(torch, inputs.complex_random_state(nx, ny, seed=2))
    ax = plan.step(x, dt, real_input=False)
    aty = plan.step_adjoint(y, dt, real_input=False)
    lhs = complex(torch.sum(torch.conj(y) * ax))
    rhs = complex(torch.sum(torch.conj(aty) * x))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_unsupported_combinations_are_refused():
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    x = to_dev(torch, inputs.complex_random_state(8, 8, seed=0))
    p = rexi.Plan(8, 8)
    p.set_coefficients("rexie")  # REXIE on the (real) shallow-water operator
    with pytest.raises(rexi.RexiError) as e:
        p.step(x, 0.01)
    assert e.value.status == rexi.REXI_EUNSUPPORTED
    with pytest.raises(rexi.RexiError) as e:
        p.set_shift("value", 3.0)
    assert e.value.status == rexi.REXI_EUNSUPPORTED
    q = rexi.Plan(8, 8)
    q.set_symbol("schrodinger")
    with pytest.raises(rexi.RexiError) as e:
        q.step(x, 0.01, real_input=True)
    assert e.value.status == rexi.REXI_EINVAL
    q.set_coefficients("rexi")  # original REXI needs a real operator
    with pytest.raises(rexi.RexiError) as e:
        q.step(x, 0.01, real_input=False)
    assert e.value.status == rexi.REXI_EUNSUPPORTED
    pl = rexi.Plan(8, 8, form="plain")
    pl.set_coefficients("rexi")
    with pytest.raises(rexi.RexiError) as e:
        pl.step(x, 0.01)
    assert e.value.status == rexi.REXI_EUNSUPPORTED
    H = torch.from_numpy(inputs.variable_depth(8, 8, seed=0)).cuda()
    kp = rexi.Plan(8, 8, depth=H)
    kp.set_coefficients("rexi")
    with pytest.raises(rexi.RexiError) as e:
        kp.step(x, 0.01)
    assert e.value.status == rexi.REXI_EUNSUPPORTED


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_step_with_library_refit_against_oracle(form):
    """A step with the library's refit of the Gaussian (Section 2.1 Step 2)
    against the oracle's sparse REXII chain with the same coefficients, and
    against the oracle's chain with the oracle's own refit."""
    torch = torch_cuda()
    from oracle import refit as RF
    from paper_2008_11607_gb300 import rexi

    nx, ny = 12, 10
    mu, a, err = rexi.gaussian_refit()
    assert err < 2e-13
    st = inputs.kminus3_field(nx, ny, seed=2)
    plan = rexi.Plan(nx, ny, form=form)
    plan.set_gaussian_fit(mu, a)
    dt = 40.0 / plan.rho
    out, info = plan.step(to_dev(torch, st), dt, want_info=True)
    out = out.cpu().numpy()
    A = O.cgrid_operator(nx, ny)
    same = R.rexii_apply_sparse(A, st.ravel(), dt, 0.5, info.M, mu=mu, a=a).reshape(st.shape)
    assert rel_l2(out, same) < TOL[form]
    muo, ao = RF.refit(mu=mu)
    other = R.rexii_apply_sparse(A, st.ravel(), dt, 0.5, info.M, mu=muo, a=ao).reshape(st.shape)
    assert rel_l2(out, other) < TOL[form]
    # restoring the table gives the table's step again
    plan.set_gaussian_fit()
    tab = R.rexii_apply_sparse(A, st.ravel(), dt, 0.5, info.M).reshape(st.shape)
    assert rel_l2(plan.step(to_dev(torch, st), dt).cpu().numpy(), tab) < TOL[form]


def test_gaussian_fit_validation():
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    mu, a = rexi.gaussian_fit_table()
    p = rexi.Plan(8, 8)
    bad = a.copy()
    bad[0] += 1e-3  # breaks a_{-l} = conj(a_l)
    with pytest.raises(rexi.RexiError) as e:
        p.set_gaussian_fit(mu, bad)
    assert e.value.status == rexi.REXI_EINVAL
    with pytest.raises(rexi.RexiError) as e:
        p.set_gaussian_fit(1.0, a)
    assert e.value.status == rexi.REXI_EINVAL
    H = torch.from_numpy(inputs.variable_depth(8, 8, seed=0)).cuda()
    kp = rexi.Plan(8, 8, depth=H)
    kp.set_gaussian_fit(mu, a)
    with pytest.raises(rexi.RexiError) as e:
        kp.step(to_dev(torch, inputs.kminus3_field(8, 8, seed=0)), 0.01)
    assert e.value.status == rexi.REXI_EUNSUPPORTED
