"""Failure paths with non-finite input, made on the host (a NaN or an Inf
written into the input state; no GPU fault is involved).

* Variable-depth path: a term whose right-hand side or residual is not finite
  stops at once (CG per term: status 3 at its first reduction), and the
  shared-Krylov method stops at its first error-bound check on non-finite
  Lanczos scalars; both return REXI_ENOCONV with the reason in
  rexi_last_error_message().
* Constant-depth (Fourier) path: values are not inspected.  The transforms mix
  every grid point into every wavenumber and back, so one non-finite input
  value makes every output value non-finite; the call returns REXI_OK.  This
  is the documented behaviour and is what is checked here.
"""
import numpy as np
import pytest

from paper_2008_11607_gb300 import inputs
from tests.gpu_util import to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _poisoned(st, value, where=(0, 3, 5)):
    bad = st.copy()
    bad[where] = value
    return bad


@pytest.mark.parametrize("form", ["fp64", "mixed", "plain"])
@pytest.mark.parametrize("real", [True, False])
@pytest.mark.parametrize("value", [np.nan, np.inf])
def test_fourier_path_propagates_non_finite_input(form, real, value):
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    nx, ny = 24, 20
    st = inputs.kminus3_field(nx, ny, seed=1) if real else inputs.complex_random_state(nx, ny, seed=1)
    plan = rexi.Plan(nx, ny, form=form)
    dt = 30.0 / plan.rho
    out = plan.step(to_dev(torch, _poisoned(st, value)), dt, real_input=real).cpu().numpy()
    assert not np.any(np.isfinite(out.real)), form
    # the plan and the stream stay usable
    good = plan.step(to_dev(torch, st), dt, real_input=real).cpu().numpy()
    assert np.all(np.isfinite(good))


@pytest.mark.parametrize("method", ["cg", "shared"])
@pytest.mark.parametrize("form", ["fp64", "mixed"])
@pytest.mark.parametrize("value", [np.nan, np.inf])
def test_krylov_path_reports_non_finite_input(method, form, value):
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    nx, ny = 12, 10
    H = torch.from_numpy(inputs.variable_depth(nx, ny, seed=3)).cuda()
    plan = rexi.Plan(nx, ny, depth=H, form=form)
    plan.set_krylov(rtol=1e-12, max_iters=2000, term_batch=16)
    plan.set_krylov_method(method)
    dt = 20.0 / plan.rho
    st = inputs.kminus3_field(nx, ny, seed=0)
    with pytest.raises(rexi.RexiError) as e:
        plan.step(to_dev(torch, _poisoned(st, value)), dt)
    assert e.value.status == rexi.REXI_ENOCONV
    assert "non-finite" in str(e.value)
    # a finite input afterwards still works on the same plan
    out = plan.step(to_dev(torch, st), dt).cpu().numpy()
    assert np.all(np.isfinite(out))
