"""rexi_step_noalloc: the constant-depth step for callers that may not allocate
device memory (no plan, no workspace; its scratch is a fixed static device
array inside the library).

Checked through the C ABI against the ordinary entry point (rexi_step with a
plan and a workspace, fused FP64 form) on two calls in a row, with the same
tolerance as the other FP64 parity tests; that a call after the first one
changes neither torch's allocator counters nor the device's free memory; that
a call on a capturing stream is refused before it copies or launches anything;
and for the clear rejection of requests larger than the fixed scratch.  This file is collected last on
purpose; it passes alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2008_11607_gb300 import inputs
from tests.gpu_util import rel_l2, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


def _noalloc(lib, torch, state, out, dt, real_input, phys, h=0.5, tol=1e-10):
    _, ny, nx = state.shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.rexi_step_noalloc(nx, ny, phys["Lx"], phys["Ly"], phys["g"], phys["f"], phys["H"], h,
                                 ctypes.c_void_p(state.data_ptr()), ctypes.c_void_p(out.data_ptr()), dt, tol,
                                 int(real_input), stream)


def test_noalloc_matches_rexi_step_twice_in_a_row():
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    lib = rexi.load()
    cases = [
        (inputs.kminus3_field(64, 48, seed=1), True, dict(Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0), 30.0),
        (inputs.complex_random_state(40, 50, seed=2), False, dict(Lx=1.3, Ly=0.8, g=2.0, f=0.6, H=0.7), 120.0),
    ]
    for state_np, real_input, phys, tau_rho in cases:
        plan = rexi.Plan(state_np.shape[2], state_np.shape[1], form="fp64", **phys)
        dt = tau_rho / plan.rho
        x = to_dev(torch, state_np)
        ref = plan.step(x, dt, real_input=real_input)
        out = torch.full_like(x, float("nan"))
        st = _noalloc(lib, torch, x, out, dt, real_input, phys)
        assert st == rexi.REXI_OK, lib.rexi_last_error_message()
        torch.cuda.synchronize()
        err = rel_l2(out.cpu().numpy(), ref.cpu().numpy())
        assert err < TOL_FP64, err


def test_noalloc_rejects_requests_beyond_its_scratch():
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    lib = rexi.load()
    phys = dict(Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0)
    big = torch.zeros((3, 256, 512), dtype=torch.complex128, device="cuda")
    assert _noalloc(lib, torch, big, big, 0.01, True, phys) == rexi.REXI_EINVAL
    assert b"65536" in lib.rexi_last_error_message()
    small = torch.zeros((3, 64, 64), dtype=torch.complex128, device="cuda")
    rho = 2 * np.sqrt(2) * 64
    assert _noalloc(lib, torch, small, small, 3000.0 / rho, True, phys) == rexi.REXI_EINVAL
    assert b"8193" in lib.rexi_last_error_message()


def test_noalloc_allocates_no_device_memory():
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    lib = rexi.load()
    phys = dict(Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0)
    x = to_dev(torch, inputs.kminus3_field(128, 96, seed=3))
    out = torch.empty_like(x)
    dt = 200.0 / (2 * np.sqrt(2) * 128)
    # the warm-up call loads the module and looks up the static array
    assert _noalloc(lib, torch, x, out, dt, True, phys) == rexi.REXI_OK, lib.rexi_last_error_message()
    torch.cuda.synchronize()
    before = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), torch.cuda.mem_get_info()[0])
    for _ in range(2):
        assert _noalloc(lib, torch, x, out, dt, True, phys) == rexi.REXI_OK, lib.rexi_last_error_message()
    torch.cuda.synchronize()
    after = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), torch.cuda.mem_get_info()[0])
    assert after == before, (before, after)


def test_noalloc_refuses_a_capturing_stream():
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    lib = rexi.load()
    phys = dict(Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0)
    x = to_dev(torch, inputs.kminus3_field(32, 32, seed=4))
    out = torch.zeros_like(x)
    y = torch.empty_like(x)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        y.copy_(x)
        st = _noalloc(lib, torch, x, out, 0.05, True, phys)
    assert st == rexi.REXI_EINVAL
    assert b"capturing" in lib.rexi_last_error_message()
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0
    # the stream is usable afterwards and a plain call still works
    assert _noalloc(lib, torch, x, out, 0.05, True, phys) == rexi.REXI_OK
    torch.cuda.synchronize()
    assert float(out.abs().max()) > 0.0
