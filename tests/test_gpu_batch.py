"""Batched serving launch: every instance of a batch must equal what the
single-instance step computes for it (and, for a small instance, the oracle),
in both the persistent (graph-replayed) mode and the per-instance mode."""
import math

import numpy as np
import pytest

from oracle import coeffs as C
from paper_2008_11607_gb300 import inputs
from tests.gpu_util import TOL, oracle_step, rel_l2, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

# The single-instance step may split the terms into slices whose partial sums
# are added in FP64, the persistent kernel sums all terms of an orbit in one
# accumulator: the same terms (bit for bit) summed in another order.  An order
# change moves the result by the accumulator's rounding: partial sums reach
# sum |term| / 2 ~ 30 |result| at tau rho = 1000, FP64 rounds each add at
# 2^-53 of that; the double-float accumulator adds its low words in plain
# FP32 (2^-24 of a low word ~ 2^-48 of the partial sum), which over ~3000
# terms gives up to ~1e-12 of the result.
SAME_SUM = {"fp64": 1e-13, "mixed": 1e-11}


def make_batch(torch, sizes, tau_rhos, form, seed0=0, real=True):
    from paper_2008_11607_gb300 import rexi

    plans = [rexi.Plan(nx, ny, form=form) for nx, ny in sizes]
    dts = [tr / p.rho for tr, p in zip(tau_rhos, plans)]
    b = rexi.Batch(sizes, dts, form=form)
    if real:
        states = [to_dev(torch, inputs.kminus3_field(nx, ny, seed=seed0 + i)) for i, (nx, ny) in enumerate(sizes)]
    else:
        states = [to_dev(torch, inputs.complex_random_state(nx, ny, seed=seed0 + i)) for i, (nx, ny) in enumerate(sizes)]
    return b, plans, dts, states


@pytest.mark.parametrize("form", ["fp64", "mixed"])
@pytest.mark.parametrize("real", [True, False])
def test_small_batch_matches_single_instance(form, real):
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    sizes = [(16, 16), (24, 20), (16, 16), (12, 18), (32, 32), (9, 15)]
    trs = [10.0, 30.0, 5.0, 20.0, 40.0, 12.0]
    b, plans, dts, states = make_batch(torch, sizes, trs, form, real=real)
    packed = b.pack(states)
    ws = b.workspace()
    refs = [p.step(s, dt, real_input=real) for p, s, dt in zip(plans, states, dts)]
    same_sum = SAME_SUM[form]
    for mode in (rexi.REXI_BATCH_PERSISTENT, rexi.REXI_BATCH_PER_INSTANCE):
        out = b.step(packed, workspace=ws, real_input=real, mode=mode)
        torch.cuda.synchronize()
        for o, r in zip(b.unpack(out), refs):
            assert rel_l2(o.cpu().numpy(), r.cpu().numpy()) < same_sum
    assert b.M == [C.pole_count_M(tr, 0.5, 1e-10) for tr in trs]
    # one instance against the oracle
    st = states[1].cpu().numpy()
    ref = oracle_step(st, dts[1], b.M[1], real_input=real)
    assert rel_l2(b.unpack(out)[1].cpu().numpy(), ref) < TOL[form]


def test_graph_replay_and_autotune():
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    sizes = [(32, 32), (48, 48), (32, 32), (20, 24)]
    trs = [25.0, 60.0, 8.0, 15.0]
    b, plans, dts, states = make_batch(torch, sizes, trs, "mixed", seed0=10)
    packed = b.pack(states)
    out = b.empty()
    ws = b.workspace()
    b.step(packed, out, ws)  # captures the graph
    # new data in the same buffers: the replayed graph must see it
    states2 = [to_dev(torch, inputs.kminus3_field(nx, ny, seed=100 + i)) for i, (nx, ny) in enumerate(sizes)]
    b.pack(states2, out=packed)
    b.step(packed, out, ws)
    torch.cuda.synchronize()
    for o, p, s, dt in zip(b.unpack(out), plans, states2, dts):
        assert rel_l2(o.cpu().numpy(), p.step(s, dt).cpu().numpy()) < SAME_SUM["mixed"]
    t, ppt, ms = b.autotune(packed, out, ws)
    assert t in (64, 128, 256) and ppt in (1, 2) and ms > 0
    b.pack(states2, out=packed)
    b.step(packed, out, ws)
    torch.cuda.synchronize()
    info = b.info()
    assert info["threads"] == t and info["orbits_per_thread"] == ppt and info["n_items"] > 0
    for o, p, s, dt in zip(b.unpack(out), plans, states2, dts):
        assert rel_l2(o.cpu().numpy(), p.step(s, dt).cpu().numpy()) < SAME_SUM["mixed"]


def test_serving_mix_96_instances():
    """The serving workload: 96 instances, D uniform from {128, 192, 256, 384,
    512}, tau rho log-uniform in [20, 800], |k|^-3 fields with seeds 0..95,
    mixed form, persistent mode (autotuned) and per-instance mode, every
    instance against the single-instance step."""
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    mix = inputs.batched_instances()
    sizes = [(m["nx"], m["ny"]) for m in mix]
    trs = [m["tau_rho"] for m in mix]
    b, plans, dts, _ = make_batch(torch, sizes, trs, "mixed")
    states = [to_dev(torch, inputs.kminus3_field(m["nx"], m["ny"], seed=m["seed"])) for m in mix]
    packed = b.pack(states)
    out = b.empty()
    ws = b.workspace()
    b.autotune(packed, out, ws)
    b.step(packed, out, ws)
    out2 = b.step(packed, workspace=ws, mode=rexi.REXI_BATCH_PER_INSTANCE)
    torch.cuda.synchronize()
    for o, o2, p, s, dt in zip(b.unpack(out), b.unpack(out2), plans, states, dts):
        r = p.step(s, dt).cpu().numpy()
        assert rel_l2(o.cpu().numpy(), r) < SAME_SUM["mixed"]
        assert rel_l2(o2.cpu().numpy(), r) < 1e-12


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_batch_with_h_off_the_split_grid(form):
    """h = 0.3: h n is not a binary fraction, so the double-float tables carry
    a low part of h n (the kernels' inexact branch).  Both launch modes against
    the oracle's sparse REXII chain."""
    torch = torch_cuda()
    from paper_2008_11607_gb300 import rexi

    sizes = [(16, 16), (12, 18), (20, 14)]
    trs = [25.0, 60.0, 15.0]
    plans = [rexi.Plan(nx, ny, form=form, h=0.3) for nx, ny in sizes]
    dts = [tr / p.rho for tr, p in zip(trs, plans)]
    b = rexi.Batch(sizes, dts, form=form, h=0.3)
    states = [to_dev(torch, inputs.kminus3_field(nx, ny, seed=40 + i)) for i, (nx, ny) in enumerate(sizes)]
    packed = b.pack(states)
    ws = b.workspace()
    for mode in (rexi.REXI_BATCH_PERSISTENT, rexi.REXI_BATCH_PER_INSTANCE):
        outs = b.unpack(b.step(packed, workspace=ws, mode=mode))
        torch.cuda.synchronize()
        for o, st, dt, M in zip(outs, states, dts, b.M):
            ref = oracle_step(st.cpu().numpy(), dt, M, h=0.3)
            assert rel_l2(o.cpu().numpy(), ref) < TOL[form]
