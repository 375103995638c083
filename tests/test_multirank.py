"""World-size-2 process-group tests (gloo, CPU) of the host logic for more than
one device: the REXII terms are split across ranks with
rexi.term_partition, each rank evaluates its slice, and one sum all-reduce
gives the full step.  Each rank computes its slice with the oracle here (no
GPU); the device side of the slicing (rexi_step term_begin/term_end summing to
the full step) is covered by the GPU tests.  Also checks the benchmark's
max-over-ranks timing reduction."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, result_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import coeffs as C
        from oracle import operator as O
        from oracle import rexi as R
        from paper_2008_11607_gb300 import inputs
        from paper_2008_11607_gb300.rexi import term_partition

        nx = ny = 8
        H = inputs.variable_depth(nx, ny, seed=2)
        A = O.cgrid_operator(nx, ny, H=H)
        f0 = inputs.kminus3_field(nx, ny, seed=5).ravel()
        rho = O.spectral_radius_bound(nx, ny, Hmax=H.max())
        dt = 15.0 / rho
        M = C.pole_count_M(15.0, 0.5, 1e-10)
        N = M + C.L
        b, e = term_partition(N + 1, world, rank)
        part = R.rexii_apply_sparse(A, f0, dt, 0.5, M, terms=set(range(b, e)))
        t = torch.from_numpy(np.stack([part.real, part.imag]))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        # max-over-ranks reduction used for timing
        tm = torch.tensor([1.0 + rank], dtype=torch.float64)
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        if rank == 0:
            np.save(result_path, np.concatenate([t.numpy().ravel(), tm.numpy()]))
    finally:
        dist.destroy_process_group()


def test_term_partition_covers_all_terms():
    from paper_2008_11607_gb300.rexi import term_partition

    for n in (1, 7, 134, 834):
        for w in (1, 2, 3, 8):
            sl = [term_partition(n, w, r) for r in range(w)]
            assert sl[0][0] == 0 and sl[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(sl[:-1], sl[1:]))
            sizes = [e - b for b, e in sl]
            assert max(sizes) - min(sizes) <= 1


def test_two_rank_term_split_allreduce(tmp_path):
    from oracle import coeffs as C
    from oracle import operator as O
    from oracle import rexi as R
    from paper_2008_11607_gb300 import inputs

    path = str(tmp_path / "res.npy")
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), path), nprocs=world, join=True)
    res = np.load(path)
    summed = res[:-1].reshape(2, -1)
    got = summed[0] + 1j * summed[1]
    assert res[-1] == 2.0  # max over ranks
    nx = ny = 8
    H = inputs.variable_depth(nx, ny, seed=2)
    A = O.cgrid_operator(nx, ny, H=H)
    f0 = inputs.kminus3_field(nx, ny, seed=5).ravel()
    dt = 15.0 / O.spectral_radius_bound(nx, ny, Hmax=H.max())
    full = R.rexii_apply_sparse(A, f0, dt, 0.5, C.pole_count_M(15.0, 0.5, 1e-10))
    assert np.linalg.norm(got - full) / np.linalg.norm(full) < 1e-13
