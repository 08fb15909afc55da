"""Multi-rank logic on CPU with gloo (world size 2).

1. The replica helpers bench.py uses under torchrun: per-rank seeds, the
   max-over-ranks step time and the whole-job throughput.
2. The channel-sharded design of the pass (each rank owns half of the
   channels; the per-channel steps of Sec. 3, Eqs. 8-12, run locally; the
   spectral step of Eqs. 13-14 needs every channel of a pixel, so D is moved
   to pixel shards by an all-to-all and T comes back the same way) computed
   with the FP64 oracle's operators, against the single-process oracle.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1602_08847_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _init(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _replica_worker(rank, world, port, out):
    _init(rank, world, port)
    step_time = 1.0 + rank                      # rank 1 is the slow one
    t = replicas.max_over_ranks(step_time, dist, "cpu")
    out[rank] = (replicas.rank_seed(3, rank), t, replicas.aggregate_throughput(100.0, world, t))
    dist.destroy_process_group()


def test_replica_timing_over_two_gloo_ranks():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_replica_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0][0] == 3 and out[1][0] == 4
    assert out[0][1] == out[1][1] == 2.0
    assert out[0][2] == pytest.approx(100.0)


def _all_to_all(recv, send):
    """All-to-all by point-to-point messages (gloo has no all_to_all)."""
    me, world = dist.get_rank(), dist.get_world_size()
    reqs = []
    for r in range(world):
        if r == me:
            recv[r].copy_(send[r])
        else:
            reqs.append(dist.isend(send[r].contiguous(), r))
            reqs.append(dist.irecv(recv[r], r))
    for q in reqs:
        q.wait()


def _sharded_worker(rank, world, port, n_iter, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle import muffin_oracle as mo
    from gpu_helpers import small_cube
    _init(rank, world, port)
    cube = small_cube(16, 6, 2, seed=91)
    p = mo.make_problem(cube.dirty, cube.psf, 2, mu_s=0.3, mu_l=0.8, tau=0.05, sigma=2.0)
    L, n, _ = p.shape
    own = slice(rank * L // world, (rank + 1) * L // world)          # channels of this rank
    npix = n * n
    pix = slice(rank * npix // world, (rank + 1) * npix // world)    # pixels of this rank (spectral step)
    X = np.zeros((own.stop - own.start, n, n))
    U = np.zeros((own.stop - own.start, p.J + 1, n, n))
    V = np.zeros((L, pix.stop - pix.start))                          # V is pixel-sharded
    T = np.zeros_like(X)
    C = mo.dct_matrix(L)
    for _ in range(n_iter):
        grad = mo.gradient(X, p.y[own], p.hhat[own], p.w[own])
        S = p.mu_s * mo.iuwt_adjoint(U, p.J, p.gen)
        Xt = mo.positive(X - p.tau * (grad + S + T))
        D = 2 * Xt - X
        U = mo.sat(U + p.sigma * p.mu_s * mo.iuwt_analysis(D, p.J, p.gen))
        X = Xt
        # channel shards -> pixel shards
        send = [torch.from_numpy(np.ascontiguousarray(D.reshape(D.shape[0], npix)[:, r * npix // world:(r + 1) * npix // world]))
                for r in range(world)]
        recv = [torch.empty((L // world, pix.stop - pix.start), dtype=torch.float64) for _ in range(world)]
        _all_to_all(recv, send)
        Dp = torch.cat(recv).numpy()                                   # [L][my pixels]
        V = mo.sat(V + p.sigma * p.mu_l * (C @ Dp))
        Tp = p.mu_l * (C.T @ V)
        # pixel shards -> channel shards
        send = [torch.from_numpy(np.ascontiguousarray(Tp[r * L // world:(r + 1) * L // world])) for r in range(world)]
        recv = [torch.empty((L // world, npix // world), dtype=torch.float64) for _ in range(world)]
        _all_to_all(recv, send)
        T = torch.cat(recv, dim=1).numpy().reshape(-1, n, n)
    out[rank] = X
    dist.destroy_process_group()


def test_channel_sharded_pass_equals_single_process():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from oracle import muffin_oracle as mo
    from gpu_helpers import small_cube
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_sharded_worker, args=(2, port, 4, out), nprocs=2, join=True)
    cube = small_cube(16, 6, 2, seed=91)
    p = mo.make_problem(cube.dirty, cube.psf, 2, mu_s=0.3, mu_l=0.8, tau=0.05, sigma=2.0)
    ref = mo.iterate(p, mo.zero_state(p), 4).X
    got = np.concatenate([out[0], out[1]])
    assert np.max(np.abs(got - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))
