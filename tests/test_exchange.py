"""The exchange step of a sharded tempering layer on CPU ranks (gloo).

Each rank holds a contiguous block of the particles.  After the exchange
every rank must hold exactly what a single process would: the gathered
potentials, the same temperature and resampling indices, the resampled rows
of its block, and the summed EM statistics.  The single-process reference is
the oracle on the unsharded arrays.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2503_16028_gb300 import exchange  # noqa: E402

N_TOTAL, D, K = 13, 3, 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _global_state():
    rng = np.random.default_rng(2503)
    X = rng.standard_normal((N_TOTAL, D))
    Phi = rng.uniform(0.0, 40.0, N_TOTAL)
    return X, Phi


def _reference():
    from oracle import smc as osmc, gm as ogm
    X, Phi = _global_state()
    h = osmc.bisect_h(Phi, 0.0, 0.5 * N_TOTAL)
    idx = osmc.systematic_indices(-h * Phi, osmc.resample_u48(7, 3))
    Xr = X[idx]
    w = np.full(K, 1.0 / K)
    m = np.stack([Xr[0], Xr[1]])
    lam = np.ones((K, D))
    g, _ = ogm.e_step(Xr, w, m, lam)
    stats = np.concatenate([g.sum(0), (g.T @ Xr).ravel(), (g.T @ Xr ** 2).ravel()])
    return h, idx, Xr, stats


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    from oracle import smc as osmc, gm as ogm
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, Phi = _global_state()
        lo, hi = exchange.block_bounds(N_TOTAL, world, rank)
        X_loc = torch.tensor(X[lo:hi])
        Phi_loc = torch.tensor(Phi[lo:hi])
        # 1. potentials
        Phi_all = exchange.allgather_rows(Phi_loc, N_TOTAL).numpy()
        # 2. temperature and indices, computed on every rank from the gathered potentials
        h = osmc.bisect_h(Phi_all, 0.0, 0.5 * N_TOTAL)
        idx = osmc.systematic_indices(-h * Phi_all, osmc.resample_u48(7, 3))
        # 3. resampled rows of this block
        X_new = exchange.exchange_rows(X_loc, idx, N_TOTAL).numpy()
        # 4. EM statistics of this block, summed over ranks (the initial means are two global rows)
        m = np.stack([exchange.allgather_rows(torch.tensor(X_new), N_TOTAL).numpy()[j] for j in (0, 1)])
        g, _ = ogm.e_step(X_new, np.full(K, 1.0 / K), m, np.ones((K, D)))
        st = torch.tensor(np.concatenate([g.sum(0), (g.T @ X_new).ravel(), (g.T @ X_new ** 2).ravel()]))
        exchange.allreduce_sum(st)
        out.put((rank, Phi_all, h, idx, lo, hi, X_new, st.numpy()))
    finally:
        dist.destroy_process_group()


def test_block_bounds_and_owner():
    for n in (1, 5, 13, 4096):
        for world in (1, 2, 3, 8):
            if world > n:
                continue
            covered = []
            for r in range(world):
                lo, hi = exchange.block_bounds(n, world, r)
                assert hi - lo in (n // world, n // world + 1)
                covered.extend(range(lo, hi))
                for i in range(lo, hi):
                    assert exchange.owner(i, n, world) == r
            assert covered == list(range(n))


def test_routing_plan_covers_every_destination_row():
    idx = np.array([12, 12, 0, 5, 5, 5, 1, 7, 3, 3, 11, 2, 9])
    plan = exchange.routing_plan(idx, N_TOTAL, 3)
    for dst in range(3):
        lo, hi = exchange.block_bounds(N_TOTAL, 3, dst)
        rows = sorted(r for src in range(3) for r in plan[src][dst][1])
        assert rows == list(range(hi - lo))
        for src in range(3):
            slo, _ = exchange.block_bounds(N_TOTAL, 3, src)
            for s_row, d_row in zip(*plan[src][dst]):
                assert idx[lo + d_row] == slo + s_row


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_layer_matches_single_process(world):
    h_ref, idx_ref, Xr_ref, stats_ref = _reference()
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    _, Phi_ref = _global_state()
    for _ in range(world):
        rank, Phi_all, h, idx, lo, hi, X_new, st = q.get()
        assert np.array_equal(Phi_all, Phi_ref)
        assert h == h_ref
        assert np.array_equal(idx, idx_ref)
        assert np.array_equal(X_new, Xr_ref[lo:hi])
        assert np.allclose(st, stats_ref, rtol=1e-13, atol=1e-13)
