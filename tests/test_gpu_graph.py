"""Batched moves in one CUDA graph (smc_batch_*) against the host-driven smc_move.

The graph runs the same kernels on the same data: the steps, the refinement
phases and the CG iterations are conditional nodes whose conditions the device
sets, and every launch between two compactions is a switch over launch sizes.
Each work item (a particle's tile, a particle) is computed by the same code
whatever the launch size, and every reduction has a fixed order, so the states,
potentials, acceptance rates, temperature schedule and solver counters must be
bit-identical to smc_move on a twin sampler (same configuration and seed).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2503_16028_gb300 import inputs, smcgm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_16028_gb300 import build
    build.build()
    smcgm.load_library()


def _twins(name, **over):
    """Two samplers of the same configuration, taken through one tempering layer and a fit."""
    wl = inputs.load_workload(name)
    out = []
    for _ in range(2):
        s = smcgm.Sampler(smcgm.make_config(wl, **over))
        s.smc_temper_step()
        s.smc_resample()
        s.gm_fit()
        out.append(s)
    return out


def _same_state(a, b):
    Xa, Pa = a.particles()
    Xb, Pb = b.particles()
    assert np.array_equal(Xa, Xb)
    assert np.array_equal(Pa, Pb)
    assert a.smc_get_schedule() == b.smc_get_schedule()


def _counters(s):
    p = s.smc_profile_query(reset=True)
    return {k: p[k] for k in ("solves", "cg_iterations", "inner_solves", "residuals")}, p["graph_launches"]


def test_single_problem_graph_equals_host_loop():
    host, graph = _twins("darcy64_bimodal", n_particles=64, n_components=2)
    host.smc_profile_query(reset=True)
    graph.smc_profile_query(reset=True)
    b = smcgm.Batch([graph], steps=3)
    acc_h, _ = host.smc_move(3)
    acc_g = b.move()
    assert acc_g[0] == acc_h
    _same_state(host, graph)
    (ch, lh), (cg, lg) = _counters(host), _counters(graph)
    assert ch == cg and cg["cg_iterations"] > 0
    assert (lh, lg) == (0, 1)
    # a second launch continues the schedule (Philox steps, beta) like a second smc_move
    acc_h, _ = host.smc_move(3)
    acc_g = b.move()
    assert acc_g[0] == acc_h
    _same_state(host, graph)
    b.close()
    host.close()
    graph.close()


def test_mixed_batch_of_uneven_problems_equals_host_loops():
    """One graph holding four problems: 64^2 and 128^2 grids, 96 and 40 particles, mixed
    precision, FP64, FP32 + BF16 smoother and a full-covariance mixture; two launches,
    each sampler against its own host-driven twin."""
    cases = [("darcy64_bimodal", dict(n_particles=96, n_components=3)),
             ("darcy64_bimodal", dict(n_particles=40, n_components=2, precision=smcgm.SMC_P_FP64)),
             ("darcy256_precision", dict(n=128, kl_modes=64, n_particles=40, n_components=2,
                                         precision=smcgm.SMC_P_BF16SMOOTH_REFINE)),
             ("darcy64_bimodal", dict(n_particles=40, n_components=2, gm_rank=8, full_cov=1, kernel=smcgm.SMC_K_GM_INDEP))]
    pairs = [_twins(name, **over) for name, over in cases]
    b = smcgm.Batch([g for _, g in pairs], steps=2)
    for _ in range(2):
        rates = b.move()
        for (h, g), r in zip(pairs, rates):
            acc_h, _ = h.smc_move(2)
            assert r == acc_h
            _same_state(h, g)
    b.close()
    for h, g in pairs:
        h.close()
        g.close()


@pytest.mark.parametrize("tile_kernel", [0, 4])
def test_metric_grid_in_graph_equals_host_loop(tile_kernel):
    """256^2 (the TMA-staged finest level and three tiled levels), 64 particles: 7 launch-size
    buckets per stage; the coarser tiled levels as warp tiles (0) or as 32 x 32 block tiles (4)."""
    host, graph = _twins("darcy256_precision", n_particles=64, n_components=2, tile_kernel=tile_kernel)
    b = smcgm.Batch([graph], steps=2)
    acc_h, _ = host.smc_move(2)
    acc_g = b.move()
    assert acc_g[0] == acc_h
    _same_state(host, graph)
    b.close()
    host.close()
    graph.close()


def test_largest_grid_in_graph_equals_host_loop():
    """512^2 (four tiled levels), 8 particles in ragged solve batches of 3."""
    host, graph = _twins("darcy256_precision", n=512, n_particles=8, n_components=2, solve_batch=3)
    b = smcgm.Batch([graph], steps=1)
    acc_h, _ = host.smc_move(1)
    acc_g = b.move()
    assert acc_g[0] == acc_h
    _same_state(host, graph)
    b.close()
    host.close()
    graph.close()


def test_batch_move_host_equals_move_host():
    """The host-buffer form of the batched move against smc_move_host on a twin: the state
    is replaced from host arrays (here the particles in reverse order), moved once and copied
    back; outputs, acceptance rates and the schedule must be identical."""
    host, graph = _twins("darcy64_bimodal", n_particles=64, n_components=2)
    X0, P0 = host.particles()
    X_in = np.ascontiguousarray(X0[::-1])
    P_in = np.ascontiguousarray(P0[::-1])
    b = smcgm.Batch([graph], steps=1)
    for _ in range(2):
        Xh, Ph = np.empty_like(X_in), np.empty_like(P_in)
        Xg, Pg = np.empty_like(X_in), np.empty_like(P_in)
        acc_h = host.smc_move_host(X_in, P_in, Xh, Ph)
        acc_g = b.move_host([X_in], [P_in], [Xg], [Pg])
        assert acc_g[0] == acc_h
        assert np.array_equal(Xg, Xh) and np.array_equal(Pg, Ph)
        assert not np.array_equal(Xg, X_in)          # the move did move particles
        _same_state(host, graph)
    with pytest.raises(ValueError):
        b.move_host([X_in, X_in], [P_in])
    b.close()
    host.close()
    graph.close()


def test_batch_rejects_unsupported_contexts():
    wl = inputs.load_workload("darcy64_bimodal")
    s = smcgm.Sampler(smcgm.make_config(wl, n_particles=8, n_components=1, kernel=smcgm.SMC_K_PCNL, gradient=1))
    with pytest.raises(smcgm.SMCError) as ei:
        smcgm.Batch([s], steps=1)
    assert ei.value.status == smcgm.SMC_EINVAL
    s2 = smcgm.Sampler(smcgm.make_config(wl, n_particles=8, n_components=1))
    with pytest.raises(smcgm.SMCError) as ei:
        smcgm.Batch([s2, s2], steps=1)
    assert ei.value.status == smcgm.SMC_EINVAL
    s3 = smcgm.Sampler(smcgm.make_config(wl, n_particles=8, n_components=1, tile_kernel=1))
    with pytest.raises(smcgm.SMCError) as ei:
        smcgm.Batch([s3], steps=1)    # the block-tile kernels are sized on the host
    assert ei.value.status == smcgm.SMC_EINVAL
    s3.close()
    b = smcgm.Batch([s2], steps=1)
    with pytest.raises(smcgm.SMCError) as ei:
        b.move()                      # no mixture fitted yet
    assert ei.value.status == smcgm.SMC_ESTATE
    b.close()
    s.close()
    s2.close()
