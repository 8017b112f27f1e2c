"""Many independent inverse problems on one GPU, and a solver-setting autotuner.

Batching: one context and one CUDA stream per problem, each driven by its own
host thread.  The library's calls release the GIL (ctypes) and synchronise
only their own stream, so while one problem's host thread waits on its
convergence checks the other problems' kernels run; small problems (64^2,
a few hundred particles) that cannot fill 152 SMs alone overlap on the GPU.
A problem's result does not depend on the others (its kernels touch only its
own workspace, and its random numbers are its own Philox streams).

One graph: `smcgm.Batch` captures the moves of many contexts (any grid size,
particle count and precision) into one CUDA graph whose loops run on the device
(`smc_batch_*`): one launch moves every problem, with no host round trip inside
the move.  `time_moves` compares it with the other two ways on the same problems.

Autotuning: the stencil tiles of the multigrid / CG passes (32 x 32 tiles per
thread block, or 16 x 16 tiles per warp with or without TMA staging), the
multigrid smoothing counts, the coarse-correction factor and the inner
tolerance are run-time settings (`smc_config`); `autotune` times `smc_move`
for each candidate on the problem itself and keeps the fastest.
Every candidate meets the same FP64 tolerance, so the choice changes speed,
not the answer beyond that tolerance.
"""
import concurrent.futures as cf
import ctypes
import json
import time

import numpy as np

from . import smcgm


def run_smc(sampler, mcmc_steps, max_layers=200, log=None):
    """Alg. 1 on one context until t = 1: reweight (ESS bisection), resample,
    fit the mixture, move.  Returns the per-layer (h, ess, log Z increment,
    acceptance) and the final particles.

    log: None, a file path or a writable text file.  With a log, each layer
    appends one JSON object: layer index, temperature t and step h, ESS, log Z
    increment, mixture log-likelihood, the beta the moves used, acceptance, the
    largest CG iteration count, CG iterations and refinement phases per solve,
    and the solves of the layer (the library's counters, reset per layer)."""
    layers = []
    fh = open(log, "a") if isinstance(log, str) else log
    try:
        for _ in range(max_layers):
            h, ess, lz, done = sampler.smc_temper_step()
            sampler.smc_resample()
            ll = sampler.gm_fit()
            if fh is not None:
                t, beta, layer, _ = sampler.smc_get_schedule()
                sampler.smc_profile_query(reset=True)
            acc, it_max = sampler.smc_move(mcmc_steps, allow_noconv=True)
            layers.append(dict(h=h, ess=ess, logz=lz, acc=acc))
            if fh is not None:
                prof = sampler.smc_profile_query(reset=True)
                solves = max(1, prof["solves"])
                fh.write(json.dumps(dict(layer=layer, t=t, h=h, ess=ess, log_z_increment=lz, gm_loglik=ll, beta=beta,
                                         acceptance=acc, cg_max=it_max, cg_per_solve=prof["cg_iterations"] / solves,
                                         refinements_per_solve=prof["inner_solves"] / solves,
                                         solves=prof["solves"])) + "\n")
                fh.flush()
            if done:
                break
    finally:
        if isinstance(log, str) and fh is not None:
            fh.close()
    X, Phi = sampler.particles()
    return dict(layers=layers, X=X, Phi=Phi)


def make_samplers(configs, device="cuda:0"):
    """One Sampler per smc_config, each on a new CUDA stream of its own."""
    import torch
    out = []
    for cfg in configs:
        stream = torch.cuda.Stream(device=device)
        out.append(smcgm.Sampler(cfg, device=device, stream=stream))
    return out


def run_batch(samplers, mcmc_steps, max_layers=200, concurrent=True):
    """run_smc on every sampler, concurrently (a thread per problem) or one by
    one.  Returns (results, seconds)."""
    steps = mcmc_steps if isinstance(mcmc_steps, (list, tuple)) else [mcmc_steps] * len(samplers)
    t0 = time.perf_counter()
    if concurrent:
        with cf.ThreadPoolExecutor(max_workers=len(samplers)) as ex:
            futs = [ex.submit(run_smc, s, k, max_layers) for s, k in zip(samplers, steps)]
            results = [f.result() for f in futs]
    else:
        results = [run_smc(s, k, max_layers) for s, k in zip(samplers, steps)]
    return results, time.perf_counter() - t0


DEFAULT_CANDIDATES = (
    dict(),                                            # the library defaults
    dict(tile_kernel=1),                               # 32 x 32 block tiles
    dict(tile_kernel=3),                               # 16 x 16 warp tiles, global loads
    dict(tile_kernel=4),                               # warp tiles on the finest level, block tiles below
    dict(smooth_sweeps=1),
    dict(fine_sweeps=2),
    dict(tol_inner=2e-4),
    dict(tol_inner=1e-3),
    dict(coarse_scale=1.8),
)


def pick_fastest(timings):
    """The candidate with the smallest time (ties: the earlier candidate)."""
    best = min(range(len(timings)), key=lambda i: (timings[i][1], i))
    return timings[best][0]


def autotune(preset, candidates=DEFAULT_CANDIDATES, n_particles=None, steps=2, reps=2, **overrides):
    """Time `steps` moves for each candidate solver setting on `preset`
    (a workload dict) and return (best overrides, [(candidate, ms per move)])."""
    import torch
    timings = []
    for cand in candidates:
        kw = dict(overrides)
        kw.update(cand)
        if n_particles:
            kw["n_particles"] = n_particles
        s = smcgm.Sampler(smcgm.make_config(preset, **kw))
        s.smc_temper_step()
        s.smc_resample()
        s.gm_fit()
        s.smc_move(1, allow_noconv=True)                     # warm-up
        best = np.inf
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.smc_move(steps, allow_noconv=True)
            torch.cuda.synchronize()
            best = min(best, (time.perf_counter() - t0) * 1e3 / steps)
        s.close()
        timings.append((cand, best))
    return pick_fastest(timings), timings


def mesh_sweep(preset, grids, n_particles, kl_modes, mcmc_steps, max_layers=200, concurrent=True, **overrides):
    """The same prior (kl_modes^2 cosine modes), data and random streams solved on
    each grid of `grids`; returns {n: cumulative temperatures per layer} (the mesh
    independence of the tempering schedule, Sec. 3.2).  The grids run as a batch."""
    configs = [smcgm.make_config(preset, n=n, kl_modes=kl_modes, n_particles=n_particles, **overrides) for n in grids]
    samplers = make_samplers(configs)
    results, seconds = run_batch(samplers, mcmc_steps, max_layers, concurrent=concurrent)
    out = {}
    for n, res in zip(grids, results):
        t, ts = 0.0, []
        for lay in res["layers"]:
            t = min(1.0, t + lay["h"])
            ts.append(t)
        out[n] = ts
    for s in samplers:
        s.close()
    return out, seconds


def capped_solve_batch(cfg, budget_bytes):
    """The largest solve batch (particles solved per launch sequence) whose share of the
    workspace fits `budget_bytes`, at most all particles; the results do not depend on it."""
    lib = smcgm.load_library()
    size = ctypes.c_size_t()

    def ws(b):
        cfg.solve_batch = int(b)
        st = lib.smc_workspace_size(ctypes.byref(cfg), ctypes.byref(size))
        if st != smcgm.SMC_OK:
            raise smcgm.SMCError(st, lib.smc_last_error(None).decode())
        return size.value
    per_particle = ws(2) - ws(1)
    return int(min(cfg.n_particles, max(1, budget_bytes // max(1, per_particle))))


def batch_configs(specs, budget_bytes=3e9):
    """smc_config of every problem of a batching workload (inputs.load_batch_workload), each
    solve batch capped so that its solver workspace stays within `budget_bytes`."""
    cfgs = []
    for sp in specs:
        cfg = smcgm.make_config(sp)
        cfg.solve_batch = capped_solve_batch(cfg, budget_bytes)
        cfgs.append(cfg)
    return cfgs


def time_moves(samplers, steps, modes=("sequential", "threads", "graph")):
    """`steps` moves of every sampler (each with a fitted mixture), timed three ways: one
    sampler after another (smc_move), concurrently with a host thread per sampler, and as
    one CUDA graph (smcgm.Batch, one launch).  Each way is warmed up once first.  Returns
    {mode: dict(seconds, solves, solves_per_s, cg_per_solve)} and, for the graph, the
    seconds its capture and instantiation took."""
    import torch
    out = {}
    for mode in modes:
        batch = None
        if mode == "graph":
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            batch = smcgm.Batch(samplers, steps)
            capture_s = time.perf_counter() - t0

        def run():
            if mode == "sequential":
                for sm in samplers:
                    sm.smc_move(steps, allow_noconv=True)
            elif mode == "threads":
                with cf.ThreadPoolExecutor(max_workers=len(samplers)) as ex:
                    list(ex.map(lambda sm: sm.smc_move(steps, allow_noconv=True), samplers))
            else:
                batch.move(allow_noconv=True)
        run()                                                  # warm-up
        for sm in samplers:
            sm.smc_profile_query(reset=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run()
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        prof = [sm.smc_profile_query(reset=True) for sm in samplers]
        solves = sum(p["solves"] for p in prof)
        out[mode] = dict(seconds=sec, solves=solves, solves_per_s=solves / sec,
                         cg_per_solve=sum(p["cg_iterations"] for p in prof) / max(1, solves))
        if batch is not None:
            out[mode]["capture_seconds"] = capture_s
            batch.close()
    return out
