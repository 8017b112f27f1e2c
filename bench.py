"""Throughput of the SMC-pCN-GM particle move on GB300.

One step = one pCN-GM mutation step (proposal, KL synthesis, Darcy solve,
observation, accept) for every particle of the 256 x 256 Darcy workload
(N = 4096 particles, 128 x 128 KL modes, K = 8 mixture components, 64
observations).  Metric: particle-move PDE solves per second with the FP32
multigrid-CG + FP64 refinement solver; the FP64 solver is timed on the same
workload beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload.  Multi-GPU: one process per GPU
(torchrun), each an independent replica of the workload (weak scaling, no
collective in the timed region), timed with a barrier and the maximum over ranks.

Beside the headline the line carries: the roofline of the dominant kernel and
the whole-move HBM byte model, the FP64 solver's rate and its agreement with the
mixed-precision path, the solver-only rate (smc_forward), the end-to-end rate
with pinned host buffers through smc_batch_move_host (each move one CUDA graph;
the smc_move_host form beside it), the adjoint-gradient rate, a whole SMC
run to t = 1 timed layer by layer with an FP64 run of the same seed in lockstep
(the posterior error of the mixed-precision run against it), the 64^2 workload on
the GPU (host-driven and as one CUDA graph) and on the CPU oracle, the 32-problem
batching workload (one after another, a host thread each, one CUDA graph), the SM
clocks sampled during the timed region and the CPU oracle baseline.
--smoother fp32 times the FP32-smoother mode as the headline; --no-fp64, --no-alt-smoother, --no-graph,
--no-e2e, --no-forward, --no-em, --no-batch, --no-autotune, --no-gradient, --no-layers, --no-small and
--no-cpu leave legs out.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "darcy256_precision"
SMALL_WORKLOAD = "darcy64_bimodal"
# ncu dram__bytes_read.sum + dram__bytes_write.sum per cell of the dominant kernel k_tpre<2,CG>, from one
# capture of the current kernel on the 512-particle case (profiles/k_tpre_darcy256_n512.md), per smoother
# face storage; None where no capture of the current kernel exists
TRAFFIC_BYTES_PER_CELL = {"fp32": 36.03, "bf16": 31.83}
METRIC = "particle-move PDE solves/sec at 256^2, fp32+refine vs fp64; HBM roofline %"
UNIT = "solves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--particles", type=int, default=0, help="override N (default: the workload's 4096)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison path")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-gradient", action="store_true", help="skip the adjoint-gradient timing")
    ap.add_argument("--no-layers", action="store_true", help="skip the whole SMC run timed layer by layer")
    ap.add_argument("--no-small", action="store_true", help="skip the 64^2 workload (GPU and CPU oracle)")
    ap.add_argument("--smoother", default="bf16", choices=["fp32", "bf16"],
                    help="face storage of the multigrid smoother in the headline (mixed-precision) sampler")
    ap.add_argument("--no-alt-smoother", action="store_true", help="skip the timing of the other smoother storage")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (host buffers)")
    ap.add_argument("--no-forward", action="store_true", help="skip the solver-only leg")
    ap.add_argument("--no-graph", action="store_true", help="skip the headline moves as one CUDA graph")
    ap.add_argument("--no-em", action="store_true", help="skip the EM-fit timing")
    ap.add_argument("--no-batch", action="store_true", help="skip the 32-problem batching workload")
    ap.add_argument("--no-autotune", action="store_true", help="skip the solver-setting autotuner on the 64^2 workload")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0, help="oracle time of the whole reference run")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# CPU oracle: bounded sample of the same workload (move steps of a few particles)
# ---------------------------------------------------------------------------
CPU_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
from paper_2503_16028_gb300 import inputs
from oracle import problem, smc, pcngm
wl = inputs.load_workload(%(name)r)
prob = problem.from_workload(wl)
S = prob.gm_modes(wl["gm_rank"])
mix = pcngm.Mixture.prior(prob.lam, S, wl["n_components"])
budget = %(budget)f
done = 0
t0 = time.perf_counter()
n = %(start)d
while True:
    x = smc.prior_draw(wl["seed"], prob.lam, n)
    phi = prob.potential(x)
    t1 = time.perf_counter()
    smc.move_particle(x, phi, mix, 0.2, 0.3, wl["seed"], n, 0, prob.potential)
    done += 1
    n += %(stride)d
    if time.perf_counter() - t0 > budget:
        break
el = time.perf_counter() - t0
print(json.dumps(dict(solves=2 * done, seconds=el)))
"""


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_rate(budget_s, procs=None, workload=WORKLOAD):
    """Solves/s of the oracle on the host cores: one process per core (BLAS pinned to one thread
    each), process i moving particles i, i + procs, ...; the rate is all their solves over the
    longest process's time."""
    procs = procs or host_cores()
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    running = []
    for i in range(procs):
        code = CPU_SNIPPET % dict(root=ROOT, name=workload, budget=budget_s, start=i, stride=procs)
        running.append(subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                                        stderr=subprocess.PIPE, text=True, env=env))
    outs = []
    for p in running:
        so, se = p.communicate(timeout=900)
        if p.returncode != 0:
            raise RuntimeError("oracle baseline failed: " + se[-500:])
        outs.append(json.loads(so.strip().splitlines()[-1]))
    solves = sum(o["solves"] for o in outs)
    seconds = max(o["seconds"] for o in outs)
    return solves / seconds, dict(solves=solves, seconds=seconds, cores=procs)


def run_reference(args, rank):
    if rank != 0:
        return
    per_step = max(1.0, args.ref_seconds / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_oracle_rate(min(per_step, 5.0))
    rates, secs, solves = [], 0.0, 0
    for _ in range(args.steps):
        r, o = cpu_oracle_rate(per_step)
        rates.append(r)
        secs += o["seconds"]
        solves += o["solves"]
    value = solves / secs
    cores = o["cores"]
    sample = ("%d oracle solves (prior draw + one pCN step per particle, 256^2 sparse LU) in %.1f s on %d processes"
              % (solves, secs, cores))
    line = dict(metric=METRIC, value=value, unit=UNIT, impl="reference", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1000.0 * secs / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=WORKLOAD, particles_per_step="bounded sample", grid="256x256", kl_modes="128x128"),
                cpu_baseline=dict(value=value, unit=UNIT, cores=cores, kind="oracle", sample=sample),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=sorted(reasons), samples=len(sm), power_w_max=max(power) if power else None)


def make_sampler(wl, precision, N, smcgm):
    cfg = smcgm.make_config(wl, precision=precision, n_particles=N)
    s = smcgm.Sampler(cfg)
    # a realistic state: one tempering layer (reweight, resample, mixture fit)
    s.smc_temper_step()
    s.smc_resample()
    s.gm_fit()
    return s


def time_gradient(wl, N, smcgm, torch, calls=2, precision=None):
    """Phi and dPhi/dx of all N particles (a forward and an adjoint solve each, mixed precision),
    timed with CUDA events on the library's stream after one untimed call."""
    mixed = smcgm.SMC_P_FP32_REFINE if precision is None else precision
    s = smcgm.Sampler(smcgm.make_config(wl, n_particles=N, gradient=1, precision=mixed))
    X = torch.tensor(s.particles()[0], dtype=torch.float64, device="cuda")
    Phi = torch.empty(N, dtype=torch.float64, device="cuda")
    G = torch.empty_like(X)
    s.smc_gradient(X, Phi, G)
    s.smc_profile_query(enable=1, reset=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    for _ in range(calls):
        s.smc_gradient(X, Phi, G)
    e1.record(s.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / calls
    prof = s.smc_profile_query(reset=True)
    s.close()
    return dict(value=N / (ms / 1000.0), unit="gradients/s", ms_per_call=ms, particles=N,
                solves_per_gradient=prof["solves"] / (N * calls), cg_per_solve=prof["cg_iterations"] / max(1, prof["solves"]))


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def time_forward(s, torch, calls=2):
    """Solver-only throughput: smc_forward (KL synthesis, Darcy solve, observation, Phi; no proposal,
    mixture terms or accept) of the sampler's N particles, CUDA events on the library's stream
    after one untimed call."""
    X = torch.tensor(s.particles()[0], dtype=torch.float64, device="cuda")
    Phi = torch.empty(X.shape[0], dtype=torch.float64, device="cuda")
    s.smc_forward(X, Phi)
    s.smc_profile_query(reset=True)
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record(s.stream)
    for _ in range(calls):
        s.smc_forward(X, Phi)
    e1.record(s.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / calls
    prof = s.smc_profile_query(reset=True)
    return dict(value=X.shape[0] / (ms / 1000.0), unit=UNIT, ms_per_call=ms,
                cg_per_solve=prof["cg_iterations"] / max(1, prof["solves"]))


def time_layers(wl, N, smcgm, torch, max_layers=60, fp64=True, precision=None):
    """A whole SMC run of the workload (Alg. 2) to t = 1: every tempering layer reweights (ESS
    bisection), resamples, fits the mixture and makes L pCN-GM moves; each layer's smc_move of the
    mixed-precision sampler is timed with CUDA events.  Returns solves/s of the first layer's
    moves, of the moves of the layers with 0.1 < t < 1 and of all layers, with the layer count and
    the run's wall time.

    With fp64, an FP64 sampler of the same workload and seed runs beside it in lockstep, and the
    result carries the error of the mixed-precision run against it: per layer the temperature
    step, the resampling indices, the acceptance rate and the potentials; at t = 1 the relative
    L2 error of the posterior mean and variance of the KL coefficients (the target is 1e-6), and
    the first layer at which any decision (an index or an accept) differs, if one does."""
    mixed = smcgm.SMC_P_FP32_REFINE if precision is None else precision
    s = smcgm.Sampler(smcgm.make_config(wl, n_particles=N, precision=mixed))
    s64 = smcgm.Sampler(smcgm.make_config(wl, n_particles=N, precision=smcgm.SMC_P_FP64)) if fp64 else None
    L = wl["mcmc_steps"]
    rows, logz = [], 0.0
    cmp = dict(max_rel_h_diff=0.0, max_rel_phi_diff=0.0, first_layer_decisions_differ=None)
    run_seconds = 0.0
    for layer in range(max_layers):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h, _, lz, done = s.smc_temper_step()
        logz += lz
        s.smc_resample()
        s.gm_fit()
        t = s.smc_get_schedule()[0]
        s.smc_profile_query(reset=True)
        e0, e1 = _events(torch)
        e0.record(s.stream)
        acc, _ = s.smc_move(L, allow_noconv=True)
        e1.record(s.stream)
        torch.cuda.synchronize()
        run_seconds += time.perf_counter() - t0
        prof = s.smc_profile_query(reset=True)
        rows.append(dict(t=t, ms=e0.elapsed_time(e1), solves=prof["solves"], cg=prof["cg_iterations"], acc=acc))
        if s64 is not None:
            h64, _, _, done64 = s64.smc_temper_step()
            s64.smc_resample()
            idx_differ = not np.array_equal(s.diagnostics()["indices"], s64.diagnostics()["indices"])
            s64.gm_fit()
            acc64, _ = s64.smc_move(L, allow_noconv=True)
            _, P = s.particles()
            _, P64 = s64.particles()
            cmp["max_rel_h_diff"] = max(cmp["max_rel_h_diff"], abs(h - h64) / h64)
            cmp["max_rel_phi_diff"] = max(cmp["max_rel_phi_diff"],
                                          float(np.max(np.abs(P - P64) / np.maximum(np.abs(P64), 1e-300))))
            if cmp["first_layer_decisions_differ"] is None and (idx_differ or acc != acc64 or done != done64):
                cmp["first_layer_decisions_differ"] = layer
            if done != done64:
                break
        if done:
            break
    if s64 is not None:
        m, v = s.smc_posterior_moments()
        m64, v64 = s64.smc_posterior_moments()
        cmp.update(layers=len(rows), posterior_mean_rel_l2=float(np.linalg.norm(m - m64) / np.linalg.norm(m64)),
                   posterior_var_rel_l2=float(np.linalg.norm(v - v64) / np.linalg.norm(v64)), target=1e-6)
        s64.close()
    s.close()

    def agg(sel):
        if not sel:
            return None
        ms = sum(r["ms"] for r in sel)
        sv = sum(r["solves"] for r in sel)
        return dict(layers=len(sel), solves_per_s=sv / (ms / 1000.0), cg_per_solve=sum(r["cg"] for r in sel) / max(1, sv),
                    acceptance=sum(r["acc"] for r in sel) / len(sel))
    first = agg(rows[:1])
    first["t"] = rows[0]["t"]
    out = dict(count=len(rows), finished=bool(rows[-1]["t"] >= 1.0), moves_per_layer=L, run_seconds=run_seconds,
               log_evidence=logz, first=first, t_between_0p1_and_1=agg([r for r in rows if 0.1 < r["t"] < 1.0]),
               all=agg(rows))
    return out, (cmp if s64 is not None else None)


def precision_agreement(s64, moves, wl, N, smcgm, precision=None):
    """The mixed-precision path against the FP64 path from the same state: a fresh mixed-precision
    sampler of the workload taken through the FP64 sampler's history (one tempering layer, then
    `moves` single moves with the same random streams).  Returns the largest absolute difference
    of the posterior mean and variance of the KL coefficients, the largest relative difference of
    Phi and the number of particles whose states differ."""
    s = make_sampler(wl, smcgm.SMC_P_FP32_REFINE if precision is None else precision, N, smcgm)
    for _ in range(moves):
        s.smc_move(1, allow_noconv=True)
    X, P = s.particles()
    X64, P64 = s64.particles()
    m, v = s.smc_posterior_moments()[:2]
    m64, v64 = s64.smc_posterior_moments()[:2]
    s.close()
    return dict(moves=moves, max_abs_posterior_mean_diff=float(np.max(np.abs(m - m64))),
                max_abs_posterior_var_diff=float(np.max(np.abs(v - v64))),
                max_rel_phi_diff=float(np.max(np.abs(P - P64) / np.maximum(np.abs(P64), 1e-300))),
                particles_differing=int(np.sum(np.any(X != X64, axis=1))), target=1e-6)


def time_small(args, smcgm, torch, barrier, precision=None):
    """GPU solves/s on the 64^2 workload (32^2 modes, N = 1024, K = 4), timed like the headline
    (host-driven smc_move, CUDA events), and the same moves as one CUDA graph (smc_batch of
    this one problem, --steps moves per launch, wall clock around the launch)."""
    from paper_2503_16028_gb300 import inputs
    wl = inputs.load_workload(SMALL_WORKLOAD)
    N = wl["n_particles"]
    s = make_sampler(wl, smcgm.SMC_P_FP32_REFINE if precision is None else precision, N, smcgm)
    ms, prof = time_moves(s, args.steps, args.warmup, torch, barrier)
    b = smcgm.Batch([s], args.steps)
    b.move(allow_noconv=True)
    s.smc_profile_query(reset=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = 3
    for _ in range(reps):
        b.move(allow_noconv=True)
    torch.cuda.synchronize()
    gsec = (time.perf_counter() - t0) / reps
    gprof = s.smc_profile_query(reset=True)
    b.close()
    s.close()
    return dict(workload=SMALL_WORKLOAD, particles=N, value=N * args.steps / (ms / 1000.0),
                unit=UNIT, cg_per_solve=prof["cg_iterations"] / max(1, prof["solves"]),
                host_syncs_per_move=prof["host_syncs"] / args.steps,
                graph=dict(value=N * args.steps / gsec, unit=UNIT, ms_per_launch=1000.0 * gsec, moves_per_launch=args.steps,
                           host_syncs_per_move=gprof["host_syncs"] / (reps * args.steps),
                           cg_per_solve=gprof["cg_iterations"] / max(1, gprof["solves"])))


def autotune_small(smcgm):
    """batch.autotune on the 64^2 workload (N = 1024): every candidate setting (stencil-tile
    kernels, smoothing counts, coarse factor, inner tolerance) timed over two moves."""
    from paper_2503_16028_gb300 import batch, inputs
    wl = inputs.load_workload(SMALL_WORKLOAD)
    best, timings = batch.autotune(wl, n_particles=wl["n_particles"], steps=2, reps=2)
    return dict(workload=SMALL_WORKLOAD, particles=wl["n_particles"], best=best,
                ms_per_move=[dict(setting=c, ms=t) for c, t in timings])


def time_batch32(smcgm, torch, steps=2, precision=None):
    """The batching workload: 32 independent Darcy problems (grids 64^2..512^2, 256..4096
    particles, 16..256 observations, sigma 0.002..0.02; inputs.batch_specs), each taken
    through one tempering layer and a mixture fit, then `steps` moves of all of them timed
    one after another, with a host thread per problem, and as one CUDA graph."""
    from paper_2503_16028_gb300 import batch, inputs
    specs = inputs.load_batch_workload(32)
    cfgs = batch.batch_configs(specs)
    if precision is not None:
        for cfg in cfgs:
            cfg.precision = precision
    samplers = batch.make_samplers(cfgs)
    for sm in samplers:
        sm.smc_temper_step()
        sm.smc_resample()
        sm.gm_fit()
    modes = batch.time_moves(samplers, steps)
    cells = sum(sp["n"] ** 2 * sp["n_particles"] for sp in specs)
    for sm in samplers:
        sm.close()
    torch.cuda.empty_cache()
    out = dict(workload="batch32: 32 independent Darcy problems, grids 64^2..512^2, 256..4096 particles",
               problems=len(specs), moves=steps, particle_solves_per_move=sum(sp["n_particles"] for sp in specs),
               cell_solves_per_move=cells, unit=UNIT, **modes)
    out["graph_vs_sequential"] = modes["graph"]["solves_per_s"] / modes["sequential"]["solves_per_s"]
    out["graph_vs_threads"] = modes["graph"]["solves_per_s"] / modes["threads"]["solves_per_s"]
    return out


def time_em(wl, N, smcgm, torch, calls=2, precision=None):
    """gm_fit (the EM fit on the r leading modes, em_iters iterations) on the workload's
    resampled particles, diagonal and full covariances, each timed with CUDA events on the
    library's stream after one untimed call."""
    out = {}
    for form, full in (("diagonal", 0), ("full_covariance", 1)):
        s = smcgm.Sampler(smcgm.make_config(wl, n_particles=N, full_cov=full,
                                            precision=smcgm.SMC_P_FP32_REFINE if precision is None else precision))
        s.smc_temper_step()
        s.smc_resample()
        s.gm_fit()
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record(s.stream)
        for _ in range(calls):
            s.gm_fit()
        e1.record(s.stream)
        torch.cuda.synchronize()
        out[form] = dict(ms_per_fit=e0.elapsed_time(e1) / calls, em_iters=int(s.cfg.em_iters), components=int(s.cfg.n_components),
                         modes=int(s.r), particles=N)
        s.close()
    return out


def time_graph(s, N, steps, torch, reps=2):
    """The same moves as the headline as one CUDA graph (smc_batch of this one problem, `steps`
    moves per launch: no host wait inside the move), wall clock around the launches after one
    untimed launch."""
    from paper_2503_16028_gb300 import smcgm
    b = smcgm.Batch([s], steps)
    b.move(allow_noconv=True)
    s.smc_profile_query(reset=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        b.move(allow_noconv=True)
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / reps
    prof = s.smc_profile_query(reset=True)
    b.close()
    return dict(value=N * steps / sec, unit=UNIT, ms_per_move=1000.0 * sec / steps, moves_per_launch=steps,
                host_syncs_per_move=prof["host_syncs"] / (reps * steps),
                cg_per_solve=prof["cg_iterations"] / max(1, prof["solves"]))


def pinned_buffers(N, d, torch):
    """The e2e legs' page-locked host buffers (X in, Phi in, X out, Phi out), allocated once when the
    bench starts, as an application would allocate its staging buffers."""
    return (torch.empty((N, d), dtype=torch.float64).pin_memory(), torch.empty(N, dtype=torch.float64).pin_memory(),
            torch.empty((N, d), dtype=torch.float64).pin_memory(), torch.empty(N, dtype=torch.float64).pin_memory())


def time_e2e(s, N, d, steps, torch, barrier, world, bufs=None):
    """End to end through the C ABI (smc_move_host): every step copies the particles and potentials
    from pinned host buffers to the device, moves them and copies them back, inside the timed region
    (wall clock over all steps, after one untimed call)."""
    Xh, Ph, Xo, Po = bufs or pinned_buffers(N, d, torch)
    X0, P0 = s.particles()
    Xh.numpy()[:] = X0
    Ph.numpy()[:] = P0
    s.smc_move_host(Xh, Ph, Xo, Po)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step_ms = []
    for _ in range(steps):
        ts = time.perf_counter()
        s.smc_move_host(Xh, Ph, Xo, Po)          # returns after its device-to-host copies
        step_ms.append((time.perf_counter() - ts) * 1000.0)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1000.0, world, "cuda")
    return dict(value=whole_job_rate(N * steps, world, e2e_ms), unit=UNIT, h2d_bytes_per_step=N * d * 8 + N * 8,
                d2h_bytes_per_step=N * d * 8 + N * 8, steps=steps,
                step_ms=dict(min=min(step_ms), median=statistics.median(step_ms), max=max(step_ms)))


def time_e2e_graph(s, N, d, steps, torch, barrier, world, smcgm, bufs=None):
    """End to end through the batched-move API with host buffers (smc_batch_move_host on a
    one-sampler batch, one move per launch): every step copies the particles and potentials in
    from pinned host buffers, runs the move as one CUDA graph (its loops on the device, one host
    wait) and copies them back, inside the timed region (wall clock over all steps)."""
    Xh, Ph, Xo, Po = bufs or pinned_buffers(N, d, torch)
    X0, P0 = s.particles()
    Xh.numpy()[:] = X0
    Ph.numpy()[:] = P0
    b = smcgm.Batch([s], steps=1)
    try:
        b.move_host([Xh], [Ph], [Xo], [Po], allow_noconv=True)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step_ms = []
        for _ in range(steps):
            ts = time.perf_counter()
            b.move_host([Xh], [Ph], [Xo], [Po], allow_noconv=True)
            step_ms.append((time.perf_counter() - ts) * 1000.0)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1000.0, world, "cuda")
    finally:
        b.close()
    return dict(value=whole_job_rate(N * steps, world, e2e_ms), unit=UNIT, h2d_bytes_per_step=N * d * 8 + N * 8,
                d2h_bytes_per_step=N * d * 8 + N * 8, steps=steps, api="smc_batch_move_host",
                step_ms=dict(min=min(step_ms), median=statistics.median(step_ms), max=max(step_ms)))


def time_moves(s, steps, warmup, torch, barrier):
    for _ in range(warmup):
        s.smc_move(1, allow_noconv=True)
    s.smc_profile_query(enable=1, reset=True)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    for _ in range(steps):
        s.smc_move(1, allow_noconv=True)
    e1.record(s.stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    prof = s.smc_profile_query(enable=0, reset=True)
    return ms, prof


def model_bytes_per_solve(prof, n, d):
    """Algorithmic DRAM bytes of the whole move per particle-solve (every array read or written once per pass)."""
    w = prof["word_bytes"]
    cells = prof["cells"]
    solves = max(1, prof["solves"])
    it = prof["cg_iterations"] / solves
    inner = prof["inner_solves"] / solves
    res = prof["residuals"] / solves
    # per V-cycle below the finest level (words per finest cell): each tiled level l >= 1 (n_l > 32)
    # pre-smoothing 4.25 words of its cells (r, Kw, Ks in; e, 1/4 restricted out) and post-smoothing
    # 5.25 (r, e, Kw, Ks, 1/4 parent in; e2 out), a fraction 4^-l of the finest cells; the coarse
    # kernel (32^2 and below) reads the coarse faces (2 words x 1/48) and its top level's r, writes e2
    n = int(round(cells ** 0.5))
    lower, l = 0.0, 1
    while (n >> l) > 32:
        lower += 9.5 * 4.0 ** -l
        l += 1
    lower += 2.0 / 48.0 + 2.0 * 4.0 ** -l
    # per CG iteration (per cell): apply 6 words, fine pre 9.25, fine post 5.25, and the levels below
    cg = (6 + 9.25 + 5.25 + lower) * w
    start = (4.25 + 5.25 + lower) * w                          # z0 = M r0 per inner solve
    refine = 24.0 + 28.0                                      # w += x (w, x in and out); residual (w, faces hi/lo in; r out)
    # set-up: synthesis passes (T^T out and in, u out: 16 B), faces (u in, faces hi/lo out: 24 B),
    # coarsening (2.7 words), w and x cleared and r = b (16 B)
    setup = 16.0 + 24.0 + 2.7 * w + 16.0
    per_cell = it * cg + inner * start + res * refine + setup
    kl = 4 * d * 8                                            # X read, V write, accept copy (worst case) and the synthesis read
    return per_cell * cells + kl


def max_over_ranks(ms, world, device):
    """The job's duration: the largest per-rank duration (all ranks started together after a barrier)."""
    if world == 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms_max):
    """Units processed by all ranks over the job's duration (weak scaling: each rank does the same work)."""
    return units_per_rank * world / (ms_max / 1000.0)


def run_native(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    from paper_2503_16028_gb300 import inputs, smcgm
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    barrier = (lambda: torch.distributed.barrier()) if world > 1 else (lambda: None)
    wl = inputs.load_workload(WORKLOAD)
    N = args.particles or wl["n_particles"]
    d = wl["kl_modes"] ** 2
    bufs = None if args.no_e2e else pinned_buffers(N, d, torch)
    # CPU oracle first (before the GPU is busy; a plain subprocess, no fork of a CUDA process)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, o = cpu_oracle_rate(args.cpu_seconds)
        cpu = dict(value=rate, unit=UNIT, cores=o["cores"], kind="oracle",
                   sample="%d solves of the 256^2 workload (prior draw + one pCN step per particle, sparse LU), "
                          "%.1f s on %d processes" % (o["solves"], o["seconds"], o["cores"]))
    cpu_small = None
    if rank == 0 and world == 1 and not args.no_cpu and not args.no_small:
        rate, o = cpu_oracle_rate(args.cpu_seconds / 3.0, workload=SMALL_WORKLOAD)
        cpu_small = dict(value=rate, unit=UNIT, cores=o["cores"], kind="oracle",
                         sample="%d solves of the 64^2 workload in %.1f s on %d processes" % (o["solves"], o["seconds"], o["cores"]))
    from paper_2503_16028_gb300 import build
    build.build()
    smcgm.load_library()
    prec_of = {"fp32": smcgm.SMC_P_FP32_REFINE, "bf16": smcgm.SMC_P_BF16SMOOTH_REFINE}
    alt = "bf16" if args.smoother == "fp32" else "fp32"
    s = make_sampler(wl, prec_of[args.smoother], N, smcgm)
    d = s.d
    clocks = ClockSampler(local)
    ms, prof = time_moves(s, args.steps, args.warmup, torch, barrier)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms, world, "cuda")
    value = whole_job_rate(N * args.steps, world, ms_max)
    # roofline of the dominant kernel (finest-level CG update + pre-smoothing + restriction)
    dom_ach = prof["dom_bytes"] / (prof["dom_ms"] / 1000.0) / 1e9 if prof["dom_ms"] > 0 else 0.0
    # DRAM bytes per cell of the dominant kernel from one ncu capture of the current kernel on
    # the 512-particle case, scaled to the average particles of a launch here
    tb = TRAFFIC_BYTES_PER_CELL.get(args.smoother)
    traffic = tb * 65536 * prof["dom_particles"] / max(1, prof["dom_launches"]) if tb else None
    roof = dict(bound="hbm", achieved=dom_ach, peak=hbm_peak, unit="GB/s", frac=dom_ach / hbm_peak, traffic=traffic,
                algorithmic_bytes_per_launch=prof["dom_bytes"] / max(1, prof["dom_launches"]),
                kernel="k_tpre<2,CG> (finest level, CG update + pre-smoothing + restriction, TMA-staged; %s smoother faces)"
                % args.smoother.upper(), peak_source=peak_src,
                launches=prof["dom_launches"], ms_per_launch=prof["dom_ms"] / max(1, prof["dom_launches"]))
    bps = model_bytes_per_solve(prof, 256, d)
    step_hbm = bps * N / (ms / args.steps / 1000.0) / 1e9
    iters = dict(cg_per_solve=prof["cg_iterations"] / max(1, prof["solves"]),
                 inner_solves_per_solve=prof["inner_solves"] / max(1, prof["solves"]),
                 residuals_per_solve=prof["residuals"] / max(1, prof["solves"]),
                 host_syncs_per_move=prof["host_syncs"] / args.steps)
    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = e2e_host = None
    if not args.no_e2e:
        e2e_host = time_e2e(s, N, d, args.steps, torch, barrier, world, bufs)
        e2e_host["api"] = "smc_move_host"
        e2e = time_e2e_graph(s, N, d, args.steps, torch, barrier, world, smcgm, bufs)
    forward = None if args.no_forward else time_forward(s, torch)
    graph = None if args.no_graph else time_graph(s, N, args.steps, torch)
    s.close()
    del s
    torch.cuda.empty_cache()
    alt_leg = None
    if not args.no_alt_smoother:
        sb = make_sampler(wl, prec_of[alt], N, smcgm)
        msb, profb = time_moves(sb, args.steps, args.warmup, torch, barrier)
        sb.close()
        msb = max_over_ranks(msb, world, "cuda")
        dom_b = profb["dom_bytes"] / (profb["dom_ms"] / 1000.0) / 1e9 if profb["dom_ms"] > 0 else 0.0
        alt_leg = dict(smoother=alt, value=whole_job_rate(N * args.steps, world, msb), unit=UNIT, ms_per_step=msb / args.steps,
                       cg_per_solve=profb["cg_iterations"] / max(1, profb["solves"]),
                       inner_solves_per_solve=profb["inner_solves"] / max(1, profb["solves"]),
                       dominant_kernel=dict(achieved=dom_b, frac=dom_b / hbm_peak,
                                            algorithmic_bytes_per_launch=profb["dom_bytes"] / max(1, profb["dom_launches"]),
                                            ms_per_launch=profb["dom_ms"] / max(1, profb["dom_launches"])))
        torch.cuda.empty_cache()
    fp64 = agree = None
    if not args.no_fp64:
        s64 = make_sampler(wl, smcgm.SMC_P_FP64, N, smcgm)
        ms64, prof64 = time_moves(s64, max(2, args.steps // 2), 1, torch, barrier)
        st64 = max(2, args.steps // 2)
        ms64 = max_over_ranks(ms64, world, "cuda")
        fp64 = dict(value=whole_job_rate(N * st64, world, ms64), ms_per_step=ms64 / st64,
                    cg_per_solve=prof64["cg_iterations"] / max(1, prof64["solves"]),
                    dominant_kernel_gbs=prof64["dom_bytes"] / (prof64["dom_ms"] / 1000.0) / 1e9 if prof64["dom_ms"] else None)
        agree = precision_agreement(s64, 1 + st64, wl, N, smcgm, precision=prec_of[args.smoother])
        s64.close()
    em = None if args.no_em else time_em(wl, N, smcgm, torch, precision=prec_of[args.smoother])
    grad = None
    if not args.no_gradient:
        grad = time_gradient(wl, N, smcgm, torch, precision=prec_of[args.smoother])
    layers = posterior = None
    if not args.no_layers:
        layers, posterior = time_layers(wl, N, smcgm, torch, fp64=not args.no_fp64, precision=prec_of[args.smoother])
    batch32 = None if args.no_batch else time_batch32(smcgm, torch, precision=prec_of[args.smoother])
    tuned = None if args.no_autotune else autotune_small(smcgm)
    small = None
    if not args.no_small:
        small = time_small(args, smcgm, torch, barrier, precision=prec_of[args.smoother])
        small["cpu_oracle"] = cpu_small
    if rank != 0:
        return
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms_max / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32+f64",
                data="synthetic",
                config=dict(workload=WORKLOAD, particles=N, grid="256x256", kl_modes="128x128", components=8,
                            observations=64, solver="FP32 MG-PCG (RB-GS 2+2, Galerkin, coarse x2; %s smoother faces) + FP64 refinement to 1e-10"
                            % args.smoother.upper(),
                            l2="inputs larger than L2 (%.1f GB device working set)" % (s_bytes(N) / 1e9),
                            parallelism="replicas" if world > 1 else "single GPU"),
                roofline=roof, hbm_roofline_step=dict(model_bytes_per_solve=bps, achieved_gbs=step_hbm,
                                                      frac=step_hbm / hbm_peak, peak=hbm_peak),
                iterations=iters, fp64=fp64,
                speedup_vs_fp64=(value / fp64["value"]) if fp64 else None, posterior_error_vs_fp64=posterior,
                fp64_agreement=agree,
                solver_only=forward, graph=graph, smoother_alternative=alt_leg, e2e=e2e, e2e_host_driven=e2e_host,
                clocks=clk, gpu_launches=prof["launches"],
                cpu_baseline=cpu,
                adjoint_gradient=grad, em_fit=em, smc_run=layers, small_workload=small, batch_workload=batch32,
                autotune=tuned)
    print(json.dumps(line), flush=True)


def s_bytes(N):
    return N * (3 * 16384 * 8 + 65536 * (4 * 8 + 12 * 4))


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if args.impl == "native" else "gloo"
        if args.impl == "native":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_native(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
