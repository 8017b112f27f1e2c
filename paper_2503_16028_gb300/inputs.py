"""Workload presets and seeded synthetic inputs.

This module holds numbers and seeded random arrays only -- no step of the
method's arithmetic -- so that both the CUDA path and the CPU oracle can
consume the same inputs.  Values that need the method (the synthetic truth
field and its noisy observations) are produced by ``tests/golden/make_workloads.py``
with the oracle and stored in ``tests/golden/workload_<name>.json``.

Presets follow the workloads of Sec. 3 of the paper (1D elliptic problem,
2D Darcy flow with point observations) at the sizes used for parity and for
the throughput measurement.
"""
import json
import os

import numpy as np

PRESETS = {
    # 1D elliptic -(e^u w')' = 1 on [0, 1], n = 128 FD intervals, 64 sine modes,
    # C = (I - 0.01 Lap)^-2, 20 equispaced observations, sigma = 0.01.
    "elliptic1d_n128": dict(dim=1, n=128, kl_modes=64, alpha=0.01, sigma=0.01,
                             source_kind=0, src_amp=1.0, src_width=0.0,
                             n_particles=256, n_components=2, gm_rank=64, mcmc_steps=5,
                             beta0=0.2, ess_frac=0.5, data_refine=2, seed=2503016028),
    # 2D Darcy on the unit square, 64 x 64 cells, 32 x 32 cosine modes,
    # C = (I - 0.02 Lap)^-2, f = 10 exp(-50 |x - c|^2), 16 observations in
    # mirror pairs (bimodal posterior), sigma = 0.005.
    "darcy64_bimodal": dict(dim=2, n=64, kl_modes=32, alpha=0.02, sigma=0.005,
                            source_kind=1, src_amp=10.0, src_width=50.0,
                            n_particles=1024, n_components=4, gm_rank=64, mcmc_steps=10,
                            beta0=0.2, ess_frac=0.5, data_refine=2, seed=2503016028),
    # 2D Darcy at 256 x 256 cells, 128 x 128 modes, 64 observations on a
    # jittered 8 x 8 lattice, sigma = 0.01, N = 4096, K = 8.
    "darcy256_precision": dict(dim=2, n=256, kl_modes=128, alpha=0.02, sigma=0.01,
                               source_kind=1, src_amp=10.0, src_width=50.0,
                               n_particles=4096, n_components=8, gm_rank=64, mcmc_steps=10,
                               beta0=0.2, ess_frac=0.5, data_refine=2, seed=2503016028),
}

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")


def observation_points(name):
    """Observation locations of a preset (seeded; no method arithmetic)."""
    p = PRESETS[name]
    if p["dim"] == 1:
        return np.arange(1, 21) / 21.0
    if name == "darcy64_bimodal":
        left = np.array([(x, y) for x in (0.2, 0.35) for y in (0.2, 0.4, 0.6, 0.8)])
        right = left.copy()
        right[:, 0] = 1.0 - right[:, 0]
        return np.concatenate([left, right])
    g = (np.arange(8) + 0.5) / 8.0
    X, Y = np.meshgrid(g, g, indexing="xy")
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    rng = np.random.default_rng(p["seed"])
    return pts + rng.uniform(-0.03, 0.03, size=pts.shape)


def load_workload(name):
    """Preset merged with the stored observation points and data."""
    with open(os.path.join(GOLDEN_DIR, "workload_%s.json" % name)) as fh:
        wl = json.load(fh)
    out = dict(PRESETS[name])
    out["name"] = name
    out["obs"] = np.asarray(wl["obs"], dtype=np.float64)
    out["data"] = np.asarray(wl["data"], dtype=np.float64)
    out["truth"] = np.asarray(wl["truth"], dtype=np.float64)
    return out


def random_particles(seed, N, d, scale=None):
    """Seeded standard-normal particle states (optionally scaled per coordinate)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, d))
    if scale is not None:
        X = X * np.asarray(scale)[None, :]
    return X


def random_potentials(seed, N, low=0.0, high=100.0):
    return np.random.default_rng(seed).uniform(low, high, size=N)


def structured_potentials(seed, N, low=0.0, high=200.0):
    """Seeded potentials with the structures that matter for reweighting and resampling:
    uniform values, the smallest value twice (a tie for the largest weight), a run of 16
    equal values (equal weights) and one value far below the rest (a dominant weight,
    at index N // 3)."""
    phi = np.random.default_rng(seed).uniform(low, high, size=N)
    lo = float(np.min(phi))
    phi[N // 2] = phi[N // 5] = lo                      # tie for the largest weight
    phi[N // 4:N // 4 + 16] = phi[N // 4]               # equal weights
    phi[N // 3] = lo - 0.05 * (high - low)              # dominant weight
    return phi


def structured_log_weights(seed, N, scale=3.0):
    """Seeded unnormalised log weights: normal values, a tie for the largest weight, a run of
    equal weights and one dominant weight (the log-weight analogue of structured_potentials)."""
    lw = np.random.default_rng(seed).normal(0.0, scale, size=N)
    hi = float(np.max(lw))
    lw[N // 2] = lw[N // 5] = hi
    lw[N // 4:N // 4 + 16] = lw[N // 4]
    lw[N // 3] = hi + 2.0
    return lw


BATCH_SEED = 20250320
BATCH_GRIDS = (64, 128, 256, 512)
BATCH_PARTICLES = (256, 1024, 4096)


def batch_specs(count=32, seed=BATCH_SEED):
    """Seeded specifications of `count` independent 2D Darcy inverse problems (the batching
    workload): grid n uniform in {64, 128, 256, 512}, particles uniform in {256, 1024, 4096},
    16 to 256 observation points uniform in [0.05, 0.95]^2, sigma uniform in [0.002, 0.02];
    the prior of the metric workload (alpha = 0.02) on min(64, n/2)^2 cosine modes, f as in
    the metric workload, K = 4 components on r = 64 modes, 10 moves per layer, and a seed per
    problem.  Numbers and seeded arrays only; the data come from tests/golden."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(BATCH_GRIDS))
        N = int(rng.choice(BATCH_PARTICLES))
        n_obs = int(rng.integers(16, 257))
        sigma = float(rng.uniform(0.002, 0.02))
        obs = rng.uniform(0.05, 0.95, size=(n_obs, 2))
        out.append(dict(index=i, dim=2, n=n, kl_modes=min(64, n // 2), alpha=0.02, sigma=sigma, source_kind=1,
                        src_amp=10.0, src_width=50.0, n_particles=N, n_components=4, gm_rank=64, mcmc_steps=10,
                        beta0=0.2, ess_frac=0.5, data_refine=2, seed=seed + 1000 + i, obs=obs))
    return out


def load_batch_workload(count=32):
    """The batching workload: batch_specs merged with the stored data of each problem."""
    with open(os.path.join(GOLDEN_DIR, "workload_batch%d.json" % count)) as fh:
        stored = json.load(fh)
    specs = batch_specs(count)
    for sp, st in zip(specs, stored["problems"]):
        assert st["index"] == sp["index"] and st["n"] == sp["n"] and len(st["data"]) == len(sp["obs"])
        sp["data"] = np.asarray(st["data"], dtype=np.float64)
    return specs
