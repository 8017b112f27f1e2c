"""Host logic of bench.py's secondary measurements, on CPU with a stand-in
sampler and event clock: the per-layer aggregation of the whole SMC run (first
layer, the layers with 0.1 < t < 1, all layers), the solver-only rate and the
mixed-precision agreement counters, and the whole-move HBM byte model."""
import os
import sys
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Clock:
    now = 0.0


class _Event:
    def __init__(self, enable_timing=True):
        self.t = None

    def record(self, stream=None):
        self.t = _Clock.now

    def elapsed_time(self, other):
        return other.t - self.t


class _Torch:
    float64 = "f64"

    class cuda:
        Event = _Event

        @staticmethod
        def synchronize():
            pass

    @staticmethod
    def tensor(a, dtype=None, device=None):
        return np.asarray(a, dtype=np.float64)

    @staticmethod
    def empty(n, dtype=None, device=None):
        return np.empty(n)


class _Sampler:
    """Temperatures 0.05, 0.15, ..., 1; the move at layer l takes (l + 1) ms for N * L solves
    and (10 + l) CG iterations per solve."""

    def __init__(self, N=8, d=4, L=10, X=None, P=None, acc_at=None):
        self.N, self.d, self.L, self.stream = N, d, L, None
        self.acc_at = acc_at or {}
        self.layer, self.t = -1, 0.0
        self.X = np.zeros((N, d)) if X is None else X
        self.P = np.ones(N) if P is None else P
        self.counts = dict(solves=0, cg=0)

    def smc_temper_step(self):
        self.layer += 1
        self.t = min(1.0, 0.05 + 0.1 * self.layer)
        return 0.1, 0.5, -0.5, self.t >= 1.0

    def smc_resample(self):
        pass

    def gm_fit(self):
        return 0.0

    def smc_get_schedule(self):
        return self.t, 0.2, self.layer, 0

    def smc_move(self, steps, allow_noconv=False):
        _Clock.now += self.layer + 1.0
        self.counts["solves"] += self.N * steps
        self.counts["cg"] += self.N * steps * (10 + self.layer)
        return self.acc_at.get(self.layer, 0.25), 20

    def diagnostics(self):
        return dict(indices=np.arange(self.N))

    def smc_forward(self, X, Phi):
        _Clock.now += 4.0
        self.counts["solves"] += X.shape[0]
        self.counts["cg"] += 12 * X.shape[0]

    def smc_profile_query(self, enable=-1, reset=False):
        out = dict(solves=self.counts["solves"], cg_iterations=self.counts["cg"])
        if reset:
            self.counts = dict(solves=0, cg=0)
        return out

    def particles(self):
        return self.X.copy(), self.P.copy()

    def smc_posterior_moments(self):
        return self.X.mean(axis=0), self.X.var(axis=0)

    def close(self):
        pass


def _smcgm(sampler, fp64_sampler=None):
    """Stand-in module: make_config returns the precision, Sampler picks the stand-in by it."""
    return types.SimpleNamespace(Sampler=lambda cfg: fp64_sampler if cfg == 0 else sampler,
                                 make_config=lambda wl, **kw: kw.get("precision", 1),
                                 SMC_P_FP32_REFINE=1, SMC_P_FP64=0)


def test_layers_aggregate_first_window_and_all():
    s = _Sampler()
    out, cmp = bench.time_layers(dict(mcmc_steps=10), 8, _smcgm(s), _Torch, fp64=False)
    assert cmp is None
    assert out["count"] == 11 and out["finished"] and out["log_evidence"] == pytest.approx(-5.5)
    # first layer: t = 0.05, 80 solves in 1 ms
    assert out["first"]["t"] == pytest.approx(0.05)
    assert out["first"]["solves_per_s"] == pytest.approx(80 / 1e-3)
    assert out["first"]["cg_per_solve"] == pytest.approx(10.0)
    # 0.1 < t < 1: layers 1..9 (t = 0.15 .. 0.95), (l + 1) ms each
    mid = out["t_between_0p1_and_1"]
    assert mid["layers"] == 9
    assert mid["solves_per_s"] == pytest.approx(9 * 80 / (sum(range(2, 11)) * 1e-3))
    assert mid["cg_per_solve"] == pytest.approx(np.mean([10 + l for l in range(1, 10)]))
    assert out["all"]["layers"] == 11
    assert out["all"]["solves_per_s"] == pytest.approx(11 * 80 / (sum(range(1, 12)) * 1e-3))


def test_forward_rate():
    s = _Sampler(N=16)
    out = bench.time_forward(s, _Torch, calls=2)
    assert out["ms_per_call"] == pytest.approx(4.0)
    assert out["value"] == pytest.approx(16 / 4e-3)
    assert out["cg_per_solve"] == pytest.approx(12.0)


def test_precision_agreement_counts(monkeypatch):
    rng = np.random.default_rng(1)
    X = rng.standard_normal((6, 3))
    P = rng.random(6) + 1.0
    X2, P2 = X.copy(), P.copy()
    X2[4, 1] += 1e-3
    P2[2] *= 1.0 + 1e-9
    mixed = _Sampler(N=6, d=3, X=X2, P=P2)
    monkeypatch.setattr(bench, "make_sampler", lambda wl, prec, N, smcgm: mixed)
    out = bench.precision_agreement(_Sampler(N=6, d=3, X=X, P=P), 3, {}, 6, _smcgm(mixed))
    assert out["particles_differing"] == 1
    assert out["max_abs_posterior_mean_diff"] == pytest.approx(1e-3 / 6)
    assert out["max_rel_phi_diff"] == pytest.approx(1e-9, rel=1e-3)
    assert mixed.counts["solves"] == 3 * 6       # the mixed sampler replays the FP64 sampler's moves


def test_whole_move_byte_model_by_hand():
    """The whole-move HBM model at 256^2 with the measured counters (14.71 CG iterations and
    3.155 refinement phases per solve, FP32 inner solver), worked out from its parts: tiled
    levels below the finest 128^2 and 64^2 (9.5 words each per own cell), the coarse kernel's
    faces and top level, 6 + 9.25 + 5.25 words per finest cell per CG iteration, 4.25 + 5.25
    per inner-solve start, 52 B per refinement, 66.8 B of set-up, 4 d doubles of KL vectors."""
    prof = dict(word_bytes=4, cells=65536, solves=100, cg_iterations=1471, inner_solves=315.5, residuals=315.5)
    lower = 9.5 / 4 + 9.5 / 16 + 2.0 / 48 + 2.0 / 64
    per_cell = (14.71 * (6 + 9.25 + 5.25 + lower) * 4 + 3.155 * (4.25 + 5.25 + lower) * 4
                + 3.155 * 52.0 + (16 + 24 + 2.7 * 4 + 16))
    expect = per_cell * 65536 + 4 * 16384 * 8
    got = bench.model_bytes_per_solve(prof, 256, 16384)
    assert got == pytest.approx(expect, rel=1e-12)
    assert got == pytest.approx(116.8e6, rel=2e-3)
    # 64^2: no tiled level below the finest; the coarse kernel starts at 32^2
    prof64 = dict(prof, cells=4096)
    lower64 = 2.0 / 48 + 2.0 / 4
    per_cell64 = (14.71 * (6 + 9.25 + 5.25 + lower64) * 4 + 3.155 * (4.25 + 5.25 + lower64) * 4
                  + 3.155 * 52.0 + (16 + 24 + 2.7 * 4 + 16))
    assert bench.model_bytes_per_solve(prof64, 64, 1024) == pytest.approx(per_cell64 * 4096 + 4 * 1024 * 8, rel=1e-12)


def test_layers_lockstep_against_fp64():
    """The mixed-precision run and the FP64 run in lockstep: identical layers give no differing
    decision; an acceptance rate that differs at layer 3 is reported as the first layer at which
    decisions differ; the posterior errors are relative L2 norms of the moment differences."""
    X = np.array([[1.0, 2.0], [3.0, 6.0]])
    same, cmp = bench.time_layers(dict(mcmc_steps=10), 2, _smcgm(_Sampler(N=2, d=2, X=X), _Sampler(N=2, d=2, X=X)),
                                  _Torch, fp64=True)
    assert cmp["first_layer_decisions_differ"] is None and cmp["layers"] == 11
    assert cmp["posterior_mean_rel_l2"] == 0.0 and cmp["posterior_var_rel_l2"] == 0.0
    X2 = X.copy()
    X2[0, 0] += 0.5
    _, cmp = bench.time_layers(dict(mcmc_steps=10), 2,
                               _smcgm(_Sampler(N=2, d=2, X=X2, acc_at={3: 0.5}), _Sampler(N=2, d=2, X=X)), _Torch, fp64=True)
    assert cmp["first_layer_decisions_differ"] == 3
    m64, m = X.mean(axis=0), X2.mean(axis=0)
    assert cmp["posterior_mean_rel_l2"] == pytest.approx(np.linalg.norm(m - m64) / np.linalg.norm(m64))
    v64, v = X.var(axis=0), X2.var(axis=0)
    assert cmp["posterior_var_rel_l2"] == pytest.approx(np.linalg.norm(v - v64) / np.linalg.norm(v64))
