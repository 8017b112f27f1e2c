"""Host logic of batch.py (no GPU): the autotuner's choice (the fastest
candidate wins, ties go to the earlier one) and the per-layer JSONL log of
run_smc, driven by a stand-in sampler."""
import io
import json

import numpy as np

from paper_2503_16028_gb300 import batch


def test_pick_fastest():
    a, b, c = dict(), dict(smooth_sweeps=1), dict(tol_inner=1e-3)
    assert batch.pick_fastest([(a, 3.0), (b, 2.0), (c, 2.5)]) is b
    assert batch.pick_fastest([(a, 2.0), (b, 2.0)]) is a


class _Sampler:
    """Temperatures 0.3, 0.6, 1; each layer's moves count 10 solves per step with 12 CG
    iterations and 3 refinement phases per solve; beta 0.2, 0.4, 0.8."""

    def __init__(self):
        self.layer, self.t, self.beta = -1, 0.0, 0.1
        self.counts = dict(solves=0, cg_iterations=0, inner_solves=0)

    def smc_temper_step(self):
        self.layer += 1
        h = min(0.3, 1.0 - self.t) if self.layer < 2 else 1.0 - self.t
        self.t = min(1.0, self.t + h)
        self.beta *= 2.0
        return h, 50.0 + self.layer, -0.5 * (self.layer + 1), self.t >= 1.0

    def smc_resample(self):
        pass

    def gm_fit(self):
        return -100.0 - self.layer

    def smc_get_schedule(self):
        return self.t, self.beta, self.layer, 0

    def smc_profile_query(self, enable=-1, reset=False):
        out = dict(self.counts)
        if reset:
            self.counts = dict(solves=0, cg_iterations=0, inner_solves=0)
        return out

    def smc_move(self, steps, allow_noconv=False):
        self.counts["solves"] += 10 * steps
        self.counts["cg_iterations"] += 120 * steps
        self.counts["inner_solves"] += 30 * steps
        return 0.25 + 0.05 * self.layer, 17

    def particles(self):
        return np.zeros((2, 3)), np.zeros(2)


def test_run_smc_writes_one_json_line_per_layer(tmp_path):
    buf = io.StringIO()
    out = batch.run_smc(_Sampler(), mcmc_steps=4, log=buf)
    rows = [json.loads(line) for line in buf.getvalue().splitlines()]
    assert len(rows) == len(out["layers"]) == 3
    assert [r["layer"] for r in rows] == [0, 1, 2]
    assert np.allclose([r["t"] for r in rows], [0.3, 0.6, 1.0])
    assert [r["beta"] for r in rows] == [0.2, 0.4, 0.8]
    assert all(r["solves"] == 40 and r["cg_per_solve"] == 12.0 and r["refinements_per_solve"] == 3.0 for r in rows)
    assert [r["acceptance"] for r in rows] == [0.25, 0.30, 0.35] and rows[0]["cg_max"] == 17
    assert [r["gm_loglik"] for r in rows] == [-100.0, -101.0, -102.0]
    # a path: appended, closed afterwards
    path = tmp_path / "layers.jsonl"
    batch.run_smc(_Sampler(), mcmc_steps=1, log=str(path))
    batch.run_smc(_Sampler(), mcmc_steps=1, log=str(path))
    assert len(path.read_text().splitlines()) == 6
    # no log: the library's counters are left alone
    s = _Sampler()
    batch.run_smc(s, mcmc_steps=2)
    assert s.counts["solves"] == 3 * 20


def test_batch_specs_are_seeded_and_in_range():
    from paper_2503_16028_gb300 import inputs
    a, b = inputs.batch_specs(), inputs.batch_specs()
    assert len(a) == 32
    for x, y in zip(a, b):
        assert x["n"] == y["n"] and x["n_particles"] == y["n_particles"] and np.array_equal(x["obs"], y["obs"])
        assert x["n"] in (64, 128, 256, 512) and x["n_particles"] in (256, 1024, 4096)
        assert 16 <= len(x["obs"]) <= 256 and 0.002 <= x["sigma"] <= 0.02
        assert np.all((x["obs"] > 0.0) & (x["obs"] < 1.0)) and x["kl_modes"] <= x["n"] // 2
    assert len({sp["n"] for sp in a}) == 4                      # every grid size drawn
    w = inputs.load_batch_workload(32)
    assert all(len(sp["data"]) == len(sp["obs"]) and np.all(np.isfinite(sp["data"])) for sp in w)


def test_capped_solve_batch_fits_the_budget():
    """The cap uses the library's workspace size (no GPU needed): the solver share of the
    workspace at the chosen batch fits the budget, one more particle would not (or all fit)."""
    import ctypes
    from paper_2503_16028_gb300 import build, inputs, smcgm
    build.build()
    lib = smcgm.load_library()
    sp = next(x for x in inputs.load_batch_workload(32) if x["n"] == 512 and x["n_particles"] == 4096)
    cfg = smcgm.make_config(sp)
    budget = 3e9
    B = batch.capped_solve_batch(cfg, budget)
    size = ctypes.c_size_t()

    def ws(b):
        cfg.solve_batch = b
        assert lib.smc_workspace_size(ctypes.byref(cfg), ctypes.byref(size)) == smcgm.SMC_OK
        return size.value
    per = ws(2) - ws(1)
    assert 1 <= B < 4096
    assert B * per <= budget < (B + 1) * per
    small = smcgm.make_config(next(x for x in inputs.load_batch_workload(32) if x["n"] == 64))
    assert batch.capped_solve_batch(small, budget) == small.n_particles
