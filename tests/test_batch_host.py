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
