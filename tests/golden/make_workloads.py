"""Writes tests/golden/workload_<name>.json: observation points, the synthetic
truth (a prior draw: Sec. 3.2 takes its true field from the prior) and its noisy
observations, computed with the oracle only.

To avoid the inverse crime (Sec. 3.2) the data come from a grid refined by the
preset's ``data_refine`` factor; noise is sigma * N(0, 1) from Philox purpose
DATA.  For the mirror-pair preset the two noisy values of each pair are
averaged, so Phi(R u) = Phi(u) for the reflection R: x -> 1 - x.

Run:  python tests/golden/make_workloads.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402
from oracle import philox, prior, problem  # noqa: E402
from paper_2503_16028_gb300 import inputs  # noqa: E402


def make(name):
    p = dict(inputs.PRESETS[name])
    seed = p["seed"]
    obs = inputs.observation_points(name)
    lam = prior.eigenvalues(p["dim"], p["kl_modes"], p["alpha"])
    truth = np.sqrt(lam) * philox.normals(seed, lam.shape[0], 0, 0, philox.TRUTH)
    fine = dict(p)
    fine["n"] = p["n"] * p["data_refine"]
    prob = problem.Problem(obs=obs, data=np.zeros(len(obs)), **fine)
    y = prob.forward(truth)
    noise = p["sigma"] * philox.normals(seed, len(obs), 0, 0, philox.DATA)
    data = y + noise
    if name == "darcy64_bimodal":
        half = len(obs) // 2
        avg = 0.5 * (data[:half] + data[half:])
        data = np.concatenate([avg, avg])
    out = dict(name=name, obs=obs.tolist(), data=data.tolist(), truth=truth.tolist(),
               recipe="truth = sqrt(lambda)*N(0,1) [Philox TRUTH]; data = F_fine(truth) + sigma*N(0,1) [Philox DATA]; "
                      "F_fine on a grid refined x%d" % p["data_refine"])
    with open(os.path.join(HERE, "workload_%s.json" % name), "w") as fh:
        json.dump(out, fh)
    return out


def make_batch(count=32):
    """workload_batch<count>.json: the data of the batching workload's problems
    (inputs.batch_specs): truth = a prior draw (Philox TRUTH, the problem's seed), data =
    its observations on a grid refined x2 up to 512^2 (a 512^2 problem's data come from its
    own grid) plus sigma * N(0, 1) (Philox DATA)."""
    out = []
    for sp in inputs.batch_specs(count):
        lam = prior.eigenvalues(2, sp["kl_modes"], sp["alpha"])
        truth = np.sqrt(lam) * philox.normals(sp["seed"], lam.shape[0], 0, 0, philox.TRUTH)
        fine = {k: v for k, v in sp.items() if k not in ("obs", "index")}
        fine["n"] = min(2 * sp["n"], 512)
        prob = problem.Problem(obs=sp["obs"], data=np.zeros(len(sp["obs"])), **fine)
        y = prob.forward(truth)
        data = y + sp["sigma"] * philox.normals(sp["seed"], len(sp["obs"]), 0, 0, philox.DATA)
        out.append(dict(index=sp["index"], n=sp["n"], data=[round(float(v), 17) for v in data]))
        print("batch problem", sp["index"], "n", sp["n"], "N", sp["n_particles"], "obs", len(data), flush=True)
    doc = dict(count=count, problems=out,
               recipe="problems from paper_2503_16028_gb300.inputs.batch_specs; truth = sqrt(lambda)*N(0,1) [Philox TRUTH]; "
                      "data = F(truth) on a grid refined x2 up to 512^2 + sigma*N(0,1) [Philox DATA]")
    with open(os.path.join(HERE, "workload_batch%d.json" % count), "w") as fh:
        json.dump(doc, fh)


if __name__ == "__main__":
    names = sys.argv[1:] or list(inputs.PRESETS) + ["batch32"]
    for nm in names:
        if nm == "batch32":
            make_batch(32)
            continue
        o = make(nm)
        print(nm, "obs", len(o["obs"]), "data[:4]", np.round(o["data"][:4], 5))
