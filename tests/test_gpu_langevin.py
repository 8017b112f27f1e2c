"""The pCN-Langevin mutation (SMC_K_PCNL) against the oracle's kernel
(oracle/langevin.py, pinned by detailed balance), with the oracle's adjoint
gradient for DPhi: one step on every particle, and a two-step call in which
the second step proposes from the gradients the first one carried over."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2503_16028_gb300 import inputs, smcgm  # noqa: E402
from oracle import adjoint as oadjoint, langevin as olangevin, pcngm as opcngm, philox as ophilox, problem as oproblem  # noqa: E402

NEAR_TIE = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_16028_gb300 import build
    build.build()
    smcgm.load_library()


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


@pytest.mark.parametrize("steps", [1, 2])
def test_pcnl_move_matches_oracle(steps):
    wl = inputs.load_workload("darcy64_bimodal")
    N = 8
    s = smcgm.Sampler(smcgm.make_config(wl, n_particles=N, n_components=1, kernel=smcgm.SMC_K_PCNL, gradient=1))
    prob = oproblem.from_workload(wl)
    pg = lambda v: oadjoint.potential_and_gradient_2d(prob, v)[:2]
    X, Phi = s.particles()
    # the explicit drift (1 - gamma) t C DPhi is a step of size ~ (beta^2/2) t lambda |DPhi|: keep
    # it below 0.5 in every coordinate, as a tempering schedule does early on (with sigma = 0.005
    # the prior draws have |DPhi| up to ~1e5, and a larger step leaves |u| < 64)
    beta, step0 = 0.25, 5
    gscale = max(np.max(np.abs(prob.lam * pg(X[n])[1])) for n in range(N))
    t = min(0.3, 0.5 / ((1.0 - np.sqrt(1.0 - beta ** 2)) * gscale))
    s.smc_set_schedule(t, beta, 0, step0)
    rate, _ = s.smc_move(steps)
    X2, Phi2 = s.particles()
    dg = s.diagnostics()
    accepted, any_tie = 0, False
    for n in range(N):
        x, ph = X[n], Phi[n]
        g = pg(x)[1]
        tie = False
        for k in range(steps):
            x, ph, g, acc, la, pv = olangevin.move_particle(x, ph, g, prob.lam, beta, t, wl["seed"], n, step0 + k, pg)
            U = float(ophilox.uniforms(wl["seed"], 0, n, step0 + k, ophilox.ACCEPT))
            tie = tie or abs(np.log(U) - la) < NEAR_TIE
            accepted += int(acc)
        if tie:
            any_tie = True
            continue
        # the last step's diagnostics
        assert abs(dg["phi_proposed"][n] - pv) <= 1e-10 * abs(pv), (n, dg["phi_proposed"][n], pv)
        assert abs(dg["log_alpha"][n] - la) <= 1e-8 * max(1.0, abs(la)), (n, dg["log_alpha"][n], la)
        assert bool(dg["accepted"][n]) == bool(acc), n
        assert _rel(X2[n], x) < 1e-12, n
        assert abs(Phi2[n] - ph) <= 1e-10 * abs(ph)
    if not any_tie:
        assert rate == pytest.approx(accepted / (N * steps))
    s.close()


def test_pcnl_needs_gradient_flag():
    wl = inputs.load_workload("darcy64_bimodal")
    with pytest.raises(smcgm.SMCError) as ei:
        smcgm.Sampler(smcgm.make_config(wl, n_particles=4, n_components=1, kernel=smcgm.SMC_K_PCNL))
    assert "gradient" in str(ei.value)


def test_gmpcnl_move_matches_oracle():
    """GMpCN-Langevin with a random 3-component mixture on the leading modes, two steps."""
    wl = inputs.load_workload("darcy64_bimodal")
    N, steps = 8, 2
    s = smcgm.Sampler(smcgm.make_config(wl, n_particles=N, n_components=3, kernel=smcgm.SMC_K_GMPCNL, gradient=1))
    prob = oproblem.from_workload(wl)
    pg = lambda v: oadjoint.potential_and_gradient_2d(prob, v)[:2]
    w, m, lam, modes = s.smc_get_mixture()
    rng = np.random.default_rng(21)
    w = rng.dirichlet(np.ones(3) * 3)
    m = rng.standard_normal(m.shape) * np.sqrt(lam) * 0.8
    lam = lam * rng.uniform(0.3, 1.5, size=lam.shape)
    s.smc_set_mixture(w, m, lam)
    mix = opcngm.Mixture(modes, w, m, lam, prob.lam)
    X, Phi = s.particles()
    beta, step0 = 0.25, 9
    gscale = max(np.max(np.abs(prob.lam * pg(X[n])[1])) for n in range(N))
    t = min(0.3, 0.5 / ((1.0 - np.sqrt(1.0 - beta ** 2)) * gscale))
    s.smc_set_schedule(t, beta, 0, step0)
    s.smc_move(steps)
    X2, Phi2 = s.particles()
    dg = s.diagnostics()
    for n in range(N):
        x, ph = X[n], Phi[n]
        g = pg(x)[1]
        tie = False
        for k in range(steps):
            x, ph, g, acc, la, pv = olangevin.gm_move_particle(x, ph, g, mix, beta, t, wl["seed"], n, step0 + k, pg)
            U = float(ophilox.uniforms(wl["seed"], 0, n, step0 + k, ophilox.ACCEPT))
            tie = tie or abs(np.log(U) - la) < NEAR_TIE
        if tie:
            continue
        assert abs(dg["phi_proposed"][n] - pv) <= 1e-10 * abs(pv), (n, dg["phi_proposed"][n], pv)
        assert abs(dg["log_alpha"][n] - la) <= 1e-8 * max(1.0, abs(la)), (n, dg["log_alpha"][n], la)
        assert bool(dg["accepted"][n]) == bool(acc), n
        assert _rel(X2[n], x) < 1e-12, n
        assert abs(Phi2[n] - ph) <= 1e-10 * abs(ph)
    s.close()
