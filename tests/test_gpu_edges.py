"""Edge cases and full-size parity of the CUDA path against the FP64 oracle.

* The metric workload at its full size and launch configuration (256^2, 4096
  particles, the solver settings bench.py times), checked on sampled particles
  that the oracle solves one by one: initial potentials and one pCN-GM move.
* Ragged solve batches: forward solves split into batches of 5 (5 + 5 + 3)
  give bit-identical results to one batch (every per-particle reduction has a
  fixed order and no particle sees another's data).
* The smallest population, two particles (one is rejected by the
  configuration check: the weights of one particle carry no information).
* A log-permeability outside the double-float range of the mixed-precision
  set-up (|u| >= 64) fails with a clear error and leaves the context usable.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2503_16028_gb300 import inputs, smcgm  # noqa: E402
from oracle import problem as oproblem, smc as osmc, pcngm as opcngm  # noqa: E402

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


def _random_mixture(s, rng, lam0):
    w, m, lam, modes = s.smc_get_mixture()
    K = w.shape[0]
    w = rng.dirichlet(np.ones(K) * 3)
    m = rng.standard_normal(m.shape) * np.sqrt(lam) * 0.8
    lam = lam * rng.uniform(0.3, 1.5, size=lam.shape)
    s.smc_set_mixture(w, m, lam)
    return opcngm.Mixture(modes, w, m, lam, lam0)


def test_full_size_metric_workload_sampled():
    wl = inputs.load_workload("darcy256_precision")
    cfg = smcgm.make_config(wl)                       # N = 4096, K = 8, the default solver settings
    s = smcgm.Sampler(cfg)
    prob = oproblem.from_workload(wl)
    X, Phi = s.particles()
    N = X.shape[0]
    assert N == 4096
    sample = (0, 1, 1365, 2730, 4095)
    for n in sample:
        assert _rel(X[n], osmc.prior_draw(wl["seed"], prob.lam, n)) < 1e-14
        ref = prob.potential(X[n])
        assert abs(Phi[n] - ref) <= 1e-10 * abs(ref), (n, Phi[n], ref)
    # one pCN-GM step with a random 8-component mixture on the 64 leading modes
    mix = _random_mixture(s, np.random.default_rng(5), prob.lam)
    t, beta, step = 0.05, 0.2, 7
    s.smc_set_schedule(t, beta, 0, step)
    s.smc_move(1)
    X2, Phi2 = s.particles()
    dg = s.diagnostics()
    for n in sample:
        x, ph, acc, la, pv = osmc.move_particle(X[n], Phi[n], mix, beta, t, wl["seed"], n, step, prob.potential)
        assert abs(dg["phi_proposed"][n] - pv) <= 1e-10 * abs(pv), (n, dg["phi_proposed"][n], pv)
        U = float(osmc.philox.uniforms(wl["seed"], 0, n, step, osmc.philox.ACCEPT))
        if abs(np.log(U) - la) < NEAR_TIE:
            continue
        assert bool(dg["accepted"][n]) == bool(acc), n
        assert _rel(X2[n], x) < 1e-13
        assert abs(Phi2[n] - ph) <= 1e-10 * abs(ph)
    s.close()


@pytest.mark.parametrize("precision", [smcgm.SMC_P_FP64, smcgm.SMC_P_FP32_REFINE, smcgm.SMC_P_BF16SMOOTH_REFINE])
def test_ragged_batches_are_bit_identical(precision):
    wl = inputs.load_workload("darcy64_bimodal")
    N = 13
    s1 = smcgm.Sampler(smcgm.make_config(wl, n_particles=N, n_components=2, precision=precision))
    s2 = smcgm.Sampler(smcgm.make_config(wl, n_particles=N, n_components=2, precision=precision, solve_batch=5))
    X1, P1 = s1.particles()
    X2, P2 = s2.particles()
    assert np.array_equal(X1, X2)
    assert np.array_equal(P1, P2)
    n = wl["n"]
    Xd = torch.tensor(X1, dtype=torch.float64, device="cuda")
    W1 = torch.empty((N, n, n), dtype=torch.float64, device="cuda")
    W2 = torch.empty_like(W1)
    F1 = torch.empty(N, dtype=torch.float64, device="cuda")
    F2 = torch.empty_like(F1)
    s1.smc_forward(Xd, F1, W1)
    s2.smc_forward(Xd, F2, W2)
    torch.cuda.synchronize()
    assert torch.equal(W1, W2) and torch.equal(F1, F2)
    prob = oproblem.from_workload(wl)
    assert _rel(W2[12].cpu().numpy(), prob.solve(X1[12])) < 1e-10
    s1.close()
    s2.close()


def test_two_particles():
    wl = inputs.load_workload("darcy64_bimodal")
    s = smcgm.Sampler(smcgm.make_config(wl, n_particles=2, n_components=1))
    prob = oproblem.from_workload(wl)
    X, Phi = s.particles()
    for n in range(2):
        ref = prob.potential(X[n])
        assert abs(Phi[n] - ref) <= 1e-10 * abs(ref)
    _random_mixture(s, np.random.default_rng(3), prob.lam)
    s.smc_set_schedule(0.1, 0.3, 0, 1)
    s.smc_move(1)
    X2, Phi2 = s.particles()
    for n in range(2):
        assert abs(Phi2[n] - prob.potential(X2[n])) <= 1e-10 * abs(Phi2[n])
    s.close()


def test_out_of_range_field_fails_cleanly():
    wl = inputs.load_workload("darcy64_bimodal")
    N = 4
    s = smcgm.Sampler(smcgm.make_config(wl, n_particles=N, n_components=1, precision=smcgm.SMC_P_FP32_REFINE))
    X, Phi = s.particles()
    bad = X.copy()
    bad[2, 0] = 80.0                                   # the constant mode: u >= 80 - |rest| > 64 everywhere
    Xd = torch.tensor(bad, dtype=torch.float64, device="cuda")
    F = torch.empty(N, dtype=torch.float64, device="cuda")
    with pytest.raises(smcgm.SMCError) as ei:
        s.smc_forward(Xd, F)
    assert "mixed-precision range" in str(ei.value)
    # the context stays usable for in-range fields
    Xd = torch.tensor(X, dtype=torch.float64, device="cuda")
    s.smc_forward(Xd, F)
    torch.cuda.synchronize()
    prob = oproblem.from_workload(wl)
    ref = prob.potential(X[1])
    assert abs(F[1].item() - ref) <= 1e-10 * abs(ref)
    s.close()


def test_move_rejects_out_of_range_proposal():
    """In a move, a proposal whose field leaves the mixed-precision range is
    rejected (Phi_v = +inf) instead of failing the call; the other particles
    move exactly as the oracle's kernel."""
    wl = inputs.load_workload("darcy64_bimodal")
    N = 6
    s = smcgm.Sampler(smcgm.make_config(wl, n_particles=N, n_components=2, precision=smcgm.SMC_P_FP32_REFINE))
    prob = oproblem.from_workload(wl)
    X, Phi = s.particles()
    X = X.copy()
    Phi = Phi.copy()
    X[2, 0] = 80.0                                    # constant mode: gamma * 80 + noise stays above 64
    Phi[2] = 1e3                                      # any finite value (the field cannot be solved in FP32 + df32)
    s.smc_set_particles(X, Phi)
    mix = _random_mixture(s, np.random.default_rng(9), prob.lam)
    t, beta, step = 0.05, 0.2, 3
    s.smc_set_schedule(t, beta, 0, step)
    s.smc_move(1)
    X2, Phi2 = s.particles()
    dg = s.diagnostics()
    assert not dg["accepted"][2] and np.isinf(dg["phi_proposed"][2])
    assert np.array_equal(X2[2], X[2]) and Phi2[2] == Phi[2]
    for n in (0, 1, 3, 4, 5):
        x, ph, acc, la, pv = osmc.move_particle(X[n], Phi[n], mix, beta, t, wl["seed"], n, step, prob.potential)
        assert abs(dg["phi_proposed"][n] - pv) <= 1e-10 * abs(pv)
        U = float(osmc.philox.uniforms(wl["seed"], 0, n, step, osmc.philox.ACCEPT))
        if abs(np.log(U) - la) < NEAR_TIE:
            continue
        assert bool(dg["accepted"][n]) == bool(acc)
        assert _rel(X2[n], x) < 1e-13
    s.close()


def test_smc_gm_does_not_take_out_of_range_proposal():
    """SMC-GM (Alg. 3, beta = 1: every mixture draw is taken) with one component whose mean
    puts the constant mode at 80: a particle that draws that component gets a field
    outside the mixed-precision range, so its proposal is not taken and its state and
    potential stay; every other particle takes its proposal, equal to the oracle's."""
    wl = inputs.load_workload("darcy64_bimodal")
    N = 8
    s = smcgm.Sampler(smcgm.make_config(wl, n_particles=N, n_components=2, precision=smcgm.SMC_P_FP32_REFINE,
                                        kernel=smcgm.SMC_K_GM_INDEP))
    prob = oproblem.from_workload(wl)
    X, Phi = s.particles()
    w, m, lam, modes = s.smc_get_mixture()
    assert modes[0] == 0                                  # the constant mode leads the mixture modes
    w = np.array([0.5, 0.5])
    m = np.zeros_like(m)
    m[1, 0] = 80.0
    s.smc_set_mixture(w, m, lam)
    mix = opcngm.Mixture(modes, w, m, lam, prob.lam)
    step = 4
    s.smc_set_schedule(0.3, 1.0, 0, step)
    s.smc_move(1)
    X2, Phi2 = s.particles()
    dg = s.diagnostics()
    far = 0
    for n in range(N):
        Uc = float(osmc.philox.uniforms(wl["seed"], 0, n, step, osmc.philox.COMP))
        j = opcngm.choose_component(w, Uc)
        if j == 1:
            far += 1
            assert not dg["accepted"][n] and np.isinf(dg["phi_proposed"][n])
            assert np.array_equal(X2[n], X[n]) and Phi2[n] == Phi[n]
        else:
            v, pv, acc, _, _ = osmc.move_particle(X[n], Phi[n], mix, 1.0, 0.3, wl["seed"], n, step, prob.potential,
                                                  always_accept=True)
            assert dg["accepted"][n]
            assert _rel(X2[n], v) < 1e-13
            assert abs(Phi2[n] - pv) <= 1e-10 * abs(pv)
    assert 0 < far < N
    s.close()
