"""Parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: Philox uniforms and every integer result (component choices,
accept decisions away from near-ties, resampling indices) must match exactly;
FP64 PDE solutions and potentials to 1e-10 relative (the solver stops at an
FP64 relative residual of 1e-10, which leaves a relative error near 1e-13; the
oracle solves exactly); KL coordinates of
moved particles to 1e-13 relative (they differ from the oracle only by
libm/CUDA transcendental rounding in the normals).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2503_16028_gb300 import inputs, smcgm  # noqa: E402
from oracle import problem as oproblem, smc as osmc, pcngm as opcngm, gm as ogm, darcy as odarcy, prior as oprior  # noqa: E402

NEAR_TIE = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_16028_gb300 import build
    build.build()
    smcgm.load_library()


def _sampler(name, **over):
    wl = inputs.load_workload(name)
    cfg = smcgm.make_config(wl, **over)
    return wl, cfg, smcgm.Sampler(cfg)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


@pytest.mark.parametrize("precision", [smcgm.SMC_P_FP64, smcgm.SMC_P_FP32_REFINE, smcgm.SMC_P_BF16SMOOTH_REFINE])
def test_init_draws_and_potentials_64(precision):
    wl, cfg, s = _sampler("darcy64_bimodal", n_particles=37, n_components=3, precision=precision)
    X, Phi = s.particles()
    prob = oproblem.from_workload(wl)
    for n in range(37):
        ref = osmc.prior_draw(wl["seed"], prob.lam, n)
        assert _rel(X[n], ref) < 1e-14
    for n in (0, 1, 17, 36):
        ref = prob.potential(X[n])
        assert abs(Phi[n] - ref) <= 1e-10 * abs(ref), (n, Phi[n], ref)
    s.close()


@pytest.mark.parametrize("tile_kernel", [0, 1, 3, 4])
@pytest.mark.parametrize("precision", [smcgm.SMC_P_FP64, smcgm.SMC_P_FP32_REFINE, smcgm.SMC_P_BF16SMOOTH_REFINE])
def test_forward_solution_matches_exact_solve(precision, tile_kernel):
    """Every stencil-tile kernel family (16 x 16 warp tiles with TMA staging, 32 x 32 block
    tiles, 16 x 16 warp tiles with global loads) in every precision."""
    wl, cfg, s = _sampler("darcy64_bimodal", n_particles=8, precision=precision, tile_kernel=tile_kernel)
    X, Phi = s.particles()
    n = cfg.n
    Xd = torch.tensor(X, dtype=torch.float64, device="cuda")
    Pd = torch.empty(8, dtype=torch.float64, device="cuda")
    Wd = torch.empty((8, n, n), dtype=torch.float64, device="cuda")
    it = s.smc_forward(Xd, Pd, Wd)
    assert it > 0
    W = Wd.cpu().numpy()
    prob = oproblem.from_workload(wl)
    for p in range(8):
        ref = prob.solve(X[p])
        assert _rel(W[p], ref) < 1e-10, (p, _rel(W[p], ref))
    s.close()


@pytest.mark.parametrize("precision", [smcgm.SMC_P_FP32_REFINE, smcgm.SMC_P_BF16SMOOTH_REFINE])
def test_forward_256_sampled_particles(precision):
    wl, cfg, s = _sampler("darcy256_precision", n_particles=6, n_components=2, precision=precision)
    X, Phi = s.particles()
    prob = oproblem.from_workload(wl)
    for p in (0, 5):
        ref = prob.potential(X[p])
        assert abs(Phi[p] - ref) <= 1e-10 * abs(ref), (p, Phi[p], ref)
    s.close()


def _random_mixture(s, rng, lam0):
    w, m, lam, modes = s.smc_get_mixture()
    K = w.shape[0]
    w = rng.dirichlet(np.ones(K) * 3)
    m = rng.standard_normal(m.shape) * np.sqrt(lam) * 0.8
    lam = lam * rng.uniform(0.3, 1.5, size=lam.shape)
    s.smc_set_mixture(w, m, lam)
    return opcngm.Mixture(modes, w, m, lam, lam0)


@pytest.mark.parametrize("precision,tile_kernel", [(smcgm.SMC_P_FP64, 0), (smcgm.SMC_P_FP32_REFINE, 0),
                                                    (smcgm.SMC_P_BF16SMOOTH_REFINE, 0), (smcgm.SMC_P_FP32_REFINE, 1),
                                                    (smcgm.SMC_P_FP32_REFINE, 3), (smcgm.SMC_P_BF16SMOOTH_REFINE, 4)])
def test_move_step_matches_oracle(precision, tile_kernel):
    N = 24
    wl, cfg, s = _sampler("darcy64_bimodal", n_particles=N, n_components=4, precision=precision, tile_kernel=tile_kernel)
    prob = oproblem.from_workload(wl)
    rng = np.random.default_rng(11)
    mix = _random_mixture(s, rng, prob.lam)
    X, Phi = s.particles()
    t, beta, step = 0.02, 0.35, 5
    s.smc_set_schedule(t, beta, 3, step)
    s.smc_move(1)
    X2, Phi2 = s.particles()
    dg = s.diagnostics()
    ties = 0
    for n in range(N):
        x, ph, acc, la, pv = osmc.move_particle(X[n], Phi[n], mix, beta, t, wl["seed"], n, step, prob.potential)
        assert abs(dg["phi_proposed"][n] - pv) <= 1e-10 * abs(pv), (n, dg["phi_proposed"][n], pv)
        assert abs(dg["log_alpha"][n] - la) <= 1e-8 * max(1.0, abs(la)), (n, dg["log_alpha"][n], la)
        U = float(osmc.philox.uniforms(wl["seed"], 0, n, step, osmc.philox.ACCEPT))
        if abs(np.log(U) - la) < NEAR_TIE:
            ties += 1
            continue
        assert bool(dg["accepted"][n]) == bool(acc), n
        assert _rel(X2[n], x) < 1e-13
        assert abs(Phi2[n] - ph) <= 1e-10 * abs(ph)
    assert ties == 0
    s.close()


def test_pcn_kernel_is_mixture_free():
    """SMC_K_PCN: log-ratio identically 0, so log alpha = t (Phi_u - Phi_v) (eq. a in pCN)."""
    wl, cfg, s = _sampler("darcy64_bimodal", n_particles=16, kernel=smcgm.SMC_K_PCN)
    X, Phi = s.particles()
    s.smc_set_schedule(0.1, 0.2, 0, 0)
    s.smc_move(1)
    dg = s.diagnostics()
    assert np.allclose(dg["log_alpha"], 0.1 * (Phi - dg["phi_proposed"]), rtol=0, atol=1e-12 * np.max(np.abs(Phi)))
    s.close()


def test_temper_resample_and_fit_match_oracle():
    N = 300
    wl, cfg, s = _sampler("darcy64_bimodal", n_particles=N, n_components=3, em_iters=25)
    X, Phi = s.particles()
    h, ess, lz, done = s.smc_temper_step()
    ref_h = osmc.bisect_h(Phi, 0.0, cfg.ess_frac * N)
    assert abs(h - ref_h) <= 1e-9 * ref_h
    assert abs(ess - osmc.ess_of_h(Phi, h)) <= 1e-9 * ess
    assert abs(lz - osmc.log_z_increment(Phi, h)) <= 1e-9 * max(1, abs(lz))
    s.smc_resample()
    idx = s.diagnostics()["indices"]
    ref_idx = osmc.systematic_indices(-h * Phi, osmc.resample_u48(wl["seed"], 0))
    assert np.array_equal(idx, ref_idx)
    X2, Phi2 = s.particles()
    assert np.array_equal(X2, X[ref_idx]) and np.array_equal(Phi2, Phi[ref_idx])
    ll = s.gm_fit()
    prob = oproblem.from_workload(wl)
    mix, hist = ogm.fit(X2, prob.gm_modes(cfg.gm_rank), prob.lam, 3, 25, wl["seed"], 0, var_floor=cfg.var_floor)
    w, m, lam, modes = s.smc_get_mixture()
    assert np.array_equal(modes, mix.S)
    assert np.allclose(w, mix.w, rtol=1e-8, atol=1e-12)
    assert np.allclose(m, mix.m, rtol=1e-7, atol=1e-9)
    assert np.allclose(lam, mix.lam, rtol=1e-7, atol=1e-12)
    assert abs(ll - hist[-1]) <= 1e-8 * abs(hist[-1])
    s.close()


def test_posterior_moments_match():
    wl, cfg, s = _sampler("darcy64_bimodal", n_particles=50)
    X, _ = s.particles()
    mean, var, mg, vg = s.smc_posterior_moments(grid=True)
    rm, rv = osmc.posterior_moments(X)
    assert np.allclose(mean, rm, rtol=1e-12, atol=1e-15) and np.allclose(var, rv, rtol=1e-11, atol=1e-15)
    assert np.allclose(mg, oprior.synthesize_2d(rm, cfg.n, cfg.kl_modes).ravel(), rtol=1e-12, atol=1e-13)
    U = oprior.synthesize_2d(X, cfg.n, cfg.kl_modes)
    assert np.allclose(vg, np.mean((U - mg.reshape(cfg.n, cfg.n)) ** 2, axis=0).ravel(), rtol=1e-10, atol=1e-13)
    s.close()


def test_elliptic_1d_full_run_matches_oracle():
    """Config-1 workload end to end (Alg. 1 with Alg. 2): layer-by-layer temperatures,
    acceptance rates and final moments agree with the oracle's own run."""
    wl = inputs.load_workload("elliptic1d_n128")
    N = 64
    cfg = smcgm.make_config(wl, n_particles=N, em_iters=20)
    s = smcgm.Sampler(cfg)
    prob = oproblem.from_workload(wl)
    ref = osmc.run(prob, N=N, K=cfg.n_components, r=cfg.gm_rank, L=wl["mcmc_steps"], beta0=wl["beta0"],
                   ess_frac=wl["ess_frac"], seed=wl["seed"], em_iters=20, max_layers=8)
    for lay in ref["layers"]:
        h, ess, lz, done = s.smc_temper_step()
        assert abs(h - lay["h"]) <= 1e-9 * lay["h"]
        s.smc_resample()
        s.gm_fit()
        acc, _ = s.smc_move(wl["mcmc_steps"])
        assert abs(acc - lay["acc"]) < 1e-12, (acc, lay["acc"])
        if done:
            break
    X, Phi = s.particles()
    assert _rel(X, ref["X"]) < 1e-10
    assert _rel(Phi, ref["Phi"]) < 1e-10
    s.close()


def test_elliptic_1d_smc_gm_full_run_matches_oracle():
    """SMC-GM (Alg. 3, SMC_K_GM_INDEP: beta = 1, every mixture draw accepted) end
    to end on the config-1 workload against the oracle's SMC-GM run."""
    wl = inputs.load_workload("elliptic1d_n128")
    N = 64
    cfg = smcgm.make_config(wl, n_particles=N, em_iters=20, kernel=smcgm.SMC_K_GM_INDEP)
    s = smcgm.Sampler(cfg)
    prob = oproblem.from_workload(wl)
    ref = osmc.run(prob, N=N, K=cfg.n_components, r=cfg.gm_rank, L=wl["mcmc_steps"], beta0=wl["beta0"],
                   ess_frac=wl["ess_frac"], seed=wl["seed"], em_iters=20, max_layers=8, kernel="gm_indep")
    for lay in ref["layers"]:
        h, ess, lz, done = s.smc_temper_step()
        assert abs(h - lay["h"]) <= 1e-9 * lay["h"]
        s.smc_resample()
        s.gm_fit()
        acc, _ = s.smc_move(wl["mcmc_steps"])
        assert acc == 1.0 and lay["acc"] == 1.0
        if done:
            break
    X, Phi = s.particles()
    assert _rel(X, ref["X"]) < 1e-10
    assert _rel(Phi, ref["Phi"]) < 1e-10
    s.close()


def test_checkpoint_roundtrip():
    wl, cfg, s = _sampler("darcy64_bimodal", n_particles=16)
    s.smc_set_schedule(0.2, 0.4, 2, 30)
    buf = s.smc_save()
    X, Phi = s.particles()
    s.smc_set_schedule(0.9, 0.1, 7, 99)
    s.smc_set_particles(np.zeros_like(X), np.zeros_like(Phi))
    s.smc_load(buf)
    X2, Phi2 = s.particles()
    assert np.array_equal(X, X2) and np.array_equal(Phi, Phi2)
    assert s.smc_get_schedule() == (0.2, 0.4, 2, 30)
    s.close()


def test_out_of_order_calls_are_rejected():
    wl, cfg, s = _sampler("darcy64_bimodal", n_particles=8)
    with pytest.raises(smcgm.SMCError) as e:
        s.smc_resample()
    assert e.value.status == smcgm.SMC_ESTATE
    with pytest.raises(smcgm.SMCError) as e:
        s.smc_move(1)                      # pCN-GM needs a fitted mixture
    assert e.value.status == smcgm.SMC_ESTATE
    s.close()


def test_bf16_smoother_matches_fp32_smoother():
    """The BF16 smoother changes only the preconditioner: at 256^2 the FP64-accurate
    solutions of both mixed-precision modes agree to the solver tolerance, and the CG
    iteration counts stay close (the V-cycle's operator differs by BF16 rounding, ~2^-9)."""
    wl = inputs.load_workload("darcy256_precision")
    N = 64
    out = {}
    for prec in (smcgm.SMC_P_FP32_REFINE, smcgm.SMC_P_BF16SMOOTH_REFINE):
        s = smcgm.Sampler(smcgm.make_config(wl, n_particles=N, n_components=2, precision=prec))
        X, _ = s.particles()
        Xd = torch.tensor(X, dtype=torch.float64, device="cuda")
        P = torch.empty(N, dtype=torch.float64, device="cuda")
        W = torch.empty((N, 256, 256), dtype=torch.float64, device="cuda")
        s.smc_profile_query(reset=True)
        s.smc_forward(Xd, P, W)
        prof = s.smc_profile_query(reset=True)
        out[prec] = (W.cpu().numpy(), P.cpu().numpy(), prof["cg_iterations"] / prof["solves"])
        s.close()
    W32, P32, it32 = out[smcgm.SMC_P_FP32_REFINE]
    W16, P16, it16 = out[smcgm.SMC_P_BF16SMOOTH_REFINE]
    for p in range(N):
        assert _rel(W16[p], W32[p]) < 2e-10
    assert np.max(np.abs(P16 - P32) / np.abs(P32)) < 2e-10
    assert it16 <= 1.15 * it32 + 1, (it16, it32)
