"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake in one oracle function on the CPU (monkeypatched
for the duration of the case: a dropped term, a wrong sign, an operand
transposed, an off-by-one, a wrong mean or scale), runs the pins written for
that function, and requires at least one of them to fail with an assertion.
The oracle's own functions look each other up through their module, so a
planted mistake also reaches the functions built on it.
"""
import numpy as np
import pytest

from oracle import adjoint, darcy, gm, langevin, observe, pcngm, philox, prior, smc

import test_oracle_adjoint as t_adj
import test_oracle_darcy as t_darcy
import test_oracle_fullcov as t_full
import test_oracle_gm as t_gm
import test_oracle_langevin as t_lang
import test_oracle_observe as t_obs
import test_oracle_philox as t_philox
import test_oracle_pcngm as t_pcngm
import test_oracle_prior as t_prior
import test_oracle_smc as t_smc


# --- the planted mistakes (each takes the original function) ------------------------------

def log_r_without_logdet(orig):
    def f(b, a, mix, beta):
        out = orig(b, a, mix, beta)
        if mix.cov is None:
            l0 = mix.lam0[mix.S]
            out = out - np.array([np.sum(0.5 * np.log(l0 / mix.lam[j])) for j in range(mix.K)])
        return out
    return f


def propose_shift_gamma(orig):
    def f(u, j, z, mix, beta):
        v = orig(u, j, z, mix, beta)
        g = pcngm.gamma_of(beta)
        v[mix.S] += (2.0 * g - 1.0) * mix.m[j]          # gamma m_j instead of (1 - gamma) m_j
        return v
    return f


def propose_full_with_covariance(orig):
    def f(u, j, z, mix, beta):
        if mix.cov is None:
            return orig(u, j, z, mix, beta)
        v = orig(u, j, z, mix, beta)
        L = np.linalg.cholesky(mix.cov[j])
        v[mix.S] += beta * ((mix.cov[j] - L) @ z[mix.S])   # C_j z instead of L_j z
        return v
    return f


def ess_without_square(orig):
    def f(phi, h):
        e = np.exp(-h * (phi - np.min(phi)))
        return np.sum(e) / np.sum(e * e)
    return f


def log_z_without_mean(orig):
    def f(phi, h):
        return orig(phi, h) + np.log(phi.shape[0])
    return f


def systematic_strict_walk(orig):
    def f(logw, u48):
        N = len(logw)
        cdf = smc.fixed_point_cdf(smc.normalised_weights(np.asarray(logw, dtype=np.float64)))
        out = np.empty(N, dtype=np.int64)
        i = 0
        for k in range(N):
            target = k * smc.RESAMPLE_T + u48
            while i < N - 1 and N * cdf[i] < target:      # '<' where the walk needs '<='
                i += 1
            out[k] = i
        return out
    return f


def arithmetic_faces(orig):
    def f(kc):
        kc = np.asarray(kc, dtype=np.float64)
        Kw = np.zeros_like(kc)
        Ks = np.zeros_like(kc)
        Kw[..., :, 1:] = 0.5 * (kc[..., :, 1:] + kc[..., :, :-1])
        Ks[..., 1:, :] = 0.5 * (kc[..., 1:, :] + kc[..., :-1, :])
        D = Kw.copy()
        D[..., :, :-1] += Kw[..., :, 1:]
        D += Ks
        D[..., :-1, :] += Ks[..., 1:, :]
        D[..., :, 0] += 2.0 * kc[..., :, 0]
        D[..., :, -1] += 2.0 * kc[..., :, -1]
        D[..., 0, :] += 2.0 * kc[..., 0, :]
        D[..., -1, :] += 2.0 * kc[..., -1, :]
        return Kw, Ks, D
    return f


def observe_transposed(orig):
    def f(w, obs_xy):
        return orig(w, np.ascontiguousarray(np.asarray(obs_xy)[:, ::-1]))
    return f


def eigenvalues_first_power(orig):
    def f(Km, alpha):
        return orig(Km, alpha) ** 0.5                   # (1 + alpha mu)^-1 instead of ^-2
    return f


def gradient_without_walls(orig):
    def f(kc, w, lam):
        g = orig(kc, w, lam)
        Kw, Ks, dWo, dWn, dSo, dSn, Ke, Kn = adjoint.face_derivatives(kc)
        g[:, 0] += dWo[:, 0] * lam[:, 0] * w[:, 0]
        g[0, :] += dSo[0, :] * lam[0, :] * w[0, :]
        g[:, -1] += Ke * lam[:, -1] * w[:, -1]
        g[-1, :] += Kn * lam[-1, :] * w[-1, :]
        return g
    return f


def e_step_without_normaliser(orig):
    def f(xs, w, m, lam):
        N, K = xs.shape[0], w.shape[0]
        logp = np.empty((N, K))
        for j in range(K):
            logp[:, j] = np.log(w[j]) + np.sum(-(xs - m[j]) ** 2 / (2.0 * lam[j]), axis=1)
        mx = np.max(logp, axis=1, keepdims=True)
        lse = mx[:, 0] + np.log(np.sum(np.exp(logp - mx), axis=1))
        return np.exp(logp - lse[:, None]), float(np.sum(lse))
    return f


def rho_sign_flipped(orig):
    def f(a, b, g_a, lam, beta, t):
        gm_ = langevin.gamma_of(beta)
        k = (1.0 - gm_) * t
        return k * float(g_a @ (b - gm_ * a)) / beta ** 2 - k * k * float(g_a @ (lam * g_a)) / (2.0 * beta ** 2)
    return f


def langevin_drift_without_t(orig):
    def f(x, g, lam, beta, t, z):
        return orig(x, g, lam, beta, 1.0 if t != 0.0 else 0.0, z)
    return f


def potential_without_half(orig):
    def f(y, data, sigma):
        return 2.0 * orig(y, data, sigma)
    return f


def cosine_basis_without_sqrt2(orig):
    def f(n, Km):
        B = orig(n, Km).copy()
        B[:, 1:] /= np.sqrt(2.0)
        return B
    return f


def analysis_transposed(orig):
    def f(g, Km):
        return orig(np.swapaxes(np.asarray(g), -1, -2), Km)
    return f


def accept_comparison_flipped(orig):
    def f(log_a, U):
        return bool(log_a >= 0.0 or np.log(U) > log_a)
    return f


def beta_rule_thresholds_swapped(orig):
    def f(beta, acc_rate):
        if acc_rate < 0.15:
            beta = 2.0 * beta
        elif acc_rate > 0.3:
            beta = 0.5 * beta
        return min(beta, 1.0)
    return f


def solve_without_h2(orig):
    def f(u, f_):
        n = u.shape[0]
        return orig(u, f_) * (n * n)
    return f


def gm_log_R_without_base(orig):
    def f(b, a, g_a, mix, beta, t):
        gm_ = langevin.gamma_of(beta)
        q0 = -0.5 * np.sum((b - gm_ * a) ** 2 / (beta ** 2 * mix.lam0) + np.log(beta ** 2 * mix.lam0))
        return orig(b, a, g_a, mix, beta, t) + q0
    return f


def sample_variance(orig):
    def f(X):
        m, v = orig(X)
        N = X.shape[0]
        return m, v * N / (N - 1)
    return f


def component_draw_closed_on_the_right(orig):
    def f(w, U):
        c = 0.0
        for j, wj in enumerate(w):
            c += wj
            if U <= c:
                return j
        return len(w) - 1
    return f


def init_indices_with_repeats(orig):
    def f(seed, layer, N, K):
        return [int((int(smc.philox.word32(seed, k, 0, layer, smc.philox.EMINIT)) * N) >> 32) for k in range(K)]
    return f


def bisection_returns_upper_bracket(orig):
    def f(phi, t, target, iters=64):
        rest = 1.0 - t
        if smc.ess_of_h(phi, rest) >= target:
            return rest
        lo, hi = 0.0, rest
        for _ in range(iters):
            mid = 0.5 * (lo + hi)
            if smc.ess_of_h(phi, mid) >= target:
                lo = mid
            else:
                hi = mid
        return hi
    return f


def prior_draw_without_sqrt(orig):
    def f(seed, lam, n):
        return orig(seed, lam, n) / np.sqrt(lam)
    return f


def solve_1d_without_h2(orig):
    def f(u_mid, f_nodes):
        n = u_mid.shape[0]
        return orig(u_mid, f_nodes) * (n * n)
    return f


def sine_basis_at_nodes(orig):
    def f(n, Km):
        x = np.arange(n) / n
        return np.sqrt(2.0) * np.sin(np.pi * np.outer(x, np.arange(1, Km + 1)))
    return f


def observe_1d_shifted(orig):
    def f(w_interior, obs_x):
        n = w_interior.shape[-1] + 1
        return orig(w_interior, np.clip(np.asarray(obs_x) + 0.5 / n, 0.0, 1.0))
    return f


def gm_propose_prior_noise(orig):
    def f(x, g, j, z, mix, beta, t):
        v = orig(x, g, j, z, mix, beta, t)
        lamj = mix.lam0.copy()
        lamj[mix.S] = mix.lam[j]
        return v + beta * (np.sqrt(mix.lam0) - np.sqrt(lamj)) * z
    return f


def box_muller_half_angle(orig):
    def f(seed, npairs, c1, c2, purpose):
        k0, k1 = philox.key_of(seed)
        m = np.arange(npairs, dtype=np.uint64)
        w = philox.philox4x32_10(m, c1, c2, purpose, k0, k1)
        u1 = philox.uniform_open(w[0], w[1])
        u2 = philox.uniform_open(w[2], w[3])
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.empty(2 * npairs)
        z[0::2] = r * np.cos(np.pi * u2)                 # pi where the angle needs 2 pi
        z[1::2] = r * np.sin(np.pi * u2)
        return z
    return f


def observation_matrix_transposed(orig):
    def f(n, obs_xy):
        perm = np.arange(n * n).reshape(n, n).T.ravel()
        return orig(n, obs_xy)[:, perm]                 # column i n + j where the grid is j n + i
    return f


def full_e_step_logdet_sign(orig):
    def f(xs, w, m, cov):
        N, r = xs.shape
        logp = np.empty((N, w.shape[0]))
        for j in range(w.shape[0]):
            _, logdet = np.linalg.slogdet(cov[j])
            dev = xs - m[j]
            q = np.sum(dev * np.linalg.solve(cov[j], dev.T).T, axis=1)
            logp[:, j] = np.log(w[j]) - 0.5 * (r * np.log(2.0 * np.pi) - logdet) - 0.5 * q
        mx = np.max(logp, axis=1, keepdims=True)
        lse = mx[:, 0] + np.log(np.sum(np.exp(logp - mx), axis=1))
        return np.exp(logp - lse[:, None]), float(np.sum(lse))
    return f


def mh_potential_sign(orig):
    def f(t, phi_u, phi_v, log_ratio):
        return t * (phi_v - phi_u) + log_ratio
    return f


def langevin_alpha_without_t(orig):
    def f(x, v, phi_x, phi_v, g_x, g_v, lam, beta, t):
        return orig(x, v, phi_x, phi_v, g_x, g_v, lam, beta, t) + (1.0 - t) * (phi_x - phi_v)
    return f


def cdf_ceil(orig):
    def f(w):
        q = [int(np.ceil(wi * smc.RESAMPLE_T)) for wi in w]      # ceil where the reading floors
        q[int(np.argmax(w))] += smc.RESAMPLE_T - sum(q)
        return list(np.cumsum(np.array(q, dtype=object)))
    return f


def cdf_remainder_to_smallest(orig):
    def f(w):
        q = [int(np.floor(wi * smc.RESAMPLE_T)) for wi in w]
        q[int(np.argmin(w))] += smc.RESAMPLE_T - sum(q)        # smallest weight takes the remainder
        return list(np.cumsum(np.array(q, dtype=object)))
    return f


def cdf_ties_to_highest_index(orig):
    def f(w):
        q = [int(np.floor(wi * smc.RESAMPLE_T)) for wi in w]
        w = np.asarray(w)
        q[len(w) - 1 - int(np.argmax(w[::-1]))] += smc.RESAMPLE_T - sum(q)   # last of the equal largest
        return list(np.cumsum(np.array(q, dtype=object)))
    return f


def _fit_variant(reseed_highest=False, collapse_weight_k=False, floor_at_lambda=False):
    """gm.fit with one planted change (the rest as the oracle's EM)."""
    def fit(X, S, lam0, K, iters, seed, layer, var_floor=1e-3):
        X = np.asarray(X, dtype=np.float64)
        N = X.shape[0]
        xs = X[:, S]
        lamS = np.asarray(lam0)[S]
        floor = lamS if floor_at_lambda else var_floor * lamS
        pm = np.mean(xs, axis=0)
        pooled = np.maximum(np.mean((xs - pm) ** 2, axis=0), floor)
        idx = gm.init_indices(seed, layer, N, K)
        w = np.full(K, 1.0 / K)
        m = xs[idx].copy()
        lam = np.tile(pooled, (K, 1))
        hist = []
        for _ in range(iters):
            g, ll = gm.e_step(xs, w, m, lam)
            hist.append(ll)
            Nj = np.sum(g, axis=0)
            for j in range(K):
                if Nj[j] < 2.0:
                    mg = np.max(g, axis=1)
                    n_star = int(np.argmax(mg)) if reseed_highest else int(np.argmin(mg))
                    m[j] = xs[n_star]
                    lam[j] = pooled
                    w[j] = 1.0 / K if collapse_weight_k else 1.0 / N
                    continue
                w[j] = Nj[j] / N
                m[j] = np.sum(g[:, j:j + 1] * xs, axis=0) / Nj[j]
                lam[j] = np.maximum(np.sum(g[:, j:j + 1] * (xs - m[j]) ** 2, axis=0) / Nj[j], floor)
            w = w / np.sum(w)
        g, ll = gm.e_step(xs, w, m, lam)
        hist.append(ll)
        return pcngm.Mixture(S, w, m, lam, lam0), hist
    return fit


def fit_reseed_at_highest(orig):
    return _fit_variant(reseed_highest=True)


def fit_collapse_weight_one_over_k(orig):
    return _fit_variant(collapse_weight_k=True)


def fit_floor_at_lambda(orig):
    return _fit_variant(floor_at_lambda=True)


CASES = {
    "log_r drops the log-determinant": (pcngm, "log_r", log_r_without_logdet,
                                        [t_pcngm.test_ratio_equals_theorem2_block_gaussian_densities,
                                         t_pcngm.test_beta_one_is_independence_sampler_ratio]),
    "proposal shifts by gamma m_j": (pcngm, "propose", propose_shift_gamma,
                                     [t_pcngm.test_proposal_mean_and_components]),
    "full-covariance proposal scales by C_j": (pcngm, "propose", propose_full_with_covariance,
                                               [t_full.test_diagonal_covariance_is_the_diagonal_kernel]),
    "ESS without the square": (smc, "ess_of_h", ess_without_square,
                               [t_smc.test_ess_limits_and_monotonicity, t_smc.test_bisection_brackets_target]),
    "log Z increment without -log N": (smc, "log_z_increment", log_z_without_mean,
                                       [t_smc.test_log_z_increment_direct_sum]),
    "resampling walk off by one": (smc, "systematic_indices", systematic_strict_walk,
                                   [t_smc.test_systematic_resampling_brute_force,
                                    t_smc.test_equal_weights_identity_and_extremes]),
    "arithmetic instead of harmonic faces": (darcy, "face_coefficients", arithmetic_faces,
                                             [t_darcy.test_assembled_operator_matches_flux_definition,
                                              t_adj.test_face_derivatives_against_central_differences]),
    "observation with x and y swapped": (observe, "observe_2d", observe_transposed,
                                         [t_obs.test_cell_centre_points_select_exactly,
                                          t_obs.test_bilinear_reproduces_affine_fields_inside]),
    "prior eigenvalues to the first power": (prior, "eigenvalues_2d", eigenvalues_first_power,
                                             [t_prior.test_cosine_modes_are_neumann_laplacian_eigenfunctions]),
    "adjoint gradient drops the wall faces": (adjoint, "grad_u_from_adjoint", gradient_without_walls,
                                              [t_adj.test_grid_gradient_matches_finite_differences_per_cell]),
    "E-step without the Gaussian normaliser": (gm, "e_step", e_step_without_normaliser,
                                               [t_gm.test_recovers_separated_mixture_and_loglik_monotone]),
    "Langevin ratio with the drift term's sign flipped": (langevin, "rho", rho_sign_flipped,
                                                          [lambda: t_lang.test_detailed_balance_direct_densities(0.3, 0.2)]),
    "Langevin drift without the temperature": (langevin, "propose", langevin_drift_without_t,
                                               [t_lang.test_propose_is_mean_plus_scaled_noise]),
    "potential without the 1/2": (observe, "potential", potential_without_half, [t_obs.test_potential]),
    "cosine basis without sqrt 2": (prior, "cosine_basis_1d", cosine_basis_without_sqrt2,
                                    [t_prior.test_basis_orthonormal_on_cell_centres,
                                     t_prior.test_synthesis_against_pointwise_sum]),
    "analysis with the grid transposed": (adjoint, "analysis_2d", analysis_transposed,
                                          [t_adj.test_analysis_is_transpose_of_synthesis]),
    "accept test inverted": (pcngm, "accept", accept_comparison_flipped,
                             [t_pcngm.test_accept_with_probability_min_one_alpha]),
    "beta rule thresholds swapped": (smc, "beta_rule", beta_rule_thresholds_swapped, [t_smc.test_beta_rule_table]),
    "Darcy solve without the h^2 scaling": (darcy, "solve_2d", solve_without_h2,
                                            [t_darcy.test_manufactured_solution_second_order]),
    "posterior variance with divisor N - 1": (smc, "posterior_moments", sample_variance,
                                              [t_smc.test_posterior_moments_closed_form]),
    "component draw closed on the right": (pcngm, "choose_component", component_draw_closed_on_the_right,
                                           [t_pcngm.test_component_draw_at_the_cumulative_boundaries]),
    "EM initial particles may repeat": (gm, "init_indices", init_indices_with_repeats,
                                        [t_gm.test_init_indices_distinct]),
    "bisection returns the upper bracket": (smc, "bisect_h", bisection_returns_upper_bracket,
                                            [t_smc.test_bisection_brackets_target]),
    "prior draw without sqrt(lambda)": (smc, "prior_draw", prior_draw_without_sqrt,
                                        [t_smc.test_prior_draws_have_the_prior_moments]),
    "1D solve without the h^2 scaling": (darcy, "solve_1d", solve_1d_without_h2,
                                         [t_darcy.test_manufactured_solution_1d_second_order]),
    "1D synthesis at the nodes instead of the midpoints": (prior, "sine_basis_midpoints", sine_basis_at_nodes,
                                                           [t_prior.test_synthesis_1d_against_pointwise_sum]),
    "1D observation half a cell off": (observe, "observe_1d", observe_1d_shifted, [t_obs.test_linear_1d]),
    "GM-Langevin noise with the prior variances": (langevin, "gm_propose", gm_propose_prior_noise,
                                                   [t_lang.test_gm_propose_is_component_mean_plus_scaled_noise]),
    "Box-Muller angle pi instead of 2 pi": (philox, "normal_pairs", box_muller_half_angle,
                                            [t_philox.test_normals_distribution]),
    "observation matrix with the grid transposed": (adjoint, "observation_matrix_2d", observation_matrix_transposed,
                                                    [t_adj.test_observation_matrix_matches_operator]),
    "full-covariance E-step with the log-determinant's sign flipped": (gm, "e_step_full", full_e_step_logdet_sign,
                                                                       [t_full.test_full_e_step_against_scipy_densities]),
    "MH ratio with the potential difference reversed": (pcngm, "log_alpha", mh_potential_sign,
                                                        [t_pcngm.test_log_alpha_is_detailed_balance_for_the_tempered_target]),
    "Langevin ratio without the temperature on Phi": (langevin, "log_alpha", langevin_alpha_without_t,
                                                      [lambda: t_lang.test_detailed_balance_direct_densities(0.3, 0.2)]),
    "GM-Langevin ratio without the pCN base density": (langevin, "gm_log_R", gm_log_R_without_base,
                                                       [lambda: t_lang.test_gm_detailed_balance_direct_densities(0.3, 0.2),
                                                        t_lang.test_gm_special_cases]),
    "fixed-point CDF rounds up": (smc, "fixed_point_cdf", cdf_ceil,
                                  [t_smc.test_fixed_point_cdf_hand_computed]),
    "fixed-point remainder on the smallest weight": (smc, "fixed_point_cdf", cdf_remainder_to_smallest,
                                                     [t_smc.test_fixed_point_cdf_hand_computed]),
    "fixed-point remainder on the last of equal largest weights": (smc, "fixed_point_cdf", cdf_ties_to_highest_index,
                                                                   [t_smc.test_fixed_point_cdf_hand_computed]),
    "EM collapse re-seeds at the highest max-responsibility": (gm, "fit", fit_reseed_at_highest,
                                                               [t_gm.test_collapse_reseeds_at_lowest_max_responsibility]),
    "EM collapse weight 1/K instead of 1/N": (gm, "fit", fit_collapse_weight_one_over_k,
                                              [t_gm.test_collapse_reseeds_at_lowest_max_responsibility]),
    "EM variance floor at lambda instead of 1e-3 lambda": (gm, "fit", fit_floor_at_lambda,
                                                           [t_gm.test_variance_floor_binds_on_a_constant_coordinate]),
}


@pytest.mark.parametrize("case", list(CASES))
def test_a_pin_catches_the_planted_mistake(case, monkeypatch):
    module, name, plant, pins = CASES[case]
    monkeypatch.setattr(module, name, plant(getattr(module, name)))
    caught = []
    for pin in pins:
        try:
            pin()
        except AssertionError:
            caught.append(getattr(pin, "__name__", "pin"))
    assert caught, "no pin caught: %s" % case


def test_the_pins_pass_on_the_unmodified_oracle():
    for case, (_, _, _, pins) in CASES.items():
        for pin in pins:
            pin()
