// pCN-GM mutation (Sec. 2.3, Alg. 2): component draw, Gaussian noise in KL
// coordinates, the proposal v = gamma u + (1 - gamma) m_j + beta sqrt(lambda_j) z
// (eq. pCN-GM proposal, per-component shift as in Thm 2), the mixture
// log-ratio terms of the acceptance ratio (eqs. auv of pCN-GMM..GMM4 in the
// prior-relative form) and the Metropolis-Hastings accept step; also the
// initial prior draws of Alg. 1.
//
// log r_j(b|a) = sum_{s in S} [ 1/2 log(lambda_s / lambda_js)
//                              - (e_s - (1-gamma) m_js)^2 / (2 beta^2 lambda_js)
//                              + e_s^2 / (2 beta^2 lambda_s) ],   e = b - gamma a,
// and log alpha = t (Phi(u) - Phi(v)) + LSE_j(log w_j + log r_j(u|v))
//                                     - LSE_j(log w_j + log r_j(v|u)).
#include "smcgm_internal.cuh"
#include "common.cuh"
#include "dfnormal.cuh"

namespace smcgm {

// Box-Muller pair m of the stream (c1, c2, purpose): U1 from words 0-1, U2 from
// words 2-3; z0 = R cos(2 pi U2), z1 = R sin(2 pi U2), R = sqrt(-2 log U1).
__device__ inline void normal_pair(uint32_t m, uint32_t c1, uint32_t c2, uint32_t purpose, Key k, double& z0, double& z1) {
    U4 w = philox(m, c1, c2, purpose, k.k0, k.k1);
    const double u1 = open53(w.x, w.y), u2 = open53(w.z, w.w);
    const double R = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z0 = R * c;
    z1 = R * s;
}

// The same pair with the logarithm and sin/cos in df32 (see dfnormal.cuh):
// agrees with normal_pair to ~1e-14 relative and keeps the proposal kernel off
// the FP64 pipe.  `tab` is the logarithm table in shared memory.
__device__ inline void normal_pair_df(uint32_t m, uint32_t c1, uint32_t c2, uint32_t purpose, Key k, const float2* tab,
                                      const NormalConsts& C, double& z0, double& z1) {
    U4 w = philox(m, c1, c2, purpose, k.k0, k.k1);
    const unsigned long long a = ((unsigned long long)(w.x >> 5) << 26) | (unsigned long long)(w.y >> 6);
    const unsigned long long b = ((unsigned long long)(w.z >> 5) << 26) | (unsigned long long)(w.w >> 6);
    const df32 lg = df_log_u54(a, tab, C);                      // log U1, U1 = (2a + 1) 2^-54
    const df32 R = df_sqrt(df32{-2.f * lg.hi, -2.f * lg.lo});
    df32 sn, cs;
    df_sincospi_u53(b, C, sn, cs);                              // of pi t, t = 2 U2 = (2b + 1) 2^-53
    const df32 r0 = df_mul(R, cs), r1 = df_mul(R, sn);
    z0 = (double)r0.hi + (double)r0.lo;
    z1 = (double)r1.hi + (double)r1.lo;
}

__global__ void k_prior_draw(int d, const double* __restrict__ sqrtlam, double* __restrict__ X, uint32_t c2, uint32_t purpose,
                             Key key) {
    const int p = blockIdx.x;
    double* x = X + (size_t)p * d;
    for (int m = threadIdx.x; m < d / 2; m += blockDim.x) {
        double z0, z1;
        normal_pair((uint32_t)m, (uint32_t)p, c2, purpose, key, z0, z1);
        x[2 * m] = sqrtlam[2 * m] * z0;
        x[2 * m + 1] = sqrtlam[2 * m + 1] * z1;
    }
    if ((d & 1) && threadIdx.x == 0) {
        double z0, z1;
        normal_pair((uint32_t)(d / 2), (uint32_t)p, c2, purpose, key, z0, z1);
        x[d - 1] = sqrtlam[d - 1] * z0;
    }
}

void launch_prior_draw(Ctx& c, double* X, int N, uint32_t counter2, uint32_t purpose) {
    k_prior_draw<<<N, 256, 0, c.stream>>>(c.d, c.sqrtlam, X, counter2, purpose, c.key); ++c.pc.launches;
    check(cudaGetLastError(), "prior draw");
}

// Proposal tables for the current beta.  Layout of `tab`:
//   [0, K r)       c0_js = 1/2 log(lambda_s / lambda_js)
//   [K r, 2K r)    a_js  = 1 / (2 beta^2 lambda_js)
//   [2K r, 3K r)   mu_js = (1 - gamma) m_js
//   [3K r, 4K r)   sq_js = beta sqrt(lambda_js)
//   [4K r, 4K r + r)         b_s = 1 / (2 beta^2 lambda_s)
//   [.. + r, .. + r + K)     log w_j
//   [.. + r + K, .. + r + 2K) cumulative w (sequential sum in index order)
__global__ void k_move_tables(int K, int r, const double* __restrict__ w, const double* __restrict__ m,
                              const double* __restrict__ lamj, const double* __restrict__ lam, const int* __restrict__ S,
                              double beta, double gamma, double* __restrict__ tab, const MoveSched* __restrict__ ms) {
    if (ms) { beta = ms->beta; gamma = ms->gamma; }
    const int Kr = K * r;
    for (int t = threadIdx.x; t < Kr; t += blockDim.x) {
        const int s = t % r;
        const double l0 = lam[S[s]], lj = lamj[t];
        tab[t] = 0.5 * log(l0 / lj);
        tab[Kr + t] = 1.0 / (2.0 * beta * beta * lj);
        tab[2 * Kr + t] = (1.0 - gamma) * m[t];
        tab[3 * Kr + t] = beta * sqrt(lj);
    }
    for (int s = threadIdx.x; s < r; s += blockDim.x) tab[4 * Kr + s] = 1.0 / (2.0 * beta * beta * lam[S[s]]);
    if (threadIdx.x == 0) {
        double cum = 0.0;
        for (int j = 0; j < K; ++j) {
            tab[4 * Kr + r + j] = log(w[j]);
            cum += w[j];
            tab[4 * Kr + r + K + j] = cum;
        }
    }
}

void launch_move_tables(Ctx& c, const MoveSched* ms) {
    const double gamma = sqrt(1.0 - c.beta * c.beta);
    k_move_tables<<<1, 256, 0, c.stream>>>(c.K, c.r, c.gw, c.gmu, c.glam, c.lam, c.S, c.beta, gamma, c.tab, ms); ++c.pc.launches;
    check(cudaGetLastError(), "move tables");
}

// One block per particle: v, then the 2K log-ratio terms.  With a gradient
// G (GMpCN-Langevin) v also takes the drift -(1 - gamma) t C_j G (kt =
// (1 - gamma) t) and the terms are left to k_gmpcnl_terms, which needs DPhi(v).
__global__ void __launch_bounds__(256) k_propose(int d, int K, int r, const double* __restrict__ X, double* __restrict__ V,
                                                 const double* __restrict__ sqrtlam, const int* __restrict__ slot,
                                                 const int* __restrict__ S, const double* __restrict__ tab, double beta, double gamma,
                                                 uint32_t step, Key key, double* __restrict__ lfwd, double* __restrict__ lrev,
                                                 const float2* __restrict__ ntab, NormalConsts nc, const double* __restrict__ G,
                                                 const double* __restrict__ lam, const double* __restrict__ glam, double kt,
                                                 const MoveSched* __restrict__ ms) {
    if (ms) { beta = ms->beta; gamma = ms->gamma; step += ms->step; }
    __shared__ int s_j;
    __shared__ float2 tab_s[NORMAL_TAB];
    for (int i = threadIdx.x; i < NORMAL_TAB; i += blockDim.x) tab_s[i] = ntab[i];
    const int p = blockIdx.x;
    const int Kr = K * r;
    const double* cumw = tab + 4 * Kr + r + K;
    if (threadIdx.x == 0) {
        U4 wc = philox(0u, (uint32_t)p, step, P_COMP, key.k0, key.k1);
        const double U = open53(wc.x, wc.y);
        int j = K - 1;
        for (int q = 0; q < K; ++q)
            if (U < cumw[q]) { j = q; break; }
        s_j = j;
    }
    __syncthreads();
    const int j = s_j;
    const double* u = X + (size_t)p * d;
    double* v = V + (size_t)p * d;
    const double* mu = tab + 2 * Kr + (size_t)j * r;
    const double* sq = tab + 3 * Kr + (size_t)j * r;
    for (int m = threadIdx.x; m < (d + 1) / 2; m += blockDim.x) {
        double z[2];
        normal_pair_df((uint32_t)m, (uint32_t)p, step, P_NORMAL, key, tab_s, nc, z[0], z[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int cidx = 2 * m + h;
            if (cidx >= d) break;
            const int sl = slot[cidx];
            const double gu = gamma * u[cidx];
            double vv = sl < 0 ? gu + (beta * sqrtlam[cidx]) * z[h] : (gu + mu[sl]) + sq[sl] * z[h];
            if (G) vv -= kt * (sl < 0 ? lam[cidx] : glam[(size_t)j * r + sl]) * G[(size_t)p * d + cidx];
            v[cidx] = vv;
        }
    }
    if (G) return;
    __syncthreads();
    // log-ratio terms: warp w handles components j = w, w + nwarps, ...
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const double* c0 = tab;
    const double* aa = tab + Kr;
    const double* mm = tab + 2 * Kr;
    const double* bb = tab + 4 * Kr;
    for (int jj = warp; jj < K; jj += nw) {
        double f = 0.0, rv = 0.0;
        for (int s = lane; s < r; s += 32) {
            const int cidx = S[s];
            const double ef = v[cidx] - gamma * u[cidx];
            const double er = u[cidx] - gamma * v[cidx];
            const int ti = jj * r + s;
            const double df = ef - mm[ti], dr = er - mm[ti];
            f += c0[ti] - df * df * aa[ti] + ef * ef * bb[s];
            rv += c0[ti] - dr * dr * aa[ti] + er * er * bb[s];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            f += __shfl_down_sync(0xffffffffu, f, o);
            rv += __shfl_down_sync(0xffffffffu, rv, o);
        }
        if (lane == 0) {
            lfwd[(size_t)p * K + jj] = f;
            lrev[(size_t)p * K + jj] = rv;
        }
    }
}

void launch_propose(Ctx& c, const MoveSched* ms, uint32_t step_off) {
    const double gamma = sqrt(1.0 - c.beta * c.beta);
    const bool drift = c.cfg.kernel == SMC_K_GMPCNL;
    k_propose<<<c.N, 256, 0, c.stream>>>(c.d, c.K, c.r, c.X, c.V, c.sqrtlam, c.slot, c.S, c.tab, c.beta, gamma,
                                         ms ? step_off : c.step, c.key, c.lfwd, c.lrev, reinterpret_cast<const float2*>(c.normtab),
                                         c.normc, drift ? c.G : nullptr, c.lam, c.glam, (1.0 - gamma) * c.t, ms); ++c.pc.launches;
    check(cudaGetLastError(), "propose");
}

// Full covariances on the mixture modes: one block per particle.  The drawn
// component j gives v_S = gamma u_S + (1-gamma) m_j + beta L_j z_S (z_S the
// same normals the diagonal proposal uses on S), the other modes the pCN move;
// then for every component
//   log r_j(b|a) = 1/2 sum_s log lambda_s - log det L_j - |L_j^{-1}(e - (1-gamma) m_j)|^2 / (2 beta^2)
//                  + sum_s e_s^2 / (2 beta^2 lambda_s),   e = b_S - gamma a_S.
__global__ void __launch_bounds__(256) k_propose_full(int d, int K, int r, const double* __restrict__ X, double* __restrict__ V,
                                                      const double* __restrict__ sqrtlam, const double* __restrict__ lam,
                                                      const int* __restrict__ slot, const int* __restrict__ S,
                                                      const double* __restrict__ tab, const double* __restrict__ L,
                                                      const double* __restrict__ Li, const double* __restrict__ logdet,
                                                      double beta, double gamma, uint32_t step, Key key, double* __restrict__ lfwd,
                                                      double* __restrict__ lrev, const float2* __restrict__ ntab, NormalConsts nc,
                                                      const MoveSched* __restrict__ ms) {
    if (ms) { beta = ms->beta; gamma = ms->gamma; step += ms->step; }
    __shared__ int s_j;
    __shared__ float2 tab_s[NORMAL_TAB];
    __shared__ double zS[MAXR], ef[MAXR], er[MAXR];
    __shared__ double red[32];
    __shared__ double s_c;
    for (int i = threadIdx.x; i < NORMAL_TAB; i += blockDim.x) tab_s[i] = ntab[i];
    const int p = blockIdx.x;
    const int Kr = K * r;
    const double* cumw = tab + 4 * Kr + r + K;
    if (threadIdx.x == 0) {
        U4 wc = philox(0u, (uint32_t)p, step, P_COMP, key.k0, key.k1);
        const double U = open53(wc.x, wc.y);
        int j = K - 1;
        for (int q = 0; q < K; ++q)
            if (U < cumw[q]) { j = q; break; }
        s_j = j;
    }
    __syncthreads();
    const int j = s_j;
    const double* u = X + (size_t)p * d;
    double* v = V + (size_t)p * d;
    const double* mu = tab + 2 * Kr;                  // (1 - gamma) m
    for (int m = threadIdx.x; m < (d + 1) / 2; m += blockDim.x) {
        double z[2];
        normal_pair_df((uint32_t)m, (uint32_t)p, step, P_NORMAL, key, tab_s, nc, z[0], z[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int cidx = 2 * m + h;
            if (cidx >= d) break;
            const int sl = slot[cidx];
            if (sl < 0) v[cidx] = gamma * u[cidx] + (beta * sqrtlam[cidx]) * z[h];
            else zS[sl] = z[h];
        }
    }
    __syncthreads();
    const double* Lj = L + (size_t)j * r * r;
    for (int s = threadIdx.x; s < r; s += blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k <= s; ++k) acc += Lj[(size_t)s * r + k] * zS[k];
        const int cidx = S[s];
        v[cidx] = (gamma * u[cidx] + mu[(size_t)j * r + s]) + beta * acc;
    }
    __syncthreads();
    double c0 = 0.0;
    for (int s = threadIdx.x; s < r; s += blockDim.x) {
        const int cidx = S[s];
        ef[s] = v[cidx] - gamma * u[cidx];
        er[s] = u[cidx] - gamma * v[cidx];
        const double l = lam[cidx];
        c0 += 0.5 * log(l);
    }
    c0 = block_sum(c0, red);
    if (threadIdx.x == 0) s_c = c0;
    __syncthreads();
    const double ib2 = 1.0 / (beta * beta);
    for (int jj = 0; jj < K; ++jj) {
        const double* Lij = Li + (size_t)jj * r * r;
        const double* muj = mu + (size_t)jj * r;
        double qf = 0.0, qr = 0.0, pf = 0.0, pr = 0.0;
        for (int i = threadIdx.x; i < r; i += blockDim.x) {
            double yf = 0.0, yr = 0.0;
            for (int k = 0; k <= i; ++k) {
                const double lik = Lij[(size_t)i * r + k];
                yf += lik * (ef[k] - muj[k]);
                yr += lik * (er[k] - muj[k]);
            }
            qf += yf * yf;
            qr += yr * yr;
            const double l = lam[S[i]];
            pf += ef[i] * ef[i] / l;
            pr += er[i] * er[i] / l;
        }
        qf = block_sum(qf, red);
        qr = block_sum(qr, red);
        pf = block_sum(pf, red);
        pr = block_sum(pr, red);
        if (threadIdx.x == 0) {
            lfwd[(size_t)p * K + jj] = s_c - logdet[jj] - 0.5 * qf * ib2 + 0.5 * pf * ib2;
            lrev[(size_t)p * K + jj] = s_c - logdet[jj] - 0.5 * qr * ib2 + 0.5 * pr * ib2;
        }
    }
}

void launch_propose_full(Ctx& c, const MoveSched* ms, uint32_t step_off) {
    const double gamma = sqrt(1.0 - c.beta * c.beta);
    k_propose_full<<<c.N, 256, 0, c.stream>>>(c.d, c.K, c.r, c.X, c.V, c.sqrtlam, c.lam, c.slot, c.S, c.tab, c.gL, c.gLi, c.glogdet,
                                              c.beta, gamma, ms ? step_off : c.step, c.key, c.lfwd, c.lrev,
                                              reinterpret_cast<const float2*>(c.normtab), c.normc, ms); ++c.pc.launches;
    check(cudaGetLastError(), "propose full");
}

__device__ inline double lse_terms(const double* lw, const double* l, int K) {
    double mx = -1.0 / 0.0;
    for (int j = 0; j < K; ++j) mx = fmax(mx, lw[j] + l[j]);
    double s = 0.0;
    for (int j = 0; j < K; ++j) s += exp(lw[j] + l[j] - mx);
    return mx + log(s);
}

// Metropolis-Hastings accept/reject and the conditional copy v -> u.
__global__ void __launch_bounds__(256) k_accept(int d, int K, int r, int kernel, double t, uint32_t step, Key key,
                                                const double* __restrict__ tab, const double* __restrict__ lfwd,
                                                const double* __restrict__ lrev, double* __restrict__ X, const double* __restrict__ V,
                                                double* __restrict__ Phi, const double* __restrict__ PhiV,
                                                double* __restrict__ logalpha, unsigned char* __restrict__ acc, int* __restrict__ count,
                                                const MoveSched* __restrict__ ms) {
    if (ms) { t = ms->t; step += ms->step; }
    __shared__ int s_acc;
    const int p = blockIdx.x;
    if (threadIdx.x == 0) {
        const double* lw = tab + 4 * K * r + r;
        double la;
        int a;
        if (kernel == SMC_K_GM_INDEP) {
            // Alg. 3 takes every proposal, except one whose potential could not be
            // evaluated (a field outside the mixed-precision range gets +inf)
            a = isfinite(PhiV[p]) ? 1 : 0;
            la = a ? 0.0 : -INFINITY;
        } else {
            const double ratio = lse_terms(lw, lrev + (size_t)p * K, K) - lse_terms(lw, lfwd + (size_t)p * K, K);
            la = t * (Phi[p] - PhiV[p]) + ratio;
            U4 wa = philox(0u, (uint32_t)p, step, P_ACCEPT, key.k0, key.k1);
            const double U = open53(wa.x, wa.y);
            a = (la >= 0.0 || log(U) < la) ? 1 : 0;
        }
        logalpha[p] = la;
        acc[p] = (unsigned char)a;
        if (a) {
            Phi[p] = PhiV[p];
            atomicAdd(count, 1);
        }
        s_acc = a;
    }
    __syncthreads();
    if (s_acc) {
        const double2* src = reinterpret_cast<const double2*>(V + (size_t)p * d);
        double2* dst = reinterpret_cast<double2*>(X + (size_t)p * d);
        for (int i = threadIdx.x; i < d / 2; i += blockDim.x) dst[i] = src[i];
        if ((d & 1) && threadIdx.x == 0) X[(size_t)p * d + d - 1] = V[(size_t)p * d + d - 1];
    }
}

void launch_accept(Ctx& c, int* acc_count, const MoveSched* ms, uint32_t step_off) {
    k_accept<<<c.N, 256, 0, c.stream>>>(c.d, c.K, c.r, c.cfg.kernel, c.t, ms ? step_off : c.step, c.key, c.tab, c.lfwd, c.lrev, c.X,
                                        c.V, c.Phi, c.PhiV, c.logalpha, c.acc, acc_count, ms); ++c.pc.launches;
    check(cudaGetLastError(), "accept");
}

// ------------------------------------------------------------------------
// pCN-Langevin mutation (App. B's Langevin equation with its drift kept for
// the tempered target exp(-t Phi) mu0; Crank-Nicolson in the linear part,
// explicit drift):
//   v = gamma u - (1 - gamma) t C g_u + beta C^{1/2} z,   g = DPhi, C = diag(lambda),
//   log alpha = t (Phi(u) - Phi(v)) + rho(v, u) - rho(u, v),
//   rho(a, b) = -(1 - gamma) t <g_a, b - gamma a> / beta^2
//               - (1 - gamma)^2 t^2 <g_a, C g_a> / (2 beta^2).
// The normals and the accept uniform are those of the pCN-GM move.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_propose_pcnl(int d, const double* __restrict__ X, const double* __restrict__ G,
                                                      double* __restrict__ V, const double* __restrict__ lam,
                                                      const double* __restrict__ sqrtlam, double beta, double gamma, double kt,
                                                      uint32_t step, Key key, const float2* __restrict__ ntab, NormalConsts nc) {
    __shared__ float2 tab_s[NORMAL_TAB];
    for (int i = threadIdx.x; i < NORMAL_TAB; i += blockDim.x) tab_s[i] = ntab[i];
    __syncthreads();
    const int p = blockIdx.x;
    const double* u = X + (size_t)p * d;
    const double* g = G + (size_t)p * d;
    double* v = V + (size_t)p * d;
    for (int m = threadIdx.x; m < (d + 1) / 2; m += blockDim.x) {
        double z[2];
        normal_pair_df((uint32_t)m, (uint32_t)p, step, P_NORMAL, key, tab_s, nc, z[0], z[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = 2 * m + h;
            if (i >= d) break;
            v[i] = (gamma * u[i] - kt * lam[i] * g[i]) + (beta * sqrtlam[i]) * z[h];
        }
    }
}

// Accept/reject of the pCN-Langevin step, one block per particle: the four
// inner products of rho by a block reduction in a fixed order, then the same
// accept rule as k_accept and the copies v -> u, g_v -> g_u, Phi_v -> Phi.
__global__ void __launch_bounds__(256) k_accept_pcnl(int d, const double* __restrict__ lam, double t, double beta, double gamma,
                                                     uint32_t step, Key key, double* __restrict__ X, const double* __restrict__ V,
                                                     double* __restrict__ G, const double* __restrict__ GV,
                                                     double* __restrict__ Phi, const double* __restrict__ PhiV,
                                                     double* __restrict__ logalpha, unsigned char* __restrict__ acc,
                                                     int* __restrict__ count) {
    __shared__ double red[32];
    __shared__ int s_acc;
    const int p = blockIdx.x;
    const double* u = X + (size_t)p * d;
    const double* v = V + (size_t)p * d;
    const double* gu = G + (size_t)p * d;
    const double* gv = GV + (size_t)p * d;
    double a = 0.0, b = 0.0, c = 0.0, e = 0.0;   // <g_u, v - gamma u>, <g_u, C g_u>, <g_v, u - gamma v>, <g_v, C g_v>
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        a += gu[i] * (v[i] - gamma * u[i]);
        b += gu[i] * lam[i] * gu[i];
        c += gv[i] * (u[i] - gamma * v[i]);
        e += gv[i] * lam[i] * gv[i];
    }
    a = block_sum(a, red);
    b = block_sum(b, red);
    c = block_sum(c, red);
    e = block_sum(e, red);
    if (threadIdx.x == 0) {
        const double k = (1.0 - gamma) * t, ib2 = 1.0 / (beta * beta);
        const double rho_uv = -k * a * ib2 - 0.5 * k * k * b * ib2;
        const double rho_vu = -k * c * ib2 - 0.5 * k * k * e * ib2;
        const double la = t * (Phi[p] - PhiV[p]) + rho_vu - rho_uv;
        U4 wa = philox(0u, (uint32_t)p, step, P_ACCEPT, key.k0, key.k1);
        const double U = open53(wa.x, wa.y);
        const int ok = (la >= 0.0 || log(U) < la) ? 1 : 0;
        logalpha[p] = la;
        acc[p] = (unsigned char)ok;
        if (ok) {
            Phi[p] = PhiV[p];
            atomicAdd(count, 1);
        }
        s_acc = ok;
    }
    __syncthreads();
    if (s_acc) {
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            X[(size_t)p * d + i] = v[i];
            G[(size_t)p * d + i] = gv[i];
        }
    }
}

// GMpCN-Langevin acceptance terms, one block per particle, after DPhi(v):
//   lfwd_j = log R_j(u, v), lrev_j = log R_j(v, u),
//   log R_j(a, b) = sum_{s in S} [ 1/2 log(lambda_s / lambda_js)
//                                  - (e_s - (1-gamma) m_js + kt lambda_js g_a,s)^2 / (2 beta^2 lambda_js)
//                                  + e_s^2 / (2 beta^2 lambda_s) ]
//                 + sum_{i not in S} [ -kt e_i g_a,i - kt^2 lambda_i g_a,i^2 / 2 ] / beta^2,
// e = b - gamma a, kt = (1 - gamma) t; the sum outside S is the same for every
// component (there C_j = C and m_j = 0) and is added to each term.
__global__ void __launch_bounds__(256) k_gmpcnl_terms(int d, int K, int r, const double* __restrict__ X,
                                                      const double* __restrict__ V, const double* __restrict__ G,
                                                      const double* __restrict__ GV, const double* __restrict__ lam,
                                                      const double* __restrict__ glam, const int* __restrict__ slot,
                                                      const int* __restrict__ S, const double* __restrict__ tab, double beta,
                                                      double gamma, double kt, double* __restrict__ lfwd, double* __restrict__ lrev) {
    __shared__ double red[32];
    __shared__ double s_tail[2];
    const int p = blockIdx.x;
    const int Kr = K * r;
    const double* u = X + (size_t)p * d;
    const double* v = V + (size_t)p * d;
    const double* gu = G + (size_t)p * d;
    const double* gv = GV + (size_t)p * d;
    const double ib2 = 1.0 / (beta * beta);
    double tf = 0.0, tr = 0.0;
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        if (slot[i] >= 0) continue;
        const double ef = v[i] - gamma * u[i], er = u[i] - gamma * v[i];
        tf += -kt * ef * gu[i] - 0.5 * kt * kt * lam[i] * gu[i] * gu[i];
        tr += -kt * er * gv[i] - 0.5 * kt * kt * lam[i] * gv[i] * gv[i];
    }
    tf = block_sum(tf, red);
    tr = block_sum(tr, red);
    if (threadIdx.x == 0) {
        s_tail[0] = tf * ib2;
        s_tail[1] = tr * ib2;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const double* c0 = tab;
    const double* aa = tab + Kr;
    const double* mm = tab + 2 * Kr;
    const double* bb = tab + 4 * Kr;
    for (int jj = warp; jj < K; jj += nw) {
        double f = 0.0, rv = 0.0;
        for (int s2 = lane; s2 < r; s2 += 32) {
            const int cidx = S[s2];
            const int ti = jj * r + s2;
            const double lj = glam[ti];
            const double ef = v[cidx] - gamma * u[cidx];
            const double er = u[cidx] - gamma * v[cidx];
            const double df = ef - mm[ti] + kt * lj * gu[cidx], dr = er - mm[ti] + kt * lj * gv[cidx];
            f += c0[ti] - df * df * aa[ti] + ef * ef * bb[s2];
            rv += c0[ti] - dr * dr * aa[ti] + er * er * bb[s2];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            f += __shfl_down_sync(0xffffffffu, f, o);
            rv += __shfl_down_sync(0xffffffffu, rv, o);
        }
        if (lane == 0) {
            lfwd[(size_t)p * K + jj] = f + s_tail[0];
            lrev[(size_t)p * K + jj] = rv + s_tail[1];
        }
    }
}

// G_u <- G_v for the accepted particles (after k_accept).
__global__ void __launch_bounds__(256) k_copy_accepted(int d, const unsigned char* __restrict__ acc, const double* __restrict__ GV,
                                                       double* __restrict__ G) {
    const int p = blockIdx.x;
    if (!acc[p]) return;
    for (int i = threadIdx.x; i < d; i += blockDim.x) G[(size_t)p * d + i] = GV[(size_t)p * d + i];
}

void launch_gmpcnl_terms(Ctx& c) {
    const double gamma = sqrt(1.0 - c.beta * c.beta);
    k_gmpcnl_terms<<<c.N, 256, 0, c.stream>>>(c.d, c.K, c.r, c.X, c.V, c.G, c.GV, c.lam, c.glam, c.slot, c.S, c.tab, c.beta, gamma,
                                              (1.0 - gamma) * c.t, c.lfwd, c.lrev); ++c.pc.launches;
    check(cudaGetLastError(), "gmpcnl terms");
}

void launch_copy_accepted_gradients(Ctx& c) {
    k_copy_accepted<<<c.N, 256, 0, c.stream>>>(c.d, c.acc, c.GV, c.G); ++c.pc.launches;
    check(cudaGetLastError(), "copy gradients");
}

void launch_propose_pcnl(Ctx& c) {
    const double gamma = sqrt(1.0 - c.beta * c.beta);
    k_propose_pcnl<<<c.N, 256, 0, c.stream>>>(c.d, c.X, c.G, c.V, c.lam, c.sqrtlam, c.beta, gamma, (1.0 - gamma) * c.t, c.step,
                                              c.key, reinterpret_cast<const float2*>(c.normtab), c.normc); ++c.pc.launches;
    check(cudaGetLastError(), "propose pcnl");
}

void launch_accept_pcnl(Ctx& c, int* acc_count) {
    const double gamma = sqrt(1.0 - c.beta * c.beta);
    k_accept_pcnl<<<c.N, 256, 0, c.stream>>>(c.d, c.lam, c.t, c.beta, gamma, c.step, c.key, c.X, c.V, c.G, c.GV, c.Phi, c.PhiV,
                                             c.logalpha, c.acc, acc_count); ++c.pc.launches;
    check(cudaGetLastError(), "accept pcnl");
}

}  // namespace smcgm
