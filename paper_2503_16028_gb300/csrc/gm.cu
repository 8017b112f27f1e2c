// Gaussian-mixture estimation of Alg. 3 / Sec. 2.4 ("estimate a Gaussian
// mixture by samples"; the paper delegates the estimator to Feng2018): EM for
// K diagonal Gaussians on the r leading KL coordinates S of the equally
// weighted particles, prior on every other coordinate.
//   E-step: log p_nj = log w_j + sum_s [-1/2 log(2 pi lambda_js) - (x_ns - m_js)^2 / (2 lambda_js)],
//           g_nj = exp(log p_nj - LSE_j), loglik = sum_n LSE_j.
//   M-step: N_j = sum_n g_nj, w_j = N_j / N, m_j = sum_n g_nj x_n / N_j,
//           lambda_js = max(sum_n g_nj (x_ns - m_js)^2 / N_j, floor * lambda_s).
//   A component with N_j < 2 is re-seeded at the particle with the lowest
//   max_j g_nj (pooled variances, w_j = 1/N); weights are renormalised.
// Initial means: K distinct particles from Philox (purpose EMINIT), variances
// the pooled population variance, w_j = 1/K.  A fixed number of iterations.
#include <cmath>
#include <vector>
#include "smcgm_internal.cuh"
#include "common.cuh"

namespace smcgm {

// xsT[s][n] = X[n][S[s]]
__global__ void k_gather_modes(int N, int d, int r, const double* __restrict__ X, const int* __restrict__ S, double* __restrict__ xsT) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)N * r) return;
    const int s = (int)(t / N), n = (int)(t % N);
    xsT[t] = X[(size_t)n * d + S[s]];
}

// pooled population variance per mode (block per s), floored.
__global__ void k_pooled(int N, int r, const double* __restrict__ xsT, const double* __restrict__ lamS, double floor_frac,
                         double* __restrict__ pooled) {
    __shared__ double red[32];
    __shared__ double s_m;
    const int s = blockIdx.x;
    const double* x = xsT + (size_t)s * N;
    double a = 0.0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) a += x[n];
    a = block_sum(a, red);
    if (threadIdx.x == 0) s_m = a / N;
    __syncthreads();
    double v = 0.0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) { const double e = x[n] - s_m; v += e * e; }
    v = block_sum(v, red);
    if (threadIdx.x == 0) pooled[s] = fmax(v / N, floor_frac * lamS[s]);
}

__global__ void k_em_init(int N, int K, int r, const int* __restrict__ init_idx, const double* __restrict__ xsT,
                          const double* __restrict__ pooled, double* __restrict__ w, double* __restrict__ m, double* __restrict__ lam) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < K * r) {
        const int j = t / r, s = t % r;
        m[t] = xsT[(size_t)s * N + init_idx[j]];
        lam[t] = pooled[s];
    }
    if (t < K) w[t] = 1.0 / K;
}

// E-step: one thread per particle.  resp[j][n], lse[n], gmax[n].
__global__ void __launch_bounds__(256) k_estep(int N, int K, int r, const double* __restrict__ xsT, const double* __restrict__ w,
                                               const double* __restrict__ m, const double* __restrict__ lam, double* __restrict__ resp,
                                               double* __restrict__ lse, double* __restrict__ gmax) {
    extern __shared__ double sh[];   // K*r means, K*r 1/(2 lam), K constants
    double* sm = sh;
    double* si = sm + K * r;
    double* sc = si + K * r;
    for (int t = threadIdx.x; t < K * r; t += blockDim.x) { sm[t] = m[t]; si[t] = 1.0 / (2.0 * lam[t]); }
    __syncthreads();
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        double c = log(w[j]);
        for (int s = 0; s < r; ++s) c += -0.5 * log(2.0 * M_PI * lam[j * r + s]);
        sc[j] = c;
    }
    __syncthreads();
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double lp[MAXK];
    for (int j = 0; j < K; ++j) lp[j] = 0.0;
    for (int s = 0; s < r; ++s) {
        const double x = xsT[(size_t)s * N + n];
        for (int j = 0; j < K; ++j) {
            const double e = x - sm[j * r + s];
            lp[j] -= e * e * si[j * r + s];
        }
    }
    double mx = -1.0 / 0.0;
    for (int j = 0; j < K; ++j) { lp[j] += sc[j]; mx = fmax(mx, lp[j]); }
    double sum = 0.0;
    for (int j = 0; j < K; ++j) sum += exp(lp[j] - mx);
    const double l = mx + log(sum);
    double gm = 0.0;
    for (int j = 0; j < K; ++j) {
        const double g = exp(lp[j] - l);
        resp[(size_t)j * N + n] = g;
        gm = fmax(gm, g);
    }
    lse[n] = l;
    gmax[n] = gm;
}

// M-step means (block per (j, s)): nj[j] and m[j][s].
__global__ void k_mstep_mean(int N, int r, const double* __restrict__ xsT, const double* __restrict__ resp, double* __restrict__ nj,
                             double* __restrict__ m) {
    __shared__ double red[32];
    __shared__ double s_n;
    const int j = blockIdx.x / r, s = blockIdx.x % r;
    const double* g = resp + (size_t)j * N;
    const double* x = xsT + (size_t)s * N;
    double a = 0.0, b = 0.0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) { a += g[n]; b += g[n] * x[n]; }
    a = block_sum(a, red);
    if (threadIdx.x == 0) s_n = a;
    __syncthreads();
    b = block_sum(b, red);
    if (threadIdx.x == 0) {
        m[j * r + s] = b / s_n;
        if (s == 0) nj[j] = s_n;
    }
}

__global__ void k_mstep_var(int N, int r, const double* __restrict__ xsT, const double* __restrict__ resp, const double* __restrict__ nj,
                            const double* __restrict__ m, const double* __restrict__ lamS, double floor_frac, double* __restrict__ lam) {
    __shared__ double red[32];
    const int j = blockIdx.x / r, s = blockIdx.x % r;
    const double* g = resp + (size_t)j * N;
    const double* x = xsT + (size_t)s * N;
    const double mu = m[j * r + s];
    double a = 0.0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) { const double e = x[n] - mu; a += g[n] * e * e; }
    a = block_sum(a, red);
    if (threadIdx.x == 0) lam[j * r + s] = fmax(a / nj[j], floor_frac * lamS[s]);
}

// Collapse handling and weights (single block).
__global__ void k_mstep_fix(int N, int K, int r, const double* __restrict__ nj, const double* __restrict__ gmax,
                            const double* __restrict__ xsT, const double* __restrict__ pooled, double* __restrict__ w,
                            double* __restrict__ m, double* __restrict__ lam) {
    __shared__ double s_v[1024];
    __shared__ int s_i[1024];
    __shared__ int s_star;
    bool any = false;
    for (int j = 0; j < K; ++j) any |= nj[j] < 2.0;
    if (any) {
        double best = 1.0 / 0.0;
        int bi = N;
        for (int n = threadIdx.x; n < N; n += blockDim.x)
            if (gmax[n] < best) { best = gmax[n]; bi = n; }
        s_v[threadIdx.x] = best;
        s_i[threadIdx.x] = bi;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = 1.0 / 0.0;
            int ib = N;
            for (int k = 0; k < (int)blockDim.x; ++k)
                if (s_v[k] < b || (s_v[k] == b && s_i[k] < ib)) { b = s_v[k]; ib = s_i[k]; }
            s_star = ib;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int j = 0; j < K; ++j) {
            if (nj[j] < 2.0) {
                for (int s = 0; s < r; ++s) { m[j * r + s] = xsT[(size_t)s * N + s_star]; lam[j * r + s] = pooled[s]; }
                w[j] = 1.0 / N;
            } else {
                w[j] = nj[j] / N;
            }
        }
        double tot = 0.0;
        for (int j = 0; j < K; ++j) tot += w[j];
        for (int j = 0; j < K; ++j) w[j] = w[j] / tot;
    }
}

__global__ void k_sum(int N, const double* __restrict__ a, double* __restrict__ out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) s += a[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) *out = s;
}

__global__ void k_lamS(int r, const double* __restrict__ lam, const int* __restrict__ S, double* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < r) out[s] = lam[S[s]];
}

// ------------------------------------------------------------------------
// Full covariances on the mixture modes (cfg.full_cov; a reading beyond the
// paper, whose C_j are diagonal in the KL basis):
//   E-step: log p_nj = log w_j - r/2 log(2 pi) - log det L_j - |L_j^{-1}(x_n - m_j)|^2 / 2,
//   M-step: C_j = sum_n g_nj (x_n - m_j)(x_n - m_j)^T / N_j + floor diag(lambda_S),
//   initial and re-seeded covariances diag(pooled variances).
// L_j (Cholesky), L_j^{-1} and log det L_j are formed on the device in FP64
// (k_factor, one block per component) after every M-step; a pivot that is not
// positive sets a device flag, read by the host once per fit.
// ------------------------------------------------------------------------

// E-step, one block per particle: for each j, y = L_j^{-1}(x_n - m_j) (a row per thread).
__global__ void __launch_bounds__(128) k_estep_full(int N, int K, int r, const double* __restrict__ xsT, const double* __restrict__ w,
                                                    const double* __restrict__ m, const double* __restrict__ Li,
                                                    const double* __restrict__ logdet, double* __restrict__ resp,
                                                    double* __restrict__ lse, double* __restrict__ gmax) {
    __shared__ double red[32];
    __shared__ double dev[MAXR];
    __shared__ double lp[MAXK];
    const int n = blockIdx.x;
    for (int j = 0; j < K; ++j) {
        for (int s = threadIdx.x; s < r; s += blockDim.x) dev[s] = xsT[(size_t)s * N + n] - m[(size_t)j * r + s];
        __syncthreads();
        double q = 0.0;
        const double* Lj = Li + (size_t)j * r * r;
        for (int i = threadIdx.x; i < r; i += blockDim.x) {
            double y = 0.0;
            for (int k = 0; k <= i; ++k) y += Lj[(size_t)i * r + k] * dev[k];
            q += y * y;
        }
        q = block_sum(q, red);
        if (threadIdx.x == 0) lp[j] = log(w[j]) - 0.5 * r * log(2.0 * M_PI) - logdet[j] - 0.5 * q;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double mx = -1.0 / 0.0;
        for (int j = 0; j < K; ++j) mx = fmax(mx, lp[j]);
        double sum = 0.0;
        for (int j = 0; j < K; ++j) sum += exp(lp[j] - mx);
        const double l = mx + log(sum);
        double gm = 0.0;
        for (int j = 0; j < K; ++j) {
            const double g = exp(lp[j] - l);
            resp[(size_t)j * N + n] = g;
            gm = fmax(gm, g);
        }
        lse[n] = l;
        gmax[n] = gm;
    }
}

// M-step covariances as a blocked SYRK: S_j = sum_n g_nj (x_n - m_j)(x_n - m_j)^T.
// The r x r output is cut into CT x CT tiles; a block computes one lower-triangle
// tile (ta >= tb) of one component over one of COV_NC chunks of the particles
// (FP64, 256 threads, 4 outputs each), staging CT particles x CT modes of the
// weighted deviations g (x_a - m_a) and of the deviations (x_b - m_b) in shared
// memory per step.  The chunk partials go to `part`; k_cov_reduce adds them in a
// fixed order (deterministic), divides by N_j, adds the ridge and writes both
// triangles.
constexpr int CT = 32;
constexpr int COV_NC = 8;
__host__ __device__ inline int cov_tiles(int r) { const int t = (r + CT - 1) / CT; return t * (t + 1) / 2; }

__global__ void __launch_bounds__(256) k_mstep_cov(int N, int r, const double* __restrict__ xsT, const double* __restrict__ resp,
                                                   const double* __restrict__ m, double* __restrict__ part) {
    __shared__ double Wa[CT][CT + 1];   // [particle][mode a]
    __shared__ double Db[CT][CT + 1];   // [particle][mode b]
    const int tile = blockIdx.x, j = blockIdx.y, chunk = blockIdx.z;
    int ta = 0, t = tile;
    while (t > ta) { t -= ta + 1; ++ta; }
    const int tb = t;                                   // tb <= ta
    const int a0 = ta * CT, b0 = tb * CT;
    const int per = (N + COV_NC - 1) / COV_NC;
    const int n_lo = chunk * per, n_hi = min(N, n_lo + per);
    const double* g = resp + (size_t)j * N;
    const int row = threadIdx.x / 8, col0 = (threadIdx.x % 8) * 4;   // outputs (a0 + row, b0 + col0 .. col0 + 3)
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int n0 = n_lo; n0 < n_hi; n0 += CT) {
        for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) {
            const int mode = e / CT, pn = e % CT;          // consecutive threads: consecutive particles
            const int n = n0 + pn;
            const bool in_n = n < n_hi;
            const int a = a0 + mode, b = b0 + mode;
            Wa[pn][mode] = (in_n && a < r) ? g[n] * (xsT[(size_t)a * N + n] - m[(size_t)j * r + a]) : 0.0;
            Db[pn][mode] = (in_n && b < r) ? xsT[(size_t)b * N + n] - m[(size_t)j * r + b] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int pn = 0; pn < CT; ++pn) {
            const double w = Wa[pn][row];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += w * Db[pn][col0 + q];
        }
        __syncthreads();
    }
    double* out = part + (((size_t)j * cov_tiles(r) + tile) * COV_NC + chunk) * CT * CT;
#pragma unroll
    for (int q = 0; q < 4; ++q) out[row * CT + col0 + q] = acc[q];
}

__global__ void k_cov_reduce(int r, const double* __restrict__ part, const double* __restrict__ nj, const double* __restrict__ lamS,
                             double floor_frac, double* __restrict__ cov) {
    const int tile = blockIdx.x, j = blockIdx.y;
    int ta = 0, t = tile;
    while (t > ta) { t -= ta + 1; ++ta; }
    const int tb = t;
    const double* p = part + ((size_t)j * cov_tiles(r) + tile) * COV_NC * CT * CT;
    for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) {
        const int a = ta * CT + e / CT, b = tb * CT + e % CT;
        if (a >= r || b >= r || b > a) continue;
        double s = 0.0;
        for (int k = 0; k < COV_NC; ++k) s += p[(size_t)k * CT * CT + e];
        const double v = s / nj[j] + (a == b ? floor_frac * lamS[a] : 0.0);
        cov[((size_t)j * r + a) * r + b] = v;
        cov[((size_t)j * r + b) * r + a] = v;
    }
}

size_t cov_partial_doubles(int K, int r) { return (size_t)K * cov_tiles(r) * COV_NC * CT * CT; }

// Cholesky factor L_j (lower), L_j^{-1} and log det L_j of every C_j, one block per
// component, FP64, in the order of the Cholesky-Banachiewicz recurrence
//   L_kk = sqrt(C_kk - sum_{q<k} L_kq^2),  L_ik = (C_ik - sum_{q<k} L_iq L_kq) / L_kk,
// a column at a time (its entries below the diagonal are independent given the earlier
// columns: a row per thread); then L^{-1} by forward substitution on the unit vectors (a
// column per thread) and log det L_j = sum_k log L_kk.  A pivot that is not positive (C_j
// not positive definite) sets *bad and is replaced by 1 so the rest stays finite.
__global__ void __launch_bounds__(256) k_factor(int r, const double* __restrict__ cov, double* __restrict__ L, double* __restrict__ Li,
                                                double* __restrict__ logdet, int* __restrict__ bad) {
    __shared__ double s_piv;
    const int j = blockIdx.x;
    const size_t rr = (size_t)r * r;
    const double* A = cov + j * rr;
    double* Lj = L + j * rr;
    double* Ij = Li + j * rr;
    for (size_t e = threadIdx.x; e < rr; e += blockDim.x)
        if ((int)(e % r) > (int)(e / r)) { Lj[e] = 0.0; Ij[e] = 0.0; }
    for (int k = 0; k < r; ++k) {
        if (threadIdx.x == 0) {
            double sum = A[(size_t)k * r + k];
            for (int q = 0; q < k; ++q) sum -= Lj[(size_t)k * r + q] * Lj[(size_t)k * r + q];
            if (!(sum > 0.0)) { atomicExch(bad, 1); sum = 1.0; }
            s_piv = sqrt(sum);
            Lj[(size_t)k * r + k] = s_piv;
        }
        __syncthreads();
        const double piv = s_piv;
        for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) {
            double sum = A[(size_t)i * r + k];
            for (int q = 0; q < k; ++q) sum -= Lj[(size_t)i * r + q] * Lj[(size_t)k * r + q];
            Lj[(size_t)i * r + k] = sum / piv;
        }
        __syncthreads();
    }
    for (int col = threadIdx.x; col < r; col += blockDim.x) {
        for (int i = col; i < r; ++i) {
            double sum = i == col ? 1.0 : 0.0;
            for (int q = col; q < i; ++q) sum -= Lj[(size_t)i * r + q] * Ij[(size_t)q * r + col];
            Ij[(size_t)i * r + col] = sum / Lj[(size_t)i * r + i];
        }
    }
    if (threadIdx.x == 0) {
        double sdet = 0.0;
        for (int k = 0; k < r; ++k) sdet += log(Lj[(size_t)k * r + k]);
        logdet[j] = sdet;
    }
}

// cov_j = diag(lam_j) for the components that are new (all) or re-seeded (N_j < 2).
__global__ void k_cov_diag(int K, int r, const double* __restrict__ nj, const double* __restrict__ lam, double* __restrict__ cov) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K * r * r) return;
    const int j = t / (r * r), a = (t / r) % r, b = t % r;
    if (nj && !(nj[j] < 2.0)) return;
    cov[t] = a == b ? lam[(size_t)j * r + a] : 0.0;
}

// lam_j = diag(C_j) (what smc_get_mixture reports in the full-covariance form).
__global__ void k_diag_of_cov(int K, int r, const double* __restrict__ cov, double* __restrict__ lam) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < K * r) lam[t] = cov[((size_t)(t / r) * r + t % r) * r + t % r];
}

// Factors every C_j on the device (k_factor) into L_j, L_j^{-1} and log det L_j; with
// cov_host the covariances are uploaded first.  check_now: wait and fail (InputError) if a
// C_j is not positive definite; otherwise the flag is read by the caller later.
static int* factor_flag(Ctx& c) { return c.icount + 40; }

static void launch_factor(Ctx& c) {
    k_factor<<<c.K, 256, 0, c.stream>>>(c.r, c.gcov, c.gL, c.gLi, c.glogdet, factor_flag(c)); ++c.pc.launches;
    check(cudaGetLastError(), "factor launch");
}

static void check_factor_flag(Ctx& c) {
    int bad = 0;
    check(cudaMemcpyAsync(&bad, factor_flag(c), sizeof(int), cudaMemcpyDeviceToHost, c.stream), "factor flag");
    sync_stream(c);
    if (bad) {
        c.fitted = false;   // the stored mixture is no longer usable
        throw InputError{"a mixture covariance is not positive definite"};
    }
}

void factor_mixture(Ctx& c, const double* cov_host) {
    const size_t n = (size_t)c.K * c.r * c.r;
    check(cudaMemsetAsync(factor_flag(c), 0, sizeof(int), c.stream), "memset");
    if (cov_host) check(cudaMemcpyAsync(c.gcov, cov_host, n * sizeof(double), cudaMemcpyHostToDevice, c.stream), "cov");
    launch_factor(c);
    check_factor_flag(c);
}

double gm_fit_device(Ctx& c) {
    const int N = c.N, K = c.K, r = c.r;
    const double fl = c.cfg.var_floor;
    double* lamS = c.pooled + r;          // second half of the pooled scratch
    int* init_idx = c.icount + 8;
    k_gather_modes<<<(unsigned)(((size_t)N * r + 255) / 256), 256, 0, c.stream>>>(N, c.d, r, c.X, c.S, c.xsT); ++c.pc.launches;
    k_lamS<<<(r + 127) / 128, 128, 0, c.stream>>>(r, c.lam, c.S, lamS); ++c.pc.launches;
    k_pooled<<<r, 256, 0, c.stream>>>(N, r, c.xsT, lamS, fl, c.pooled); ++c.pc.launches;
    // initial picks (host Philox, the same definition as on the device)
    std::vector<int> picks;
    for (int k = 0; k < K; ++k) {
        const U4 w = philox((uint32_t)k, 0u, (uint32_t)c.layer, P_EMINIT, c.key.k0, c.key.k1);
        int cidx = (int)(((unsigned long long)w.x * (unsigned long long)N) >> 32);
        bool clash = true;
        while (clash) {
            clash = false;
            for (int q : picks) if (q == cidx) { clash = true; break; }
            if (clash) cidx = (cidx + 1) % N;
        }
        picks.push_back(cidx);
    }
    check(cudaMemcpyAsync(init_idx, picks.data(), K * sizeof(int), cudaMemcpyHostToDevice, c.stream), "em picks");
    k_em_init<<<(K * r + 127) / 128, 128, 0, c.stream>>>(N, K, r, init_idx, c.xsT, c.pooled, c.gw, c.gmu, c.glam); ++c.pc.launches;
    const size_t esm = sizeof(double) * (2 * (size_t)K * r + K);
    if (esm > 48 * 1024) check(cudaFuncSetAttribute(k_estep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)esm), "attr");
    const int eg = (N + 255) / 256;
    if (c.cfg.full_cov) {
        const int kr2 = K * r * r;
        const dim3 cg(cov_tiles(r), K, COV_NC);
        check(cudaMemsetAsync(factor_flag(c), 0, sizeof(int), c.stream), "memset");
        k_cov_diag<<<(kr2 + 255) / 256, 256, 0, c.stream>>>(K, r, nullptr, c.glam, c.gcov); ++c.pc.launches;
        for (int it = 0; it < c.cfg.em_iters; ++it) {
            launch_factor(c);
            k_estep_full<<<N, 128, 0, c.stream>>>(N, K, r, c.xsT, c.gw, c.gmu, c.gLi, c.glogdet, c.resp, c.lse, c.gmax); ++c.pc.launches;
            k_mstep_mean<<<K * r, 256, 0, c.stream>>>(N, r, c.xsT, c.resp, c.nj, c.gmu); ++c.pc.launches;
            k_mstep_cov<<<cg, 256, 0, c.stream>>>(N, r, c.xsT, c.resp, c.gmu, c.covpart); ++c.pc.launches;
            k_cov_reduce<<<dim3(cov_tiles(r), K), 256, 0, c.stream>>>(r, c.covpart, c.nj, lamS, fl, c.gcov); ++c.pc.launches;
            k_diag_of_cov<<<(K * r + 255) / 256, 256, 0, c.stream>>>(K, r, c.gcov, c.glam); ++c.pc.launches;
            k_mstep_fix<<<1, 1024, 0, c.stream>>>(N, K, r, c.nj, c.gmax, c.xsT, c.pooled, c.gw, c.gmu, c.glam); ++c.pc.launches;
            k_cov_diag<<<(kr2 + 255) / 256, 256, 0, c.stream>>>(K, r, c.nj, c.glam, c.gcov); ++c.pc.launches;   // re-seeded ones
        }
        launch_factor(c);
        k_estep_full<<<N, 128, 0, c.stream>>>(N, K, r, c.xsT, c.gw, c.gmu, c.gLi, c.glogdet, c.resp, c.lse, c.gmax); ++c.pc.launches;
        k_sum<<<1, 1024, 0, c.stream>>>(N, c.lse, c.dscal + 8); ++c.pc.launches;
        double ll = 0.0;
        check(cudaMemcpyAsync(&ll, c.dscal + 8, sizeof(double), cudaMemcpyDeviceToHost, c.stream), "ll");
        check_factor_flag(c);                            // one wait for the whole fit
        return ll;
    }
    for (int it = 0; it < c.cfg.em_iters; ++it) {
        k_estep<<<eg, 256, esm, c.stream>>>(N, K, r, c.xsT, c.gw, c.gmu, c.glam, c.resp, c.lse, c.gmax); ++c.pc.launches;
        k_mstep_mean<<<K * r, 256, 0, c.stream>>>(N, r, c.xsT, c.resp, c.nj, c.gmu); ++c.pc.launches;
        k_mstep_var<<<K * r, 256, 0, c.stream>>>(N, r, c.xsT, c.resp, c.nj, c.gmu, lamS, fl, c.glam); ++c.pc.launches;
        k_mstep_fix<<<1, 1024, 0, c.stream>>>(N, K, r, c.nj, c.gmax, c.xsT, c.pooled, c.gw, c.gmu, c.glam); ++c.pc.launches;
    }
    k_estep<<<eg, 256, esm, c.stream>>>(N, K, r, c.xsT, c.gw, c.gmu, c.glam, c.resp, c.lse, c.gmax); ++c.pc.launches;
    k_sum<<<1, 1024, 0, c.stream>>>(N, c.lse, c.dscal + 8); ++c.pc.launches;
    double ll = 0.0;
    check(cudaMemcpyAsync(&ll, c.dscal + 8, sizeof(double), cudaMemcpyDeviceToHost, c.stream), "ll");
    sync_stream(c);
    return ll;
}

}  // namespace smcgm
