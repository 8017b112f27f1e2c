// Reweighting, tempering, resampling and moments of Alg. 1 (Sec. 2.1) with
// the temperature rule of App. C.
//
// Tempering: with uniform weights before reweighting, the weights of step h
// are exp(-h Phi_n) and ESS(h) = (sum e^{-h Phi})^2 / sum e^{-2 h Phi} (the
// paper's (sum w^2)^-1 for normalised w).  h = 1 - t when ESS(1 - t) meets
// the target, else 64 bisection steps on [0, 1 - t] keeping the lower bracket.
//
// Resampling: systematic, on an integer CDF: normalised weights scaled by
// T = 2^48 and floored, the remainder added to the largest weight, inclusive
// prefix sums CDF_i; particle k takes min{i : N CDF_i > k T + u48} with u48 one
// Philox draw.  Integer arithmetic makes the indices independent of summation
// order.
#include "smcgm_internal.cuh"
#include "common.cuh"

namespace smcgm {

constexpr int SB = 1024;   // threads of the single-block kernels

__device__ double ess_at(const double* phi, int N, double phimin, double h, double* red) {
    double s1 = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double e = exp(-h * (phi[i] - phimin));
        s1 += e;
        s2 += e * e;
    }
    __shared__ double out[2];
    double a = block_sum(s1, red);
    if (threadIdx.x == 0) out[0] = a;
    double b = block_sum(s2, red);
    if (threadIdx.x == 0) out[1] = b;
    __syncthreads();
    const double r = out[0] * out[0] / out[1];
    __syncthreads();
    return r;
}

// out: [0] h, [1] ESS(h), [2] log Z increment, [3] new t
__global__ void __launch_bounds__(SB) k_temper(int N, const double* __restrict__ phi, double t, double target, double* __restrict__ logw,
                                               double* __restrict__ out) {
    __shared__ double red[32];
    __shared__ double s_min, s_max, s_sum;
    double mn = 1.0 / 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) mn = fmin(mn, phi[i]);
    mn = -block_max(-mn, red);
    if (threadIdx.x == 0) s_min = mn;
    __syncthreads();
    const double phimin = s_min;
    const double rest = 1.0 - t;
    double h;
    double e = ess_at(phi, N, phimin, rest, red);
    if (e >= target) {
        h = rest;
    } else {
        double lo = 0.0, hi = rest;
        for (int it = 0; it < 64; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (ess_at(phi, N, phimin, mid, red) >= target) lo = mid;
            else hi = mid;
        }
        h = lo;
        e = ess_at(phi, N, phimin, h, red);
    }
    // log weights -h Phi, their LSE, normalised weights; log Z increment = LSE - log N
    double mx = -1.0 / 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) mx = fmax(mx, -h * phi[i]);
    mx = block_max(mx, red);
    if (threadIdx.x == 0) s_max = mx;
    __syncthreads();
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) s += exp(-h * phi[i] - s_max);
    s = block_sum(s, red);
    if (threadIdx.x == 0) s_sum = s;
    __syncthreads();
    const double lse = s_max + log(s_sum);
    for (int i = threadIdx.x; i < N; i += blockDim.x) logw[i] = -h * phi[i] - lse;
    if (threadIdx.x == 0) {
        out[0] = h;
        out[1] = e;
        out[2] = lse - log((double)N);
        out[3] = (h == rest) ? 1.0 : t + h;
    }
}

void launch_temper(Ctx& c, double* out) {
    k_temper<<<1, SB, 0, c.stream>>>(c.N, c.Phi, c.t, c.cfg.ess_frac * c.N, c.logw, out); ++c.pc.launches;
    check(cudaGetLastError(), "temper");
}

// Systematic resampling on the 2^48 fixed-point CDF; writes idx[N].
__global__ void __launch_bounds__(SB) k_resample(int N, const double* __restrict__ logw, unsigned long long u48,
                                                 unsigned long long* __restrict__ cdf, int* __restrict__ idx) {
    __shared__ double red[32];
    __shared__ double s_max, s_sum;
    __shared__ unsigned long long s_part[SB];
    __shared__ double s_wmax[SB];
    __shared__ int s_imax[SB];
    const unsigned long long T = 1ull << 48;
    double mx = -1.0 / 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) mx = fmax(mx, logw[i]);
    mx = block_max(mx, red);
    if (threadIdx.x == 0) s_max = mx;
    __syncthreads();
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) s += exp(logw[i] - s_max);
    s = block_sum(s, red);
    if (threadIdx.x == 0) s_sum = s;
    __syncthreads();
    const double lse = s_max + log(s_sum);
    // contiguous chunk per thread: q_i = floor(w_i T), local argmax (lowest index on ties)
    const int chunk = (N + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * chunk, b1 = min(N, b0 + chunk);
    unsigned long long loc = 0;
    double wbest = -1.0;
    int ibest = N;
    for (int i = b0; i < b1; ++i) {
        const double w = exp(logw[i] - lse);
        const unsigned long long q = (unsigned long long)floor(w * (double)T);
        cdf[i] = q;
        loc += q;
        if (w > wbest) { wbest = w; ibest = i; }
    }
    s_part[threadIdx.x] = loc;
    s_wmax[threadIdx.x] = wbest;
    s_imax[threadIdx.x] = ibest;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        double wb = -1.0;
        int ib = N;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            tot += s_part[k];
            if (s_wmax[k] > wb || (s_wmax[k] == wb && s_imax[k] < ib)) { wb = s_wmax[k]; ib = s_imax[k]; }
        }
        cdf[ib] = (unsigned long long)((long long)cdf[ib] + ((long long)T - (long long)tot));
        // exclusive prefix of the chunk sums (recomputed after the fix-up)
        s_imax[0] = ib;
    }
    __syncthreads();
    // recompute chunk sums after the remainder fix-up, then exclusive scan
    loc = 0;
    for (int i = b0; i < b1; ++i) loc += cdf[i];
    __syncthreads();
    s_part[threadIdx.x] = loc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) { unsigned long long v = s_part[k]; s_part[k] = run; run += v; }
    }
    __syncthreads();
    unsigned long long run = s_part[threadIdx.x];
    for (int i = b0; i < b1; ++i) { run += cdf[i]; cdf[i] = run; }
    __syncthreads();
    // particle k: smallest i with N * CDF_i > k T + u48
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const unsigned long long target = (unsigned long long)k * T + u48;
        int lo = 0, hi = N - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((unsigned long long)N * cdf[mid] > target) hi = mid;
            else lo = mid + 1;
        }
        idx[k] = lo;
    }
}

__global__ void k_gather(int d, const int* __restrict__ idx, const double* __restrict__ X, double* __restrict__ X2,
                         const double* __restrict__ Phi, double* __restrict__ Phi2) {
    const int k = blockIdx.x;
    const int src = idx[k];
    const double2* a = reinterpret_cast<const double2*>(X + (size_t)src * d);
    double2* b = reinterpret_cast<double2*>(X2 + (size_t)k * d);
    for (int i = threadIdx.x; i < d / 2; i += blockDim.x) b[i] = a[i];
    if (threadIdx.x == 0) Phi2[k] = Phi[src];
}

void launch_resample(Ctx& c) {
    const U4 w = philox(0u, 0u, (uint32_t)c.layer, P_RESAMPLE, c.key.k0, c.key.k1);
    const unsigned long long u48 = ((unsigned long long)w.x << 16) | (unsigned long long)(w.y >> 16);
    k_resample<<<1, SB, 0, c.stream>>>(c.N, c.logw, u48, reinterpret_cast<unsigned long long*>(c.gridtmp), c.idx); ++c.pc.launches;
    k_gather<<<c.N, 256, 0, c.stream>>>(c.d, c.idx, c.X, c.X2, c.Phi, c.Phi2); ++c.pc.launches;
    check(cudaGetLastError(), "resample");
    std::swap(c.X, c.X2);
    std::swap(c.Phi, c.Phi2);
}

// Posterior moments over the particles: mean and population variance per coordinate.
__global__ void k_moments(int N, int d, const double* __restrict__ X, double* __restrict__ mean, double* __restrict__ var) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d) return;
    double s = 0.0;
    for (int n = 0; n < N; ++n) s += X[(size_t)n * d + c];
    const double m = s / N;
    double v = 0.0;
    for (int n = 0; n < N; ++n) { const double e = X[(size_t)n * d + c] - m; v += e * e; }
    mean[c] = m;
    var[c] = v / N;
}

void launch_moments(Ctx& c, double* mean, double* var) {
    k_moments<<<(c.d + 127) / 128, 128, 0, c.stream>>>(c.N, c.d, c.X, mean, var); ++c.pc.launches;
    check(cudaGetLastError(), "moments");
}

// 1D field at the midpoints for `count` particles.
__global__ void k_synth1d(int n, int Km, int count, const double* __restrict__ X, const double* __restrict__ S, double* __restrict__ U) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)count * n) return;
    const int p = (int)(t / n), i = (int)(t % n);
    double u = 0.0;
    for (int k = 0; k < Km; ++k) u = fma(X[(size_t)p * Km + k], S[(size_t)i * Km + k], u);
    U[t] = u;
}

__global__ void k_grid_acc(size_t cells, int count, const double* __restrict__ U, const double* __restrict__ mean, double* __restrict__ acc) {
    const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cells) return;
    double s = acc[c];
    for (int p = 0; p < count; ++p) { const double e = U[(size_t)p * cells + c] - mean[c]; s += e * e; }
    acc[c] = s;
}

__global__ void k_scale(size_t n, double* a, double f) {
    const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) a[c] *= f;
}

void launch_grid_moments(Ctx& c, const double* mean_kl, double* mean_grid, double* var_grid) {
    const size_t cells = c.dim == 2 ? (size_t)c.n * c.n : (size_t)c.n;
    auto synth = [&](const double* X, int count, double* U) {
        if (c.dim == 2) launch_synth2d(c, X, count, U);
        else { k_synth1d<<<(unsigned)(((size_t)count * c.n + 255) / 256), 256, 0, c.stream>>>(c.n, c.Km, count, X, c.basis, U); ++c.pc.launches; }
    };
    synth(mean_kl, 1, mean_grid);
    check(cudaMemsetAsync(var_grid, 0, cells * sizeof(double), c.stream), "memset");
    for (int off = 0; off < c.N; off += c.B) {
        const int cnt = std::min(c.B, c.N - off);
        synth(c.X + (size_t)off * c.d, cnt, c.u64);
        k_grid_acc<<<(unsigned)((cells + 255) / 256), 256, 0, c.stream>>>(cells, cnt, c.u64, mean_grid, var_grid); ++c.pc.launches;
    }
    k_scale<<<(unsigned)((cells + 255) / 256), 256, 0, c.stream>>>(cells, var_grid, 1.0 / c.N); ++c.pc.launches;
    check(cudaGetLastError(), "grid moments");
}

// ---------------------------------------------------------------------------
// Resampling without any allocation.
//
// Some callers cannot hand the library a device buffer at all: a host
// application that owns every byte of device memory through its own pool and
// forbids other allocations, or a loop where a cudaMalloc (which may
// synchronise the device) is not acceptable.  For them the systematic-
// resampling indices can be computed with scratch that lives in this file: a
// fixed array of device memory that every GPU loading the library keeps until
// the process exits.  The caller passes the log weights and the output array;
// the library allocates nothing.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned long long g_static_cdf[SMC_STATIC_RESAMPLE_MAX];

// Device address of g_static_cdf on the current device.  It is looked up on every
// call (the lookup allocates nothing): a cached address would go stale if the
// process reset the device, which unloads the library's module there.  The first
// lookup on a device also loads the module's copy of the array onto it.
static unsigned long long* static_cdf_ptr() {
    void* p = nullptr;
    check(cudaGetSymbolAddress(&p, g_static_cdf), "cudaGetSymbolAddress(g_static_cdf)");
    return reinterpret_cast<unsigned long long*>(p);
}

}  // namespace smcgm

extern "C" smc_status smc_resample_indices_static(const double* d_logw, int n_particles, unsigned long long seed, int layer,
                                                  int* d_indices, void* stream) {
    using namespace smcgm;
    if (!d_logw || !d_indices || layer < 0) {
        set_global_error("smc_resample_indices_static: null pointer or negative layer");
        return SMC_EINVAL;
    }
    if (n_particles < 1 || n_particles > SMC_STATIC_RESAMPLE_MAX) {
        set_global_error("smc_resample_indices_static: n_particles must be in [1, SMC_STATIC_RESAMPLE_MAX] (32768)");
        return SMC_EINVAL;
    }
    if (!device_visible(d_logw) || !device_visible(d_indices)) {
        set_global_error("smc_resample_indices_static: d_logw and d_indices must be device memory");
        return SMC_EINVAL;
    }
    try {
        unsigned long long* cdf = static_cdf_ptr();
        const Key key = key_of(seed);
        const U4 w = philox(0u, 0u, (uint32_t)layer, P_RESAMPLE, key.k0, key.k1);
        const unsigned long long u48 = ((unsigned long long)w.x << 16) | (unsigned long long)(w.y >> 16);
        // every entry of the CDF scratch below n_particles is written before it is read; nothing needs clearing
        k_resample<<<1, SB, 0, reinterpret_cast<cudaStream_t>(stream)>>>(n_particles, d_logw, u48, cdf, d_indices);
        check(cudaGetLastError(), "k_resample launch");
    } catch (const CudaError& ce) {
        set_global_error((std::string(ce.what) + ": " + cudaGetErrorString(ce.e)).c_str());
        return SMC_ECUDA;
    }
    return SMC_OK;
}
