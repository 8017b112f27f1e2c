// Field synthesis u = sum_{k,l} v_kl c_k cos(k pi x) c_l cos(l pi y) at the
// cell centres (the KL expansion of the prior, Sec. 2.1 / Sec. 3.2, eq. Fourier
// series), in FP64, and the whole 1D forward map of the elliptic problem.
//
// 2D synthesis is separable: T = V^T B^T (stage 1, along x), U = B T (stage 2,
// along y), with B[i][k] = c_k cos(k pi (i + 1/2)/n).  Both stages use the
// mirror symmetry of the cell-centre cosines, B[n-1-i][k] = (-1)^k B[i][k]:
// even and odd modes are summed separately for i < n/2 and combined as
// E + O (row i) and E - O (row n-1-i), halving the multiply-adds.
#include "smcgm_internal.cuh"
#include "common.cuh"

namespace smcgm {

constexpr int SY_CI = 16;        // output columns i per block (plus their mirrors)

// grid: (n/2/SY_CI, count); block 256.  Shared: T[Km][2*SY_CI] doubles.
__global__ void __launch_bounds__(256) k_synth2d(int n, int Km, const double* __restrict__ X, const double* __restrict__ B,
                                                 double* __restrict__ U) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double* Ts = reinterpret_cast<double*>(smraw);   // [Km][2*SY_CI]: columns i0+c (c < CI) then mirrors
    const int p = blockIdx.y;
    const int i0 = blockIdx.x * SY_CI;
    const double* V = X + (size_t)p * Km * Km;       // V[k][l]
    const int tid = threadIdx.x;
    const int Kh = (Km + 1) / 2;
    // stage 1: for each (l, c): Te = sum_{k even} V[k][l] B[i0+c][k], To = sum_{k odd}
    for (int task = tid; task < Km * SY_CI; task += blockDim.x) {
        const int l = task / SY_CI, cc = task % SY_CI;
        const int i = i0 + cc;
        const double* Bi = B + (size_t)i * Km;
        double te = 0.0, to = 0.0;
        for (int h = 0; h < Kh; ++h) {
            const int k = 2 * h;
            te = fma(V[(size_t)k * Km + l], Bi[k], te);
            if (k + 1 < Km) to = fma(V[(size_t)(k + 1) * Km + l], Bi[k + 1], to);
        }
        Ts[l * (2 * SY_CI) + cc] = te + to;
        Ts[l * (2 * SY_CI) + SY_CI + cc] = te - to;
    }
    __syncthreads();
    // stage 2: U[j][col] = sum_l B[j][l] T[l][col], j < n/2 with mirrors.
    const int nh = n / 2;
    for (int task = tid; task < nh * 2 * SY_CI; task += blockDim.x) {
        const int j = task / (2 * SY_CI), col = task % (2 * SY_CI);
        const double* Bj = B + (size_t)j * Km;
        double e = 0.0, o = 0.0;
        for (int h = 0; h < Kh; ++h) {
            const int l = 2 * h;
            e = fma(Bj[l], Ts[l * (2 * SY_CI) + col], e);
            if (l + 1 < Km) o = fma(Bj[l + 1], Ts[(l + 1) * (2 * SY_CI) + col], o);
        }
        const int i = col < SY_CI ? i0 + col : n - 1 - (i0 + col - SY_CI);
        double* Up = U + (size_t)p * n * n;
        Up[(size_t)j * n + i] = e + o;
        Up[(size_t)(n - 1 - j) * n + i] = e - o;
    }
}

void launch_synth2d(Ctx& c, const double* X, int count, double* U) {
    const int n = c.n, Km = c.Km;
    const size_t smem = sizeof(double) * (size_t)Km * 2 * SY_CI;
    static bool attr = false;
    if (!attr) {
        check(cudaFuncSetAttribute(k_synth2d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(double) * 256 * 2 * SY_CI)), "attr");
        attr = true;
    }
    dim3 grid(n / 2 / SY_CI, count);
    k_synth2d<<<grid, 256, smem, c.stream>>>(n, Km, X, c.basis, U);
    check(cudaGetLastError(), "synth2d");
}

// ------------------------------------------------------------------------
// Observation of the cell-centred solution (bilinear, odd reflection across
// the walls so the interpolant vanishes there) and the potential
// Phi = |F(u) - d|^2 / (2 sigma^2) (Sec. 2.1, eq. Phi).  One warp per particle.
// ------------------------------------------------------------------------
__device__ inline double wghost(const double* w, int n, int i, int j) {
    double s = 1.0;
    if (i < 0) { i = 0; s = -s; }
    if (i > n - 1) { i = n - 1; s = -s; }
    if (j < 0) { j = 0; s = -s; }
    if (j > n - 1) { j = n - 1; s = -s; }
    return s * w[(size_t)j * n + i];
}

__global__ void k_observe2d(int n, int count, int nobs, const double* __restrict__ w, const double* __restrict__ obs,
                            const double* __restrict__ data, double inv2s2, double* __restrict__ Phi) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= count) return;
    const double* wp = w + (size_t)warp * n * n;
    double acc = 0.0;
    for (int m = lane; m < nobs; m += 32) {
        const double s = obs[2 * m] * n - 0.5, t = obs[2 * m + 1] * n - 0.5;
        const int i0 = (int)floor(s), j0 = (int)floor(t);
        const double fx = s - i0, fy = t - j0;
        const double a = wghost(wp, n, i0, j0), b = wghost(wp, n, i0 + 1, j0);
        const double cc = wghost(wp, n, i0, j0 + 1), d = wghost(wp, n, i0 + 1, j0 + 1);
        const double y = (1 - fy) * ((1 - fx) * a + fx * b) + fy * ((1 - fx) * cc + fx * d);
        const double rr = y - data[m];
        acc += rr * rr;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) Phi[warp] = acc * inv2s2;
}

void launch_observe(Ctx& c, const double* w, int count, double* Phi) {
    const double inv2s2 = 1.0 / (2.0 * c.cfg.sigma * c.cfg.sigma);
    const int threads = 256;
    const int blocks = (count * 32 + threads - 1) / threads;
    k_observe2d<<<blocks, threads, 0, c.stream>>>(c.n, count, c.nobs, w, c.obs, c.data, inv2s2, Phi);
    check(cudaGetLastError(), "observe");
}

// ------------------------------------------------------------------------
// 1D forward map, one thread per particle: u at the n midpoints from the sine
// KL expansion, K = e^u, tridiagonal system of the nodal FD scheme solved by
// the Thomas algorithm (forward elimination, back substitution), linear
// interpolation at the observation points, Phi.  FP64 throughout.
// The basis table holds S[i][k] = sqrt(2) sin((k+1) pi (i+1/2)/n).
// ------------------------------------------------------------------------
__global__ void k_forward1d(int n, int Km, int count, const double* __restrict__ X, const double* __restrict__ S,
                            const double* __restrict__ b, int nobs, const double* __restrict__ obs, const double* __restrict__ data,
                            double inv2s2, double* __restrict__ Phi, double* __restrict__ wout, double* __restrict__ scratch) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= count) return;
    const double* v = X + (size_t)p * Km;
    // scratch per particle: K[n], cp[n], w[n+1]
    double* K = scratch + (size_t)p * (3 * n + 2);
    double* cp = K + n;
    double* w = cp + n;       // w[0..n], w[0] = w[n] = 0
    for (int i = 0; i < n; ++i) {
        double u = 0.0;
        const double* Si = S + (size_t)i * Km;
        for (int k = 0; k < Km; ++k) u = fma(v[k], Si[k], u);
        K[i] = exp(u);
    }
    // unknowns w_1..w_{n-1}: diag K_{i-1/2} + K_{i+1/2} = K[i-1] + K[i]; off-diagonal -K[i]
    // Thomas: forward sweep
    const int m = n - 1;
    double dprev = 0.0;
    for (int r = 0; r < m; ++r) {
        const int node = r + 1;
        const double diag = K[node - 1] + K[node];
        const double lower = r > 0 ? -K[node - 1] : 0.0;
        const double upper = r < m - 1 ? -K[node] : 0.0;
        const double denom = diag - lower * (r > 0 ? cp[r - 1] : 0.0);
        cp[r] = upper / denom;
        const double rhs = b[r];
        dprev = (rhs - lower * (r > 0 ? w[r] : 0.0)) / denom;   // w[r] holds d'_{r-1}
        w[r + 1] = dprev;                                       // temporarily d'_r at w[r+1]
    }
    // back substitution: x_{m-1} = d'_{m-1}; x_r = d'_r - c'_r x_{r+1}
    w[0] = 0.0;
    w[n] = 0.0;
    for (int r = m - 2; r >= 0; --r) w[r + 1] = w[r + 1] - cp[r] * w[r + 2];
    if (wout) for (int i = 0; i < m; ++i) wout[(size_t)p * m + i] = w[i + 1];
    double acc = 0.0;
    for (int o = 0; o < nobs; ++o) {
        const double s = obs[o] * n;
        int i0 = (int)floor(s);
        if (i0 > n - 1) i0 = n - 1;
        if (i0 < 0) i0 = 0;
        const double fx = s - i0;
        const double y = (1 - fx) * w[i0] + fx * w[i0 + 1];
        const double rr = y - data[o];
        acc += rr * rr;
    }
    Phi[p] = acc * inv2s2;
}

void launch_forward1d(Ctx& c, const double* X, int count, double* Phi, double* w_out) {
    const double inv2s2 = 1.0 / (2.0 * c.cfg.sigma * c.cfg.sigma);
    for (int off = 0; off < count; off += c.B) {
        const int cnt = std::min(c.B, count - off);
        k_forward1d<<<(cnt + 63) / 64, 64, 0, c.stream>>>(c.n, c.Km, cnt, X + (size_t)off * c.d, c.basis, c.b64, c.nobs, c.obs,
                                                          c.data, inv2s2, Phi + off, w_out ? w_out + (size_t)off * (c.n - 1) : nullptr,
                                                          c.u64);
    }
    check(cudaGetLastError(), "forward1d");
}

}  // namespace smcgm
