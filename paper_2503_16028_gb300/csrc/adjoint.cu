// Gradient of the potential with respect to the KL coordinates by the adjoint
// of the discrete forward model (the drift D Phi of the Langevin equation of
// App. B; see smc_gradient in smcgm.h for the formulas):
//   1. forward solve A(u) w = b and Phi (the forward map's own kernels);
//   2. adjoint right-hand side O^T (O w - d) / sigma^2, one thread per particle
//      scattering its observation stencils in a fixed order (deterministic);
//   3. adjoint solve A lam = that right-hand side with the same solver;
//   4. dPhi/du per cell from w, lam, the faces and e^{-u} (k_grad_u);
//   5. dPhi/dx = S^T dPhi/du (launch_analysis2d, the transposed cosine transform).
#include <algorithm>
#include "smcgm_internal.cuh"
#include "common.cuh"

namespace smcgm {

// The four cells and signed bilinear weights of an observation at (x, y), with
// the odd reflection across the walls of k_observe2d.
__device__ inline void obs_stencil(int n, double x, double y, int* cell, double* wgt) {
    const double s = x * n - 0.5, t = y * n - 0.5;
    const int i0 = (int)floor(s), j0 = (int)floor(t);
    const double fx = s - i0, fy = t - j0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int di = k & 1, dj = k >> 1;
        int i = i0 + di, j = j0 + dj;
        double sg = 1.0;
        if (i < 0) { i = 0; sg = -sg; }
        if (i > n - 1) { i = n - 1; sg = -sg; }
        if (j < 0) { j = 0; sg = -sg; }
        if (j > n - 1) { j = n - 1; sg = -sg; }
        cell[k] = j * n + i;
        wgt[k] = sg * (di ? fx : 1.0 - fx) * (dj ? fy : 1.0 - fy);
    }
}

// rhs (zeroed, FP64 [count][n][n]) += O^T (O w - d) / sigma^2, one thread per particle.
__global__ void k_adjoint_scatter(int n, int count, int nobs, const double* __restrict__ w, const double* __restrict__ obs,
                                  const double* __restrict__ data, double inv_s2, double* __restrict__ rhs) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= count) return;
    const size_t base = (size_t)p * n * n;
    for (int m = 0; m < nobs; ++m) {
        int cell[4];
        double wgt[4];
        obs_stencil(n, obs[2 * m], obs[2 * m + 1], cell, wgt);
        double y = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) y += wgt[k] * w[base + cell[k]];
        const double r = (y - data[m]) * inv_s2;
#pragma unroll
        for (int k = 0; k < 4; ++k) rhs[base + cell[k]] += wgt[k] * r;
    }
}

// |rhs|^2 per particle and, for the mixed-precision solver, the right-hand
// side rewritten in place as df32 pairs (each 8-byte cell by its own thread).
__global__ void __launch_bounds__(256) k_rhs_finish(int nn, int as_df32, double* __restrict__ rhs, double* __restrict__ b2) {
    __shared__ double red[32];
    const int p = blockIdx.x;
    double* b = rhs + (size_t)p * nn;
    double acc = 0.0;
    for (int i = threadIdx.x; i < nn; i += blockDim.x) {
        const double v = b[i];
        acc += v * v;
        if (as_df32) {
            const df32 d = df_from_double_bits(v);
            reinterpret_cast<float2*>(b)[i] = make_float2(d.hi, d.lo);
        }
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) b2[p] = acc;
}

// Face coefficient and its derivative with respect to the cell's own log
// permeability: harmonic face K^2 e^{-u} / 2, wall face K.
struct FaceD {
    double K, dK;
};

template <bool MIXED>
struct GradSrc;

template <>
struct GradSrc<true> {   // df32 field and faces of the mixed-precision set-up
    const float2* u;
    const float *kwh, *kwl, *ksh, *ksl, *eh, *el, *nh, *nl;
    const float2* tab;
    ExpConsts ec;
    __device__ df32 emu(size_t c) const {
        const float2 v = u[c];
        return df_exp(df32{-v.x, -v.y}, tab, ec);
    }
    __device__ static FaceD face(float kh, float kl, df32 e, bool wall) {
        const df32 K{kh, kl};
        if (wall) return FaceD{(double)kh + (double)kl, (double)kh + (double)kl};
        const df32 d = df_mul(df_mul(K, K), e);
        return FaceD{(double)kh + (double)kl, 0.5 * ((double)d.hi + (double)d.lo)};
    }
    __device__ FaceD west(size_t c, df32 e, bool wall) const { return face(kwh[c], kwl[c], e, wall); }
    __device__ FaceD south(size_t c, df32 e, bool wall) const { return face(ksh[c], ksl[c], e, wall); }
    __device__ FaceD east_wall(size_t r) const { return face(eh[r], el[r], df32{0.f, 0.f}, true); }
    __device__ FaceD north_wall(size_t r) const { return face(nh[r], nl[r], df32{0.f, 0.f}, true); }
};

template <>
struct GradSrc<false> {  // FP64 faces; the FP64 set-up leaves e^{-u} in the field's array (k_exp_neg)
    const double* s;
    const double *kw, *ks, *E, *N;
    __device__ double emu(size_t c) const { return s[c]; }
    __device__ static FaceD face(double K, double e, bool wall) { return FaceD{K, wall ? K : 0.5 * K * K * e}; }
    __device__ FaceD west(size_t c, double e, bool wall) const { return face(kw[c], e, wall); }
    __device__ FaceD south(size_t c, double e, bool wall) const { return face(ks[c], e, wall); }
    __device__ FaceD east_wall(size_t r) const { return face(E[r], 0.0, true); }
    __device__ FaceD north_wall(size_t r) const { return face(N[r], 0.0, true); }
};

// dPhi/du_c = -sum over the faces of cell c of (dK_f/du_c)(lam_c - lam_nb)(w_c - w_nb),
// lam_nb = w_nb = 0 across a wall.  A 32 x 32 tile per block, 4 cells a thread;
// the east / north face of a cell is its neighbour's west / south face, whose
// derivative with respect to this cell takes this cell's e^{-u}.
template <bool MIXED>
__global__ void __launch_bounds__(256) k_grad_u(int n, GradSrc<MIXED> S, const double* __restrict__ w,
                                                const double* __restrict__ lam, double* __restrict__ g) {
    const int p = blockIdx.y;
    const int tpr = n / TILE;
    const int tx = blockIdx.x % tpr, ty = blockIdx.x / tpr;
    const size_t nn = (size_t)n * n, base = (size_t)p * nn;
    const int li = threadIdx.x % TILE, lj0 = threadIdx.x / TILE;
    for (int lj = lj0; lj < TILE; lj += blockDim.x / TILE) {
        const int i = tx * TILE + li, j = ty * TILE + lj;
        const size_t c = base + (size_t)j * n + i;
        const auto e = S.emu(c);
        const double wc = w[c], lc = lam[c];
        double acc = 0.0;
        {   // west
            const FaceD f = S.west(c, e, i == 0);
            acc += f.dK * (i > 0 ? (lc - lam[c - 1]) * (wc - w[c - 1]) : lc * wc);
        }
        {   // east
            const FaceD f = i + 1 < n ? S.west(c + 1, e, false) : S.east_wall((size_t)p * n + j);
            acc += f.dK * (i + 1 < n ? (lc - lam[c + 1]) * (wc - w[c + 1]) : lc * wc);
        }
        {   // south
            const FaceD f = S.south(c, e, j == 0);
            acc += f.dK * (j > 0 ? (lc - lam[c - n]) * (wc - w[c - n]) : lc * wc);
        }
        {   // north
            const FaceD f = j + 1 < n ? S.south(c + n, e, false) : S.north_wall((size_t)p * n + i);
            acc += f.dK * (j + 1 < n ? (lc - lam[c + n]) * (wc - w[c + n]) : lc * wc);
        }
        g[c] = -acc;
    }
}

int gradient_batch(Ctx& c, const double* X, int count, double* Phi_out, double* grad_out) {
    const int n = c.n;
    const size_t nn = (size_t)n * n;
    const bool mixed = c.cfg.precision == SMC_P_FP32_REFINE;
    int itmax = 0;
    for (int off = 0; off < count; off += c.B) {
        const int cnt = std::min(c.B, count - off);
        // 1. forward: field, coefficients, w, Phi
        if (mixed) launch_synth2d_df(c, X + (size_t)off * c.d, cnt, reinterpret_cast<float2*>(c.u64));
        else launch_synth2d(c, X + (size_t)off * c.d, cnt, c.u64);
        launch_setup_coeffs(c, cnt);
        itmax = std::max(itmax, solve_batch(c, cnt, shared_rhs(c), c.w64));
        launch_observe(c, c.w64, cnt, Phi_out + off);
        launch_mark_out_of_range(c, cnt, Phi_out + off);
        // 2. adjoint right-hand side
        check(cudaMemsetAsync(c.rhs, 0, (size_t)cnt * nn * sizeof(double), c.stream), "memset rhs");
        k_adjoint_scatter<<<(cnt + 127) / 128, 128, 0, c.stream>>>(n, cnt, c.nobs, c.w64, c.obs, c.data,
                                                                  1.0 / (c.cfg.sigma * c.cfg.sigma), c.rhs); ++c.pc.launches;
        k_rhs_finish<<<cnt, 256, 0, c.stream>>>((int)nn, mixed ? 1 : 0, c.rhs, c.rhs_b2); ++c.pc.launches;
        // 3. adjoint solve
        const Rhs R{mixed ? nullptr : c.rhs, mixed ? reinterpret_cast<const float2*>(c.rhs) : nullptr, nn, c.rhs_b2, 0.0};
        itmax = std::max(itmax, solve_batch(c, cnt, R, c.lam64));
        // 4. dPhi/du into the right-hand side's storage (no longer needed)
        const dim3 grid((n / TILE) * (n / TILE), cnt);
        if (mixed) {
            LevelArrays<float>& f0 = c.s32.lv[0];
            GradSrc<true> S{reinterpret_cast<const float2*>(c.u64), f0.Kw, c.Kwlo, f0.Ks, c.Kslo, f0.E, c.Elo, f0.Nn, c.Nlo,
                            reinterpret_cast<const float2*>(c.exptab), c.expc};
            k_grad_u<true><<<grid, 256, 0, c.stream>>>(n, S, c.w64, c.lam64, c.rhs); ++c.pc.launches;
        } else {
            GradSrc<false> S{c.u64, c.Kw64, c.Ks64, c.E64, c.N64};
            k_grad_u<false><<<grid, 256, 0, c.stream>>>(n, S, c.w64, c.lam64, c.rhs); ++c.pc.launches;
        }
        // 5. dPhi/dx
        launch_analysis2d(c, c.rhs, cnt, grad_out + (size_t)off * c.d);
    }
    check(cudaGetLastError(), "gradient");
    return itmax;
}

}  // namespace smcgm
