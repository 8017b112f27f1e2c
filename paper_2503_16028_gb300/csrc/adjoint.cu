// Gradient of the potential with respect to the KL coordinates by the adjoint
// of the discrete forward model (the drift D Phi of the Langevin equation of
// App. B; see smc_gradient in smcgm.h for the formulas):
//   1. forward solve A(u) w = b and Phi (the forward map's own kernels);
//   2. adjoint right-hand side O^T (O w - d) / sigma^2, one thread per particle
//      scattering its observation stencils in a fixed order (deterministic);
//   3. adjoint solve A lam = that right-hand side with the same solver;
//   4. dPhi/du per cell from w, lam, the faces and e^{-u} (k_grad_u_df, k_grad_u64);
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

// FP64 context: dPhi/du_c = -sum over the faces of cell c of
// (dK_f/du_c)(lam_c - lam_nb)(w_c - w_nb), lam_nb = w_nb = 0 across a wall, with
// dK_f/du_c = K_f^2 e^{-u_c} / 2 for a harmonic face and K_f for a wall face.
// The FP64 set-up leaves e^{-u} in the field's array (k_exp_neg).  A 32 x 32
// tile per block, 4 cells a thread; the east / north face of a cell is its
// neighbour's west / south face.
__global__ void __launch_bounds__(256) k_grad_u64(int n, const double* __restrict__ s, const double* __restrict__ kw,
                                                  const double* __restrict__ ks, const double* __restrict__ E,
                                                  const double* __restrict__ N, const double* __restrict__ w,
                                                  const double* __restrict__ lam, double* __restrict__ g) {
    const int p = blockIdx.y;
    const int tpr = n / TILE;
    const int tx = blockIdx.x % tpr, ty = blockIdx.x / tpr;
    const size_t nn = (size_t)n * n, base = (size_t)p * nn;
    const int li = threadIdx.x % TILE, lj0 = threadIdx.x / TILE;
    for (int lj = lj0; lj < TILE; lj += blockDim.x / TILE) {
        const int i = tx * TILE + li, j = ty * TILE + lj;
        const size_t c = base + (size_t)j * n + i;
        const double e = s[c], wc = w[c], lc = lam[c];
        auto dk = [e](double K) { return 0.5 * K * K * e; };
        double acc = 0.0;
        acc += i > 0 ? dk(kw[c]) * (lc - lam[c - 1]) * (wc - w[c - 1]) : kw[c] * lc * wc;
        acc += i + 1 < n ? dk(kw[c + 1]) * (lc - lam[c + 1]) * (wc - w[c + 1]) : E[(size_t)p * n + j] * lc * wc;
        acc += j > 0 ? dk(ks[c]) * (lc - lam[c - n]) * (wc - w[c - n]) : ks[c] * lc * wc;
        acc += j + 1 < n ? dk(ks[c + n]) * (lc - lam[c + n]) * (wc - w[c + n]) : N[(size_t)p * n + i] * lc * wc;
        g[c] = -acc;
    }
}

// Mixed precision: the same gradient with the face terms formed once per face
// and in df32.  For a harmonic face dK_f/du_c = K_f^2 e^{-u_c} / 2, and for a
// wall face K_f = 2 k_c gives K_f = K_f^2 e^{-u_c} / 2 as well, so
//   dPhi/du_c = -e^{-u_c} sum over the faces of c of P_f,
//   P_f = K_f^2 (lam_a - lam_b)(w_a - w_b) / 2   (lam_b = w_b = 0 across a wall),
// symmetric in the face's two cells.  A 32 x 32 tile puts the west and south
// P of its cells (and those of the next column and row) in shared memory; the
// differences use the FP64 unit once per face (exact for neighbours), the rest
// runs in df32 on the FP32 pipes.
__global__ void __launch_bounds__(256) k_grad_u_df(int n, const float2* __restrict__ u, const float* __restrict__ Kwh,
                                                   const float* __restrict__ Kwl, const float* __restrict__ Ksh,
                                                   const float* __restrict__ Ksl, const float* __restrict__ Eh,
                                                   const float* __restrict__ El, const float* __restrict__ Nh,
                                                   const float* __restrict__ Nl, const float2* __restrict__ exptab, ExpConsts ec,
                                                   const double* __restrict__ w, const double* __restrict__ lam, double* __restrict__ g) {
    __shared__ float2 tab[64];
    __shared__ float2 PW[TILE][TILE + 1];
    __shared__ float2 PS[TILE + 1][TILE];
    const int p = blockIdx.y;
    const int tpr = n / TILE;
    const int tx = blockIdx.x % tpr, ty = blockIdx.x / tpr;
    const int x0 = tx * TILE, y0 = ty * TILE;
    const size_t nn = (size_t)n * n, base = (size_t)p * nn;
    const double* wp = w + base;
    const double* lp = lam + base;
    const int li = threadIdx.x % TILE, lj0 = threadIdx.x / TILE;
    if (threadIdx.x < 64) tab[threadIdx.x] = exptab[threadIdx.x];
    auto P = [](float kh, float kl, double dl, double dw) {
        const df32 K{kh, kl};
        const df32 r = df_mul(df_mul(K, K), df_mul(df_from_double_bits(dl), df_from_double_bits(dw)));
        return make_float2(0.5f * r.hi, 0.5f * r.lo);
    };
    for (int lj = lj0; lj < TILE; lj += blockDim.x / TILE) {
        const int i = x0 + li, j = y0 + lj;
        const size_t c = base + (size_t)j * n + i;
        const size_t cl = c - base;
        const double wc = wp[cl], lc = lp[cl];
        PW[lj][li] = i > 0 ? P(Kwh[c], Kwl[c], lc - lp[cl - 1], wc - wp[cl - 1]) : P(Kwh[c], Kwl[c], lc, wc);
        PS[lj][li] = j > 0 ? P(Ksh[c], Ksl[c], lc - lp[cl - n], wc - wp[cl - n]) : P(Ksh[c], Ksl[c], lc, wc);
        if (li == TILE - 1)
            PW[lj][TILE] = i + 1 < n ? P(Kwh[c + 1], Kwl[c + 1], lp[cl + 1] - lc, wp[cl + 1] - wc)
                                     : P(Eh[(size_t)p * n + j], El[(size_t)p * n + j], lc, wc);
        if (lj == TILE - 1)
            PS[TILE][li] = j + 1 < n ? P(Ksh[c + n], Ksl[c + n], lp[cl + n] - lc, wp[cl + n] - wc)
                                     : P(Nh[(size_t)p * n + i], Nl[(size_t)p * n + i], lc, wc);
    }
    __syncthreads();
    for (int lj = lj0; lj < TILE; lj += blockDim.x / TILE) {
        const size_t c = base + (size_t)(y0 + lj) * n + x0 + li;
        const float2 a = PW[lj][li], b = PW[lj][li + 1], d = PS[lj][li], e = PS[lj + 1][li];
        const df32 sum = df_add(df_add(df32{a.x, a.y}, df32{b.x, b.y}), df_add(df32{d.x, d.y}, df32{e.x, e.y}));
        const float2 uv = u[c];
        const df32 r = df_mul(df_exp(df32{-uv.x, -uv.y}, tab, ec), sum);
        g[c] = -((double)r.hi + (double)r.lo);
    }
}

int gradient_batch(Ctx& c, const double* X, int count, double* Phi_out, double* grad_out) {
    const int n = c.n;
    const size_t nn = (size_t)n * n;
    const bool mixed = mixed_precision(c.cfg);
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
            k_grad_u_df<<<grid, 256, 0, c.stream>>>(n, reinterpret_cast<const float2*>(c.u64), f0.Kw, c.Kwlo, f0.Ks, c.Kslo, f0.E,
                                                    c.Elo, f0.Nn, c.Nlo, reinterpret_cast<const float2*>(c.exptab), c.expc, c.w64,
                                                    c.lam64, c.rhs); ++c.pc.launches;
        } else {
            k_grad_u64<<<grid, 256, 0, c.stream>>>(n, c.u64, c.Kw64, c.Ks64, c.E64, c.N64, c.w64, c.lam64, c.rhs); ++c.pc.launches;
        }
        // 5. dPhi/dx
        launch_analysis2d(c, c.rhs, cnt, grad_out + (size_t)off * c.d);
    }
    check(cudaGetLastError(), "gradient");
    return itmax;
}

}  // namespace smcgm
