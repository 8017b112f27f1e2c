// Forward PDE solve of the Darcy problem (Sec. 3.2, eq. example2:PDE),
// -div(e^u grad w) = f on (0,1)^2, w = 0 on the boundary, for a batch of
// particles: cell-centred 5-point finite volumes with harmonic face means,
// multigrid-preconditioned conjugate gradients, optional FP64 iterative
// refinement around FP32 inner solves.
//
// Multigrid: Galerkin coarse operators for piecewise-constant prolongation
// (coarse face coefficient = sum of the two fine faces it covers), R = P^T,
// coarse correction scaled by `coarse_scale` (2 makes up for the energy of the
// piecewise-constant interpolant), symmetric red-black Gauss-Seidel smoothing
// (pre: red, black; post: black, red), so the V-cycle is a symmetric
// preconditioner for CG.
//
// Memory layout: every array is particle-major, row-major inside a particle
// (x fastest).  The fine levels are swept by tiled kernels: one block per
// 32 x 32 tile and particle, the tile plus a halo of 2*nu cells staged in
// shared memory, all smoothing sweeps of one pre- or post-smoothing done in
// shared memory (the halo shrinks by one cell per half-sweep), so each
// multigrid pass reads its inputs from HBM once.  Levels at or below
// `coarse_top` cells per side run the rest of the V-cycle in one block per
// particle entirely in shared memory.
#include <cstdio>
#include <algorithm>
#include <cudaTypedefs.h>
#include "smcgm_internal.cuh"
#include "common.cuh"
#include "tma.cuh"
#include "df32.cuh"

namespace smcgm {

// ------------------------------------------------------------------------
// Setup: s = exp(-u); face coefficients 2/(s_a + s_b) (harmonic mean of e^u),
// wall faces 2 e^u (Dirichlet 0 half a cell away).
// ------------------------------------------------------------------------
__global__ void k_exp_neg(double* __restrict__ u, size_t total) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i < total; i += stride) u[i] = exp(-u[i]);
}

// Stores one face coefficient: FP64, or (mixed precision) its df32 split into
// the inner solver's FP32 face hi = round(v) and lo = round(v - hi).
struct FaceOut {
    double* f64;
    float *hi, *lo;
    __nv_bfloat16* bf = nullptr;   // the BF16 smoother's copy of hi (interior faces)
    __device__ void put(size_t i, double v) const {
        if (f64) f64[i] = v;
        if (hi) {
            const float h = __double2float_rn(v);
            hi[i] = h;
            if (lo) lo[i] = __double2float_rn(v - (double)h);
            if (bf) bf[i] = __float2bfloat16_rn(h);
        }
    }
};

// Harmonic face coefficients from s = exp(-u): west and south faces
// 2 / (s_c + s_nb), wall faces 2 / s_c (Dirichlet ghost on the wall).
__global__ void k_faces(int n, int count, const double* __restrict__ s, FaceOut Kw, FaceOut Ks, FaceOut E, FaceOut Nn) {
    const size_t nn = (size_t)n * n;
    const size_t total = nn * count;
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; t < total; t += stride) {
        const size_t p = t / nn;
        const int c = (int)(t - p * nn);
        const int i = c % n, j = c / n;
        const double* sp = s + p * nn;
        const double sc = sp[c];
        Kw.put(t, (i == 0) ? 2.0 * recip_nr(sc) : 2.0 * recip_nr(sc + sp[c - 1]));
        Ks.put(t, (j == 0) ? 2.0 * recip_nr(sc) : 2.0 * recip_nr(sc + sp[c - n]));
        if (i == n - 1) E.put(p * n + j, 2.0 * recip_nr(sc));
        if (j == n - 1) Nn.put(p * n + i, 2.0 * recip_nr(sc));
    }
}

// Mixed precision: s = exp(-u) and the harmonic faces in df32 (FP32 pipes
// only; the FP64 unit of GB300 is ~58x slower).  A block covers a 32 x 8 tile
// of one particle: s on the tile plus its west column and south row goes to
// shared memory, then each thread forms its cell's west and south faces
// 2 / (s_c + s_nb) (2 / s_c on a wall) and the east / north wall faces.  The
// high parts are the inner solver's FP32 faces, the low parts complete them
// to ~1e-14 relative for the FP64-accurate residual.  |u| >= 64 (beyond the
// FP32 range of e^u) sets err[1] and is reported by the host.  With Kwb, Ksb
// (the BF16 smoother faces) the interior faces are also stored rounded to BF16.
constexpr int FX = 32, FY = 8;
__global__ void __launch_bounds__(FX * FY) k_faces_df(int n, const float2* __restrict__ u, const float2* __restrict__ exptab,
                                                      ExpConsts ec, float* __restrict__ Kwh, float* __restrict__ Kwl,
                                                      float* __restrict__ Ksh, float* __restrict__ Ksl, float* __restrict__ Eh,
                                                      float* __restrict__ El, float* __restrict__ Nh, float* __restrict__ Nl,
                                                      __nv_bfloat16* __restrict__ Kwb, __nv_bfloat16* __restrict__ Ksb,
                                                      int* __restrict__ err, int* __restrict__ badp) {
    __shared__ float2 tab[64];
    __shared__ float2 S[FY + 1][FX + 1];
    const int p = blockIdx.y;
    const int tpr = n / FX;
    const int tx = blockIdx.x % tpr, ty = blockIdx.x / tpr;
    if (threadIdx.x < 64) tab[threadIdx.x] = exptab[threadIdx.x];
    __syncthreads();
    const size_t nn = (size_t)n * n, base = (size_t)p * nn;
    const float2* up = u + base;
    bool bad = false;
    for (int idx = threadIdx.x; idx < (FY + 1) * (FX + 1); idx += blockDim.x) {
        const int ly = idx / (FX + 1), lx = idx % (FX + 1);
        const int gi = tx * FX + lx - 1, gj = ty * FY + ly - 1;
        float2 v = make_float2(1.f, 0.f);
        if (gi >= 0 && gj >= 0) {
            const float2 uv = up[(size_t)gj * n + gi];
            if (!(fabsf(uv.x) < 64.f)) {
                bad = true;
            } else {
                const df32 sv = df_exp(df32{-uv.x, -uv.y}, tab, ec);
                v = make_float2(sv.hi, sv.lo);
            }
        }
        S[ly][lx] = v;
    }
    if (bad) {
        atomicExch(&err[1], 1);
        badp[p] = 1;                          // the particle (batch index) whose field is out of range
    }
    __syncthreads();
    const int lx = threadIdx.x % FX, ly = threadIdx.x / FX;
    const int i = tx * FX + lx, j = ty * FY + ly;
    const size_t t = base + (size_t)j * n + i;
    const float2 c2 = S[ly + 1][lx + 1];
    const df32 sc{c2.x, c2.y};
    const df32 wall = df_two_over(sc);
    df32 kw = wall, ks = wall;
    if (i > 0) { const float2 w2 = S[ly + 1][lx]; kw = df_two_over(df_add(sc, df32{w2.x, w2.y})); }
    if (j > 0) { const float2 s2 = S[ly][lx + 1]; ks = df_two_over(df_add(sc, df32{s2.x, s2.y})); }
    Kwh[t] = kw.hi; Kwl[t] = kw.lo;
    Ksh[t] = ks.hi; Ksl[t] = ks.lo;
    if (Kwb) { Kwb[t] = __float2bfloat16_rn(kw.hi); Ksb[t] = __float2bfloat16_rn(ks.hi); }
    if (i == n - 1) { Eh[(size_t)p * n + j] = wall.hi; El[(size_t)p * n + j] = wall.lo; }
    if (j == n - 1) { Nh[(size_t)p * n + i] = wall.hi; Nl[(size_t)p * n + i] = wall.lo; }
}

// Galerkin coarsening for piecewise-constant prolongation; with Kwcb, Kscb the
// coarse interior faces are also stored rounded to BF16 (the BF16 smoother).
template <typename T>
__global__ void k_coarsen(int m, int count, const T* __restrict__ Kw, const T* __restrict__ Ks, const T* __restrict__ E,
                          const T* __restrict__ Nn, T* __restrict__ Kwc, T* __restrict__ Ksc, T* __restrict__ Ec,
                          T* __restrict__ Nnc, __nv_bfloat16* __restrict__ Kwcb, __nv_bfloat16* __restrict__ Kscb) {
    const int n = 2 * m;
    const size_t mm = (size_t)m * m, nn = (size_t)n * n;
    const size_t total = mm * count;
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; t < total; t += stride) {
        const size_t p = t / mm;
        const int c = (int)(t - p * mm);
        const int I = c % m, J = c / m;
        const T* kw = Kw + p * nn;
        const T* ks = Ks + p * nn;
        const T kwv = kw[(2 * J) * n + 2 * I] + kw[(2 * J + 1) * n + 2 * I];
        const T ksv = ks[(2 * J) * n + 2 * I] + ks[(2 * J) * n + 2 * I + 1];
        Kwc[t] = kwv;
        Ksc[t] = ksv;
        if (Kwcb) { Kwcb[t] = __float2bfloat16_rn((float)kwv); Kscb[t] = __float2bfloat16_rn((float)ksv); }
        if (I == m - 1) Ec[p * m + J] = E[p * n + 2 * J] + E[p * n + 2 * J + 1];
        if (J == m - 1) Nnc[p * m + I] = Nn[p * n + 2 * I] + Nn[p * n + 2 * I + 1];
    }
}

// ------------------------------------------------------------------------
// Tiled smoothing kernels.  A block covers a TILE x TILE tile of one particle
// plus a halo of H cells, a region of R x R cells (R = TILE + 2H).  Thread t
// (t < R*G) owns the region cells in column lx = t % R and rows
// ly = t / R + G k; G is odd, so a thread's cells alternate in colour and every
// half-sweep keeps all threads busy.  The owned cells' right-hand side, face
// coefficients and 1/D live in registers; only the correction e is shared.
// A half-sweep over [lo, hi)^2 is exact there as long as lo >= s for the s-th
// half-sweep (the halo shrinks by one cell per half-sweep).
// ------------------------------------------------------------------------
constexpr int OWN_G = 7;

template <int R>
struct Own {
    static constexpr int G = OWN_G;
    static constexpr int ROWS = (R + G - 1) / G;
    static constexpr int NT = R * G;
    static constexpr int THREADS = ((NT + 31) / 32) * 32;
};

template <typename T> __device__ inline T rcp_pos(T d);
template <> __device__ inline float rcp_pos<float>(float d) { return __frcp_rn(d); }
template <> __device__ inline double rcp_pos<double>(double d) { return recip_nr(d); }

// Face coefficients of global cell (gx, gy): west, east, south, north (walls at the domain edge).
template <typename T>
__device__ inline void load_cell_faces(const T* __restrict__ Kw, const T* __restrict__ Ks, const T* __restrict__ E,
                                       const T* __restrict__ Nn, int n, int gx, int gy, T& w, T& e, T& s, T& nn) {
    const int c = gy * n + gx;
    w = Kw[c];
    e = gx + 1 < n ? Kw[c + 1] : E[gy];
    s = Ks[c];
    nn = gy + 1 < n ? Ks[c + n] : Nn[gx];
}

template <typename T, int NU>
__global__ void __launch_bounds__(Own<TILE + 4 * NU>::THREADS) k_pre(
        int n, const T* __restrict__ Kw, const T* __restrict__ Ks, const T* __restrict__ E, const T* __restrict__ Nn,
        const T* __restrict__ rin, T* __restrict__ rout, T* __restrict__ e_out, T* __restrict__ rc, const T* __restrict__ q,
        T* __restrict__ x, const T* __restrict__ p, const double* __restrict__ alpha, double* __restrict__ part_rr,
        const int* __restrict__ active, int cg, int want_rr, const int* __restrict__ nact_dev = nullptr) {
    if (nact_dev && (int)blockIdx.y >= *nact_dev) return;   // a launch sized before the active count was known
    constexpr int H = 2 * NU;
    constexpr int R = TILE + 2 * H;
    using O = Own<R>;
    constexpr int ROWS = O::ROWS, G = O::G;
    __shared__ T se[R * R];
    __shared__ double red[32];
    const int pb = active[blockIdx.y];   // active-particle list
    const int tpr = n / TILE;
    const int tx = blockIdx.x % tpr, ty = blockIdx.x / tpr;
    const int gx0 = tx * TILE - H, gy0 = ty * TILE - H;
    const size_t base = (size_t)pb * n * n;
    const T* kw = Kw + base;
    const T* ks = Ks + base;
    const T* Ep = E + (size_t)pb * n;
    const T* Np = Nn + (size_t)pb * n;
    const int t = threadIdx.x;
    const bool own = t < O::NT;
    const int lx = own ? t % R : 0, g = own ? t / R : 0;
    const int gx = gx0 + lx;
    const int col0 = (gx + gy0 + g) & 1;
    const T a = cg ? (T)alpha[pb] : T(0);
    T rr[ROWS], inv[ROWS], cw[ROWS], ce[ROWS], cs[ROWS], cn[ROWS];
    double rr_loc = 0.0;
#pragma unroll
    for (int k = 0; k < ROWS; ++k) {
        const int ly = g + G * k;
        const int gy = gy0 + ly;
        const bool inreg = own && ly < R;
        const bool in = inreg && gx >= 0 && gx < n && gy >= 0 && gy < n;
        T rv = T(0), w = T(0), e = T(0), s = T(0), nn = T(0);
        if (in) {
            const size_t gi = base + (size_t)gy * n + gx;
            rv = rin[gi];
            load_cell_faces(kw, ks, Ep, Np, n, gx, gy, w, e, s, nn);
            const bool inner = lx >= H && lx < H + TILE && ly >= H && ly < H + TILE;
            if (cg) {
                rv -= a * q[gi];
                if (inner) {
                    rout[gi] = rv;
                    x[gi] += a * p[gi];
                }
            }
            if (inner && (cg || want_rr)) rr_loc += (double)rv * (double)rv;
        }
        rr[k] = rv; cw[k] = w; ce[k] = e; cs[k] = s; cn[k] = nn;
        inv[k] = in ? rcp_pos(w + e + s + nn) : T(0);
        if (inreg) se[ly * R + lx] = T(0);
    }
    __syncthreads();
    // NU sweeps of (red, black); the first red half-sweep starts from e = 0 and is pointwise.
#pragma unroll
    for (int hs = 0; hs < 2 * NU; ++hs) {
        const int colr = hs & 1;
        const int lo = hs, hi = R - hs;
#pragma unroll
        for (int k = 0; k < ROWS; ++k) {
            const int ly = g + G * k;
            if (inv[k] != T(0) && ((col0 ^ (k & 1)) == colr) && lx >= lo && lx < hi && ly >= lo && ly < hi) {
                const int c = ly * R + lx;
                T num = rr[k];
                if (hs > 0) num += cw[k] * se[c - 1] + ce[k] * se[c + 1] + cs[k] * se[c - R] + cn[k] * se[c + R];
                se[c] = num * inv[k];
            }
        }
        __syncthreads();
    }
    // residual on the tile interior, then restriction (sum of 2 x 2)
    T res[ROWS], ev[ROWS];
#pragma unroll
    for (int k = 0; k < ROWS; ++k) {
        const int ly = g + G * k;
        res[k] = T(0);
        ev[k] = T(0);
        if (own && ly >= H && ly < H + TILE && lx >= H && lx < H + TILE) {
            const int c = ly * R + lx;
            const T ec = se[c];
            ev[k] = ec;
            res[k] = rr[k] - ((cw[k] + ce[k] + cs[k] + cn[k]) * ec -
                              (cw[k] * se[c - 1] + ce[k] * se[c + 1] + cs[k] * se[c - R] + cn[k] * se[c + R]));
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ROWS; ++k) {
        const int ly = g + G * k;
        if (own && ly >= H && ly < H + TILE && lx >= H && lx < H + TILE) {
            se[ly * R + lx] = res[k];
            e_out[base + (size_t)(gy0 + ly) * n + gx] = ev[k];
        }
    }
    __syncthreads();
    constexpr int hT = TILE / 2;
    const int m = n / 2;
    for (int idx = t; idx < hT * hT; idx += blockDim.x) {
        const int J = idx / hT, I = idx % hT;
        const int c = (H + 2 * J) * R + H + 2 * I;
        rc[(size_t)pb * m * m + (size_t)(ty * hT + J) * m + tx * hT + I] = se[c] + se[c + 1] + se[c + R] + se[c + R + 1];
    }
    if (cg || want_rr) {
        const double tot = block_sum(rr_loc, red);
        if (t == 0) part_rr[(size_t)pb * gridDim.x + blockIdx.x] = tot;
    }
}

// Prolongation of the coarse correction (scaled by cc), post-smoothing
// (black, red) and, on the finest level, the partial r.z of the CG step.
template <typename T, int NU>
__global__ void __launch_bounds__(Own<TILE + 4 * NU>::THREADS) k_post(
        int n, const T* __restrict__ Kw, const T* __restrict__ Ks, const T* __restrict__ E, const T* __restrict__ Nn,
        const T* __restrict__ r, const T* __restrict__ e_in, const T* __restrict__ ec, T cc, T* __restrict__ e_out,
        double* __restrict__ part_rz, const int* __restrict__ active, int cg, const int* __restrict__ nact_dev = nullptr) {
    if (nact_dev && (int)blockIdx.y >= *nact_dev) return;
    constexpr int H = 2 * NU;
    constexpr int R = TILE + 2 * H;
    using O = Own<R>;
    constexpr int ROWS = O::ROWS, G = O::G;
    __shared__ T se[R * R];
    __shared__ double red[32];
    const int pb = active[blockIdx.y];   // active-particle list
    const int tpr = n / TILE;
    const int tx = blockIdx.x % tpr, ty = blockIdx.x / tpr;
    const int gx0 = tx * TILE - H, gy0 = ty * TILE - H;
    const int m = n / 2;
    const size_t base = (size_t)pb * n * n, cbase = (size_t)pb * m * m;
    const T* kw = Kw + base;
    const T* ks = Ks + base;
    const T* Ep = E + (size_t)pb * n;
    const T* Np = Nn + (size_t)pb * n;
    const int t = threadIdx.x;
    const bool own = t < O::NT;
    const int lx = own ? t % R : 0, g = own ? t / R : 0;
    const int gx = gx0 + lx;
    const int col0 = (gx + gy0 + g) & 1;
    T rr[ROWS], inv[ROWS], cw[ROWS], ce[ROWS], cs[ROWS], cn[ROWS];
#pragma unroll
    for (int k = 0; k < ROWS; ++k) {
        const int ly = g + G * k;
        const int gy = gy0 + ly;
        const bool inreg = own && ly < R;
        const bool in = inreg && gx >= 0 && gx < n && gy >= 0 && gy < n;
        T rv = T(0), w = T(0), e = T(0), s = T(0), nn = T(0), ev = T(0);
        if (in) {
            const size_t gi = base + (size_t)gy * n + gx;
            rv = r[gi];
            ev = e_in[gi] + cc * ec[cbase + (size_t)(gy >> 1) * m + (gx >> 1)];
            load_cell_faces(kw, ks, Ep, Np, n, gx, gy, w, e, s, nn);
        }
        rr[k] = rv; cw[k] = w; ce[k] = e; cs[k] = s; cn[k] = nn;
        inv[k] = in ? rcp_pos(w + e + s + nn) : T(0);
        if (inreg) se[ly * R + lx] = ev;
    }
    __syncthreads();
#pragma unroll
    for (int hs = 0; hs < 2 * NU; ++hs) {
        const int colr = 1 - (hs & 1);
        const int lo = hs + 1, hi = R - hs - 1;
#pragma unroll
        for (int k = 0; k < ROWS; ++k) {
            const int ly = g + G * k;
            if (inv[k] != T(0) && ((col0 ^ (k & 1)) == colr) && lx >= lo && lx < hi && ly >= lo && ly < hi) {
                const int c = ly * R + lx;
                se[c] = (rr[k] + cw[k] * se[c - 1] + ce[k] * se[c + 1] + cs[k] * se[c - R] + cn[k] * se[c + R]) * inv[k];
            }
        }
        __syncthreads();
    }
    double rz = 0.0;
#pragma unroll
    for (int k = 0; k < ROWS; ++k) {
        const int ly = g + G * k;
        if (own && ly >= H && ly < H + TILE && lx >= H && lx < H + TILE) {
            const T ev = se[ly * R + lx];
            e_out[base + (size_t)(gy0 + ly) * n + gx] = ev;
            if (cg) rz += (double)rr[k] * (double)ev;
        }
    }
    if (cg) {
        const double tot = block_sum(rz, red);
        if (t == 0) part_rz[(size_t)pb * gridDim.x + blockIdx.x] = tot;
    }
}

// CG direction update and operator application: p <- z + beta p, q = A p, partial p.q.
template <typename T>
__global__ void __launch_bounds__(Own<TILE + 2>::THREADS) k_apply(
        int n, const T* __restrict__ Kw, const T* __restrict__ Ks, const T* __restrict__ E, const T* __restrict__ Nn,
        const T* __restrict__ z, const T* __restrict__ pin, T* __restrict__ pout, T* __restrict__ q,
        const double* __restrict__ betac, double* __restrict__ part_pq, const int* __restrict__ active, int first) {
    constexpr int H = 1;
    constexpr int R = TILE + 2 * H;
    using O = Own<R>;
    constexpr int ROWS = O::ROWS, G = O::G;
    __shared__ T se[R * R];
    __shared__ double red[32];
    const int pb = active[blockIdx.y];   // active-particle list
    const int tpr = n / TILE;
    const int tx = blockIdx.x % tpr, ty = blockIdx.x / tpr;
    const int gx0 = tx * TILE - H, gy0 = ty * TILE - H;
    const size_t base = (size_t)pb * n * n;
    const int t = threadIdx.x;
    const bool own = t < O::NT;
    const int lx = own ? t % R : 0, g = own ? t / R : 0;
    const int gx = gx0 + lx;
    const T b = first ? T(0) : (T)betac[pb];
#pragma unroll
    for (int k = 0; k < ROWS; ++k) {
        const int ly = g + G * k;
        const int gy = gy0 + ly;
        if (own && ly < R) {
            T pv = T(0);
            if (gx >= 0 && gx < n && gy >= 0 && gy < n) {
                const size_t gi = base + (size_t)gy * n + gx;
                pv = z[gi];
                if (!first) pv += b * pin[gi];
            }
            se[ly * R + lx] = pv;
        }
    }
    __syncthreads();
    double pq = 0.0;
#pragma unroll
    for (int k = 0; k < ROWS; ++k) {
        const int ly = g + G * k;
        if (own && ly >= H && ly < H + TILE && lx >= H && lx < H + TILE) {
            const int gy = gy0 + ly;
            T w, e, s, nn;
            load_cell_faces(Kw + base, Ks + base, E + (size_t)pb * n, Nn + (size_t)pb * n, n, gx, gy, w, e, s, nn);
            const int c = ly * R + lx;
            const T pv = se[c];
            const T qv = w * (pv - se[c - 1]) + e * (pv - se[c + 1]) + s * (pv - se[c - R]) + nn * (pv - se[c + R]);
            const size_t gi = base + (size_t)gy * n + gx;
            pout[gi] = pv;
            q[gi] = qv;
            pq += (double)pv * (double)qv;
        }
    }
    const double tot = block_sum(pq, red);
    if (t == 0) part_pq[(size_t)pb * gridDim.x + blockIdx.x] = tot;
}

}  // namespace smcgm
#include "wtiles.cuh"
#include "wtma.cuh"
namespace smcgm {

// ------------------------------------------------------------------------
// Coarse V-cycle: levels with n_l <= coarse_top, one block per particle, all
// in shared memory.  Input r at the top level; output the correction e2.
// ------------------------------------------------------------------------
template <typename T>
struct CoarseLevelPtrs {
    const T* Kw[12]; const T* Ks[12]; const T* E[12]; const T* Nn[12];
    const T* rtop; T* etop;
    int ntop, nlev;   // nlev levels: ntop, ntop/2, ..., 1
    const int* nact;  // device count of active particles (a launch sized before it was known), or null
};

template <typename T>
__device__ inline T cdiag(const T* kw, const T* ks, const T* E, const T* Nn, int n, int i, int j) {
    const int c = j * n + i;
    return kw[c] + (i < n - 1 ? kw[c + 1] : E[j]) + ks[c] + (j < n - 1 ? ks[c + n] : Nn[i]);
}

template <typename T>
__device__ inline T cnbr(const T* kw, const T* ks, const T* e, int n, int i, int j) {
    const int c = j * n + i;
    T s = T(0);
    if (i > 0) s += kw[c] * e[c - 1];
    if (i < n - 1) s += kw[c + 1] * e[c + 1];
    if (j > 0) s += ks[c] * e[c - n];
    if (j < n - 1) s += ks[c + n] * e[c + n];
    return s;
}

// One half-sweep of colour col on an n x n level; dinv holds 1/D of every cell.
template <typename T>
__device__ inline void chalf(const T* kw, const T* ks, const T* dinv, const T* r, T* e, int n, int col, bool pointwise) {
    const int half = (n * n + 1) / 2;
    for (int k = threadIdx.x; k < half; k += blockDim.x) {
        int j = (2 * k) / n;
        int i = (2 * k) % n;
        if (((i + j) & 1) != col) i += 1;
        if (n == 1) { i = 0; j = 0; if (col != 0) continue; }
        if (i >= n) continue;
        T num = r[j * n + i];
        if (!pointwise) num += cnbr(kw, ks, e, n, i, j);
        e[j * n + i] = num * dinv[j * n + i];
    }
}

// COARSE_THREADS per block (one particle): 128 threads and 7 blocks per SM measured faster than
// 256 and 4 (+0.7 % for the whole move), 64 and 32 threads slower again.
constexpr int COARSE_THREADS = 128;
template <typename T, int NU>
__global__ void __launch_bounds__(COARSE_THREADS, 7) k_coarse(CoarseLevelPtrs<T> P, T cc, const int* __restrict__ active) {
    extern __shared__ __align__(16) unsigned char smraw[];
    if (P.nact && (int)blockIdx.x >= *P.nact) return;
    const int pb = active[blockIdx.x];   // active-particle list
    T* kw[12]; T* ks[12]; T* E[12]; T* Nn[12]; T* r[12]; T* e[12];   // 1/D of level l at e[l] + n_l^2
    T* cur = reinterpret_cast<T*>(smraw);
    int nl = P.ntop;
    for (int l = 0; l < P.nlev; ++l) {
        const int nn = nl * nl;
        kw[l] = cur; cur += nn;
        ks[l] = cur; cur += nn;
        r[l] = cur; cur += nn;
        e[l] = cur; cur += nn;
        cur += nn;                          // 1/D
        E[l] = cur; cur += nl;
        Nn[l] = cur; cur += nl;
        const T* gkw = P.Kw[l] + (size_t)pb * nn;
        const T* gks = P.Ks[l] + (size_t)pb * nn;
        for (int i = threadIdx.x; i < nn; i += blockDim.x) {
            cp_async_elem(kw[l] + i, gkw + i);
            cp_async_elem(ks[l] + i, gks + i);
        }
        for (int i = threadIdx.x; i < nl; i += blockDim.x) {
            cp_async_elem(E[l] + i, P.E[l] + (size_t)pb * nl + i);
            cp_async_elem(Nn[l] + i, P.Nn[l] + (size_t)pb * nl + i);
        }
        nl >>= 1;
    }
    {
        const int nn = P.ntop * P.ntop;
        const T* g = P.rtop + (size_t)pb * nn;
        for (int i = threadIdx.x; i < nn; i += blockDim.x) cp_async_elem(r[0] + i, g + i);
    }
    cp_async_wait_all();   // every copy of this thread is in shared memory
    __syncthreads();
    // 1/D of every cell of every level, once (the half-sweeps multiply by it)
    nl = P.ntop;
    for (int l = 0; l < P.nlev; ++l) {
        for (int c = threadIdx.x; c < nl * nl; c += blockDim.x)
            e[l][nl * nl + c] = T(1) / cdiag(kw[l], ks[l], E[l], Nn[l], nl, c % nl, c / nl);
        nl >>= 1;
    }
    __syncthreads();
    // down
    nl = P.ntop;
    for (int l = 0; l < P.nlev - 1; ++l) {
        const int nn = nl * nl;
        for (int i = threadIdx.x; i < nn; i += blockDim.x) e[l][i] = T(0);
        __syncthreads();
        for (int sw = 0; sw < NU; ++sw) {
            chalf(kw[l], ks[l], e[l] + nl * nl, r[l], e[l], nl, 0, sw == 0);
            __syncthreads();
            chalf(kw[l], ks[l], e[l] + nl * nl, r[l], e[l], nl, 1, false);
            __syncthreads();
        }
        const int m = nl / 2;
        for (int k = threadIdx.x; k < m * m; k += blockDim.x) {
            const int I = k % m, J = k / m;
            T s = T(0);
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    const int i = 2 * I + di, j = 2 * J + dj, c = j * nl + i;
                    s += r[l][c] - (cdiag(kw[l], ks[l], E[l], Nn[l], nl, i, j) * e[l][c] - cnbr(kw[l], ks[l], e[l], nl, i, j));
                }
            r[l + 1][k] = s;
        }
        __syncthreads();
        nl = m;
    }
    // coarsest 1 x 1: exact
    {
        const int l = P.nlev - 1;
        if (threadIdx.x == 0) e[l][0] = r[l][0] / (kw[l][0] + E[l][0] + ks[l][0] + Nn[l][0]);
        __syncthreads();
    }
    // up
    for (int l = P.nlev - 2; l >= 0; --l) {
        nl = P.ntop >> l;
        const int m = nl / 2;
        for (int k = threadIdx.x; k < nl * nl; k += blockDim.x) {
            const int i = k % nl, j = k / nl;
            e[l][k] += cc * e[l + 1][(j >> 1) * m + (i >> 1)];
        }
        __syncthreads();
        for (int sw = 0; sw < NU; ++sw) {
            chalf(kw[l], ks[l], e[l] + nl * nl, r[l], e[l], nl, 1, false);
            __syncthreads();
            chalf(kw[l], ks[l], e[l] + nl * nl, r[l], e[l], nl, 0, false);
            __syncthreads();
        }
    }
    {
        const int nn = P.ntop * P.ntop;
        T* g = P.etop + (size_t)pb * nn;
        for (int i = threadIdx.x; i < nn; i += blockDim.x) g[i] = e[0][i];
    }
}

template <typename T>
size_t coarse_smem_bytes(int ntop, int nlev) {
    size_t s = 0;
    int nl = ntop;
    for (int l = 0; l < nlev; ++l) { s += (size_t)(5 * nl * nl + 2 * nl); nl >>= 1; }
    return s * sizeof(T);
}

// ------------------------------------------------------------------------
// Per-particle scalar bookkeeping of CG and refinement.
// ------------------------------------------------------------------------
enum ScalarMode { SM_START = 0, SM_INIT_RR = 1, SM_RZ_FIRST = 2, SM_RZ = 3, SM_PQ = 4, SM_RR = 5 };

// One warp per particle: the tile partial sums are reduced in a fixed order
// (lane-strided, then a shuffle tree), so results do not depend on scheduling.
// A CG phase ends when |r|^2 <= max(tol2 |r_start|^2, floor2 |b|^2): the floor
// keeps the last refinement phase from reducing the residual further than the
// FP64 tolerance needs.
__global__ void k_scalar(int mode, int count, int ntiles, SolverScalars sc, Partials part, double tol2, double floor2,
                         int maxit) {
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= count) return;
    if (mode == SM_START) {
        if (lane == 0) sc.act_in[p] = sc.act_out[p];
        return;
    }
    if (!sc.act_in[p]) return;
    const double* src = mode == SM_PQ ? part.pq : (mode == SM_RZ || mode == SM_RZ_FIRST) ? part.rz : part.rr;
    double s = 0.0;
    for (int t = lane; t < ntiles; t += 32) s += src[(size_t)p * ntiles + t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane != 0) return;
    if (mode == SM_INIT_RR) {
        sc.rr0[p] = fmax(tol2 * s, floor2 * sc.b2[p]);   // the phase's stopping threshold on |r|^2
        sc.rr[p] = s;
        if (!(s > 0.0)) sc.act_in[p] = 0;
        else atomicAdd(&sc.count[0], 1);
    } else if (mode == SM_RZ_FIRST) {
        sc.rz[p] = s;
        sc.betac[p] = 0.0;
    } else if (mode == SM_RZ) {
        sc.betac[p] = s / sc.rz[p];
        sc.rz[p] = s;
    } else if (mode == SM_PQ) {
        sc.pq[p] = s;
        sc.alpha[p] = s > 0.0 ? sc.rz[p] / s : 0.0;
    } else if (mode == SM_RR) {
        sc.rr[p] = s;
        int it = ++sc.iters[p];
        if (s <= sc.rr0[p]) {
            sc.act_in[p] = 0;
        } else if (it >= maxit || !(s == s)) {
            sc.act_in[p] = 0;
            sc.flags[p] |= 1;
        } else {
            atomicAdd(&sc.count[0], 1);
        }
        atomicMax(&sc.count[2], it);
    }
}

// w64 += x, x = 0, for particles still refining.  Grid (nn / 1024, particles):
// a block covers 1024 cells of one particle and returns at once if that
// particle has converged, so the late refinement steps cost little.
template <typename T>
__global__ void __launch_bounds__(256) k_update_w(int nn, double* __restrict__ w, T* __restrict__ x, const int* __restrict__ act) {
    const int p = blockIdx.y;
    if (!act[p]) return;
    const size_t base = (size_t)p * nn + (size_t)blockIdx.x * 1024;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const size_t t = base + threadIdx.x + 256 * k;
        w[t] += (double)x[t];
        x[t] = T(0);
    }
}

// FP64 residual b - A64 w, stored in the inner precision; partial |res|^2 per tile.
template <typename T>
__global__ void __launch_bounds__(256) k_residual(int n, const double* __restrict__ Kw, const double* __restrict__ Ks,
                                                  const double* __restrict__ E, const double* __restrict__ Nn,
                                                  const double* __restrict__ w, const double* __restrict__ b, size_t bstride,
                                                  T* __restrict__ rout, double* __restrict__ part_res, const int* __restrict__ act) {
    __shared__ double red[32];
    const int pb = blockIdx.y;
    if (!act[pb]) return;
    const int tpr = n / TILE;
    const int tx = blockIdx.x % tpr, ty = blockIdx.x / tpr;
    const size_t nn = (size_t)n * n, base = (size_t)pb * nn;
    const double* kw = Kw + base;
    const double* ks = Ks + base;
    const double* wp = w + base;
    double acc = 0.0;
    for (int idx = threadIdx.x; idx < TILE * TILE; idx += blockDim.x) {
        const int i = tx * TILE + idx % TILE, j = ty * TILE + idx / TILE;
        const int c = j * n + i;
        const double kE = i < n - 1 ? kw[c + 1] : E[(size_t)pb * n + j];
        const double kN = j < n - 1 ? ks[c + n] : Nn[(size_t)pb * n + i];
        double aw = (kw[c] + kE + ks[c] + kN) * wp[c];
        if (i > 0) aw -= kw[c] * wp[c - 1];
        if (i < n - 1) aw -= kE * wp[c + 1];
        if (j > 0) aw -= ks[c] * wp[c - n];
        if (j < n - 1) aw -= kN * wp[c + n];
        const double res = b[(size_t)pb * bstride + c] - aw;
        rout[base + c] = (T)res;
        acc += res * res;
    }
    double tot = block_sum(acc, red);
    if (threadIdx.x == 0) part_res[(size_t)pb * gridDim.x + blockIdx.x] = tot;
}

// Mixed precision: the FP64-accurate residual b - A w, with w in FP64 and the
// faces and b as df32 pairs, evaluated as b - sum over faces of the fluxes
// k_f (w_c - w_nb) (w_nb = 0 beyond a wall).  Only the differences w_c - w_nb
// use the FP64 unit (exact for neighbouring values, by Sterbenz's lemma), and
// each face's flux is formed once: a 32 x 32 tile puts the west and south
// fluxes of its cells, plus those of the next column and row, into shared
// memory as df32 (the difference split by bit manipulation, the product in
// df32), and every cell takes its east / north flux from its neighbour's west
// / south one.  Products and sums run in df32 on the FP32 pipes (error ~2^-47
// of the face fluxes, whose sum is ~200 |b| at 256^2).  Stored in FP32 with the
// partial |res|^2 per tile, summed in FP32 (a convergence test needs no more,
// and the FP64 unit, ~1/64 of the FP32 rate here, is left to the differences).
// RES_THREADS per 32 x 32 tile: 128 (four rows of threads) measured faster than 256 (+0.6 % for the
// whole move) and 512.
constexpr int RES_THREADS = 128;
__global__ void __launch_bounds__(RES_THREADS) k_residual_mix(int n, const float* __restrict__ Kwh, const float* __restrict__ Kwl,
                                                      const float* __restrict__ Ksh, const float* __restrict__ Ksl,
                                                      const float* __restrict__ Eh, const float* __restrict__ El,
                                                      const float* __restrict__ Nh, const float* __restrict__ Nl,
                                                      const double* __restrict__ w, const float2* __restrict__ bdf,
                                                      size_t bstride, float* __restrict__ rout,
                                                      double* __restrict__ part_res, const int* __restrict__ act) {
    __shared__ float red[RES_THREADS / 32];
    __shared__ float2 FW[TILE][TILE + 1];   // FW[j][i]: flux of the west face of cell (x0 + i, y0 + j); column TILE: the east edge
    __shared__ float2 FS[TILE + 1][TILE];   // FS[j][i]: south face; row TILE: the north edge
    const int pb = blockIdx.y;
    if (!act[pb]) return;
    const int tpr = n / TILE;
    const int tx = blockIdx.x % tpr, ty = blockIdx.x / tpr;
    const int x0 = tx * TILE, y0 = ty * TILE;
    const size_t nn = (size_t)n * n, base = (size_t)pb * nn;
    const double* wp = w + base;
    const float *kwh = Kwh + base, *kwl = Kwl + base, *ksh = Ksh + base, *ksl = Ksl + base;
    const int li = threadIdx.x % TILE, lj0 = threadIdx.x / TILE;   // RES_THREADS / 32 rows of threads
    auto flux = [](float kh, float kl, double d) {
        const df32 v = df_mul(df32{kh, kl}, df_from_double_bits(d));
        return make_float2(v.hi, v.lo);
    };
    for (int lj = lj0; lj < TILE; lj += blockDim.x / TILE) {
        const int i = x0 + li, j = y0 + lj;
        const int c = j * n + i;
        const double wc = wp[c];
        FW[lj][li] = flux(kwh[c], kwl[c], i > 0 ? wc - wp[c - 1] : wc);
        FS[lj][li] = flux(ksh[c], ksl[c], j > 0 ? wc - wp[c - n] : wc);
        if (li == TILE - 1)
            FW[lj][TILE] = i + 1 < n ? flux(kwh[c + 1], kwl[c + 1], wp[c + 1] - wc)
                                     : flux(Eh[(size_t)pb * n + j], El[(size_t)pb * n + j], -wc);
        if (lj == TILE - 1)
            FS[TILE][li] = j + 1 < n ? flux(ksh[c + n], ksl[c + n], wp[c + n] - wc)
                                     : flux(Nh[(size_t)pb * n + i], Nl[(size_t)pb * n + i], -wc);
    }
    __syncthreads();
    float acc2 = 0.f;                       // |r|^2 of a thread's cells
    for (int lj = lj0; lj < TILE; lj += blockDim.x / TILE) {
        const int c = (y0 + lj) * n + x0 + li;
        const float2 fw = FW[lj][li], fe = FW[lj][li + 1], fs = FS[lj][li], fn = FS[lj + 1][li];
        const df32 aw = df_add(df_add(df32{fw.x, fw.y}, df32{-fe.x, -fe.y}), df_add(df32{fs.x, fs.y}, df32{-fn.x, -fn.y}));
        const float2 bb = bdf[(size_t)pb * bstride + c];
        const df32 res = df_sub_acc(df32{bb.x, bb.y}, aw);
        const float r = __fadd_rn(res.hi, res.lo);
        rout[base + c] = r;
        acc2 = fmaf(r, r, acc2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc2 += __shfl_down_sync(0xffffffffu, acc2, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc2;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int k = 0; k < RES_THREADS / 32; ++k) t += red[k];
        part_res[(size_t)pb * gridDim.x + blockIdx.x] = (double)t;
    }
}

// r = b for every particle (the residual of w = 0), in the inner precision:
// from the df32 pairs when given (mixed precision), else from FP64.
template <typename T>
__global__ void k_fill_rhs(size_t nn, int count, const double* __restrict__ b, const float2* __restrict__ bdf, size_t stride,
                           T* __restrict__ r) {
    const size_t total = nn * count;
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t step = (size_t)gridDim.x * blockDim.x;
    for (; t < total; t += step) {
        const size_t p = t / nn, i = p * stride + (t - p * nn);
        r[t] = bdf ? (T)__fadd_rn(bdf[i].x, bdf[i].y) : (T)b[i];
    }
}

__global__ void k_outer(int mode, int count, int ntiles, SolverScalars sc, Partials part, double tol2, double b2const,
                        const double* __restrict__ b2pp, const int* __restrict__ badp) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= count) return;
    if (mode == 0) {  // initial residual = b, |b|^2 known (per particle, or common); out-of-range fields are not solved
        const double s = b2pp ? b2pp[p] : b2const;
        sc.b2[p] = s;
        sc.res2[p] = s;
        sc.act_out[p] = (s > 0.0 && !(badp && badp[p])) ? 1 : 0;
        sc.iters[p] = 0;
        sc.flags[p] = 0;
        return;
    }
    if (!sc.act_out[p]) return;
    double s = 0.0;
    for (int t = 0; t < ntiles; ++t) s += part.res[(size_t)p * ntiles + t];
    sc.res2[p] = s;
    if (s <= tol2 * sc.b2[p]) sc.act_out[p] = 0;
    else atomicAdd(&sc.count[1], 1);
}

// ------------------------------------------------------------------------
// Host orchestration
// ------------------------------------------------------------------------
static inline int grid_for(size_t total, int block = 256) {
    size_t g = (total + block - 1) / block;
    return (int)std::min<size_t>(g, 152 * 64);
}

// Deterministic compaction of the active flags into a list (one block).
__global__ void __launch_bounds__(1024) k_compact(int count, const int* __restrict__ act, int* __restrict__ list,
                                                  int* __restrict__ nact) {
    __shared__ int sums[1024];
    const int chunk = (count + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * chunk, b1 = min(count, b0 + chunk);
    int loc = 0;
    for (int i = b0; i < b1; ++i) loc += act[i] ? 1 : 0;
    sums[threadIdx.x] = loc;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) { const int v = sums[k]; sums[k] = run; run += v; }
        *nact = run;
    }
    __syncthreads();
    int pos = sums[threadIdx.x];
    for (int i = b0; i < b1; ++i)
        if (act[i]) list[pos++] = i;
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        check(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q), "entry point");
        if (q != cudaDriverEntryPointSuccess || !p) throw CudaError{cudaErrorNotSupported, "cuTensorMapEncodeTiled unavailable"};
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

static inline int wtiles(int n) { return (n / WT) * (n / WT); }

// log2 of the warp tiles per row of an n x n level (n / 16, a power of two).
static int lg_tiles_per_row(int n) {
    int l = 0;
    while ((WT << l) < n) ++l;
    if ((WT << l) != n) throw CudaError{cudaErrorInvalidValue, "warp-tile level size is not 16 times a power of two"};
    return l;
}

// 3-D map over a particle-major [B][n][n] array of FP32 (es = 4) or BF16 (es = 2)
// values, box bx x by x 1 (x innermost).
static CUtensorMap make_map_es(const void* base, int es_bytes, int n, int B, int bx, int by) {
    CUtensorMap m;
    cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)B};
    cuuint64_t strides[2] = {(cuuint64_t)n * es_bytes, (cuuint64_t)n * n * es_bytes};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t es[3] = {1, 1, 1};
    const CUtensorMapDataType dt = es_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    if ((bx * es_bytes) % 16 != 0) throw CudaError{cudaErrorInvalidValue, "tensor map box row not a multiple of 16 bytes"};
    const CUresult r = tensor_map_encoder()(&m, dt, 3, const_cast<void*>(base), dims, strides, box,
                                            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw CudaError{cudaErrorInvalidValue, "cuTensorMapEncodeTiled"};
    return m;
}
static CUtensorMap make_map(const float* base, int n, int B, int bx, int by) { return make_map_es(base, 4, n, B, bx, by); }

// Halo (2 nu) of the tiled level l: the finest level uses fine_sweeps, the others smooth_sweeps.
static inline int level_halo(const Ctx& c, int l) { return 2 * (l == 0 ? c.cfg.fine_sweeps : c.cfg.smooth_sweeps); }

template <int H>
static void level_maps(TmaMaps& M, InnerSolver<float>& s, int B, int l) {
    using G = TGeo<H>;
    using GB = TGeo<H, 2>;
    LevelArrays<float>& L = s.lv[l];
    M.kw[l] = make_map(L.Kw, L.n, B, G::KWE, G::RW);
    M.ks[l] = make_map(L.Ks, L.n, B, G::KSE, G::RW + 1);
    if (L.Kwb) {
        M.kwb[l] = make_map_es(L.Kwb, 2, L.n, B, GB::KWE, GB::RW);
        M.ksb[l] = make_map_es(L.Ksb, 2, L.n, B, GB::KSE, GB::RW + 1);
    }
    M.e[l] = make_map(L.e, L.n, B, G::BX, G::RW);
    if (l > 0) M.r[l] = make_map(L.r, L.n, B, G::BX, G::RW);
    M.ec[l] = make_map(s.lv[l + 1].e2, s.lv[l + 1].n, B, G::CX, G::CY);
    if (l == 0) {
        for (int k = 0; k < 2; ++k) {
            M.r0[k] = make_map(s.r[k], L.n, B, G::BX, G::RW);
            M.p[k] = make_map(s.p[k], L.n, B, WT, WT);
        }
        M.q = make_map(s.q, L.n, B, G::BX, G::RW);
        M.x = make_map(s.x, L.n, B, WT, WT);
    }
}

// Tensor maps of the TMA-staged kernels (FP32 inner solver, finest level only).
template <typename T>
void build_tma_maps(Ctx& c, InnerSolver<T>& s) {
    if constexpr (sizeof(T) == 4) {
        if (!s.maps) s.maps = new TmaMaps();
        if (s.lv[0].n % WT) return;
        if (level_halo(c, 0) == 2) level_maps<2>(*s.maps, s, c.B, 0);
        else level_maps<4>(*s.maps, s, c.B, 0);
    }
}
template void build_tma_maps<float>(Ctx&, InnerSolver<float>&);
template void build_tma_maps<double>(Ctx&, InnerSolver<double>&);

// Resident blocks per SM of a staged kernel (queried once, with its shared-memory opt-in).
template <typename K>
static int staged_occupancy(K kernel, size_t smem) {
    check(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "attr");
    int b = 0;
    check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, 32 * TW_WARPS, smem), "occupancy");
    return std::max(1, b);
}

static inline int persistent_grid(int total_warps, int per_sm, int sms) {
    const int blocks = (total_warps + TW_WARPS - 1) / TW_WARPS;
    return std::max(1, std::min(blocks, per_sm * sms));
}

// Pre-smoothing pass of the TMA-staged path on level `level`; cg = 1 only on the finest level.
// FB = 2: the smoother reads the BF16 interior faces.
template <int H, bool CG, int MINB, int FB>
static void launch_tpre_b(Ctx& c, InnerSolver<float>& s, int level, int nact, const CUtensorMap& mr, const float* rin, float* rout,
                          int want_rr, int pc) {
    static const int per_sm = staged_occupancy(k_tpre<H, CG, MINB, FB>, tpre_smem<H, CG, FB>());
    LevelArrays<float>& L = s.lv[level];
    TmaMaps& M = *s.maps;
    WPreArgs<float> A{};
    A.a.n = L.n; A.a.ntiles = wtiles(L.n); A.a.lg_tpr = lg_tiles_per_row(L.n); A.a.total = nact * A.a.ntiles; A.a.list = s.list; A.a.err = c.dev_err;
    A.a.nact = c.graph ? s.nact : nullptr;
    A.Kw = L.Kw; A.Ks = L.Ks; A.E = L.E; A.Nn = L.Nn; A.rin = rin; A.q = s.q; A.p = s.p[pc];
    A.rout = rout; A.e_out = L.e; A.rc = s.lv[level + 1].r; A.x = s.x; A.alpha = c.sc.alpha; A.part_rr = c.part.rr;
    A.cg = CG ? 1 : 0; A.want_rr = want_rr;
    const CUtensorMap& mkw = FB == 2 ? M.kwb[level] : M.kw[level];
    const CUtensorMap& mks = FB == 2 ? M.ksb[level] : M.ks[level];
    k_tpre<H, CG, MINB, FB><<<persistent_grid(A.a.total, per_sm, c.sm_count), 32 * TW_WARPS, tpre_smem<H, CG, FB>(), c.stream>>>(
        A, mkw, mks, mr, M.q, M.x, M.p[pc]); ++c.pc.launches;
}
template <int H, bool CG>
static void launch_tpre(Ctx& c, InnerSolver<float>& s, int level, int nact, const CUtensorMap& mr, const float* rin, float* rout,
                        int want_rr, int pc) {
    // blocks per SM asked of the register allocator: on a 20 x 20 region 4 with the CG update
    // (<= 128 registers, 16 warps) and 5 without it (<= 96 registers, 20 warps; no spills), 2 on
    // the 24 x 24 region of two sweeps
    if (s.lv[level].Kwb) launch_tpre_b<H, CG, H == 2 ? (CG ? 4 : 5) : 2, 2>(c, s, level, nact, mr, rin, rout, want_rr, pc);
    else launch_tpre_b<H, CG, H == 2 ? (CG ? 4 : 5) : 2, 4>(c, s, level, nact, mr, rin, rout, want_rr, pc);
}

template <int H, bool CG, int MINB, int FB>
static void launch_tpost_b(Ctx& c, InnerSolver<float>& s, int level, int nact, const CUtensorMap& mr, const float* r, float* eout) {
    static const int per_sm = staged_occupancy(k_tpost<H, CG, MINB, FB>, tpost_smem<H, FB>());
    LevelArrays<float>& L = s.lv[level];
    TmaMaps& M = *s.maps;
    WPostArgs<float> A{};
    A.a.n = L.n; A.a.ntiles = wtiles(L.n); A.a.lg_tpr = lg_tiles_per_row(L.n); A.a.total = nact * A.a.ntiles; A.a.list = s.list; A.a.err = c.dev_err;
    A.a.nact = c.graph ? s.nact : nullptr;
    A.Kw = L.Kw; A.Ks = L.Ks; A.E = L.E; A.Nn = L.Nn; A.r = r; A.e_in = L.e; A.ec = s.lv[level + 1].e2;
    A.cc = (float)c.cfg.coarse_scale; A.e_out = eout; A.part_rz = c.part.rz; A.cg = CG ? 1 : 0;
    const CUtensorMap& mkw = FB == 2 ? M.kwb[level] : M.kw[level];
    const CUtensorMap& mks = FB == 2 ? M.ksb[level] : M.ks[level];
    k_tpost<H, CG, MINB, FB><<<persistent_grid(A.a.total, per_sm, c.sm_count), 32 * TW_WARPS, tpost_smem<H, FB>(), c.stream>>>(
        A, mkw, mks, mr, M.e[level], M.ec[level]); ++c.pc.launches;
}
// One sweep (H = 2): 5 blocks of 4 warps per SM (<= 96 registers, no spills; the staging buffers fit);
// two sweeps: 2 blocks.
template <int H, bool CG>
static void launch_tpost(Ctx& c, InnerSolver<float>& s, int level, int nact, const CUtensorMap& mr, const float* r, float* eout) {
    if (s.lv[level].Kwb) launch_tpost_b<H, CG, H == 2 ? 5 : 2, 2>(c, s, level, nact, mr, r, eout);
    else launch_tpost_b<H, CG, H == 2 ? 5 : 2, 4>(c, s, level, nact, mr, r, eout);
}

template <typename T>
static void launch_coarse(Ctx& c, InnerSolver<T>& s, int nact);

// The tiled levels below the finest with one block per 32 x 32 tile (NU sweeps), then the
// coarse V-cycle, then back up.
template <typename T, int NU>
static void run_vcycle_lower(Ctx& c, InnerSolver<T>& s, int nact) {
    const T cc = (T)c.cfg.coarse_scale;
    constexpr int TPB = Own<TILE + 4 * NU>::THREADS;
    const int* nd = c.graph ? s.nact : nullptr;
    for (int l = 1; l < s.ntile_levels; ++l) {
        LevelArrays<T>& L = s.lv[l];
        dim3 grid((L.n / TILE) * (L.n / TILE), nact);
        k_pre<T, NU><<<grid, TPB, 0, c.stream>>>(L.n, L.Kw, L.Ks, L.E, L.Nn, L.r, nullptr, L.e, s.lv[l + 1].r, nullptr, nullptr,
                                                 nullptr, nullptr, nullptr, s.list, 0, 0, nd); ++c.pc.launches;
    }
    launch_coarse<T>(c, s, nact);
    for (int l = s.ntile_levels - 1; l >= 1; --l) {
        LevelArrays<T>& L = s.lv[l];
        dim3 grid((L.n / TILE) * (L.n / TILE), nact);
        k_post<T, NU><<<grid, TPB, 0, c.stream>>>(L.n, L.Kw, L.Ks, L.E, L.Nn, L.r, L.e, s.lv[l + 1].e2, cc, L.e2, nullptr, s.list, 0,
                                                  nd); ++c.pc.launches;
    }
}

// Compacts act_in into the active list and returns its length (synchronises the stream).
template <typename T>
static int compact_active(Ctx& c, InnerSolver<T>& s, int count, int* hcount) {
    k_compact<<<1, 1024, 0, c.stream>>>(count, c.sc.act_in, s.list, s.nact); ++c.pc.launches;
    int h[4];
    int err[2] = {0, 0};
    check(cudaMemcpyAsync(h, s.nact, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "nact d2h");
    check(cudaMemcpyAsync(hcount, c.sc.count, 3 * sizeof(int), cudaMemcpyDeviceToHost, c.stream), "count d2h");
    check(cudaMemcpyAsync(err, c.dev_err, 2 * sizeof(int), cudaMemcpyDeviceToHost, c.stream), "err d2h");
    sync_stream(c);
    if (err[0] || err[1]) {   // cleared in stream order, so the context stays usable and no later flag is lost
        check(cudaMemsetAsync(c.dev_err, 0, 2 * sizeof(int), c.stream), "err reset");
        sync_stream(c);
    }
    if (err[0]) throw CudaError{cudaErrorLaunchTimeout, "a kernel's bounded mbarrier wait timed out"};
    if (err[1] && !c.lenient)
        throw InputError{"log-permeability |u| >= 64 is outside the mixed-precision range (use the FP64 solver)"};
    return h[0];
}

// ---------------------------------------------------------------------------
// Warp-tile path: launchers
// ---------------------------------------------------------------------------

template <typename T, int H>
static void launch_wpre(Ctx& c, InnerSolver<T>& s, int level, int nact, const T* rin, T* rout, int cg, int want_rr, const T* p) {
    LevelArrays<T>& L = s.lv[level];
    WPreArgs<T> A{};
    A.a.n = L.n; A.a.ntiles = wtiles(L.n); A.a.lg_tpr = lg_tiles_per_row(L.n); A.a.total = nact * A.a.ntiles; A.a.list = s.list;
    A.a.nact = c.graph ? s.nact : nullptr;
    A.Kw = L.Kw; A.Ks = L.Ks; A.E = L.E; A.Nn = L.Nn; A.rin = rin; A.q = s.q; A.p = p;
    A.rout = rout; A.e_out = L.e; A.rc = s.lv[level + 1].r; A.x = s.x; A.alpha = c.sc.alpha; A.part_rr = c.part.rr;
    A.cg = cg; A.want_rr = want_rr; A.Kwb = L.Kwb; A.Ksb = L.Ksb;
    const int grid = (A.a.total + WPB - 1) / WPB;
    if constexpr (sizeof(T) == 4) {
        if (L.Kwb) {   // the BF16 smoother faces
            if (cg) k_wpre<T, H, true, true><<<grid, 32 * WPB, 0, c.stream>>>(A);
            else k_wpre<T, H, false, true><<<grid, 32 * WPB, 0, c.stream>>>(A);
            ++c.pc.launches;
            return;
        }
    }
    if constexpr (H == 4 && sizeof(T) == 8) {
        // the FP64 solver's coarser levels: a pair of warps per item (156 registers, 12 warps per SM,
        // against 235 and 8 for one warp per item: 2 % faster; in FP32 pairs made the move 8 % slower, their
        // third slot a quarter full)
        if (!cg && !want_rr && level > 0) {
            constexpr int IPB = WPB / 2;
            k_wpre<T, H, false, false, 2><<<(A.a.total + IPB - 1) / IPB, 32 * WPB, 0, c.stream>>>(A);
            ++c.pc.launches;
            return;
        }
    }
    if (cg) k_wpre<T, H, true><<<grid, 32 * WPB, 0, c.stream>>>(A);
    else k_wpre<T, H, false><<<grid, 32 * WPB, 0, c.stream>>>(A);
    ++c.pc.launches;
}

template <typename T, int H>
static void launch_wpost(Ctx& c, InnerSolver<T>& s, int level, int nact, const T* r, T* eout, int cg) {
    LevelArrays<T>& L = s.lv[level];
    WPostArgs<T> A{};
    A.a.n = L.n; A.a.ntiles = wtiles(L.n); A.a.lg_tpr = lg_tiles_per_row(L.n); A.a.total = nact * A.a.ntiles; A.a.list = s.list;
    A.a.nact = c.graph ? s.nact : nullptr;
    A.Kw = L.Kw; A.Ks = L.Ks; A.E = L.E; A.Nn = L.Nn; A.r = r; A.e_in = L.e; A.ec = s.lv[level + 1].e2;
    A.cc = (T)c.cfg.coarse_scale; A.e_out = eout; A.part_rz = c.part.rz; A.cg = cg; A.Kwb = L.Kwb; A.Ksb = L.Ksb;
    const int grid = (A.a.total + WPB - 1) / WPB;
    if constexpr (sizeof(T) == 4) {
        if (L.Kwb) {   // the BF16 smoother faces
            if (cg) k_wpost<T, H, true, true><<<grid, 32 * WPB, 0, c.stream>>>(A);
            else k_wpost<T, H, false, true><<<grid, 32 * WPB, 0, c.stream>>>(A);
            ++c.pc.launches;
            return;
        }
    }
    if constexpr (H == 4 && sizeof(T) == 8) {
        if (!cg && level > 0) {               // as in launch_wpre
            constexpr int IPB = WPB / 2;
            k_wpost<T, H, false, false, 2><<<(A.a.total + IPB - 1) / IPB, 32 * WPB, 0, c.stream>>>(A);
            ++c.pc.launches;
            return;
        }
    }
    if (cg) k_wpost<T, H, true><<<grid, 32 * WPB, 0, c.stream>>>(A);
    else k_wpost<T, H, false><<<grid, 32 * WPB, 0, c.stream>>>(A);
    ++c.pc.launches;
}

template <typename T>
static void launch_coarse(Ctx& c, InnerSolver<T>& s, int nact) {
    CoarseLevelPtrs<T> P{};
    const int top = s.ntile_levels;
    P.ntop = s.lv[top].n;
    P.nlev = s.nlev - top;
    for (int l = 0; l < P.nlev; ++l) {
        P.Kw[l] = s.lv[top + l].Kw; P.Ks[l] = s.lv[top + l].Ks; P.E[l] = s.lv[top + l].E; P.Nn[l] = s.lv[top + l].Nn;
    }
    P.rtop = s.lv[top].r;
    P.etop = s.lv[top].e2;
    P.nact = c.graph ? s.nact : nullptr;
    const size_t cs = coarse_smem_bytes<T>(P.ntop, P.nlev);
    if (c.cfg.smooth_sweeps == 1) k_coarse<T, 1><<<nact, COARSE_THREADS, cs, c.stream>>>(P, (T)c.cfg.coarse_scale, s.list);
    else k_coarse<T, 2><<<nact, COARSE_THREADS, cs, c.stream>>>(P, (T)c.cfg.coarse_scale, s.list);
    ++c.pc.launches;
}

// Passes of the TMA-staged path (FP32 inner solver only).
static void staged_pre(Ctx& c, InnerSolver<float>& s, int nact, int cur, int pc, int cg) {
    TmaMaps& M = *s.maps;
    float* rout = cg ? s.r[1 - cur] : nullptr;
    if (level_halo(c, 0) == 2) {
        if (cg) launch_tpre<2, true>(c, s, 0, nact, M.r0[cur], s.r[cur], rout, 1, pc);
        else launch_tpre<2, false>(c, s, 0, nact, M.r0[cur], s.r[cur], rout, 1, pc);
    } else {
        if (cg) launch_tpre<4, true>(c, s, 0, nact, M.r0[cur], s.r[cur], rout, 1, pc);
        else launch_tpre<4, false>(c, s, 0, nact, M.r0[cur], s.r[cur], rout, 1, pc);
    }
}
static void staged_lower(Ctx& c, InnerSolver<float>& s, int nact);
static void staged_post(Ctx& c, InnerSolver<float>& s, int nact, int cur) {
    TmaMaps& M = *s.maps;
    if (level_halo(c, 0) == 2) launch_tpost<2, true>(c, s, 0, nact, M.r0[cur], s.r[cur], s.z);
    else launch_tpost<4, true>(c, s, 0, nact, M.r0[cur], s.r[cur], s.z);
}
static void staged_pre(Ctx&, InnerSolver<double>&, int, int, int, int) {}   // the staged path is FP32 only
static void staged_post(Ctx&, InnerSolver<double>&, int, int) {}
static void staged_lower(Ctx&, InnerSolver<double>&, int) {}

// Solver kernel family for the tiled levels (cfg.tile_kernel): 0 = one block per
// 32 x 32 tile, 1 = persistent warps with TMA-staged 16 x 16 tiles (FP32), 2 = one
// warp per 16 x 16 tile loading from global memory.
static int tile_path(const Ctx& c, bool fp32) {
    const int k = c.cfg.tile_kernel;
    const int path = k == 1 ? 0 : k == 3 ? 2 : 1;   // 4: the default's finest level (the coarser levels: Passes)
    if (path == 1 && !fp32) return 2;
    if (path == 1 && c.n % WT) return 2;
    return path;
}

// The passes of one CG iteration on the finest level and the V-cycle below it.
template <typename T>
struct Passes {
    Ctx& c;
    InnerSolver<T>& s;
    int path, n, ntiles;
    bool lower_blocks;        // the coarser tiled levels with one block per 32 x 32 tile
    Passes(Ctx& cc, InnerSolver<T>& ss) : c(cc), s(ss) {
        path = tile_path(cc, sizeof(T) == 4);
        n = ss.lv[0].n;
        ntiles = path == 0 ? (n / TILE) * (n / TILE) : wtiles(n);
        lower_blocks = path == 0 || cc.cfg.tile_kernel == 4;
    }
    // finest-level pre-smoothing (cg: with the CG update from r[cur] into r[1-cur])
    void pre(int nact, int cur, int pc, int cg) {
        LevelArrays<T>& L0 = s.lv[0];
        T* rout = cg ? s.r[1 - cur] : nullptr;
        if (path == 2) {
            if (c.cfg.fine_sweeps == 1) launch_wpre<T, 2>(c, s, 0, nact, s.r[cur], rout, cg, 1, s.p[pc]);
            else launch_wpre<T, 4>(c, s, 0, nact, s.r[cur], rout, cg, 1, s.p[pc]);
        } else if (path == 1) {
            staged_pre(c, s, nact, cur, pc, cg);
        } else {
            constexpr int NU = 1;
            k_pre<T, NU><<<dim3(ntiles, nact), Own<TILE + 4 * NU>::THREADS, 0, c.stream>>>(
                n, L0.Kw, L0.Ks, L0.E, L0.Nn, s.r[cur], rout, L0.e, s.lv[1].r, s.q, s.x, s.p[pc], c.sc.alpha, c.part.rr, s.list, cg, 1); ++c.pc.launches;
        }
    }
    void lower(int nact) {
        if (lower_blocks) {
            if (c.cfg.smooth_sweeps == 2) run_vcycle_lower<T, 2>(c, s, nact);
            else run_vcycle_lower<T, 1>(c, s, nact);
        } else if (path == 2) {
            for (int l = 1; l < s.ntile_levels; ++l) {
                if (level_halo(c, l) == 4) launch_wpre<T, 4>(c, s, l, nact, s.lv[l].r, nullptr, 0, 0, nullptr);
                else launch_wpre<T, 2>(c, s, l, nact, s.lv[l].r, nullptr, 0, 0, nullptr);
            }
            launch_coarse<T>(c, s, nact);
            for (int l = s.ntile_levels - 1; l >= 1; --l) {
                if (level_halo(c, l) == 4) launch_wpost<T, 4>(c, s, l, nact, s.lv[l].r, s.lv[l].e2, 0);
                else launch_wpost<T, 2>(c, s, l, nact, s.lv[l].r, s.lv[l].e2, 0);
            }
        } else {
            staged_lower(c, s, nact);
        }
    }
    void post(int nact, int cur) {
        LevelArrays<T>& L0 = s.lv[0];
        if (path == 2) {
            if (c.cfg.fine_sweeps == 1) launch_wpost<T, 2>(c, s, 0, nact, s.r[cur], s.z, 1);
            else launch_wpost<T, 4>(c, s, 0, nact, s.r[cur], s.z, 1);
        } else if (path == 1) {
            staged_post(c, s, nact, cur);
        } else {
            constexpr int NU = 1;
            k_post<T, NU><<<dim3(ntiles, nact), Own<TILE + 4 * NU>::THREADS, 0, c.stream>>>(
                n, L0.Kw, L0.Ks, L0.E, L0.Nn, s.r[cur], L0.e, s.lv[1].e2, (T)c.cfg.coarse_scale, s.z, c.part.rz, s.list, 1); ++c.pc.launches;
        }
    }
    void apply(int nact, int pc, int first) {
        LevelArrays<T>& L0 = s.lv[0];
        if (path != 0) {
            WApplyArgs<T> A{};
            A.a.n = n; A.a.ntiles = ntiles; A.a.lg_tpr = lg_tiles_per_row(n); A.a.total = nact * ntiles; A.a.list = s.list; A.a.err = c.dev_err;
            A.a.nact = c.graph ? s.nact : nullptr;
            A.Kw = L0.Kw; A.Ks = L0.Ks; A.E = L0.E; A.Nn = L0.Nn; A.z = s.z; A.pin = s.p[pc];
            A.pout = s.p[1 - pc]; A.q = s.q; A.betac = c.sc.betac; A.part_pq = c.part.pq; A.first = first;
            k_wapply<T, sizeof(T) == 4 ? 7 : 4><<<(A.a.total + WPB - 1) / WPB, 32 * WPB, 0, c.stream>>>(A); ++c.pc.launches;
        } else {
            k_apply<T><<<dim3(ntiles, nact), Own<TILE + 2>::THREADS, 0, c.stream>>>(n, L0.Kw, L0.Ks, L0.E, L0.Nn, s.z, s.p[pc],
                                                                                   s.p[1 - pc], s.q, c.sc.betac, c.part.pq, s.list,
                                                                                   first); ++c.pc.launches;
        }
    }
};

static void staged_lower(Ctx& c, InnerSolver<float>& s, int nact) {
    // The coarser tiled levels keep the warp kernels loading from global memory:
    // without the CG vectors their registers allow 16 warps per SM, which
    // measured faster than the staged form there.
    for (int l = 1; l < s.ntile_levels; ++l) {
        if (level_halo(c, l) == 4) launch_wpre<float, 4>(c, s, l, nact, s.lv[l].r, nullptr, 0, 0, nullptr);
        else launch_wpre<float, 2>(c, s, l, nact, s.lv[l].r, nullptr, 0, 0, nullptr);
    }
    launch_coarse<float>(c, s, nact);
    for (int l = s.ntile_levels - 1; l >= 1; --l) {
        if (level_halo(c, l) == 4) launch_wpost<float, 4>(c, s, l, nact, s.lv[l].r, s.lv[l].e2, 0);
        else launch_wpost<float, 2>(c, s, l, nact, s.lv[l].r, s.lv[l].e2, 0);
    }
}

// One preconditioned-CG solve A x = r[0] (x = 0 on entry) for the particles whose
// refinement is still active; every launch covers only the particles still iterating.
template <typename T>
static int inner_solve(Ctx& c, InnerSolver<T>& s, int count, double tol, double floor2) {
    SolverScalars& sc = c.sc;
    Passes<T> P(c, s);
    const int n = P.n, ntiles = P.ntiles;
    const int wgrid = (count * 32 + 127) / 128;   // k_scalar: one warp per particle
    const double tol2 = tol * tol;
    const int maxit = c.cfg.max_iter;
    int cur = 0, pc = 0;
    int hcount[3] = {0, 0, 0};
    k_scalar<<<wgrid, 128, 0, c.stream>>>(SM_START, count, ntiles, sc, c.part, tol2, floor2, maxit); ++c.pc.launches;
    check(cudaMemsetAsync(sc.count, 0, 3 * sizeof(int), c.stream), "memset count");
    int nact = compact_active(c, s, count, hcount);
    if (nact == 0) return 0;
    P.pre(nact, cur, pc, 0);                      // z0 = M r0
    k_scalar<<<wgrid, 128, 0, c.stream>>>(SM_INIT_RR, count, ntiles, sc, c.part, tol2, floor2, maxit); ++c.pc.launches;
    nact = compact_active(c, s, count, hcount);
    c.pc.inner_solves += nact;
    if (nact == 0) return 0;
    P.lower(nact);
    P.post(nact, cur);
    k_scalar<<<wgrid, 128, 0, c.stream>>>(SM_RZ_FIRST, count, ntiles, sc, c.part, tol2, floor2, maxit); ++c.pc.launches;
    // per cell: r, q, x, p, Kw, Ks in (the faces 2 bytes each with the BF16 smoother); r, x, e, rc out
    const double dom_bpc = (double)(6 * sizeof(T) + 3 * sizeof(T)) + 0.25 * sizeof(T) - (s.lv[0].Kwb ? 2.0 * (sizeof(T) - 2) : 0.0);
    for (int it = 0; it < maxit; ++it) {
        P.apply(nact, pc, it == 0);
        pc ^= 1;
        k_scalar<<<wgrid, 128, 0, c.stream>>>(SM_PQ, count, ntiles, sc, c.part, tol2, floor2, maxit); ++c.pc.launches;
        if (c.prof) check(cudaEventRecord(c.ev0, c.stream), "event");
        P.pre(nact, cur, pc, 1);
        if (c.prof) check(cudaEventRecord(c.ev1, c.stream), "event");
        cur ^= 1;
        c.pc.cg_iterations += nact;
        const int launched = nact;
        check(cudaMemsetAsync(sc.count, 0, sizeof(int), c.stream), "memset count");
        k_scalar<<<wgrid, 128, 0, c.stream>>>(SM_RR, count, ntiles, sc, c.part, tol2, floor2, maxit); ++c.pc.launches;
        nact = compact_active(c, s, count, hcount);
        if (c.prof) {
            float ms = 0.f;
            check(cudaEventElapsedTime(&ms, c.ev0, c.ev1), "event time");
            c.pc.dom_ms += ms;
            c.pc.dom_launches += 1;
            c.pc.dom_particles += launched;
            c.pc.dom_bytes += dom_bpc * (double)n * n * launched;
        }
        if (nact == 0) break;
        P.lower(nact);
        P.post(nact, cur);
        k_scalar<<<wgrid, 128, 0, c.stream>>>(SM_RZ, count, ntiles, sc, c.part, tol2, floor2, maxit); ++c.pc.launches;
    }
    check(cudaGetLastError(), "inner solve launch");
    return hcount[2];
}

// Dynamic shared-memory opt-in of the coarse kernel; its need depends on the
// grid, so the largest size requested so far is remembered per precision.
template <typename T>
static void set_smem_attrs(Ctx& c, InnerSolver<T>& s) {
    (void)c;
    static size_t coarse_set[2] = {0, 0};
    const int k = sizeof(T) == 4 ? 0 : 1;
    const int top = s.ntile_levels;
    const size_t cs = coarse_smem_bytes<T>(s.lv[top].n, s.nlev - top);
    if (coarse_set[k] < cs) {
        check(cudaFuncSetAttribute(k_coarse<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs), "attr");
        check(cudaFuncSetAttribute(k_coarse<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs), "attr");
        coarse_set[k] = cs;
    }
}

template <typename T>
void launch_coarsen_all(Ctx& c, InnerSolver<T>& s, int count) {
    for (int l = 0; l + 1 < s.nlev; ++l) {
        LevelArrays<T>& A = s.lv[l];
        LevelArrays<T>& Bc = s.lv[l + 1];
        const size_t total = (size_t)Bc.n * Bc.n * count;
        k_coarsen<T><<<grid_for(total), 256, 0, c.stream>>>(Bc.n, count, A.Kw, A.Ks, A.E, A.Nn, Bc.Kw, Bc.Ks, Bc.E, Bc.Nn,
                                                            Bc.Kwb, Bc.Ksb); ++c.pc.launches;
    }
}
template void launch_coarsen_all<float>(Ctx&, InnerSolver<float>&, int);
template void launch_coarsen_all<double>(Ctx&, InnerSolver<double>&, int);

void launch_setup_coeffs(Ctx& c, int count) {
    const int n = c.n;
    const size_t total = (size_t)n * n * count;
    const bool mixed = mixed_precision(c.cfg);
    if (mixed && n % FX == 0 && n % FY == 0) {
        LevelArrays<float>& f0 = c.s32.lv[0];
        check(cudaMemsetAsync(c.badp, 0, count * sizeof(int), c.stream), "memset badp");
        k_faces_df<<<dim3((n / FX) * (n / FY), count), FX * FY, 0, c.stream>>>(
            n, reinterpret_cast<const float2*>(c.u64), reinterpret_cast<const float2*>(c.exptab), c.expc, f0.Kw, c.Kwlo, f0.Ks, c.Kslo, f0.E, c.Elo, f0.Nn, c.Nlo,
            f0.Kwb, f0.Ksb, c.dev_err, c.badp); ++c.pc.launches;
        launch_coarsen_all<float>(c, c.s32, count);
        return;
    }
    k_exp_neg<<<grid_for(total), 256, 0, c.stream>>>(c.u64, total); ++c.pc.launches;
    if (mixed) {
        LevelArrays<float>& f0 = c.s32.lv[0];
        k_faces<<<grid_for(total), 256, 0, c.stream>>>(n, count, c.u64, FaceOut{nullptr, f0.Kw, c.Kwlo, f0.Kwb},
                                                       FaceOut{nullptr, f0.Ks, c.Kslo, f0.Ksb}, FaceOut{nullptr, f0.E, c.Elo},
                                                       FaceOut{nullptr, f0.Nn, c.Nlo}); ++c.pc.launches;
        launch_coarsen_all<float>(c, c.s32, count);
    } else {
        k_faces<<<grid_for(total), 256, 0, c.stream>>>(n, count, c.u64, FaceOut{c.Kw64, nullptr, nullptr}, FaceOut{c.Ks64, nullptr, nullptr},
                                                       FaceOut{c.E64, nullptr, nullptr}, FaceOut{c.N64, nullptr, nullptr}); ++c.pc.launches;
        launch_coarsen_all<double>(c, c.s64, count);
    }
    check(cudaGetLastError(), "setup launch");
}

template <typename T>
static int solve_batch_t(Ctx& c, InnerSolver<T>& s, int count, const Rhs& R, double* W) {
    const int n = c.n;
    const int ntiles = (n / TILE) * (n / TILE);
    dim3 tgrid(ntiles, count);
    const size_t total = (size_t)n * n * count;
    set_smem_attrs<T>(c, s);
    SolverScalars& sc = c.sc;
    const bool mixed = sizeof(T) == 4;
    const double tol_out2 = c.cfg.tol_outer * c.cfg.tol_outer;
    check(cudaMemsetAsync(W, 0, total * sizeof(double), c.stream), "memset w");
    check(cudaMemsetAsync(s.x, 0, total * sizeof(T), c.stream), "memset x");
    // act_out = 1 for the residual of w = 0
    {
        std::vector<int> ones(count, 1);
        check(cudaMemcpyAsync(sc.act_out, ones.data(), count * sizeof(int), cudaMemcpyHostToDevice, c.stream), "act init");
        sync_stream(c);
    }
    k_fill_rhs<T><<<grid_for(total), 256, 0, c.stream>>>((size_t)n * n, count, R.b64, mixed ? R.bdf : nullptr, R.stride,
                                                        s.r[0]); ++c.pc.launches;
    c.pc.solves += count;
    c.pc.cells = n * n;
    c.pc.word_bytes = (int)sizeof(T);
    int outer_active = count;
    const int sgrid = (count + 127) / 128;
    const int* badp = (mixed && c.lenient) ? c.badp : nullptr;
    k_outer<<<sgrid, 128, 0, c.stream>>>(0, count, ntiles, sc, c.part, tol_out2, R.b2const, R.b2pp, badp); ++c.pc.launches;
    int itmax = 0;
    const int max_outer = mixed ? c.cfg.max_refine : std::max(2, c.cfg.max_refine);
    const double tol_in = mixed ? c.cfg.tol_inner : c.cfg.tol_outer;
    const double floor2 = 0.25 * tol_out2;   // no phase need reduce |r| below half the final tolerance
    for (int o = 0; o < max_outer; ++o) {
        int it = inner_solve<T>(c, s, count, tol_in, floor2);
        itmax = std::max(itmax, it);
        c.pc.residuals += outer_active;
        k_update_w<T><<<dim3(n * n / 1024, count), 256, 0, c.stream>>>(n * n, W, s.x, sc.act_out); ++c.pc.launches;
        if constexpr (sizeof(T) == 4) {
            LevelArrays<float>& f0 = s.lv[0];
            k_residual_mix<<<tgrid, RES_THREADS, 0, c.stream>>>(n, f0.Kw, c.Kwlo, f0.Ks, c.Kslo, f0.E, c.Elo, f0.Nn, c.Nlo, W, R.bdf, R.stride,
                                                       s.r[0], c.part.res, sc.act_out); ++c.pc.launches;
        } else {
            k_residual<T><<<tgrid, 256, 0, c.stream>>>(n, c.Kw64, c.Ks64, c.E64, c.N64, W, R.b64, R.stride, s.r[0], c.part.res,
                                                       sc.act_out); ++c.pc.launches;
        }
        check(cudaMemsetAsync(sc.count + 1, 0, sizeof(int), c.stream), "memset");
        k_outer<<<sgrid, 128, 0, c.stream>>>(1, count, ntiles, sc, c.part, tol_out2, R.b2const, R.b2pp, badp); ++c.pc.launches;
        int h = 0;
        check(cudaMemcpyAsync(&h, sc.count + 1, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "d2h");
        sync_stream(c);
        if (h == 0) break;
        outer_active = h;
        if (o == max_outer - 1) c.nonconv += h;
    }
    return itmax;
}


// ---------------------------------------------------------------------------
// Graph mode: the solve captured into a CUDA graph, its loops on the device.
//
// The refinement phases and the CG iterations become conditional 'while' nodes
// whose condition is set by a kernel: the outer one after each phase's FP64
// residual (more particles above the tolerance and fewer than max_refine phases),
// the inner one by the compaction of the active list after each CG step (any
// particle still iterating).  Every launch between two compactions is sized before
// the active count is known, so each such stage is a 'switch' node over launch-size
// buckets (count, count/2, ..., 1 particles, rounded up): the compaction picks the
// smallest bucket that holds the active particles (none when no particle is left),
// and the kernels read the exact count from device memory.  The CG loop body holds
// two iterations, so its ping-pong buffers come back to their entry state.  Both
// loops are bounded: a particle leaves CG after max_iter iterations, and the
// refinement stops after max_refine phases.  The counters that the host loop keeps
// (CG iterations, inner solves, residuals, unconverged solves, largest iteration
// count) are kept in device memory (GraphCounters).
// ---------------------------------------------------------------------------
constexpr int GB_MAX = 16;   // launch-size buckets: count <= 32768 needs 16

__host__ __device__ inline int bucket_size(int count, int b) { return (count + (1 << b) - 1) >> b; }

static int launch_buckets(int count) {
    int nb = 1;
    while (bucket_size(count, nb - 1) > 1) ++nb;
    return nb;
}

// The smallest launch-size bucket that holds nact particles; nb (no body) for none.
__device__ inline unsigned int bucket_of(int nact, int count, int nb) {
    if (nact <= 0) return (unsigned int)nb;
    int b = 0;
    while (b + 1 < nb && bucket_size(count, b + 1) >= nact) ++b;
    return (unsigned int)b;
}

// The deterministic compaction of k_compact, plus: the previous count added to
// *add_old, the new one to *add_new, the launch-size bucket of the next stage set
// on hsw (flags & 1) and 'any active' set on hw (flags & 2).
__global__ void __launch_bounds__(1024) k_compact_graph(int count, const int* __restrict__ act, int* __restrict__ list,
                                                        int* __restrict__ nact, unsigned long long* __restrict__ add_old,
                                                        unsigned long long* __restrict__ add_new, cudaGraphConditionalHandle hsw,
                                                        int nb, cudaGraphConditionalHandle hw, int flags) {
    __shared__ int sums[1024];
    __shared__ int s_run;
    const int chunk = (count + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * chunk, b1 = min(count, b0 + chunk);
    int loc = 0;
    for (int i = b0; i < b1; ++i) loc += act[i] ? 1 : 0;
    sums[threadIdx.x] = loc;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) { const int v = sums[k]; sums[k] = run; run += v; }
        const int old = *nact;
        *nact = run;
        s_run = run;
        if (add_old) *add_old += (unsigned long long)old;
        if (add_new) *add_new += (unsigned long long)run;
        if (flags & 1) cudaGraphSetConditional(hsw, bucket_of(run, count, nb));
        if (flags & 2) cudaGraphSetConditional(hw, run > 0 ? 1u : 0u);
    }
    __syncthreads();
    int pos = sums[threadIdx.x];
    for (int i = b0; i < b1; ++i)
        if (act[i]) list[pos++] = i;
}

__global__ void k_fill_int(int* __restrict__ a, int count, int v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) a[i] = v;
}

// Before the refinement loop: phase 0, `count` particles entering it, the loop taken.
__global__ void k_outer_init(cudaGraphConditionalHandle h, int* __restrict__ gouter, int count) {
    gouter[0] = 0;
    gouter[1] = count;
    cudaGraphSetConditional(h, 1u);
}

// After a refinement phase's residual: its counters, and whether another phase runs.
__global__ void k_outer_cond(cudaGraphConditionalHandle h, const int* __restrict__ scount, int* __restrict__ gouter, int max_outer,
                             GraphCounters* __restrict__ g) {
    const int active = scount[1];                 // particles still above the FP64 tolerance
    const int o = ++gouter[0];
    g->residuals += (unsigned long long)gouter[1];
    gouter[1] = active;
    g->itmax = max(g->itmax, scount[2]);
    if (active > 0 && o >= max_outer) g->nonconv += (unsigned long long)active;
    cudaGraphSetConditional(h, (active > 0 && o < max_outer) ? 1u : 0u);
}

static cudaGraphConditionalHandle make_handle(cudaStream_t st) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    check(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr), "capture info");
    if (cs != cudaStreamCaptureStatusActive || !g) throw CudaError{cudaErrorStreamCaptureInvalidated, "stream not capturing"};
    cudaGraphConditionalHandle h;
    check(cudaGraphConditionalHandleCreate(&h, g, 0, 0), "conditional handle");
    return h;
}

// Adds a conditional node (while: 1 body; switch: `size` bodies) at the capture
// position of `st` and makes it the stream's dependency; returns the bodies.
static void add_conditional_node(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type, unsigned int size,
                                 cudaGraph_t* bodies) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    check(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd), "capture info");
    if (cs != cudaStreamCaptureStatusActive || !g) throw CudaError{cudaErrorStreamCaptureInvalidated, "stream not capturing"};
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = size;
    cudaGraphNode_t node;
    check(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p), "conditional node");
    for (unsigned int i = 0; i < size; ++i) bodies[i] = p.conditional.phGraph_out[i];
    check(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies), "capture dependencies");
}

// Captures fn()'s launches into `body` on the auxiliary stream of the next depth
// (the context's launchers use c.stream, which points there meanwhile).
template <class F>
static void capture_body(Ctx& c, cudaGraph_t body, F&& fn) {
    if (c.gdepth >= 4 || !c.gaux[c.gdepth]) throw CudaError{cudaErrorInvalidValue, "graph nesting deeper than the auxiliary streams"};
    cudaStream_t aux = c.gaux[c.gdepth];
    check(cudaStreamBeginCaptureToGraph(aux, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed), "body capture");
    cudaStream_t saved = c.stream;
    c.stream = aux;
    ++c.gdepth;
    try {
        fn();
    } catch (...) {
        --c.gdepth;
        c.stream = saved;
        cudaGraph_t tmp = nullptr;
        (void)cudaStreamEndCapture(aux, &tmp);
        (void)cudaGetLastError();
        throw;
    }
    --c.gdepth;
    c.stream = saved;
    cudaGraph_t out = nullptr;
    check(cudaStreamEndCapture(aux, &out), "end body capture");
}

template <typename T>
static void inner_solve_graph(Ctx& c, InnerSolver<T>& s, int count, double tol, double floor2) {
    SolverScalars& sc = c.sc;
    Passes<T> P(c, s);
    if (P.path == 0) throw CudaError{cudaErrorNotSupported, "graph capture needs the warp-tile solver kernels"};
    const int ntiles = P.ntiles;
    const int wgrid = (count * 32 + 127) / 128;
    const double tol2 = tol * tol;
    const int maxit = c.cfg.max_iter;
    const int nb = launch_buckets(count);
    GraphCounters* g = c.gcnt;
    auto scalar = [&](int mode) {
        k_scalar<<<wgrid, 128, 0, c.stream>>>(mode, count, ntiles, sc, c.part, tol2, floor2, maxit); ++c.pc.launches;
    };
    auto compact = [&](unsigned long long* add_old, unsigned long long* add_new, cudaGraphConditionalHandle hsw,
                       cudaGraphConditionalHandle hw, int flags) {
        k_compact_graph<<<1, 1024, 0, c.stream>>>(count, sc.act_in, s.list, s.nact, add_old, add_new, hsw, nb, hw, flags);
        ++c.pc.launches;
    };
    auto switch_stage = [&](cudaGraphConditionalHandle h, auto&& stage) {
        cudaGraph_t bodies[GB_MAX];
        add_conditional_node(c.stream, h, cudaGraphCondTypeSwitch, (unsigned int)nb, bodies);
        for (int b = 0; b < nb; ++b) capture_body(c, bodies[b], [&] { stage(bucket_size(count, b)); });
    };
    auto rr_step = [&]() {
        check(cudaMemsetAsync(sc.count, 0, sizeof(int), c.stream), "memset count");
        scalar(SM_RR);
    };
    scalar(SM_START);
    check(cudaMemsetAsync(sc.count, 0, 3 * sizeof(int), c.stream), "memset count");
    const cudaGraphConditionalHandle h0 = make_handle(c.stream);
    compact(nullptr, nullptr, h0, 0, 1);
    switch_stage(h0, [&](int L) { P.pre(L, 0, 0, 0); });          // z0 = M r0: the first V-cycle's pre-smoothing
    scalar(SM_INIT_RR);
    const cudaGraphConditionalHandle h1 = make_handle(c.stream);
    compact(nullptr, &g->inner_solves, h1, 0, 1);
    switch_stage(h1, [&](int L) {                                 // rest of the first V-cycle, then the first CG step
        P.lower(L); P.post(L, 0); scalar(SM_RZ_FIRST);
        P.apply(L, 0, 1); scalar(SM_PQ); P.pre(L, 0, 1, 1);
    });
    rr_step();
    const cudaGraphConditionalHandle hA = make_handle(c.stream), hw = make_handle(c.stream);
    compact(&g->cg_iterations, nullptr, hA, hw, 3);
    cudaGraph_t wbody;
    add_conditional_node(c.stream, hw, cudaGraphCondTypeWhile, 1, &wbody);
    capture_body(c, wbody, [&] {
        switch_stage(hA, [&](int L) {
            P.lower(L); P.post(L, 1); scalar(SM_RZ);
            P.apply(L, 1, 0); scalar(SM_PQ); P.pre(L, 1, 0, 1);
        });
        rr_step();
        const cudaGraphConditionalHandle hB = make_handle(c.stream);
        compact(&g->cg_iterations, nullptr, hB, 0, 1);
        switch_stage(hB, [&](int L) {
            P.lower(L); P.post(L, 0); scalar(SM_RZ);
            P.apply(L, 0, 0); scalar(SM_PQ); P.pre(L, 0, 1, 1);
        });
        rr_step();
        compact(&g->cg_iterations, nullptr, hA, hw, 3);
    });
}

template <typename T>
static void solve_batch_graph(Ctx& c, InnerSolver<T>& s, int count, const Rhs& R, double* W) {
    const int n = c.n;
    const int ntiles = (n / TILE) * (n / TILE);
    dim3 tgrid(ntiles, count);
    const size_t total = (size_t)n * n * count;
    set_smem_attrs<T>(c, s);
    SolverScalars& sc = c.sc;
    const bool mixed = sizeof(T) == 4;
    const double tol_out2 = c.cfg.tol_outer * c.cfg.tol_outer;
    check(cudaMemsetAsync(W, 0, total * sizeof(double), c.stream), "memset w");
    check(cudaMemsetAsync(s.x, 0, total * sizeof(T), c.stream), "memset x");
    k_fill_int<<<(count + 255) / 256, 256, 0, c.stream>>>(sc.act_out, count, 1); ++c.pc.launches;
    k_fill_rhs<T><<<grid_for(total), 256, 0, c.stream>>>((size_t)n * n, count, R.b64, mixed ? R.bdf : nullptr, R.stride,
                                                        s.r[0]); ++c.pc.launches;
    const int sgrid = (count + 127) / 128;
    const int* badp = (mixed && c.lenient) ? c.badp : nullptr;
    k_outer<<<sgrid, 128, 0, c.stream>>>(0, count, ntiles, sc, c.part, tol_out2, R.b2const, R.b2pp, badp); ++c.pc.launches;
    const int max_outer = mixed ? c.cfg.max_refine : std::max(2, c.cfg.max_refine);
    const double tol_in = mixed ? c.cfg.tol_inner : c.cfg.tol_outer;
    const double floor2 = 0.25 * tol_out2;
    const cudaGraphConditionalHandle ho = make_handle(c.stream);
    k_outer_init<<<1, 1, 0, c.stream>>>(ho, c.gouter, count); ++c.pc.launches;
    cudaGraph_t obody;
    add_conditional_node(c.stream, ho, cudaGraphCondTypeWhile, 1, &obody);
    capture_body(c, obody, [&] {
        inner_solve_graph<T>(c, s, count, tol_in, floor2);
        k_update_w<T><<<dim3(n * n / 1024, count), 256, 0, c.stream>>>(n * n, W, s.x, sc.act_out); ++c.pc.launches;
        if constexpr (sizeof(T) == 4) {
            LevelArrays<float>& f0 = s.lv[0];
            k_residual_mix<<<tgrid, RES_THREADS, 0, c.stream>>>(n, f0.Kw, c.Kwlo, f0.Ks, c.Kslo, f0.E, c.Elo, f0.Nn, c.Nlo, W, R.bdf, R.stride,
                                                       s.r[0], c.part.res, sc.act_out); ++c.pc.launches;
        } else {
            k_residual<T><<<tgrid, 256, 0, c.stream>>>(n, c.Kw64, c.Ks64, c.E64, c.N64, W, R.b64, R.stride, s.r[0], c.part.res,
                                                       sc.act_out); ++c.pc.launches;
        }
        check(cudaMemsetAsync(sc.count + 1, 0, sizeof(int), c.stream), "memset");
        k_outer<<<sgrid, 128, 0, c.stream>>>(1, count, ntiles, sc, c.part, tol_out2, R.b2const, R.b2pp, badp); ++c.pc.launches;
        k_outer_cond<<<1, 1, 0, c.stream>>>(ho, sc.count, c.gouter, max_outer, c.gcnt); ++c.pc.launches;
    });
}

// The forward map of `count` particles (synthesis, set-up, solve, observation) into
// the graph being captured on c.stream; Phi of an out-of-range field is +inf.
void forward_solve_graph(Ctx& c, const double* X, int count, double* Phi_out) {
    if (c.dim != 2) throw CudaError{cudaErrorNotSupported, "graph capture is built for the 2D solver"};
    for (int off = 0; off < count; off += c.B) {
        const int cnt = std::min(c.B, count - off);
        if (mixed_precision(c.cfg) && c.n % FX == 0 && c.n % FY == 0)
            launch_synth2d_df(c, X + (size_t)off * c.d, cnt, reinterpret_cast<float2*>(c.u64));
        else
            launch_synth2d(c, X + (size_t)off * c.d, cnt, c.u64);
        launch_setup_coeffs(c, cnt);
        if (mixed_precision(c.cfg)) solve_batch_graph<float>(c, c.s32, cnt, shared_rhs(c), c.w64);
        else solve_batch_graph<double>(c, c.s64, cnt, shared_rhs(c), c.w64);
        launch_observe(c, c.w64, cnt, Phi_out + off);
        launch_mark_out_of_range(c, cnt, Phi_out + off);
    }
}

// Graph-mode move steps (pCN-GM, pCN and SMC-GM kernels): the proposal tables, then a
// 'while' node over the steps; each step proposes, solves, accepts and advances the
// Philox step in the device schedule.
__global__ void k_steps_init(cudaGraphConditionalHandle h, int* __restrict__ left, int steps) {
    *left = steps;
    cudaGraphSetConditional(h, steps > 0 ? 1u : 0u);
}

__global__ void k_step_next(cudaGraphConditionalHandle h, int* __restrict__ left, MoveSched* __restrict__ ms) {
    ms->step += 1u;
    const int l = --(*left);
    cudaGraphSetConditional(h, l > 0 ? 1u : 0u);
}

void capture_move_steps(Ctx& c, int steps, int* acc_count) {
    if (c.cfg.kernel != SMC_K_PCN_GM && c.cfg.kernel != SMC_K_PCN && c.cfg.kernel != SMC_K_GM_INDEP)
        throw InputError{"graph capture covers the pCN, pCN-GM and SMC-GM kernels"};
    launch_move_tables(c, c.msched);
    const cudaGraphConditionalHandle hs = make_handle(c.stream);
    k_steps_init<<<1, 1, 0, c.stream>>>(hs, c.gsteps, steps); ++c.pc.launches;
    cudaGraph_t body;
    add_conditional_node(c.stream, hs, cudaGraphCondTypeWhile, 1, &body);
    capture_body(c, body, [&] {
        if (c.cfg.full_cov) launch_propose_full(c, c.msched, 0);
        else launch_propose(c, c.msched, 0);
        forward_solve_graph(c, c.V, c.N, c.PhiV);
        launch_accept(c, acc_count, c.msched, 0);
        k_step_next<<<1, 1, 0, c.stream>>>(hs, c.gsteps, c.msched); ++c.pc.launches;
    });
}

Rhs shared_rhs(const Ctx& c) { return Rhs{c.b64, c.bdf, 0, nullptr, c.b2}; }

// In a move (c.lenient) a proposal whose field is outside the mixed-precision
// range is not solved; Phi = +inf makes the accept step reject it.
__global__ void k_mark_out_of_range(int count, const int* __restrict__ badp, double* __restrict__ Phi) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < count && badp[p]) Phi[p] = 1.0 / 0.0;
}

void launch_mark_out_of_range(Ctx& c, int count, double* Phi) {
    if (!c.lenient || !c.badp || !mixed_precision(c.cfg)) return;
    k_mark_out_of_range<<<(count + 127) / 128, 128, 0, c.stream>>>(count, c.badp, Phi); ++c.pc.launches;
}

int solve_batch(Ctx& c, int count, const Rhs& R, double* W) {
    return mixed_precision(c.cfg) ? solve_batch_t<float>(c, c.s32, count, R, W)
                                                 : solve_batch_t<double>(c, c.s64, count, R, W);
}

int forward_solve(Ctx& c, const double* X, int count, double* Phi_out, double* w_out) {
    if (c.dim == 1) {
        launch_forward1d(c, X, count, Phi_out, w_out);
        return 0;
    }
    int itmax = 0;
    const size_t nn = (size_t)c.n * c.n;
    for (int off = 0; off < count; off += c.B) {
        const int cnt = std::min(c.B, count - off);
        {
            NvtxRange nvtx("synthesis and set-up");
            // the mixed-precision set-up takes the field as df32 pairs (in the FP64 field's storage)
            if (mixed_precision(c.cfg) && c.n % FX == 0 && c.n % FY == 0)
                launch_synth2d_df(c, X + (size_t)off * c.d, cnt, reinterpret_cast<float2*>(c.u64));
            else
                launch_synth2d(c, X + (size_t)off * c.d, cnt, c.u64);
            launch_setup_coeffs(c, cnt);
        }
        int it = 0;
        {
            NvtxRange nvtx("MG-PCG solve");
            it = solve_batch(c, cnt, shared_rhs(c), c.w64);
        }
        itmax = std::max(itmax, it);
        NvtxRange nvtx("observation");
        launch_observe(c, c.w64, cnt, Phi_out + off);
        launch_mark_out_of_range(c, cnt, Phi_out + off);
        if (w_out) check(cudaMemcpyAsync(w_out + off * nn, c.w64, cnt * nn * sizeof(double), cudaMemcpyDeviceToDevice, c.stream), "w copy");
    }
    check(cudaGetLastError(), "forward");
    c.last_iters = itmax;
    return itmax;
}

}  // namespace smcgm
