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
#include "smcgm_internal.cuh"
#include "common.cuh"

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

__global__ void k_faces(int n, int count, const double* __restrict__ s, double* __restrict__ Kw, double* __restrict__ Ks,
                        double* __restrict__ E, double* __restrict__ Nn, float* __restrict__ Kw32, float* __restrict__ Ks32,
                        float* __restrict__ E32, float* __restrict__ Nn32) {
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
        double kw = (i == 0) ? 2.0 * recip_nr(sc) : 2.0 * recip_nr(sc + sp[c - 1]);
        double ks = (j == 0) ? 2.0 * recip_nr(sc) : 2.0 * recip_nr(sc + sp[c - n]);
        Kw[t] = kw;
        Ks[t] = ks;
        if (Kw32) { Kw32[t] = (float)kw; Ks32[t] = (float)ks; }
        if (i == n - 1) {
            double e = 2.0 * recip_nr(sc);
            E[p * n + j] = e;
            if (E32) E32[p * n + j] = (float)e;
        }
        if (j == n - 1) {
            double e = 2.0 * recip_nr(sc);
            Nn[p * n + i] = e;
            if (Nn32) Nn32[p * n + i] = (float)e;
        }
    }
}

// Galerkin coarsening for piecewise-constant prolongation.
template <typename T>
__global__ void k_coarsen(int m, int count, const T* __restrict__ Kw, const T* __restrict__ Ks, const T* __restrict__ E,
                          const T* __restrict__ Nn, T* __restrict__ Kwc, T* __restrict__ Ksc, T* __restrict__ Ec,
                          T* __restrict__ Nnc) {
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
        Kwc[t] = kw[(2 * J) * n + 2 * I] + kw[(2 * J + 1) * n + 2 * I];
        Ksc[t] = ks[(2 * J) * n + 2 * I] + ks[(2 * J) * n + 2 * I + 1];
        if (I == m - 1) Ec[p * m + J] = E[p * n + 2 * J] + E[p * n + 2 * J + 1];
        if (J == m - 1) Nnc[p * m + I] = Nn[p * n + 2 * I] + Nn[p * n + 2 * I + 1];
    }
}

// ------------------------------------------------------------------------
// Tiled smoothing kernels.  Shared layout for a region of R x R cells
// (R = TILE + 2H): r, e, D (R*R each), Kw (R rows of R+1), Ks (R+1 rows of R).
// ------------------------------------------------------------------------
template <typename T>
struct TileSmem {
    T *r, *e, *d, *kw, *ks;
    __device__ TileSmem(T* base, int R) {
        r = base; e = r + R * R; d = e + R * R; kw = d + R * R; ks = kw + R * (R + 1);
    }
};

template <typename T>
__host__ __device__ inline size_t tile_smem_bytes(int R) { return sizeof(T) * (size_t)(3 * R * R + 2 * R * (R + 1)); }

// Load the face coefficients of a region whose origin is (gx0, gy0).
// skw(ly, lx) is the west face of region cell (lx, ly), lx = 0..R (lx = R: the
// east face of the last column); global column n maps to the east wall E.
template <typename T>
__device__ inline void load_faces(TileSmem<T>& sm, int R, int n, int gx0, int gy0, const T* __restrict__ Kw,
                                  const T* __restrict__ Ks, const T* __restrict__ E, const T* __restrict__ Nn) {
    for (int idx = threadIdx.x; idx < R * (R + 1); idx += blockDim.x) {
        int ly = idx / (R + 1), lx = idx - ly * (R + 1);
        int gx = gx0 + lx, gy = gy0 + ly;
        T v = T(0);
        if (gy >= 0 && gy < n) {
            if (gx >= 0 && gx < n) v = Kw[gy * n + gx];
            else if (gx == n) v = E[gy];
        }
        sm.kw[ly * (R + 1) + lx] = v;
    }
    for (int idx = threadIdx.x; idx < (R + 1) * R; idx += blockDim.x) {
        int ly = idx / R, lx = idx - ly * R;
        int gx = gx0 + lx, gy = gy0 + ly;
        T v = T(0);
        if (gx >= 0 && gx < n) {
            if (gy >= 0 && gy < n) v = Ks[gy * n + gx];
            else if (gy == n) v = Nn[gx];
        }
        sm.ks[ly * R + lx] = v;
    }
}

template <typename T>
__device__ inline T nbr_sum(const TileSmem<T>& sm, int R, int lx, int ly) {
    const int c = ly * R + lx;
    return sm.kw[ly * (R + 1) + lx] * sm.e[c - 1] + sm.kw[ly * (R + 1) + lx + 1] * sm.e[c + 1] +
           sm.ks[ly * R + lx] * sm.e[c - R] + sm.ks[(ly + 1) * R + lx] * sm.e[c + R];
}

// One red-black half-sweep of colour `col` over region cells [lo, hi)^2 that lie
// in the domain; zero start allows a pointwise update when `pointwise`.
template <typename T>
__device__ inline void half_sweep(TileSmem<T>& sm, int R, int n, int gx0, int gy0, int lo, int hi, int col, bool pointwise) {
    const int w = hi - lo;
    if (w <= 0) return;
    const int half = (w + 1) / 2;
    for (int idx = threadIdx.x; idx < w * half; idx += blockDim.x) {
        int ly = lo + idx / half;
        int k = idx - (idx / half) * half;
        // first lx in [lo, hi) with (gx0 + lx + gy0 + ly) % 2 == col
        int lx = lo + ((((gx0 + lo + gy0 + ly) & 1) == col) ? 0 : 1) + 2 * k;
        if (lx >= hi) continue;
        int gx = gx0 + lx, gy = gy0 + ly;
        if (gx < 0 || gx >= n || gy < 0 || gy >= n) continue;
        const int c = ly * R + lx;
        T num = sm.r[c];
        if (!pointwise) num += nbr_sum(sm, R, lx, ly);
        sm.e[c] = num / sm.d[c];
    }
}

template <typename T>
__device__ inline void compute_diag(TileSmem<T>& sm, int R, int n, int gx0, int gy0) {
    for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
        int ly = idx / R, lx = idx - ly * R;
        int gx = gx0 + lx, gy = gy0 + ly;
        T dv = T(1);
        if (gx >= 0 && gx < n && gy >= 0 && gy < n)
            dv = sm.kw[ly * (R + 1) + lx] + sm.kw[ly * (R + 1) + lx + 1] + sm.ks[ly * R + lx] + sm.ks[(ly + 1) * R + lx];
        sm.d[idx] = dv;
    }
}

// Pre-smoothing + residual + restriction.  cg = 1 (finest level): first applies
// the CG update r' = r - alpha q (whole region), x += alpha p and stores r'
// (tile interior), accumulating |r'|^2 per tile.
template <typename T, int NU>
__global__ void __launch_bounds__(256) k_pre(int n, const T* __restrict__ Kw, const T* __restrict__ Ks, const T* __restrict__ E,
                                             const T* __restrict__ Nn, const T* __restrict__ rin, T* __restrict__ rout,
                                             T* __restrict__ e_out, T* __restrict__ rc, const T* __restrict__ q, T* __restrict__ x,
                                             const T* __restrict__ p, const double* __restrict__ alpha, double* __restrict__ part_rr,
                                             const int* __restrict__ active, int cg, int want_rr) {
    constexpr int H = 2 * NU;
    constexpr int R = TILE + 2 * H;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[32];
    const int pb = blockIdx.y;
    if (!active[pb]) return;
    const int tpr = n / TILE;
    const int tx = blockIdx.x % tpr, ty = blockIdx.x / tpr;
    const int gx0 = tx * TILE - H, gy0 = ty * TILE - H;
    const size_t nn = (size_t)n * n;
    const size_t base = (size_t)pb * nn;
    TileSmem<T> sm(reinterpret_cast<T*>(smraw), R);
    load_faces(sm, R, n, gx0, gy0, Kw + base, Ks + base, E + (size_t)pb * n, Nn + (size_t)pb * n);
    const T a = cg ? (T)alpha[pb] : T(0);
    double rr_loc = 0.0;
    for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
        int ly = idx / R, lx = idx - ly * R;
        int gx = gx0 + lx, gy = gy0 + ly;
        T rv = T(0);
        if (gx >= 0 && gx < n && gy >= 0 && gy < n) {
            const size_t gi = base + (size_t)gy * n + gx;
            rv = rin[gi];
            if (cg) {
                rv -= a * q[gi];
                if (lx >= H && lx < H + TILE && ly >= H && ly < H + TILE) {
                    rout[gi] = rv;
                    x[gi] += a * p[gi];
                    rr_loc += (double)rv * (double)rv;
                }
            } else if (want_rr && lx >= H && lx < H + TILE && ly >= H && ly < H + TILE) {
                rr_loc += (double)rv * (double)rv;
            }
        }
        sm.r[idx] = rv;
        sm.e[idx] = T(0);
    }
    __syncthreads();
    compute_diag(sm, R, n, gx0, gy0);
    __syncthreads();
    // NU sweeps of (red, black); the first red half-sweep starts from e = 0.
    int s = 0;
#pragma unroll
    for (int sw = 0; sw < NU; ++sw) {
        half_sweep(sm, R, n, gx0, gy0, s == 0 ? 0 : s, s == 0 ? R : R - s, 0, s == 0);
        __syncthreads();
        ++s;
        half_sweep(sm, R, n, gx0, gy0, s, R - s, 1, false);
        __syncthreads();
        ++s;
    }
    // residual on the interior (after 2NU half-sweeps the valid region is [2NU-1, R-2NU+1)).
    T res[4];
    int cnt = 0;
    for (int idx = threadIdx.x; idx < TILE * TILE; idx += blockDim.x) {
        int ly = H + idx / TILE, lx = H + idx % TILE;
        int gx = gx0 + lx, gy = gy0 + ly;
        T rv = T(0);
        if (gx < n && gy < n) {
            const int c = ly * R + lx;
            rv = sm.r[c] - (sm.d[c] * sm.e[c] - nbr_sum(sm, R, lx, ly));
        }
        res[cnt++] = rv;
    }
    __syncthreads();
    cnt = 0;
    for (int idx = threadIdx.x; idx < TILE * TILE; idx += blockDim.x) {
        int ly = H + idx / TILE, lx = H + idx % TILE;
        sm.r[ly * R + lx] = res[cnt++];
    }
    __syncthreads();
    // write e (interior) and the restricted residual (TILE/2)^2
    for (int idx = threadIdx.x; idx < TILE * TILE; idx += blockDim.x) {
        int ly = H + idx / TILE, lx = H + idx % TILE;
        int gx = gx0 + lx, gy = gy0 + ly;
        e_out[base + (size_t)gy * n + gx] = sm.e[ly * R + lx];
    }
    const int m = n / 2;
    const int hT = TILE / 2;
    for (int idx = threadIdx.x; idx < hT * hT; idx += blockDim.x) {
        int J = idx / hT, I = idx % hT;
        int lx = H + 2 * I, ly = H + 2 * J;
        T v = sm.r[ly * R + lx] + sm.r[ly * R + lx + 1] + sm.r[(ly + 1) * R + lx] + sm.r[(ly + 1) * R + lx + 1];
        int GX = tx * hT + I, GY = ty * hT + J;
        rc[(size_t)pb * m * m + (size_t)GY * m + GX] = v;
    }
    if (cg || want_rr) {
        double tot = block_sum(rr_loc, red);
        if (threadIdx.x == 0) part_rr[(size_t)pb * gridDim.x + blockIdx.x] = tot;
    }
}

// Prolongation of the coarse correction, post-smoothing (black, red) and,
// on the finest level, the partial r.z of the CG step.
template <typename T, int NU>
__global__ void __launch_bounds__(256) k_post(int n, const T* __restrict__ Kw, const T* __restrict__ Ks, const T* __restrict__ E,
                                              const T* __restrict__ Nn, const T* __restrict__ r, const T* __restrict__ e_in,
                                              const T* __restrict__ ec, T cc, T* __restrict__ e_out, double* __restrict__ part_rz,
                                              const int* __restrict__ active, int cg) {
    constexpr int H = 2 * NU;
    constexpr int R = TILE + 2 * H;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[32];
    const int pb = blockIdx.y;
    if (!active[pb]) return;
    const int tpr = n / TILE;
    const int tx = blockIdx.x % tpr, ty = blockIdx.x / tpr;
    const int gx0 = tx * TILE - H, gy0 = ty * TILE - H;
    const int m = n / 2;
    const size_t nn = (size_t)n * n, base = (size_t)pb * nn, cbase = (size_t)pb * m * m;
    TileSmem<T> sm(reinterpret_cast<T*>(smraw), R);
    load_faces(sm, R, n, gx0, gy0, Kw + base, Ks + base, E + (size_t)pb * n, Nn + (size_t)pb * n);
    for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
        int ly = idx / R, lx = idx - ly * R;
        int gx = gx0 + lx, gy = gy0 + ly;
        T rv = T(0), ev = T(0);
        if (gx >= 0 && gx < n && gy >= 0 && gy < n) {
            const size_t gi = base + (size_t)gy * n + gx;
            rv = r[gi];
            ev = e_in[gi] + cc * ec[cbase + (size_t)(gy >> 1) * m + (gx >> 1)];
        }
        sm.r[idx] = rv;
        sm.e[idx] = ev;
    }
    __syncthreads();
    compute_diag(sm, R, n, gx0, gy0);
    __syncthreads();
    int s = 1;
#pragma unroll
    for (int sw = 0; sw < NU; ++sw) {
        half_sweep(sm, R, n, gx0, gy0, s, R - s, 1, false);
        __syncthreads();
        ++s;
        half_sweep(sm, R, n, gx0, gy0, s, R - s, 0, false);
        __syncthreads();
        ++s;
    }
    double rz = 0.0;
    for (int idx = threadIdx.x; idx < TILE * TILE; idx += blockDim.x) {
        int ly = H + idx / TILE, lx = H + idx % TILE;
        int gx = gx0 + lx, gy = gy0 + ly;
        const int c = ly * R + lx;
        T ev = sm.e[c];
        e_out[base + (size_t)gy * n + gx] = ev;
        if (cg) rz += (double)sm.r[c] * (double)ev;
    }
    if (cg) {
        double tot = block_sum(rz, red);
        if (threadIdx.x == 0) part_rz[(size_t)pb * gridDim.x + blockIdx.x] = tot;
    }
}

// CG direction update and operator application: p <- z + beta p, q = A p, partial p.q.
template <typename T>
__global__ void __launch_bounds__(256) k_apply(int n, const T* __restrict__ Kw, const T* __restrict__ Ks, const T* __restrict__ E,
                                               const T* __restrict__ Nn, const T* __restrict__ z, const T* __restrict__ pin,
                                               T* __restrict__ pout, T* __restrict__ q, const double* __restrict__ betac,
                                               double* __restrict__ part_pq, const int* __restrict__ active, int first) {
    constexpr int H = 1;
    constexpr int R = TILE + 2 * H;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[32];
    const int pb = blockIdx.y;
    if (!active[pb]) return;
    const int tpr = n / TILE;
    const int tx = blockIdx.x % tpr, ty = blockIdx.x / tpr;
    const int gx0 = tx * TILE - H, gy0 = ty * TILE - H;
    const size_t nn = (size_t)n * n, base = (size_t)pb * nn;
    TileSmem<T> sm(reinterpret_cast<T*>(smraw), R);
    load_faces(sm, R, n, gx0, gy0, Kw + base, Ks + base, E + (size_t)pb * n, Nn + (size_t)pb * n);
    const T b = first ? T(0) : (T)betac[pb];
    for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
        int ly = idx / R, lx = idx - ly * R;
        int gx = gx0 + lx, gy = gy0 + ly;
        T pv = T(0);
        if (gx >= 0 && gx < n && gy >= 0 && gy < n) {
            const size_t gi = base + (size_t)gy * n + gx;
            pv = z[gi];
            if (!first) pv += b * pin[gi];
        }
        sm.e[idx] = pv;
    }
    __syncthreads();
    double pq = 0.0;
    for (int idx = threadIdx.x; idx < TILE * TILE; idx += blockDim.x) {
        int ly = H + idx / TILE, lx = H + idx % TILE;
        int gx = gx0 + lx, gy = gy0 + ly;
        const int c = ly * R + lx;
        T dv = sm.kw[ly * (R + 1) + lx] + sm.kw[ly * (R + 1) + lx + 1] + sm.ks[ly * R + lx] + sm.ks[(ly + 1) * R + lx];
        T pv = sm.e[c];
        T qv = dv * pv - nbr_sum(sm, R, lx, ly);
        const size_t gi = base + (size_t)gy * n + gx;
        pout[gi] = pv;
        q[gi] = qv;
        pq += (double)pv * (double)qv;
    }
    double tot = block_sum(pq, red);
    if (threadIdx.x == 0) part_pq[(size_t)pb * gridDim.x + blockIdx.x] = tot;
}

// ------------------------------------------------------------------------
// Coarse V-cycle: levels with n_l <= coarse_top, one block per particle, all
// in shared memory.  Input r at the top level; output the correction e2.
// ------------------------------------------------------------------------
template <typename T>
struct CoarseLevelPtrs {
    const T* Kw[12]; const T* Ks[12]; const T* E[12]; const T* Nn[12];
    const T* rtop; T* etop;
    int ntop, nlev;   // nlev levels: ntop, ntop/2, ..., 1
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

template <typename T>
__device__ inline void chalf(const T* kw, const T* ks, const T* E, const T* Nn, const T* r, T* e, int n, int col, bool pointwise) {
    const int half = (n * n + 1) / 2;
    for (int k = threadIdx.x; k < half; k += blockDim.x) {
        int j = (2 * k) / n;
        int i = (2 * k) % n;
        if (((i + j) & 1) != col) i += 1;
        if (n == 1) { i = 0; j = 0; if (col != 0) continue; }
        if (i >= n) continue;
        T num = r[j * n + i];
        if (!pointwise) num += cnbr(kw, ks, e, n, i, j);
        e[j * n + i] = num / cdiag(kw, ks, E, Nn, n, i, j);
    }
}

template <typename T, int NU>
__global__ void __launch_bounds__(256) k_coarse(CoarseLevelPtrs<T> P, T cc, const int* __restrict__ active) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int pb = blockIdx.x;
    if (!active[pb]) return;
    T* kw[12]; T* ks[12]; T* E[12]; T* Nn[12]; T* r[12]; T* e[12];
    T* cur = reinterpret_cast<T*>(smraw);
    int nl = P.ntop;
    for (int l = 0; l < P.nlev; ++l) {
        const int nn = nl * nl;
        kw[l] = cur; cur += nn;
        ks[l] = cur; cur += nn;
        r[l] = cur; cur += nn;
        e[l] = cur; cur += nn;
        E[l] = cur; cur += nl;
        Nn[l] = cur; cur += nl;
        const T* gkw = P.Kw[l] + (size_t)pb * nn;
        const T* gks = P.Ks[l] + (size_t)pb * nn;
        for (int i = threadIdx.x; i < nn; i += blockDim.x) { kw[l][i] = gkw[i]; ks[l][i] = gks[i]; }
        for (int i = threadIdx.x; i < nl; i += blockDim.x) { E[l][i] = P.E[l][(size_t)pb * nl + i]; Nn[l][i] = P.Nn[l][(size_t)pb * nl + i]; }
        nl >>= 1;
    }
    {
        const int nn = P.ntop * P.ntop;
        const T* g = P.rtop + (size_t)pb * nn;
        for (int i = threadIdx.x; i < nn; i += blockDim.x) r[0][i] = g[i];
    }
    __syncthreads();
    // down
    nl = P.ntop;
    for (int l = 0; l < P.nlev - 1; ++l) {
        const int nn = nl * nl;
        for (int i = threadIdx.x; i < nn; i += blockDim.x) e[l][i] = T(0);
        __syncthreads();
        for (int sw = 0; sw < NU; ++sw) {
            chalf(kw[l], ks[l], E[l], Nn[l], r[l], e[l], nl, 0, sw == 0);
            __syncthreads();
            chalf(kw[l], ks[l], E[l], Nn[l], r[l], e[l], nl, 1, false);
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
            chalf(kw[l], ks[l], E[l], Nn[l], r[l], e[l], nl, 1, false);
            __syncthreads();
            chalf(kw[l], ks[l], E[l], Nn[l], r[l], e[l], nl, 0, false);
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
    for (int l = 0; l < nlev; ++l) { s += (size_t)(4 * nl * nl + 2 * nl); nl >>= 1; }
    return s * sizeof(T);
}

// ------------------------------------------------------------------------
// Per-particle scalar bookkeeping of CG and refinement.
// ------------------------------------------------------------------------
enum ScalarMode { SM_START = 0, SM_INIT_RR = 1, SM_RZ_FIRST = 2, SM_RZ = 3, SM_PQ = 4, SM_RR = 5 };

__global__ void k_scalar(int mode, int count, int ntiles, SolverScalars sc, Partials part, double tol2, int maxit) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= count) return;
    if (mode == SM_START) {
        sc.act_in[p] = sc.act_out[p];
        return;
    }
    if (!sc.act_in[p]) return;
    const double* src = mode == SM_PQ ? part.pq : (mode == SM_RZ || mode == SM_RZ_FIRST) ? part.rz : part.rr;
    double s = 0.0;
    for (int t = 0; t < ntiles; ++t) s += src[(size_t)p * ntiles + t];
    if (mode == SM_INIT_RR) {
        sc.rr0[p] = s;
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
        if (s <= tol2 * sc.rr0[p]) {
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

// w64 += x, x = 0, for particles still refining.
template <typename T>
__global__ void k_update_w(int nn, int count, double* __restrict__ w, T* __restrict__ x, const int* __restrict__ act) {
    const size_t total = (size_t)nn * count;
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; t < total; t += stride) {
        const int p = (int)(t / nn);
        if (!act[p]) continue;
        w[t] += (double)x[t];
        x[t] = T(0);
    }
}

// FP64 residual b - A64 w, stored in the inner precision; partial |res|^2 per tile.
template <typename T>
__global__ void __launch_bounds__(256) k_residual(int n, const double* __restrict__ Kw, const double* __restrict__ Ks,
                                                  const double* __restrict__ E, const double* __restrict__ Nn,
                                                  const double* __restrict__ w, const double* __restrict__ b, T* __restrict__ rout,
                                                  double* __restrict__ part_res, const int* __restrict__ act) {
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
        const double res = b[c] - aw;
        rout[base + c] = (T)res;
        acc += res * res;
    }
    double tot = block_sum(acc, red);
    if (threadIdx.x == 0) part_res[(size_t)pb * gridDim.x + blockIdx.x] = tot;
}

__global__ void k_outer(int mode, int count, int ntiles, SolverScalars sc, Partials part, double tol2) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= count) return;
    if (mode == 0) {  // initial residual = b
        double s = 0.0;
        for (int t = 0; t < ntiles; ++t) s += part.res[(size_t)p * ntiles + t];
        sc.b2[p] = s;
        sc.res2[p] = s;
        sc.act_out[p] = s > 0.0 ? 1 : 0;
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

template <typename T, int NU>
static void run_vcycle_lower(Ctx& c, InnerSolver<T>& s, int count, const int* act) {
    // levels 1 .. ntile_levels-1 (pre), coarse, then post back up to level 1
    const T cc = (T)c.cfg.coarse_scale;
    constexpr int R = TILE + 4 * NU;
    const size_t smem = tile_smem_bytes<T>(R);
    for (int l = 1; l < s.ntile_levels; ++l) {
        LevelArrays<T>& L = s.lv[l];
        dim3 grid((L.n / TILE) * (L.n / TILE), count);
        k_pre<T, NU><<<grid, 256, smem, c.stream>>>(L.n, L.Kw, L.Ks, L.E, L.Nn, L.r, nullptr, L.e, s.lv[l + 1].r, nullptr,
                                                    nullptr, nullptr, nullptr, nullptr, act, 0, 0);
    }
    {
        CoarseLevelPtrs<T> P{};
        const int top = s.ntile_levels;
        P.ntop = s.lv[top].n;
        P.nlev = s.nlev - top;
        for (int l = 0; l < P.nlev; ++l) {
            P.Kw[l] = s.lv[top + l].Kw; P.Ks[l] = s.lv[top + l].Ks; P.E[l] = s.lv[top + l].E; P.Nn[l] = s.lv[top + l].Nn;
        }
        P.rtop = s.lv[top].r;
        P.etop = s.lv[top].e2;
        const size_t cs = coarse_smem_bytes<T>(P.ntop, P.nlev);
        k_coarse<T, NU><<<count, 256, cs, c.stream>>>(P, cc, act);
    }
    for (int l = s.ntile_levels - 1; l >= 1; --l) {
        LevelArrays<T>& L = s.lv[l];
        dim3 grid((L.n / TILE) * (L.n / TILE), count);
        k_post<T, NU><<<grid, 256, smem, c.stream>>>(L.n, L.Kw, L.Ks, L.E, L.Nn, L.r, L.e, s.lv[l + 1].e2, cc, L.e2, nullptr,
                                                     act, 0);
    }
}

template <typename T, int NU>
static int inner_solve(Ctx& c, InnerSolver<T>& s, int count, double tol) {
    SolverScalars& sc = c.sc;
    LevelArrays<T>& L0 = s.lv[0];
    const int n = L0.n;
    const int ntiles = (n / TILE) * (n / TILE);
    dim3 tgrid(ntiles, count);
    constexpr int R = TILE + 4 * NU;
    const size_t smem = tile_smem_bytes<T>(R);
    const size_t smem_apply = tile_smem_bytes<T>(TILE + 2);
    const T cc = (T)c.cfg.coarse_scale;
    const int sgrid = (count + 127) / 128;
    const double tol2 = tol * tol;
    const int maxit = c.cfg.max_iter;
    int cur = 0, pc = 0;
    k_scalar<<<sgrid, 128, 0, c.stream>>>(SM_START, count, ntiles, sc, c.part, tol2, maxit);
    check(cudaMemsetAsync(sc.count, 0, 3 * sizeof(int), c.stream), "memset count");
    // z0 = M r0
    k_pre<T, NU><<<tgrid, 256, smem, c.stream>>>(n, L0.Kw, L0.Ks, L0.E, L0.Nn, s.r[cur], nullptr, L0.e, s.lv[1].r, nullptr,
                                                 nullptr, nullptr, nullptr, c.part.rr, sc.act_in, 0, 1);
    k_scalar<<<sgrid, 128, 0, c.stream>>>(SM_INIT_RR, count, ntiles, sc, c.part, tol2, maxit);
    int hcount[3] = {0, 0, 0};
    check(cudaMemcpyAsync(hcount, sc.count, 3 * sizeof(int), cudaMemcpyDeviceToHost, c.stream), "count d2h");
    check(cudaStreamSynchronize(c.stream), "sync");
    int active = hcount[0];
    c.pc.inner_solves += active;
    if (active == 0) return 0;
    run_vcycle_lower<T, NU>(c, s, count, sc.act_in);
    k_post<T, NU><<<tgrid, 256, smem, c.stream>>>(n, L0.Kw, L0.Ks, L0.E, L0.Nn, s.r[cur], L0.e, s.lv[1].e2, cc, s.z, c.part.rz,
                                                  sc.act_in, 1);
    k_scalar<<<sgrid, 128, 0, c.stream>>>(SM_RZ_FIRST, count, ntiles, sc, c.part, tol2, maxit);
    const double dom_bpc = (double)(6 * sizeof(T) + 3 * sizeof(T)) + 0.25 * sizeof(T);   // per cell: r,q,x,p,Kw,Ks in; r,x,e,rc out
    for (int it = 0; it < maxit; ++it) {
        k_apply<T><<<tgrid, 256, smem_apply, c.stream>>>(n, L0.Kw, L0.Ks, L0.E, L0.Nn, s.z, s.p[pc], s.p[1 - pc], s.q, sc.betac,
                                                        c.part.pq, sc.act_in, it == 0);
        pc ^= 1;
        k_scalar<<<sgrid, 128, 0, c.stream>>>(SM_PQ, count, ntiles, sc, c.part, tol2, maxit);
        if (c.prof) check(cudaEventRecord(c.ev0, c.stream), "event");
        k_pre<T, NU><<<tgrid, 256, smem, c.stream>>>(n, L0.Kw, L0.Ks, L0.E, L0.Nn, s.r[cur], s.r[1 - cur], L0.e, s.lv[1].r, s.q,
                                                     s.x, s.p[pc], sc.alpha, c.part.rr, sc.act_in, 1, 1);
        if (c.prof) check(cudaEventRecord(c.ev1, c.stream), "event");
        cur ^= 1;
        c.pc.cg_iterations += active;
        check(cudaMemsetAsync(sc.count, 0, sizeof(int), c.stream), "memset count");
        k_scalar<<<sgrid, 128, 0, c.stream>>>(SM_RR, count, ntiles, sc, c.part, tol2, maxit);
        check(cudaMemcpyAsync(hcount, sc.count, 3 * sizeof(int), cudaMemcpyDeviceToHost, c.stream), "count d2h");
        check(cudaStreamSynchronize(c.stream), "sync");
        if (c.prof) {
            float ms = 0.f;
            check(cudaEventElapsedTime(&ms, c.ev0, c.ev1), "event time");
            c.pc.dom_ms += ms;
            c.pc.dom_launches += 1;
            c.pc.dom_particles += active;
            c.pc.dom_bytes += dom_bpc * (double)n * n * active;
        }
        active = hcount[0];
        if (active == 0) break;
        run_vcycle_lower<T, NU>(c, s, count, sc.act_in);
        k_post<T, NU><<<tgrid, 256, smem, c.stream>>>(n, L0.Kw, L0.Ks, L0.E, L0.Nn, s.r[cur], L0.e, s.lv[1].e2, cc, s.z, c.part.rz,
                                                      sc.act_in, 1);
        k_scalar<<<sgrid, 128, 0, c.stream>>>(SM_RZ, count, ntiles, sc, c.part, tol2, maxit);
    }
    check(cudaGetLastError(), "inner solve launch");
    return hcount[2];
}

// Dynamic shared-memory opt-in; the coarse kernel's need depends on the grid, so
// the largest size requested so far is remembered per precision.
template <typename T>
static void set_smem_attrs(Ctx& c, InnerSolver<T>& s) {
    static size_t tile_set[2] = {0, 0}, coarse_set[2] = {0, 0};
    const int k = sizeof(T) == 4 ? 0 : 1;
    const size_t t2 = tile_smem_bytes<T>(TILE + 8);
    if (tile_set[k] < t2) {
        const size_t t1 = tile_smem_bytes<T>(TILE + 4);
        check(cudaFuncSetAttribute(k_pre<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t1), "attr");
        check(cudaFuncSetAttribute(k_post<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t1), "attr");
        check(cudaFuncSetAttribute(k_pre<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t2), "attr");
        check(cudaFuncSetAttribute(k_post<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t2), "attr");
        tile_set[k] = t2;
    }
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
        k_coarsen<T><<<grid_for(total), 256, 0, c.stream>>>(Bc.n, count, A.Kw, A.Ks, A.E, A.Nn, Bc.Kw, Bc.Ks, Bc.E, Bc.Nn);
    }
}
template void launch_coarsen_all<float>(Ctx&, InnerSolver<float>&, int);
template void launch_coarsen_all<double>(Ctx&, InnerSolver<double>&, int);

void launch_setup_coeffs(Ctx& c, int count) {
    const int n = c.n;
    const size_t total = (size_t)n * n * count;
    k_exp_neg<<<grid_for(total), 256, 0, c.stream>>>(c.u64, total);
    const bool mixed = c.cfg.precision == SMC_P_FP32_REFINE;
    if (mixed) {
        LevelArrays<float>& f0 = c.s32.lv[0];
        k_faces<<<grid_for(total), 256, 0, c.stream>>>(n, count, c.u64, c.Kw64, c.Ks64, c.E64, c.N64, f0.Kw, f0.Ks, f0.E, f0.Nn);
        launch_coarsen_all<float>(c, c.s32, count);
    } else {
        k_faces<<<grid_for(total), 256, 0, c.stream>>>(n, count, c.u64, c.Kw64, c.Ks64, c.E64, c.N64, nullptr, nullptr, nullptr,
                                                       nullptr);
        launch_coarsen_all<double>(c, c.s64, count);
    }
    check(cudaGetLastError(), "setup launch");
}

template <typename T>
static int solve_batch_t(Ctx& c, InnerSolver<T>& s, int count) {
    const int n = c.n;
    const int ntiles = (n / TILE) * (n / TILE);
    dim3 tgrid(ntiles, count);
    const size_t total = (size_t)n * n * count;
    set_smem_attrs<T>(c, s);
    SolverScalars& sc = c.sc;
    const bool mixed = sizeof(T) == 4;
    const double tol_out2 = c.cfg.tol_outer * c.cfg.tol_outer;
    check(cudaMemsetAsync(c.w64, 0, total * sizeof(double), c.stream), "memset w");
    check(cudaMemsetAsync(s.x, 0, total * sizeof(T), c.stream), "memset x");
    // act_out = 1 for the residual of w = 0
    {
        std::vector<int> ones(count, 1);
        check(cudaMemcpyAsync(sc.act_out, ones.data(), count * sizeof(int), cudaMemcpyHostToDevice, c.stream), "act init");
        check(cudaStreamSynchronize(c.stream), "sync");
    }
    k_residual<T><<<tgrid, 256, 0, c.stream>>>(n, c.Kw64, c.Ks64, c.E64, c.N64, c.w64, c.b64, s.r[0], c.part.res, sc.act_out);
    c.pc.residuals += count;
    c.pc.solves += count;
    c.pc.cells = n * n;
    c.pc.word_bytes = (int)sizeof(T);
    int outer_active = count;
    const int sgrid = (count + 127) / 128;
    k_outer<<<sgrid, 128, 0, c.stream>>>(0, count, ntiles, sc, c.part, tol_out2);
    int itmax = 0;
    const int nu = c.cfg.smooth_sweeps;
    const int max_outer = mixed ? c.cfg.max_refine : std::max(2, c.cfg.max_refine);
    const double tol_in = mixed ? c.cfg.tol_inner : c.cfg.tol_outer;
    for (int o = 0; o < max_outer; ++o) {
        int it = nu == 1 ? inner_solve<T, 1>(c, s, count, tol_in) : inner_solve<T, 2>(c, s, count, tol_in);
        itmax = std::max(itmax, it);
        c.pc.residuals += outer_active;
        k_update_w<T><<<grid_for(total), 256, 0, c.stream>>>(n * n, count, c.w64, s.x, sc.act_out);
        k_residual<T><<<tgrid, 256, 0, c.stream>>>(n, c.Kw64, c.Ks64, c.E64, c.N64, c.w64, c.b64, s.r[0], c.part.res, sc.act_out);
        check(cudaMemsetAsync(sc.count + 1, 0, sizeof(int), c.stream), "memset");
        k_outer<<<sgrid, 128, 0, c.stream>>>(1, count, ntiles, sc, c.part, tol_out2);
        int h = 0;
        check(cudaMemcpyAsync(&h, sc.count + 1, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "d2h");
        check(cudaStreamSynchronize(c.stream), "sync");
        if (h == 0) break;
        outer_active = h;
        if (o == max_outer - 1) c.nonconv += h;
    }
    return itmax;
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
        launch_synth2d(c, X + (size_t)off * c.d, cnt, c.u64);
        launch_setup_coeffs(c, cnt);
        int it = c.cfg.precision == SMC_P_FP32_REFINE ? solve_batch_t<float>(c, c.s32, cnt) : solve_batch_t<double>(c, c.s64, cnt);
        itmax = std::max(itmax, it);
        launch_observe(c, c.w64, cnt, Phi_out + off);
        if (w_out) check(cudaMemcpyAsync(w_out + off * nn, c.w64, cnt * nn * sizeof(double), cudaMemcpyDeviceToDevice, c.stream), "w copy");
    }
    check(cudaGetLastError(), "forward");
    c.last_iters = itmax;
    return itmax;
}

}  // namespace smcgm
