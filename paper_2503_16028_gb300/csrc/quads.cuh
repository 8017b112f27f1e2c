// Quad-owned, TMA-pipelined smoothing kernels of the tiled multigrid levels.
//
// A work item is one 32 x 32 tile of one active particle.  The smoothing
// region is the tile plus a halo of H = 2 nu cells (nu red-black sweeps); the
// staged boxes are 40 columns wide from x = 32 tx - 4 (16-byte aligned) and
// 32 + 2H rows from y = 32 ty - H.  Thread t owns one 2 x 2 quad of the
// region: its cells (0,0), (1,1) are red and (1,0), (0,1) black (tile origins
// are even), so a half-sweep updates exactly two cells per thread with no
// colour test, the quad's four residuals sum to its restricted value, and the
// quad shares one parent for the prolongation.  Every half-sweep updates the
// whole region; the shared correction array has a zero border, so an error
// can only enter at the region edge and moves one cell inward per half-sweep,
// which H = 2 nu keeps outside the tile interior (the first pre-smoothing
// half-sweep starts from zero and is pointwise, so it introduces none).
// Cells outside the grid have 1/D = 0 and stay zero.
#pragma once
#include "tma.cuh"

namespace smcgm {

template <typename T, int H>
struct QGeo {
    static constexpr int QN = (TT + 2 * H) / 2;       // quads per row / column of the region
    static constexpr int NQ = QN * QN;
    static constexpr int THREADS = ((NQ + 31) / 32) * 32;
    static constexpr int RY = TT + 2 * H;              // region rows (= staged rows)
    static constexpr int BX = 40;                      // staged columns (x0 = 32 tx - 4)
    static constexpr int CX = 4 - H;                   // first region column inside the box
    static constexpr int KWX = 44;                     // staged west-face columns
    static constexpr int EW = TT + 2 * H + 2;          // correction array row length (zero border)
    static constexpr int EH = TT + 2 * H + 2;
    // stage layout (bytes)
    static constexpr int R_OFF = 0;
    static constexpr int Q_OFF = R_OFF + align_elems(RY * BX * (int)sizeof(T));
    static constexpr int KW_OFF = Q_OFF + align_elems(RY * BX * (int)sizeof(T));
    static constexpr int KS_OFF = KW_OFF + align_elems(RY * KWX * (int)sizeof(T));
    static constexpr int X_OFF = KS_OFF + align_elems((RY + 1) * BX * (int)sizeof(T));
    static constexpr int P_OFF = X_OFF + align_elems(TT * TT * (int)sizeof(T));
    static constexpr int PRE_BYTES = P_OFF + align_elems(TT * TT * (int)sizeof(T));
    static constexpr uint32_t PRE_TX_BASE = (uint32_t)sizeof(T) * (RY * BX + RY * KWX + (RY + 1) * BX);
    static constexpr uint32_t PRE_TX_CG = (uint32_t)sizeof(T) * (RY * BX + 2 * TT * TT);
    // post stage: e_in, ec (coarse box CW x QN), r, Kw, Ks
    static constexpr int CW = 24;
    static constexpr int PE_OFF = 0;
    static constexpr int PEC_OFF = PE_OFF + align_elems(RY * BX * (int)sizeof(T));
    static constexpr int PR_OFF = PEC_OFF + align_elems(QN * CW * (int)sizeof(T));
    static constexpr int PKW_OFF = PR_OFF + align_elems(RY * BX * (int)sizeof(T));
    static constexpr int PKS_OFF = PKW_OFF + align_elems(RY * KWX * (int)sizeof(T));
    static constexpr int POST_BYTES = PKS_OFF + align_elems((RY + 1) * BX * (int)sizeof(T));
    static constexpr uint32_t POST_TX = (uint32_t)sizeof(T) * (2 * RY * BX + QN * CW + RY * KWX + (RY + 1) * BX);
};

template <typename T, int H, int STAGES> constexpr size_t qpre_smem() {
    return (size_t)STAGES * QGeo<T, H>::PRE_BYTES + 256 + (size_t)QGeo<T, H>::EW * QGeo<T, H>::EH * sizeof(T);
}
template <typename T, int H, int STAGES> constexpr size_t qpost_smem() {
    return (size_t)STAGES * QGeo<T, H>::POST_BYTES + 256 + (size_t)QGeo<T, H>::EW * QGeo<T, H>::EH * sizeof(T);
}

// Per-quad coefficients: index 0..3 = cells (0,0), (1,0), (0,1), (1,1).
template <typename T>
struct Quad {
    T r[4], w[4], e[4], s[4], n[4], inv[4];
};

// Loads the quad's right-hand side (minus a q if cg) and faces from the staged
// boxes; out-of-grid cells get inv = 0.
template <typename T, int H>
__device__ inline void load_quad(Quad<T>& Q, const T* sr, const T* sq, const T* skw, const T* sks, T a, bool cg, int bx, int by,
                                 int gx, int gy, int n) {
    using G = QGeo<T, H>;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int dx = k & 1, dy = k >> 1;
        const int c = (by + dy) * G::BX + bx + dx;
        const bool in = (gx + dx) >= 0 && (gx + dx) < n && (gy + dy) >= 0 && (gy + dy) < n;
        T rv = sr[c];
        if (cg) rv -= a * sq[c];
        Q.r[k] = rv;
        Q.w[k] = skw[(by + dy) * G::KWX + bx + dx];
        Q.e[k] = skw[(by + dy) * G::KWX + bx + dx + 1];
        Q.s[k] = sks[c];
        Q.n[k] = sks[c + G::BX];
        Q.inv[k] = in ? rcp_pos(Q.w[k] + Q.e[k] + Q.s[k] + Q.n[k]) : T(0);
    }
}

// Gauss-Seidel update of quad cell k (index in e of cell (0,0) is ec0).
template <typename T, int EW>
__device__ inline void gs_cell(T* se, int ec0, const Quad<T>& Q, int k, bool pointwise) {
    const int c = ec0 + (k >> 1) * EW + (k & 1);
    T num = Q.r[k];
    if (!pointwise) num += Q.w[k] * se[c - 1] + Q.e[k] * se[c + 1] + Q.s[k] * se[c - EW] + Q.n[k] * se[c + EW];
    se[c] = num * Q.inv[k];
}

template <typename T>
struct QPreArgs {
    PipeCommon pc;
    const T* E; const T* Nn;
    T* rout; T* e_out; T* rc; T* x;
    const double* alpha; double* part_rr;
    int cg, want_rr;
};

template <typename T>
struct QPostArgs {
    PipeCommon pc;
    const T* E; const T* Nn;
    T cc; T* e_out; double* part_rz; int cg;
};

// Pre-smoothing (nu = H/2 red-black sweeps from zero), residual, restriction;
// on the finest level also the CG update r' = r - alpha q, x' = x + alpha p and |r'|^2.
template <typename T, int H, int STAGES>
__global__ void __launch_bounds__(QGeo<T, H>::THREADS) k_qpre(QPreArgs<T> a, const __grid_constant__ CUtensorMap m_r,
                                                             const __grid_constant__ CUtensorMap m_kw,
                                                             const __grid_constant__ CUtensorMap m_ks,
                                                             const __grid_constant__ CUtensorMap m_q,
                                                             const __grid_constant__ CUtensorMap m_x,
                                                             const __grid_constant__ CUtensorMap m_p) {
    using G = QGeo<T, H>;
    constexpr int NU = H / 2;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = align128(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * G::PRE_BYTES);
    T* se = reinterpret_cast<T*>(smem + STAGES * G::PRE_BYTES + 128);
    __shared__ double red[32];
    const PipeCommon& pc = a.pc;
    const int n = pc.n, t = threadIdx.x;
    const uint32_t txb = G::PRE_TX_BASE + (a.cg ? G::PRE_TX_CG : 0u);
    auto issue = [&](int item, int s) {
        int p, tx, ty;
        item_tile(pc, item, p, tx, ty);
        unsigned char* st = smem + s * G::PRE_BYTES;
        fence_proxy_async();
        mbar_expect_tx(&bars[s], txb);
        const int X0 = tx * TT - 4, Y0 = ty * TT - H;
        tma_load_3d(st + G::R_OFF, &m_r, X0, Y0, p, &bars[s]);
        tma_load_3d(st + G::KW_OFF, &m_kw, X0, Y0, p, &bars[s]);
        tma_load_3d(st + G::KS_OFF, &m_ks, X0, Y0, p, &bars[s]);
        if (a.cg) {
            tma_load_3d(st + G::Q_OFF, &m_q, X0, Y0, p, &bars[s]);
            tma_load_3d(st + G::X_OFF, &m_x, tx * TT, ty * TT, p, &bars[s]);
            tma_load_3d(st + G::P_OFF, &m_p, tx * TT, ty * TT, p, &bars[s]);
        }
    };
    if (t == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    for (int i = t; i < G::EW * G::EH; i += blockDim.x) se[i] = T(0);   // zero border stays zero
    __syncthreads();
    if (t == 0)
        for (int s = 0; s < STAGES - 1; ++s) {
            const int item = blockIdx.x + s * gridDim.x;
            if (item < pc.total) issue(item, s);
        }
    const bool own = t < G::NQ;
    const int qx = own ? t % G::QN : 0, qy = own ? t / G::QN : 0;
    const int bx = G::CX + 2 * qx, by = 2 * qy;                  // quad origin in the staged boxes
    const int ec0 = (2 * qy + 1) * G::EW + 2 * qx + 1;           // quad origin in the correction array
    const bool inner = own && qx >= H / 2 && qx < H / 2 + TT / 2 && qy >= H / 2 && qy < H / 2 + TT / 2;
    uint32_t used[STAGES];
    for (int s = 0; s < STAGES; ++s) used[s] = 0;
    int it = 0;
    for (int item = blockIdx.x; item < pc.total; item += gridDim.x, ++it) {
        const int s = it % STAGES;
        if (t == 0) {
            const int ahead = item + (STAGES - 1) * gridDim.x;
            if (ahead < pc.total) issue(ahead, (it + STAGES - 1) % STAGES);
        }
        if (!mbar_wait_bounded(&bars[s], used[s] & 1u)) {
            if (t == 0) atomicExch(pc.err, 1);
            drain(bars, STAGES, used);
            return;
        }
        used[s]++;
        int p, tx, ty;
        item_tile(pc, item, p, tx, ty);
        unsigned char* st = smem + s * G::PRE_BYTES;
        const T* sr = reinterpret_cast<const T*>(st + G::R_OFF);
        const T* sq = reinterpret_cast<const T*>(st + G::Q_OFF);
        T* skw = reinterpret_cast<T*>(st + G::KW_OFF);
        T* sks = reinterpret_cast<T*>(st + G::KS_OFF);
        const T* sx = reinterpret_cast<const T*>(st + G::X_OFF);
        const T* sp = reinterpret_cast<const T*>(st + G::P_OFF);
        const int X0 = tx * TT - 4, Y0 = ty * TT - H;
        const int tpr = n / TT;
        if (tx == tpr - 1 || ty == tpr - 1) {
            patch_walls(skw, G::KWX, G::RY, X0, Y0, sks, G::BX, G::RY + 1, X0, Y0, n, a.E + (size_t)p * n, a.Nn + (size_t)p * n);
            __syncthreads();
        }
        const T al = a.cg ? (T)a.alpha[p] : T(0);
        const int gx = X0 + bx, gy = Y0 + by;
        Quad<T> Q;
        if (own) load_quad<T, H>(Q, sr, sq, skw, sks, al, a.cg != 0, bx, by, gx, gy, n);
        const size_t base = (size_t)p * n * n;
        double rr_loc = 0.0;
        if (inner) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int dx = k & 1, dy = k >> 1;
                const size_t gi = base + (size_t)(gy + dy) * n + gx + dx;
                if (a.cg) {
                    const int ci = (by + dy - H) * TT + (bx + dx - 4);
                    a.rout[gi] = Q.r[k];
                    a.x[gi] = sx[ci] + al * sp[ci];
                }
                rr_loc += (double)Q.r[k] * (double)Q.r[k];
            }
        }
        // nu sweeps (red, black); the first red half-sweep is pointwise from zero
#pragma unroll
        for (int sw = 0; sw < NU; ++sw) {
            if (own) { gs_cell<T, G::EW>(se, ec0, Q, 0, sw == 0); gs_cell<T, G::EW>(se, ec0, Q, 3, sw == 0); }
            __syncthreads();
            if (own) { gs_cell<T, G::EW>(se, ec0, Q, 1, false); gs_cell<T, G::EW>(se, ec0, Q, 2, false); }
            __syncthreads();
        }
        if (inner) {
            T rsum = T(0);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = ec0 + (k >> 1) * G::EW + (k & 1);
                const T ev = se[c];
                rsum += Q.r[k] - ((Q.w[k] + Q.e[k] + Q.s[k] + Q.n[k]) * ev -
                                  (Q.w[k] * se[c - 1] + Q.e[k] * se[c + 1] + Q.s[k] * se[c - G::EW] + Q.n[k] * se[c + G::EW]));
                a.e_out[base + (size_t)(gy + (k >> 1)) * n + gx + (k & 1)] = ev;
            }
            const int m = n / 2;
            a.rc[(size_t)p * m * m + (size_t)(gy >> 1) * m + (gx >> 1)] = rsum;
        }
        if (a.cg || a.want_rr) {
            const double tot = block_sum(rr_loc, red);
            if (t == 0) a.part_rr[(size_t)p * pc.ntiles + (ty * tpr + tx)] = tot;
        }
        __syncthreads();
        // the next item starts from a zero correction
        if (own) {
#pragma unroll
            for (int k = 0; k < 4; ++k) se[ec0 + (k >> 1) * G::EW + (k & 1)] = T(0);
        }
    }
}

// Prolongation (e + cc P ec), nu sweeps (black, red), and on the finest level r.z.
template <typename T, int H, int STAGES>
__global__ void __launch_bounds__(QGeo<T, H>::THREADS) k_qpost(QPostArgs<T> a, const __grid_constant__ CUtensorMap m_e,
                                                              const __grid_constant__ CUtensorMap m_ec,
                                                              const __grid_constant__ CUtensorMap m_r,
                                                              const __grid_constant__ CUtensorMap m_kw,
                                                              const __grid_constant__ CUtensorMap m_ks) {
    using G = QGeo<T, H>;
    constexpr int NU = H / 2;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = align128(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * G::POST_BYTES);
    T* se = reinterpret_cast<T*>(smem + STAGES * G::POST_BYTES + 128);
    __shared__ double red[32];
    const PipeCommon& pc = a.pc;
    const int n = pc.n, t = threadIdx.x;
    auto issue = [&](int item, int s) {
        int p, tx, ty;
        item_tile(pc, item, p, tx, ty);
        unsigned char* st = smem + s * G::POST_BYTES;
        fence_proxy_async();
        mbar_expect_tx(&bars[s], G::POST_TX);
        const int X0 = tx * TT - 4, Y0 = ty * TT - H;
        tma_load_3d(st + G::PE_OFF, &m_e, X0, Y0, p, &bars[s]);
        tma_load_3d(st + G::PEC_OFF, &m_ec, tx * (TT / 2) - 4, ty * (TT / 2) - H / 2, p, &bars[s]);
        tma_load_3d(st + G::PR_OFF, &m_r, X0, Y0, p, &bars[s]);
        tma_load_3d(st + G::PKW_OFF, &m_kw, X0, Y0, p, &bars[s]);
        tma_load_3d(st + G::PKS_OFF, &m_ks, X0, Y0, p, &bars[s]);
    };
    if (t == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    for (int i = t; i < G::EW * G::EH; i += blockDim.x) se[i] = T(0);
    __syncthreads();
    if (t == 0)
        for (int s = 0; s < STAGES - 1; ++s) {
            const int item = blockIdx.x + s * gridDim.x;
            if (item < pc.total) issue(item, s);
        }
    const bool own = t < G::NQ;
    const int qx = own ? t % G::QN : 0, qy = own ? t / G::QN : 0;
    const int bx = G::CX + 2 * qx, by = 2 * qy;
    const int ec0 = (2 * qy + 1) * G::EW + 2 * qx + 1;
    const bool inner = own && qx >= H / 2 && qx < H / 2 + TT / 2 && qy >= H / 2 && qy < H / 2 + TT / 2;
    uint32_t used[STAGES];
    for (int s = 0; s < STAGES; ++s) used[s] = 0;
    int it = 0;
    for (int item = blockIdx.x; item < pc.total; item += gridDim.x, ++it) {
        const int s = it % STAGES;
        if (t == 0) {
            const int ahead = item + (STAGES - 1) * gridDim.x;
            if (ahead < pc.total) issue(ahead, (it + STAGES - 1) % STAGES);
        }
        if (!mbar_wait_bounded(&bars[s], used[s] & 1u)) {
            if (t == 0) atomicExch(pc.err, 1);
            drain(bars, STAGES, used);
            return;
        }
        used[s]++;
        int p, tx, ty;
        item_tile(pc, item, p, tx, ty);
        unsigned char* st = smem + s * G::POST_BYTES;
        const T* sein = reinterpret_cast<const T*>(st + G::PE_OFF);
        const T* sec = reinterpret_cast<const T*>(st + G::PEC_OFF);
        const T* sr = reinterpret_cast<const T*>(st + G::PR_OFF);
        T* skw = reinterpret_cast<T*>(st + G::PKW_OFF);
        T* sks = reinterpret_cast<T*>(st + G::PKS_OFF);
        const int X0 = tx * TT - 4, Y0 = ty * TT - H;
        const int tpr = n / TT;
        if (tx == tpr - 1 || ty == tpr - 1) {
            patch_walls(skw, G::KWX, G::RY, X0, Y0, sks, G::BX, G::RY + 1, X0, Y0, n, a.E + (size_t)p * n, a.Nn + (size_t)p * n);
            __syncthreads();
        }
        const int gx = X0 + bx, gy = Y0 + by;
        Quad<T> Q;
        if (own) {
            load_quad<T, H>(Q, sr, nullptr, skw, sks, T(0), false, bx, by, gx, gy, n);
            // quad parent: coarse (gx/2, gy/2); box origin (16 tx - 4, 16 ty - H/2)
            const T ecv = a.cc * sec[qy * G::CW + qx + 4 - H / 2];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = (by + (k >> 1)) * G::BX + bx + (k & 1);
                se[ec0 + (k >> 1) * G::EW + (k & 1)] = Q.inv[k] != T(0) ? sein[c] + ecv : T(0);
            }
        }
        __syncthreads();
#pragma unroll
        for (int sw = 0; sw < NU; ++sw) {
            if (own) { gs_cell<T, G::EW>(se, ec0, Q, 1, false); gs_cell<T, G::EW>(se, ec0, Q, 2, false); }
            __syncthreads();
            if (own) { gs_cell<T, G::EW>(se, ec0, Q, 0, false); gs_cell<T, G::EW>(se, ec0, Q, 3, false); }
            __syncthreads();
        }
        const size_t base = (size_t)p * n * n;
        double rz = 0.0;
        if (inner) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const T ev = se[ec0 + (k >> 1) * G::EW + (k & 1)];
                a.e_out[base + (size_t)(gy + (k >> 1)) * n + gx + (k & 1)] = ev;
                rz += (double)Q.r[k] * (double)ev;
            }
        }
        if (a.cg) {
            const double tot = block_sum(rz, red);
            if (t == 0) a.part_rz[(size_t)p * pc.ntiles + (ty * tpr + tx)] = tot;
        }
        __syncthreads();
    }
}

}  // namespace smcgm
