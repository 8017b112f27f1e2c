// TMA-pipelined tile kernels of the finest CG level: the shared pipeline
// pieces and the operator application p <- z + beta p, q = A p.
//
// Each block is persistent: it walks the work items (active particle, 32 x 32
// tile) with a grid stride, and while it works on the current tile the TMA
// unit is already copying the next tiles' inputs into the other shared-memory
// stages (an mbarrier per stage counts the bytes in).  Boxes start at
// x = 32 tx - 4 (16-byte aligned for any element size) and at any y; cells
// outside the grid arrive as zeros.  The east and north wall faces live in
// separate 1-D arrays and are patched into the staged face tiles.
#pragma once
#include "tma.cuh"

namespace smcgm {

constexpr int TT = 32;              // tile edge
constexpr int TH = 4;               // halo (2 nu, nu = 2)
constexpr int TR = TT + 2 * TH;     // region edge (40)
constexpr int TKW = TR + 4;         // staged west-face columns (44 >= 41, multiple of 4)
constexpr int TPRE = Own<TR>::THREADS;   // 288

__host__ __device__ constexpr int align_elems(int bytes) { return (bytes + 127) / 128 * 128; }

// TMA destinations are kept 128-byte aligned whatever the dynamic shared-memory base.
__device__ inline unsigned char* align128(unsigned char* p) {
    return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 127) & ~uintptr_t(127));
}



template <typename T>
struct ApplyStage {   // z and p: 34 rows x 40 columns from (32 tx - 4, 32 ty - 1); faces of the tile only
    static constexpr int AR = TT + 2, AC = TR;
    static constexpr int FKW = TT + 4;        // west faces, columns 32 tx .. 32 tx + 35 (need 33)
    static constexpr int Z_OFF = 0;
    static constexpr int P_OFF = Z_OFF + align_elems(AR * AC * (int)sizeof(T));
    static constexpr int KW_OFF = P_OFF + align_elems(AR * AC * (int)sizeof(T));
    static constexpr int KS_OFF = KW_OFF + align_elems(TT * FKW * (int)sizeof(T));
    static constexpr int BYTES = KS_OFF + align_elems((TT + 1) * TT * (int)sizeof(T));
    static constexpr uint32_t TX_BASE = (uint32_t)sizeof(T) * (AR * AC + TT * FKW + (TT + 1) * TT);
    static constexpr uint32_t TX_P = (uint32_t)sizeof(T) * (AR * AC);
};

struct PipeCommon {
    int n, ntiles, total;        // total = active particles x tiles
    const int* list;             // active particle indices
    int* err;                    // set to 1 when an mbarrier wait times out
};



template <typename T>
struct ApplyArgs {
    PipeCommon pc;
    const T* E; const T* Nn;
    T* pout; T* q; const double* betac; double* part_pq; int first;
};

__device__ inline void item_tile(const PipeCommon& pc, int item, int& p, int& tx, int& ty) {
    const int pi = item / pc.ntiles, tile = item - pi * pc.ntiles;
    p = pc.list[pi];
    const int tpr = pc.n / TT;
    tx = tile % tpr;
    ty = tile / tpr;
}

// Wall faces that TMA cannot fetch (they are not in the face arrays): the east
// wall column of the west-face tile and the north wall row of the south-face tile.
template <typename T>
__device__ inline void patch_walls(T* skw, int kwcols, int kwrows, int kwx0, int kwy0, T* sks, int kscols, int ksrows, int ksx0,
                                   int ksy0, int n, const T* E, const T* Nn) {
    const int col = n - kwx0;
    if (col >= 0 && col < kwcols)
        for (int ly = threadIdx.x; ly < kwrows; ly += blockDim.x) {
            const int gy = kwy0 + ly;
            if (gy >= 0 && gy < n) skw[ly * kwcols + col] = E[gy];
        }
    const int row = n - ksy0;
    if (row >= 0 && row < ksrows)
        for (int lx = threadIdx.x; lx < kscols; lx += blockDim.x) {
            const int gx = ksx0 + lx;
            if (gx >= 0 && gx < n) sks[row * kscols + lx] = Nn[gx];
        }
}

// Bounded drain of the stages still in flight after a timeout.
__device__ inline void drain(uint64_t* bars, int stages, const uint32_t* phase_used) {
    for (int s = 0; s < stages; ++s) mbar_wait_bounded(&bars[s], phase_used[s] & 1u, 1u << 20);
}

// ---------------------------------------------------------------------------
// p <- z + beta p, q = A p, partial p.q.
// ---------------------------------------------------------------------------
template <typename T, int STAGES>
__global__ void __launch_bounds__(256) k_apply_tma(ApplyArgs<T> a, const __grid_constant__ CUtensorMap m_z,
                                                   const __grid_constant__ CUtensorMap m_p, const __grid_constant__ CUtensorMap m_kw,
                                                   const __grid_constant__ CUtensorMap m_ks) {
    using S = ApplyStage<T>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = align128(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * S::BYTES);
    T* sp = reinterpret_cast<T*>(smem + STAGES * S::BYTES + 128);   // p_new, AR x AC
    __shared__ double red[32];
    const PipeCommon& pc = a.pc;
    const int n = pc.n, t = threadIdx.x;
    const uint32_t txb = S::TX_BASE + (a.first ? 0u : S::TX_P);
    auto issue = [&](int item, int s) {
        int p, tx, ty;
        item_tile(pc, item, p, tx, ty);
        unsigned char* st = smem + s * S::BYTES;
        fence_proxy_async();
        mbar_expect_tx(&bars[s], txb);
        tma_load_3d(st + S::Z_OFF, &m_z, tx * TT - 4, ty * TT - 1, p, &bars[s]);
        if (!a.first) tma_load_3d(st + S::P_OFF, &m_p, tx * TT - 4, ty * TT - 1, p, &bars[s]);
        tma_load_3d(st + S::KW_OFF, &m_kw, tx * TT, ty * TT, p, &bars[s]);
        tma_load_3d(st + S::KS_OFF, &m_ks, tx * TT, ty * TT, p, &bars[s]);
    };
    if (t == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (t == 0)
        for (int s = 0; s < STAGES - 1; ++s) {
            const int item = blockIdx.x + s * gridDim.x;
            if (item < pc.total) issue(item, s);
        }
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
        unsigned char* st = smem + s * S::BYTES;
        const T* sz = reinterpret_cast<T*>(st + S::Z_OFF);
        const T* spi = reinterpret_cast<T*>(st + S::P_OFF);
        T* skw = reinterpret_cast<T*>(st + S::KW_OFF);
        T* sks = reinterpret_cast<T*>(st + S::KS_OFF);
        const int tpr = n / TT;
        if (tx == tpr - 1 || ty == tpr - 1) {
            patch_walls(skw, S::FKW, TT, tx * TT, ty * TT, sks, TT, TT + 1, tx * TT, ty * TT, n, a.E + (size_t)p * n,
                        a.Nn + (size_t)p * n);
        }
        const T b = a.first ? T(0) : (T)a.betac[p];
        const int X0 = tx * TT - 4, Y0 = ty * TT - 1;
        for (int idx = t; idx < S::AR * S::AC; idx += blockDim.x) {
            const int ly = idx / S::AC, lx = idx - ly * S::AC;
            const int gxx = X0 + lx, gyy = Y0 + ly;
            T v = T(0);
            if (gxx >= 0 && gxx < n && gyy >= 0 && gyy < n) v = a.first ? sz[idx] : sz[idx] + b * spi[idx];
            sp[idx] = v;
        }
        __syncthreads();
        const size_t base = (size_t)p * n * n;
        double pq = 0.0;
        for (int idx = t; idx < TT * TT; idx += blockDim.x) {
            const int j = idx / TT, i = idx - j * TT;
            const int c = (j + 1) * S::AC + (i + 4);
            const T w = skw[j * S::FKW + i], e = skw[j * S::FKW + i + 1];
            const T so = sks[j * TT + i], no = sks[(j + 1) * TT + i];
            const T pv = sp[c];
            const T qv = (w + e + so + no) * pv - (w * sp[c - 1] + e * sp[c + 1] + so * sp[c - S::AC] + no * sp[c + S::AC]);
            const size_t gi = base + (size_t)(ty * TT + j) * n + tx * TT + i;
            a.pout[gi] = pv;
            a.q[gi] = qv;
            pq += (double)pv * (double)qv;
        }
        const double tot = block_sum(pq, red);
        if (t == 0) a.part_pq[(size_t)p * pc.ntiles + (ty * tpr + tx)] = tot;
        __syncthreads();
    }
}

// dynamic shared memory: stages + mbarriers (128 B) + scratch + 128 B alignment slack
template <typename T, int STAGES> constexpr size_t apply_tma_smem() {
    return STAGES * ApplyStage<T>::BYTES + 256 + ApplyStage<T>::AR * ApplyStage<T>::AC * sizeof(T);
}

}  // namespace smcgm
