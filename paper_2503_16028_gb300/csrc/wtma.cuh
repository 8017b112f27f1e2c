// TMA-staged warp-tile kernels (FP32) of the tiled multigrid/CG levels.
//
// The work item, quad ownership and smoothing arithmetic are those of the
// warp-tile kernels (wpre_item / wpost_item), but a tile's inputs arrive in
// shared memory by TMA.  Each warp is persistent: it owns one staging buffer
// with an mbarrier and walks the work items with a grid-wide stride.  As soon
// as it has read a tile's inputs out of the buffer into registers, it starts
// the copies of its next tile into the same buffer, so the DRAM latency of
// that tile overlaps the smoothing of this one, and every resident warp keeps
// a whole tile of loads in flight.  Warps never wait for one another.
//
// Boxes start at x = 16 tx - 4 (16-byte aligned) and y = 16 ty - H; cells
// outside the grid arrive as zeros, and the wall faces (east and north) are
// read from the 1-D wall arrays.  The parent box of the prolongation starts at
// x = 8 tx - 4, y = 8 ty - H/2 on the next coarser grid.  With the BF16
// smoother the interior-face boxes hold 2-byte values; a box must start on a
// 16-byte boundary, so they start at x = 16 tx - 8 (a multiple of 8 values)
// and span 40 values (80 bytes) per row.
#pragma once
#include "tma.cuh"
#include "wtiles.cuh"

namespace smcgm {

constexpr int TW_WARPS = 4;       // warps per block of the staged kernels

__host__ __device__ constexpr int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Staged box geometry of a region with halo H; FB: bytes per stored interior
// face (4: FP32, 2: BF16).  Offsets count floats from the staging buffer's start.
template <int H, int FB = 4>
struct TGeo {
    static_assert(FB == 4 || FB == 2, "FP32 or BF16 faces");
    static constexpr int RW = WT + 2 * H;                    // region edge
    static constexpr int BX = round_up(WT + H + 4, 4);       // r, q, e: columns 16 tx - 4 .. 16 tx + 15 + H
    static constexpr int FXO = FB == 4 ? 4 : 8;              // face boxes start at column 16 tx - FXO
    static constexpr int FA = 16 / FB;                       // values per 16 bytes
    // west faces: columns 16 tx - FXO .. 16 tx + 16 + H; south faces: to column 16 tx + 15 + H.
    // BF16 rows are 40 values (80 bytes): the four quad rows a warp reads at once lie two
    // box rows apart, 160 bytes = 40 banks = 8 mod 32, so their 8-bank spans start on banks
    // 0, 8, 16, 24 and never share one (32-value rows would put all four on the same banks);
    // the extra columns are the next tile's, served by L2.
    static constexpr int KWE = FB == 4 ? round_up(WT + H + 1 + FXO, FA) : 40;
    static constexpr int KSE = FB == 4 ? round_up(WT + H + FXO, FA) : 40;
    static constexpr int CX = 16;                            // parent box: columns 8 tx - 4 .. 8 tx + 11
    static constexpr int CY = RW / 2;                        // parent box rows
    static constexpr int KW_OFF = 0;                                          // every box 128-byte aligned
    static constexpr int KS_OFF = KW_OFF + round_up(RW * KWE * FB / 4, 32);   // south faces: RW + 1 rows
    static constexpr int R_OFF = KS_OFF + round_up((RW + 1) * KSE * FB / 4, 32);
    static constexpr int V_OFF = R_OFF + round_up(RW * BX, 32);        // pre: q; post: e_in
    static constexpr int X_OFF = V_OFF + round_up(RW * BX, 32);        // pre: x (tile); post: parent e
    static constexpr int P_OFF = X_OFF + round_up(WT * WT, 32);        // pre: p (tile)
    static constexpr int PRE_STAGE = V_OFF;                            // without the CG vectors
    static constexpr int PRE_CG_STAGE = P_OFF + round_up(WT * WT, 32);
    static constexpr int POST_STAGE = X_OFF + round_up(CY * CX, 32);
    static constexpr uint32_t FACE_BYTES = (uint32_t)FB * (RW * KWE + (RW + 1) * KSE);
    static constexpr uint32_t REGION_BYTES = 4u * (RW * BX);
    static_assert((KWE * FB) % 16 == 0 && (KSE * FB) % 16 == 0, "box rows are whole 16-byte units");
    static_assert((FXO * FB) % 16 == 0, "face box origin 16 tx - FXO on a 16-byte boundary");
};

// Per-warp shared memory: the staging buffer, the correction array, the mbarrier.
template <int H, int STAGE>
struct TLayout {
    static constexpr int SE_OFF = STAGE;
    static constexpr int BAR_OFF = SE_OFF + round_up(WGeo<float, H>::EN, 32);
    // after the mbarrier (8 bytes): the next item's particle index (int) and its CG step
    // alpha (8-byte aligned), written by the lane that starts the item's copies
    static constexpr int NEXT_P_OFF = BAR_OFF + 2;
    static constexpr int NEXT_ALPHA_OFF = BAR_OFF + 4;
    static constexpr int WARP = BAR_OFF + 32;                          // floats per warp
    static constexpr size_t block_bytes() { return (size_t)TW_WARPS * WARP * 4 + 128; }
};

// Inputs of one work item read from its staging buffer.  F: the storage type
// of the interior faces (float, or BF16 for the BF16 smoother).
template <int H, typename F = float>
struct StagedSrc {
    static constexpr bool COMBINE_EARLY = true;
    using G = TGeo<H, (int)sizeof(F)>;
    const F *kw, *ks;                       // interior-face boxes (origin column x0 + 4 - FXO)
    const float *a, *b, *x, *p;             // a: r; b: q (pre) or e_in (post); x: x (pre) or parent e (post)
    const float *Ep, *Np;                   // wall faces of the particle (global)
    int n, x0, y0, tx0, ty0, cx0, cy0;     // box origins: region, tile, parent
    __device__ void faces(WRaw<float>& R, int gx, int gy) const {
        const int bx = gx - x0 + (G::FXO - 4), by = gy - y0;
        const F* k0 = kw + by * G::KWE + bx;
        ldf2(k0, R.a0, R.a1);
        ldf2(k0 + G::KWE, R.b0, R.b1);
        R.ea = gx + 2 < n ? ldf1(k0 + 2) : Ep[gy];
        R.eb = gx + 2 < n ? ldf1(k0 + G::KWE + 2) : Ep[gy + 1];
        const F* s0 = ks + by * G::KSE + bx;
        ldf2(s0, R.s0, R.s1);
        ldf2(s0 + G::KSE, R.m0, R.m1);
        if (gy + 2 < n) ldf2(s0 + 2 * G::KSE, R.t0, R.t1);
        else { R.t0 = Np[gx]; R.t1 = Np[gx + 1]; }
    }
    __device__ void va(float* v, int gx, int gy) const {
        const float* c = a + (gy - y0) * G::BX + gx - x0;
        ld2(c, v[0], v[1]);
        ld2(c + G::BX, v[2], v[3]);
    }
    __device__ void vb(float* v, int gx, int gy) const {
        const float* c = b + (gy - y0) * G::BX + gx - x0;
        ld2(c, v[0], v[1]);
        ld2(c + G::BX, v[2], v[3]);
    }
    __device__ void xp(float* v, int gx, int gy) const {
        const int c = (gy - ty0) * WT + gx - tx0;
        ld2(x + c, v[0], v[1]);
        ld2(x + c + WT, v[2], v[3]);
        ld2(p + c, v[4], v[5]);
        ld2(p + c + WT, v[6], v[7]);
    }
    __device__ float parent(int, int gx, int gy) const { return x[((gy >> 1) - cy0) * G::CX + (gx >> 1) - cx0]; }
    // right-hand side (and q) and the four faces of the single cell (gx, gy)
    __device__ void cell(int gx, int gy, bool withq, float& rv, float& qv, float& fw, float& fe, float& fs, float& fn) const {
        const int bx = gx - x0, by = gy - y0, fx = bx + (G::FXO - 4);
        rv = a[by * G::BX + bx];
        qv = withq ? b[by * G::BX + bx] : 0.f;
        fw = ldf1(kw + by * G::KWE + fx);
        fe = gx + 1 < n ? ldf1(kw + by * G::KWE + fx + 1) : Ep[gy];
        fs = ldf1(ks + by * G::KSE + fx);
        fn = gy + 1 < n ? ldf1(ks + (by + 1) * G::KSE + fx) : Np[gx];
    }
};

__device__ inline void item_decode(const WArgs& a, int item, int& p, int& tile, int& tx, int& ty) {
    int pi;
    item_tile(a, item, pi, tile, tx, ty);
    p = a.list[pi];
}

// The persistent pipeline of one warp: `issue(item)` (lane 0) starts the
// copies of an item into the staging buffer; `work(item, lane, refill)` reads
// them into registers, calls refill() (which starts the next item's copies)
// and computes.  A wait that does not complete within its limit sets *err,
// waits (again bounded) for the copies in flight and ends the warp.
template <class Issue, class Work>
__device__ inline void warp_pipeline(const WArgs& a, uint64_t* bar, int lane, Issue issue, Work work) {
    const int nw = gridDim.x * TW_WARPS;
    const int total = work_total(a);
    int item = blockIdx.x * TW_WARPS + (threadIdx.x >> 5);
    if (item >= total) return;
    if (lane == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
        issue(item);
    }
    __syncwarp();
    uint32_t ph = 0u;
    for (; item < total; item += nw) {
        const bool more = item + nw < total;
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar, ph));
        if (!ok) {
            if (lane == 0) {
                atomicExch(a.err, 1);
                mbar_wait_bounded(bar, ph, 1u << 20);
            }
            return;
        }
        ph ^= 1u;
        const int next = item + nw;
        auto refill = [&]() {
            __syncwarp();                 // every lane has read the buffer
            if (more && lane == 0) {
                fence_proxy_async();      // those reads come before the new copies
                issue(next);
            }
        };
        // The lane index is made opaque per item so that the per-quad positions
        // derived from it are recomputed instead of held in registers across items.
        int ln = lane;
        asm volatile("" : "+r"(ln));
        work(item, ln, refill);
        __syncwarp();
    }
}

// Pre-smoothing (see wpre_item); CG stages q, x and p as well.  FB: bytes per
// stored interior face (m_kw, m_ks map FP32 or BF16 faces).
template <int H, bool CG, int MINB, int FB = 4>
__global__ void __launch_bounds__(32 * TW_WARPS, MINB) k_tpre(WPreArgs<float> A, const __grid_constant__ CUtensorMap m_kw,
                                                        const __grid_constant__ CUtensorMap m_ks,
                                                        const __grid_constant__ CUtensorMap m_r,
                                                        const __grid_constant__ CUtensorMap m_q,
                                                        const __grid_constant__ CUtensorMap m_x,
                                                        const __grid_constant__ CUtensorMap m_p) {
    using G = TGeo<H, FB>;
    using F = typename std::conditional<FB == 2, __nv_bfloat16, float>::type;
    constexpr int STAGE = CG ? G::PRE_CG_STAGE : G::PRE_STAGE;
    using L = TLayout<H, STAGE>;
    constexpr uint32_t TX = G::FACE_BYTES + G::REGION_BYTES + (CG ? G::REGION_BYTES + 8u * WT * WT : 0u);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* wb = reinterpret_cast<float*>(align128(smem_raw)) + (threadIdx.x >> 5) * L::WARP;
    uint64_t* bar = reinterpret_cast<uint64_t*>(wb + L::BAR_OFF);
    const int lane = threadIdx.x & 31;
    const int n = A.a.n;
    int* next_p = reinterpret_cast<int*>(wb + L::NEXT_P_OFF);
    double* next_alpha = reinterpret_cast<double*>(wb + L::NEXT_ALPHA_OFF);
    auto issue = [&](int item) {
        int p, tile, tx, ty;
        item_decode(A.a, item, p, tile, tx, ty);
        mbar_expect_tx(bar, TX);
        const int x0 = tx * WT - 4, y0 = ty * WT - H;
        tma_load_3d(wb + G::KW_OFF, &m_kw, tx * WT - G::FXO, y0, p, bar);
        tma_load_3d(wb + G::KS_OFF, &m_ks, tx * WT - G::FXO, y0, p, bar);
        tma_load_3d(wb + G::R_OFF, &m_r, x0, y0, p, bar);
        if (CG) {
            tma_load_3d(wb + G::V_OFF, &m_q, x0, y0, p, bar);
            tma_load_3d(wb + G::X_OFF, &m_x, tx * WT, ty * WT, p, bar);
            tma_load_3d(wb + G::P_OFF, &m_p, tx * WT, ty * WT, p, bar);
            cp_async8(next_alpha, A.alpha + p);       // the item's alpha, in flight with its tiles
        }
        *next_p = p;
    };
    auto work = [&](int item, int ln, auto refill) {
        // the particle index and alpha were fetched when the item's copies started (its issue)
        if (CG && ln == 0) cp_async_wait_all_groups();
        __syncwarp();
        const int p = *next_p;
        const double al = CG ? *next_alpha : 0.0;
        int pi, tile, tx, ty;
        item_tile(A.a, item, pi, tile, tx, ty);
        const float* st = wb;
        StagedSrc<H, F> S{reinterpret_cast<const F*>(st + G::KW_OFF), reinterpret_cast<const F*>(st + G::KS_OFF),
                          st + G::R_OFF, st + G::V_OFF, st + G::X_OFF, st + G::P_OFF,
                          A.E + (size_t)p * n, A.Nn + (size_t)p * n, n, tx * WT - 4, ty * WT - H, tx * WT, ty * WT, 0, 0};
        // the border is zeroed per item here (once per warp in k_tpost): measured faster for this pass
        zero_border<float, WGeo<float, H>>(wb + L::SE_OFF, ln);
        wpre_item<float, H, CG>(A, S, wb + L::SE_OFF, ln, p, tile, tx, ty, refill, CG ? &al : nullptr);
    };
    warp_pipeline(A.a, bar, lane, issue, work);
}

// Prolongation and post-smoothing (see wpost_item); FB as for k_tpre.
template <int H, bool CG, int MINB, int FB = 4>
__global__ void __launch_bounds__(32 * TW_WARPS, MINB) k_tpost(WPostArgs<float> A, const __grid_constant__ CUtensorMap m_kw,
                                                         const __grid_constant__ CUtensorMap m_ks,
                                                         const __grid_constant__ CUtensorMap m_r,
                                                         const __grid_constant__ CUtensorMap m_e,
                                                         const __grid_constant__ CUtensorMap m_ec) {
    using G = TGeo<H, FB>;
    using F = typename std::conditional<FB == 2, __nv_bfloat16, float>::type;
    constexpr int STAGE = G::POST_STAGE;
    using L = TLayout<H, STAGE>;
    constexpr uint32_t TX = G::FACE_BYTES + 2u * G::REGION_BYTES + 4u * G::CY * G::CX;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* wb = reinterpret_cast<float*>(align128(smem_raw)) + (threadIdx.x >> 5) * L::WARP;
    uint64_t* bar = reinterpret_cast<uint64_t*>(wb + L::BAR_OFF);
    int* next_p = reinterpret_cast<int*>(wb + L::NEXT_P_OFF);
    const int lane = threadIdx.x & 31;
    const int n = A.a.n;
    auto issue = [&](int item) {
        int p, tile, tx, ty;
        item_decode(A.a, item, p, tile, tx, ty);
        mbar_expect_tx(bar, TX);
        const int x0 = tx * WT - 4, y0 = ty * WT - H;
        tma_load_3d(wb + G::KW_OFF, &m_kw, tx * WT - G::FXO, y0, p, bar);
        tma_load_3d(wb + G::KS_OFF, &m_ks, tx * WT - G::FXO, y0, p, bar);
        tma_load_3d(wb + G::R_OFF, &m_r, x0, y0, p, bar);
        tma_load_3d(wb + G::V_OFF, &m_e, x0, y0, p, bar);
        tma_load_3d(wb + G::X_OFF, &m_ec, tx * (WT / 2) - 4, ty * (WT / 2) - H / 2, p, bar);
        *next_p = p;
    };
    auto work = [&](int item, int ln, auto refill) {
        __syncwarp();
        const int p = *next_p;                       // written when the item's copies started
        int pi, tile, tx, ty;
        item_tile(A.a, item, pi, tile, tx, ty);
        const float* st = wb;
        StagedSrc<H, F> S{reinterpret_cast<const F*>(st + G::KW_OFF), reinterpret_cast<const F*>(st + G::KS_OFF),
                          st + G::R_OFF, st + G::V_OFF, st + G::X_OFF, nullptr,
                          A.E + (size_t)p * n, A.Nn + (size_t)p * n, n, tx * WT - 4, ty * WT - H, tx * WT, ty * WT,
                          tx * (WT / 2) - 4, ty * (WT / 2) - H / 2};
        wpost_item<float, H, CG>(A, S, wb + L::SE_OFF, ln, p, tile, tx, ty, refill);
    };
    zero_border<float, WGeo<float, H>>(wb + L::SE_OFF, lane);   // once: no item writes it
    warp_pipeline(A.a, bar, lane, issue, work);
}

template <int H, bool CG, int FB = 4> constexpr size_t tpre_smem() {
    return TLayout<H, CG ? TGeo<H, FB>::PRE_CG_STAGE : TGeo<H, FB>::PRE_STAGE>::block_bytes();
}
template <int H, int FB = 4> constexpr size_t tpost_smem() { return TLayout<H, TGeo<H, FB>::POST_STAGE>::block_bytes(); }

}  // namespace smcgm
