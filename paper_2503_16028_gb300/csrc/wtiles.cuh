// Warp-per-tile kernels of the tiled multigrid/CG levels.
//
// A work item is one 16 x 16 tile of one active particle and is processed by
// one warp on its own: the warp's lanes own the 2 x 2 quads of the smoothing
// region (tile plus a halo of H = 2 nu cells), hold each quad's right-hand
// side, face coefficients and 1/D in registers, and keep only the correction
// in a per-warp shared array with a zero border.  Warps never wait for one
// another (__syncwarp only), so an SM keeps ~16 tiles in flight and their
// global loads -- all issued up front -- overlap the smoothing of other tiles.
//
// Quad cells (0,0), (1,1) are red and (1,0), (0,1) black (tile origins are
// even), so each half-sweep updates two cells per quad with no colour test;
// the quad's residuals sum to its restricted value and it shares one parent
// for the prolongation.  Tile origins are even and n is even, so a quad lies
// wholly inside or wholly outside the grid; outside quads keep e = 0.  Every
// half-sweep updates the whole region: an error can enter only at the region
// edge and moves one cell per half-sweep, which the halo H = 2 nu keeps out of
// the tile interior (the first pre-smoothing half-sweep is pointwise from zero).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <type_traits>

namespace smcgm {

constexpr int WT = 16;            // tile edge of the warp kernels
constexpr int WPB = 4;            // warps per block

// WI: warps per work item (1, or 2 for the FP64 solver's coarser levels: the item's quads spread
// over 64 lanes, so each lane holds fewer slots and registers).
template <typename T, int H, int WI = 1>
struct WGeo {
    static constexpr int LANES = 32 * WI;              // lanes that share the item
    static constexpr int RW = WT + 2 * H;              // region edge
    static constexpr int QW = RW / 2;                  // quads per region edge
    static constexpr int NQ = QW * QW;
    // With one sweep (H = 2) the region's four corner quads feed the tile only
    // through one red cell each (two of them, none for the other two corners),
    // so they leave the slots and are handled by a short separate step: the
    // remaining 96 quads fill exactly three slots.
    static constexpr bool CORNERS = (H == 2);
    static constexpr int NQM = CORNERS ? NQ - 4 : NQ;  // quads kept in the slots
    static constexpr int SLOTS = (NQM + LANES - 1) / LANES;   // quads per lane
    static constexpr int IQ = WT / 2;                  // tile quads per edge
    static constexpr int ISL = IQ * IQ / LANES;        // slots that hold tile quads (the rest: halo)
    // The correction lives in four planes, one per quad cell k, each a grid of
    // quads with a zero border: cell k of the quad at (qx, qy) is at
    // k PL + (qy + 1) QS + qx + 1.  With the quad-row stride QS = 24 (= 24 mod
    // 32) the 8 x 4 quads of a tile slot fall on 32 distinct banks, so the
    // same-colour accesses of a half-sweep are conflict-free.
    static constexpr int QS = 24;
    static constexpr int QR = QW + 2;
    static constexpr int PL = QS * QR;
    // When two planes fit side by side in a quad row (H = 2: 2 x 12 <= 24),
    // planes 1 and 3 sit 12 words to the right of planes 0 and 2 (a constant
    // shift keeps the accesses conflict-free) and the array halves.
    static constexpr bool PACK = 2 * QR <= QS;
    static constexpr int PO1 = PACK ? QR : PL;            // offset of plane 1 from plane 0
    static constexpr int PO2 = PACK ? PL : 2 * PL;        // plane 2
    static constexpr int PO3 = PO2 + PO1;                 // plane 3
    static constexpr int EN = PACK ? 2 * PL : 4 * PL;
    static constexpr __host__ __device__ int po(int k) { return k == 0 ? 0 : k == 1 ? PO1 : k == 2 ? PO2 : PO3; }
    static_assert(QW + 2 <= QS, "quad row fits the plane stride");
    static_assert(IQ * IQ % LANES == 0, "tile quads fill whole slots");
};

// Synchronisation of the lanes that share a work item: the warp, or its pair of
// warps (named barrier 1 + pair index, 64 threads; both warps of a pair hold the
// same item and reach every barrier of it, so no barrier waits on an absent warp).
template <int WI> __device__ __forceinline__ void item_sync();
template <> __device__ __forceinline__ void item_sync<1>() { __syncwarp(); }
template <> __device__ __forceinline__ void item_sync<2>() {
    asm volatile("bar.sync %0, 64;" ::"r"(1 + (int)(threadIdx.x >> 6)) : "memory");
}

// Position (qx, qy) in the region of a warp's quad qi: the tile's quads come
// first (slots 0 .. ISL-1, always inside the grid), then the halo ring.  Keeping
// the tile quads in their own slots lets the per-slot CG update, stores and
// restriction be decided at compile time and their registers exist only for
// those slots.  H = 2: the ring without its corners (low band, high band, west
// side, east side; 8 quads each).  Otherwise the whole ring as the band of
// lowest rows, the band of highest rows and the two side bands.
template <int H>
__host__ __device__ inline void quad_pos(int qi, int& qx, int& qy) {
    constexpr int QW = (WT + 2 * H) / 2, HB = H / 2, IQ = WT / 2;
    if (qi < IQ * IQ) { qx = HB + qi % IQ; qy = HB + qi / IQ; return; }
    int h = qi - IQ * IQ;
    if (H == 2) {
        const int side = h / IQ, j = 1 + h % IQ;
        qx = side == 0 || side == 1 ? j : side == 2 ? 0 : QW - 1;
        qy = side == 2 || side == 3 ? j : side == 0 ? 0 : QW - 1;
        return;
    }
    if (h < HB * QW) { qx = h % QW; qy = h / QW; return; }
    h -= HB * QW;
    if (h < HB * QW) { qx = h % QW; qy = QW - HB + h / QW; return; }
    h -= HB * QW;
    const int c = h % (2 * HB);
    qy = HB + h / (2 * HB);
    qx = c < HB ? c : IQ + c;
}

struct WArgs {
    int n, ntiles, total;   // total = active particles x tiles (when nact is null)
    int lg_tpr;             // log2 of the tiles per row, n / 16 (n is a power of two)
    const int* list;        // active particle indices
    int* err;               // set to 1 by a staged kernel whose bounded wait timed out
    const int* nact;        // device count of active particles: total = *nact x ntiles
};

// Work items of a launch: the active particles' tiles, counted on the device when the
// launch was sized before the count was known (a launch inside a CUDA graph).
__device__ inline int work_total(const WArgs& a) { return a.nact ? *a.nact * a.ntiles : a.total; }

// Work item -> index in the active list, tile of the particle and its coordinates.
// The tiles per row and per particle are powers of two, so these are shifts and
// masks rather than divisions by run-time values.
__device__ inline void item_tile(const WArgs& a, int item, int& pi, int& tile, int& tx, int& ty) {
    const int lt = a.lg_tpr;
    pi = item >> (2 * lt);
    tile = item & ((1 << (2 * lt)) - 1);
    tx = tile & ((1 << lt) - 1);
    ty = tile >> lt;
}

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

template <typename T>
__device__ inline void ld2(const T* p, T& a, T& b) {
    const typename Vec2<T>::type v = *reinterpret_cast<const typename Vec2<T>::type*>(p);
    a = v.x;
    b = v.y;
}
template <typename T>
__device__ inline void st2(T* p, T a, T b) {
    typename Vec2<T>::type v;
    v.x = a;
    v.y = b;
    *reinterpret_cast<typename Vec2<T>::type*>(p) = v;
}

// Face coefficients as stored (the solver's own type, or BF16 for the BF16
// smoother) read as the solver's type: a pair at an even cell, or one value.
template <typename T>
__device__ inline void ldf2(const T* p, T& a, T& b) { ld2(p, a, b); }
__device__ inline void ldf2(const __nv_bfloat16* p, float& a, float& b) {
    const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
    a = v.x;
    b = v.y;
}
template <typename T>
__device__ inline T ldf1(const T* p) { return *p; }
__device__ inline float ldf1(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// Sum over the warp in the solver's own precision (a tile's partial of a CG
// dot product: FP32 for the FP32 solver, keeping the FP64 pipe free), widened
// to double for the per-particle sums over tiles.
template <typename T>
__device__ inline double warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return (double)v;
}

// Quad data: cells k = 0..3 are (0,0), (1,0), (0,1), (1,1).
template <typename T>
struct WQuad {
    T r[4], w[4], e[4], s[4], n[4], inv[4];
};

// Raw loads of a quad at global (gx, gy) (inside the grid): west faces of its
// two columns and of the column to the east (wall E at the grid edge), south
// faces of its two rows and of the row to the north (wall Nn at the edge).
template <typename T>
struct WRaw {
    T a0, a1, ea, b0, b1, eb;      // west faces rows gy, gy+1; east face of column gx+1
    T s0, s1, m0, m1, t0, t1;      // south faces rows gy, gy+1, gy+2 (north of gy+1)
};

template <typename T, typename F>
__device__ inline void load_faces_raw(WRaw<T>& R, const F* kw, const F* ks, const T* E, const T* Nn, int n, int gx, int gy) {
    ldf2(kw + (size_t)gy * n + gx, R.a0, R.a1);
    ldf2(kw + (size_t)(gy + 1) * n + gx, R.b0, R.b1);
    R.ea = gx + 2 < n ? ldf1(kw + (size_t)gy * n + gx + 2) : E[gy];
    R.eb = gx + 2 < n ? ldf1(kw + (size_t)(gy + 1) * n + gx + 2) : E[gy + 1];
    ldf2(ks + (size_t)gy * n + gx, R.s0, R.s1);
    ldf2(ks + (size_t)(gy + 1) * n + gx, R.m0, R.m1);
    if (gy + 2 < n) ldf2(ks + (size_t)(gy + 2) * n + gx, R.t0, R.t1);
    else { R.t0 = Nn[gx]; R.t1 = Nn[gx + 1]; }
}

// 1/D of the smoother.  The smoother only has to be a fixed symmetric
// preconditioner, so FP32 uses the one-instruction approximate reciprocal.
template <typename T> __device__ inline T smoother_rcp(T d);
template <> __device__ inline float smoother_rcp<float>(float d) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    return r;
}
template <> __device__ inline double smoother_rcp<double>(double d) { return recip_nr(d); }

template <typename T>
__device__ inline void faces_from_raw(WQuad<T>& Q, const WRaw<T>& R) {
    Q.w[0] = R.a0; Q.e[0] = R.a1; Q.w[1] = R.a1; Q.e[1] = R.ea;
    Q.w[2] = R.b0; Q.e[2] = R.b1; Q.w[3] = R.b1; Q.e[3] = R.eb;
    Q.s[0] = R.s0; Q.n[0] = R.m0; Q.s[1] = R.s1; Q.n[1] = R.m1;
    Q.s[2] = R.m0; Q.n[2] = R.t0; Q.s[3] = R.m1; Q.n[3] = R.t1;
#pragma unroll
    for (int k = 0; k < 4; ++k) Q.inv[k] = smoother_rcp(Q.w[k] + Q.e[k] + Q.s[k] + Q.n[k]);
}

// Offset, from the quad base b = (qy + 1) QS + qx + 1, of cell k of the quad
// (dir = 4) or of its west, east, south, north neighbour (dir = 0..3).
template <class G>
__device__ __forceinline__ constexpr int qoff(int k, int dir) {
    // cells: 0 = (0,0), 1 = (1,0), 2 = (0,1), 3 = (1,1)
    constexpr int QS = G::QS, P1 = G::PO1, P2 = G::PO2, P3 = G::PO3;
    return dir == 4 ? G::po(k)
         : k == 0 ? (dir == 0 ? P1 - 1 : dir == 1 ? P1 : dir == 2 ? P2 - QS : P2)
         : k == 1 ? (dir == 0 ? 0 : dir == 1 ? 1 : dir == 2 ? P3 - QS : P3)
         : k == 2 ? (dir == 0 ? P3 - 1 : dir == 1 ? P3 : dir == 2 ? 0 : QS)
                  : (dir == 0 ? P2 : dir == 1 ? P2 + 1 : dir == 2 ? P1 : P1 + QS);
}

// Zeroes the border quads of the correction planes that the region's edge
// cells read (west border: planes 1, 3; east: 0, 2; south: 2, 3; north: 0, 1).
// Interior quads are always written before they are read, or belong to quads
// outside the grid, which their owners zero; no item writes the border, so a
// warp that keeps its array across items zeroes it once.
template <typename T, class G>
__device__ inline void zero_border(T* se, int lane) {
    constexpr int QW = G::QW, QS = G::QS;
    for (int i = lane; i < 8 * QW; i += G::LANES) {
        const int side = i / (2 * QW), rem = i % (2 * QW), which = rem / QW, j = rem % QW;
        int plane, pos;
        if (side == 0) { plane = which ? 3 : 1; pos = (j + 1) * QS; }
        else if (side == 1) { plane = which ? 2 : 0; pos = (j + 1) * QS + QW + 1; }
        else if (side == 2) { plane = which ? 3 : 2; pos = j + 1; }
        else { plane = which ? 1 : 0; pos = (QW + 1) * QS + j + 1; }
        se[G::po(plane) + pos] = T(0);
    }
}

template <typename T, class G>
__device__ __forceinline__ void wgs(T* se, int b, const WQuad<T>& Q, int k, bool pointwise) {
    T num = Q.r[k];
    if (!pointwise)
        num += Q.w[k] * se[b + qoff<G>(k, 0)] + Q.e[k] * se[b + qoff<G>(k, 1)] + Q.s[k] * se[b + qoff<G>(k, 2)] +
               Q.n[k] * se[b + qoff<G>(k, 3)];
    se[b + qoff<G>(k, 4)] = num * Q.inv[k];
}

template <typename T>
struct WPreArgs {
    WArgs a;
    const T *Kw, *Ks, *E, *Nn, *rin, *q, *p;
    T *rout, *e_out, *rc, *x;
    const double* alpha;
    double* part_rr;
    int cg, want_rr;
    const __nv_bfloat16 *Kwb, *Ksb;   // BF16 smoother faces (kernels instantiated for them)
};

template <typename T>
struct WPostArgs {
    WArgs a;
    const T *Kw, *Ks, *E, *Nn, *r, *e_in, *ec;
    T cc;
    T* e_out;
    double* part_rz;
    int cg;
    const __nv_bfloat16 *Kwb, *Ksb;
};

// Inputs of one work item read straight from global memory.  (x0, y0) is the
// tile origin; every quad asked for lies inside the grid.  F: the storage
// type of the interior faces kw, ks (T, or BF16 for the BF16 smoother).
template <typename T, typename F = T>
struct GlobalSrc {
    static constexpr bool COMBINE_EARLY = false;
    const F *kw, *ks;
    const T *Ep, *Np, *a, *b, *x, *p;   // a: r, b: q (pre) or e_in (post)
    int n;
    __device__ void faces(WRaw<T>& R, int gx, int gy) const { load_faces_raw(R, kw, ks, Ep, Np, n, gx, gy); }
    __device__ void va(T* v, int gx, int gy) const {
        const int gi = gy * n + gx;
        ld2(a + gi, v[0], v[1]);
        ld2(a + gi + n, v[2], v[3]);
    }
    __device__ void vb(T* v, int gx, int gy) const {
        const int gi = gy * n + gx;
        ld2(b + gi, v[0], v[1]);
        ld2(b + gi + n, v[2], v[3]);
    }
    __device__ void xp(T* v, int gx, int gy) const {
        const int gi = gy * n + gx;
        ld2(x + gi, v[0], v[1]);
        ld2(x + gi + n, v[2], v[3]);
        ld2(p + gi, v[4], v[5]);
        ld2(p + gi + n, v[6], v[7]);
    }
    __device__ T parent(int m, int gx, int gy) const { return x[(gy >> 1) * m + (gx >> 1)]; }
    // right-hand side (and q) and the four faces of the single cell (gx, gy)
    __device__ void cell(int gx, int gy, bool withq, T& rv, T& qv, T& fw, T& fe, T& fs, T& fn) const {
        const int gi = gy * n + gx;
        rv = a[gi];
        qv = withq ? b[gi] : T(0);
        fw = ldf1(kw + gi);
        fe = gx + 1 < n ? ldf1(kw + gi + 1) : Ep[gy];
        fs = ldf1(ks + gi);
        fn = gy + 1 < n ? ldf1(ks + gi + n) : Np[gx];
    }
};

// Called once every input of a work item has been read from its source.
struct NoHook {
    __device__ void operator()() const {}
};

// Pre-smoothing of one work item (particle p, tile (tx, ty)) by one warp:
// nu = H/2 sweeps (red, black) from zero, residual, restriction; with CG
// (finest level, a compile-time switch) first r' = r - alpha q, x += alpha p,
// and |r'|^2.  The border of se is zero on entry (zero_border).
template <typename T, int H, bool CG, class Src, class Hook = NoHook, int WI = 1>
__device__ inline void wpre_item(const WPreArgs<T>& A, const Src& S, T* se, int lane, int p, int tile, int tx, int ty,
                                 Hook loaded = Hook(), const double* alpha_src = nullptr) {
    static_assert(WI == 1 || !CG, "the CG update and its sums are one warp's");
    using G = WGeo<T, H, WI>;
    constexpr int NU = H / 2;
    const int n = A.a.n;
    const size_t base = (size_t)p * n * n;
    const T al = CG ? (T)(alpha_src ? *alpha_src : A.alpha[p]) : T(0);   // alpha_src: a copy fetched ahead
    T* xg = A.x + base;
    T* routg = A.rout + base;
    WQuad<T> Q[G::SLOTS];
    int c0[G::SLOTS], gq[G::SLOTS];
    bool live[G::SLOTS];
    T rr = T(0);
    // phase 1: every load of every owned quad is issued before any is used
    // A source in shared memory combines r' = r - alpha q and x + alpha p as it
    // reads (fewer live registers); a global source keeps the raw loads until
    // phase 2 so that all of them are in flight together.
    constexpr bool early = Src::COMBINE_EARLY;
    constexpr int RQ = early ? 4 : 8, XP = early ? 4 : 8;
    WRaw<T> Rw[G::SLOTS];
    T rq[G::SLOTS][RQ];           // r (and q, unless combined)
    T xp[G::ISL][XP];             // x + alpha p, or x and p, on the tile quads (cg)
#pragma unroll
    for (int sl = 0; sl < G::SLOTS; ++sl) {
        const int qi = lane + G::LANES * sl;
        int qx, qy;
        quad_pos<H>(qi, qx, qy);
        const int gx = tx * WT - H + 2 * qx, gy = ty * WT - H + 2 * qy;
        live[sl] = sl < G::ISL || (qi < G::NQM && gx >= 0 && gx < n && gy >= 0 && gy < n);
        c0[sl] = (qy + 1) * G::QS + qx + 1;
        gq[sl] = gy * n + gx;
        if (live[sl]) {
            S.faces(Rw[sl], gx, gy);
            S.va(rq[sl], gx, gy);
            if (CG) {
                if constexpr (early) {
                    T qv[4], v[8];
                    S.vb(qv, gx, gy);
#pragma unroll
                    for (int k = 0; k < 4; ++k) rq[sl][k] -= al * qv[k];
                    if (sl < G::ISL) {
                        S.xp(v, gx, gy);
#pragma unroll
                        for (int k = 0; k < 4; ++k) xp[sl][k] = v[k] + al * v[4 + k];
                    }
                } else {
                    S.vb(&rq[sl][4], gx, gy);
                    if (sl < G::ISL) S.xp(xp[sl], gx, gy);
                }
            }
        } else if (qi < G::NQM) {
            const int c = c0[sl];
            se[c] = T(0); se[c + G::PO1] = T(0); se[c + G::PO2] = T(0); se[c + G::PO3] = T(0);
        }
    }
    if constexpr (G::CORNERS) {
        // Corner quads (lane 0: west-south, 1: east-south, 2: west-north, 3: east-north).
        // Only the red cells diagonal to the tile's corners, region (1, 1) and
        // (RW-2, RW-2), are ever read (by the black half-sweep next to the tile);
        // they get their pointwise first half-sweep value, the rest zeros.
        if (lane < 4) {
            const int qx = (lane & 1) ? G::QW - 1 : 0, qy = (lane & 2) ? G::QW - 1 : 0;
            T val = T(0);
            if (lane == 0 || lane == 3) {
                const int d = lane == 0 ? 1 : 0;          // cell (1,1) of the west-south quad, (0,0) of the east-north one
                const int gx = tx * WT - H + 2 * qx + d, gy = ty * WT - H + 2 * qy + d;
                if (gx >= 0 && gx < n && gy >= 0 && gy < n) {
                    T rv, qv, fw, fe, fs, fn;
                    S.cell(gx, gy, CG, rv, qv, fw, fe, fs, fn);
                    val = (CG ? rv - al * qv : rv) * smoother_rcp(fw + fe + fs + fn);
                }
            }
            const int c = (qy + 1) * G::QS + qx + 1;
            se[c] = lane == 3 ? val : T(0);
            se[c + G::PO1] = T(0);
            se[c + G::PO2] = T(0);
            se[c + G::PO3] = lane == 0 ? val : T(0);
        }
    }
    loaded();
    // phase 2: derived quantities and the CG update
#pragma unroll
    for (int sl = 0; sl < G::SLOTS; ++sl) {
        if (!live[sl]) continue;
        faces_from_raw(Q[sl], Rw[sl]);
#pragma unroll
        for (int k = 0; k < 4; ++k) Q[sl].r[k] = (early || !CG) ? rq[sl][k] : rq[sl][k] - al * rq[sl][4 + k];
        if (sl < G::ISL) {
            if (CG) {
                const int gi = gq[sl];
                T xv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) xv[k] = early ? xp[sl][k] : xp[sl][k] + al * xp[sl][4 + k];
                st2(xg + gi, xv[0], xv[1]);
                st2(xg + gi + n, xv[2], xv[3]);
                st2(routg + gi, Q[sl].r[0], Q[sl].r[1]);
                st2(routg + gi + n, Q[sl].r[2], Q[sl].r[3]);
            }
            if (CG || A.want_rr) {
#pragma unroll
                for (int k = 0; k < 4; ++k) rr += Q[sl].r[k] * Q[sl].r[k];
            }
        }
    }
    item_sync<WI>();
#pragma unroll
    for (int sw = 0; sw < NU; ++sw) {
#pragma unroll
        for (int sl = 0; sl < G::SLOTS; ++sl)
            if (live[sl]) { wgs<T, G>(se, c0[sl], Q[sl], 0, sw == 0); wgs<T, G>(se, c0[sl], Q[sl], 3, sw == 0); }
        item_sync<WI>();
#pragma unroll
        for (int sl = 0; sl < G::SLOTS; ++sl)
            if (live[sl]) { wgs<T, G>(se, c0[sl], Q[sl], 1, false); wgs<T, G>(se, c0[sl], Q[sl], 2, false); }
        item_sync<WI>();
    }
    const int m = n / 2;
#pragma unroll
    for (int sl = 0; sl < G::ISL; ++sl) {
        const int gi = gq[sl];
        const int qi = lane + G::LANES * sl;
        const int gx = tx * WT + 2 * (qi % G::IQ), gy = ty * WT + 2 * (qi / G::IQ);
        T rsum = T(0), ev[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int b = c0[sl];
            const WQuad<T>& q = Q[sl];
            ev[k] = se[b + qoff<G>(k, 4)];
            rsum += q.r[k] - ((q.w[k] + q.e[k] + q.s[k] + q.n[k]) * ev[k] -
                              (q.w[k] * se[b + qoff<G>(k, 0)] + q.e[k] * se[b + qoff<G>(k, 1)] +
                               q.s[k] * se[b + qoff<G>(k, 2)] + q.n[k] * se[b + qoff<G>(k, 3)]));
        }
        st2(A.e_out + base + gi, ev[0], ev[1]);
        st2(A.e_out + base + gi + n, ev[2], ev[3]);
        A.rc[(size_t)p * m * m + (gy >> 1) * m + (gx >> 1)] = rsum;
    }
    if constexpr (WI == 1) {
        if (CG || A.want_rr) {
            const double tot = warp_sum<T>(rr);
            if (lane == 0) A.part_rr[(size_t)p * A.a.ntiles + tile] = tot;
        }
    }
}

// Prolongation e + cc P ec, nu = H/2 sweeps (black, red), and with CG (the
// finest level) r.z, for one work item by one warp.  The border of se is zero
// on entry (zero_border).
template <typename T, int H, bool CG, class Src, class Hook = NoHook, int WI = 1>
__device__ inline void wpost_item(const WPostArgs<T>& A, const Src& S, T* se, int lane, int p, int tile, int tx, int ty,
                                  Hook loaded = Hook()) {
    static_assert(WI == 1 || !CG, "the r.z sum is one warp's");
    using G = WGeo<T, H, WI>;
    constexpr int NU = H / 2;
    const int n = A.a.n, m = n / 2;
    const size_t base = (size_t)p * n * n;
    WQuad<T> Q[G::SLOTS];
    int c0[G::SLOTS], gq[G::SLOTS];
    bool live[G::SLOTS];
    WRaw<T> Rw[G::SLOTS];
    T ev[G::SLOTS][5];            // e_in (4) and the parent correction
    // phase 1: all loads first
#pragma unroll
    for (int sl = 0; sl < G::SLOTS; ++sl) {
        const int qi = lane + G::LANES * sl;
        int qx, qy;
        quad_pos<H>(qi, qx, qy);
        const int gx = tx * WT - H + 2 * qx, gy = ty * WT - H + 2 * qy;
        live[sl] = sl < G::ISL || (qi < G::NQM && gx >= 0 && gx < n && gy >= 0 && gy < n);
        c0[sl] = (qy + 1) * G::QS + qx + 1;
        gq[sl] = gy * n + gx;
        if (live[sl]) {
            S.faces(Rw[sl], gx, gy);
            S.va(Q[sl].r, gx, gy);
            S.vb(ev[sl], gx, gy);
            ev[sl][4] = S.parent(m, gx, gy);
        } else if (qi < G::NQM) {
            const int c = c0[sl];
            se[c] = T(0); se[c + G::PO1] = T(0); se[c + G::PO2] = T(0); se[c + G::PO3] = T(0);
        }
    }
    if constexpr (G::CORNERS) {
        // Corner quads: only their prolongated values are read (by the black
        // half-sweep next to the tile); no corner cell is updated.
        if (lane < 4) {
            const int qx = (lane & 1) ? G::QW - 1 : 0, qy = (lane & 2) ? G::QW - 1 : 0;
            const int gx = tx * WT - H + 2 * qx, gy = ty * WT - H + 2 * qy;
            T v[4] = {T(0), T(0), T(0), T(0)};
            if (gx >= 0 && gx < n && gy >= 0 && gy < n) {
                S.vb(v, gx, gy);
                const T up = A.cc * S.parent(m, gx, gy);
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k] += up;
            }
            const int c = (qy + 1) * G::QS + qx + 1;
            se[c] = v[0]; se[c + G::PO1] = v[1]; se[c + G::PO2] = v[2]; se[c + G::PO3] = v[3];
        }
    }
    loaded();
    // phase 2: prolongation into the correction array, faces and 1/D
#pragma unroll
    for (int sl = 0; sl < G::SLOTS; ++sl) {
        if (!live[sl]) continue;
        faces_from_raw(Q[sl], Rw[sl]);
        const T up = A.cc * ev[sl][4];
        const int c = c0[sl];
        se[c] = ev[sl][0] + up;
        se[c + G::PO1] = ev[sl][1] + up;
        se[c + G::PO2] = ev[sl][2] + up;
        se[c + G::PO3] = ev[sl][3] + up;
    }
    item_sync<WI>();
#pragma unroll
    for (int sw = 0; sw < NU; ++sw) {
#pragma unroll
        for (int sl = 0; sl < G::SLOTS; ++sl)
            if (live[sl]) { wgs<T, G>(se, c0[sl], Q[sl], 1, false); wgs<T, G>(se, c0[sl], Q[sl], 2, false); }
        item_sync<WI>();
        // the last (red) half-sweep matters only on the tile: no later update reads the halo
#pragma unroll
        for (int sl = 0; sl < G::SLOTS; ++sl)
            if (live[sl] && (sw < NU - 1 || sl < G::ISL)) {
                wgs<T, G>(se, c0[sl], Q[sl], 0, false);
                wgs<T, G>(se, c0[sl], Q[sl], 3, false);
            }
        item_sync<WI>();
    }
    T rz = T(0);
#pragma unroll
    for (int sl = 0; sl < G::ISL; ++sl) {
        const int c = c0[sl];
        const T e0 = se[c], e1 = se[c + G::PO1], e2 = se[c + G::PO2], e3 = se[c + G::PO3];
        const int gi = gq[sl];
        st2(A.e_out + base + gi, e0, e1);
        st2(A.e_out + base + gi + n, e2, e3);
        if (CG) rz += Q[sl].r[0] * e0 + Q[sl].r[1] * e1 + Q[sl].r[2] * e2 + Q[sl].r[3] * e3;
    }
    if (CG) {
        const double tot = warp_sum<T>(rz);
        if (lane == 0) A.part_rz[(size_t)p * A.a.ntiles + tile] = tot;
    }
}

template <typename F>
struct FacePtrs {
    const F *kw, *ks;
};
template <typename F>
__device__ inline FacePtrs<F> make_pair_ptr(const F* kw, const F* ks) { return FacePtrs<F>{kw, ks}; }

// The interior faces a warp kernel reads: the solver's own, or the BF16 copies.
template <typename T, bool BF, class A>
__device__ inline auto smoother_faces(const A& args, size_t base) {
    if constexpr (BF) return make_pair_ptr(args.Kwb + base, args.Ksb + base);
    else return make_pair_ptr(args.Kw + base, args.Ks + base);
}

// One warp per work item, inputs loaded from global memory.  BF: the
// smoother's interior faces are the BF16 copies (FP32 solver only); the
// lower levels' BF16 pre-smoothing is held to 128 registers (16 warps per SM,
// as the FP32 kernel).
// WI = 2: a pair of warps per item (the FP64 solver's coarser levels, 3 blocks per SM; 6 for FP32).
template <typename T, int H, bool CG, bool BF = false, int WI = 1>
__global__ void __launch_bounds__(32 * WPB, WI == 2 ? (sizeof(T) == 4 ? 6 : 3) : (BF && !CG) ? 4 : 0) k_wpre(WPreArgs<T> A) {
    using G = WGeo<T, H, WI>;
    using F = typename std::conditional<BF, __nv_bfloat16, T>::type;
    constexpr int IPB = WPB / WI;                      // items per block
    __shared__ T sme[IPB][G::EN];
    const int slot = threadIdx.x / G::LANES, lane = threadIdx.x % G::LANES;
    const int item = blockIdx.x * IPB + slot;
    if (item >= work_total(A.a)) return;              // both warps of a pair leave together
    const int n = A.a.n;
    int pi, tile, tx, ty;
    item_tile(A.a, item, pi, tile, tx, ty);
    const int p = A.a.list[pi];
    const size_t base = (size_t)p * n * n;
    const auto fc = smoother_faces<T, BF>(A, base);
    GlobalSrc<T, F> S{fc.kw, fc.ks, A.E + (size_t)p * n, A.Nn + (size_t)p * n, A.rin + base, A.q + base,
                      A.x + base, A.p + base, n};
    zero_border<T, G>(sme[slot], lane);
    wpre_item<T, H, CG, GlobalSrc<T, F>, NoHook, WI>(A, S, sme[slot], lane, p, tile, tx, ty);
}

template <typename T, int H, bool CG, bool BF = false, int WI = 1>
__global__ void __launch_bounds__(32 * WPB, WI == 2 ? (sizeof(T) == 4 ? 6 : 3) : 0) k_wpost(WPostArgs<T> A) {
    using G = WGeo<T, H, WI>;
    using F = typename std::conditional<BF, __nv_bfloat16, T>::type;
    constexpr int IPB = WPB / WI;
    __shared__ T sme[IPB][G::EN];
    const int slot = threadIdx.x / G::LANES, lane = threadIdx.x % G::LANES;
    const int item = blockIdx.x * IPB + slot;
    if (item >= work_total(A.a)) return;              // both warps of a pair leave together
    const int n = A.a.n, m = n / 2;
    int pi, tile, tx, ty;
    item_tile(A.a, item, pi, tile, tx, ty);
    const int p = A.a.list[pi];
    const size_t base = (size_t)p * n * n;
    const auto fc = smoother_faces<T, BF>(A, base);
    GlobalSrc<T, F> S{fc.kw, fc.ks, A.E + (size_t)p * n, A.Nn + (size_t)p * n, A.r + base, A.e_in + base,
                      A.ec + (size_t)p * m * m, nullptr, n};
    zero_border<T, G>(sme[slot], lane);
    wpost_item<T, H, CG, GlobalSrc<T, F>, NoHook, WI>(A, S, sme[slot], lane, p, tile, tx, ty);
}

template <typename T>
struct WApplyArgs {
    WArgs a;
    const T *Kw, *Ks, *E, *Nn, *z, *pin;
    T *pout, *q;
    const double* betac;
    double* part_pq;
    int first;
};

// p <- z + beta p on the tile plus a one-cell ring, then q = A p and p.q on the tile.
// Lane l covers column l % 16 of rows l / 16 + 2 k (k < 8), so one warp access
// touches 16 consecutive words of two rows: in global memory two 64-byte row
// segments, in the staged p (row stride 48 = 16 mod 32) 32 distinct banks.
// All global loads (z, p, ring, faces) are issued before any is used.
// q is formed as the sum of the face fluxes k_f (p_c - p_nb), not as
// diag p_c - sum k_f p_nb: for a smooth p the differences are exact and the
// rounding error stays at the size of the fluxes, where the diagonal form
// loses it to cancellation.  CG's recursive residual r - alpha q then tracks
// the true residual of the FP32 iterate closely, and each refinement phase's
// reduction holds for the FP64 residual too.
// MINB: resident blocks per SM asked of the register allocator (7 for FP32:
// 72 registers without spills, 28 warps per SM to cover the load latency;
// 4 for FP64: 128 registers).
constexpr int WAPPLY_PW = 48;                 // staged p row stride (tile + ring: 18 columns used)
constexpr int WAPPLY_PR = WT + 2;             // staged rows

template <typename T>
__device__ inline void wapply_item(const WApplyArgs<T>& A, T* sp, int lane, int item) {
    constexpr int PW = WAPPLY_PW;
    constexpr int PR = WAPPLY_PR;
    const int n = A.a.n;
    int pi, tile, tx, ty;
    item_tile(A.a, item, pi, tile, tx, ty);
    const int p = A.a.list[pi];
    const size_t base = (size_t)p * n * n;
    const T* zg = A.z + base;
    const T* pg = A.pin + base;
    const T* kw = A.Kw + base;
    const T* ks = A.Ks + base;
    const bool first = A.first != 0;
    const T b = first ? T(0) : (T)A.betac[p];
    const int cx = lane & 15, ry = lane >> 4;
    const int gx = tx * WT + cx;
    // phase 1: loads
    T pv[8], pold[8], fw[8], fe[8], fs[8], fn[8], rz[2], rp[2];
    int rgi[2];
    bool rin[2];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int gy = ty * WT + ry + 2 * k;
        const int gi = gy * n + gx;
        pv[k] = zg[gi];
        pold[k] = first ? T(0) : pg[gi];
        fw[k] = kw[gi];
        fe[k] = gx + 1 < n ? kw[gi + 1] : A.E[(size_t)p * n + gy];
        fs[k] = ks[gi];
        fn[k] = gy + 1 < n ? ks[gi + n] : A.Nn[(size_t)p * n + gx];
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        const int side = i / WT, j = i % WT;
        int gxx, gyy;
        if (side == 0) { gxx = tx * WT - 1; gyy = ty * WT + j; }
        else if (side == 1) { gxx = tx * WT + WT; gyy = ty * WT + j; }
        else if (side == 2) { gxx = tx * WT + j; gyy = ty * WT - 1; }
        else { gxx = tx * WT + j; gyy = ty * WT + WT; }
        rin[h] = gxx >= 0 && gxx < n && gyy >= 0 && gyy < n;
        rgi[h] = gyy * n + gxx;
        rz[h] = rin[h] ? zg[rgi[h]] : T(0);
        rp[h] = (rin[h] && !first) ? pg[rgi[h]] : T(0);
    }
    // phase 2: p_new into shared memory
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        pv[k] += b * pold[k];
        sp[(ry + 2 * k + 1) * PW + cx + 1] = pv[k];
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        const int side = i / WT, j = i % WT;
        const int lx = side == 0 ? 0 : side == 1 ? PR - 1 : j + 1;
        const int ly = side == 2 ? 0 : side == 3 ? PR - 1 : j + 1;
        sp[ly * PW + lx] = rz[h] + b * rp[h];
    }
    __syncwarp();
    T pq = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int yy = ry + 2 * k;
        const int c = (yy + 1) * PW + cx + 1;
        const T q = fw[k] * (pv[k] - sp[c - 1]) + fe[k] * (pv[k] - sp[c + 1]) + fs[k] * (pv[k] - sp[c - PW]) +
                    fn[k] * (pv[k] - sp[c + PW]);
        const size_t gi = base + (size_t)(ty * WT + yy) * n + gx;
        A.pout[gi] = pv[k];
        A.q[gi] = q;
        pq += pv[k] * q;
    }
    const double tot = warp_sum<T>(pq);
    if (lane == 0) A.part_pq[(size_t)p * A.a.ntiles + tile] = tot;
}

template <typename T, int MINB>
__global__ void __launch_bounds__(32 * WPB, MINB) k_wapply(WApplyArgs<T> A) {
    __shared__ T smp[WPB][WAPPLY_PR * WAPPLY_PW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * WPB + warp;
    if (item >= work_total(A.a)) return;
    wapply_item<T>(A, smp[warp], lane, item);
}

}  // namespace smcgm
