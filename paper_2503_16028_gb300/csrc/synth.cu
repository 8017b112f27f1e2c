// Field synthesis u = sum_{k,l} v_kl c_k cos(k pi x) c_l cos(l pi y) at the
// cell centres (the KL expansion of the prior, Sec. 2.1 / Sec. 3.2, eq. Fourier
// series), in FP64, and the whole 1D forward map of the elliptic problem.
// At cell centres x_i = (i + 1/2)/n the synthesis along one axis is a DCT-III
// of length n, so the separable 2D synthesis is two passes of fast cosine
// transforms (stage 1 along x, stage 2 along y).
#include "smcgm_internal.cuh"
#include "common.cuh"

namespace smcgm {

// ------------------------------------------------------------------------
// Fast cosine synthesis.  Both stages are DCT-III transforms of length n,
// X[i] = sum_k x_k cos(pi k (2i + 1) / (2n)), with x_k = c_k v_k for k < Km and
// 0 above, evaluated by Lee's recursive factorisation (B. G. Lee, "A new
// algorithm to compute the discrete cosine transform", IEEE Trans. ASSP 32,
// 1984): with x_e[m] = x_{2m} and y[m] = x_{2m+1} + x_{2m-1},
//   X[i] = G[i] + H[i],  X[n-1-i] = G[i] - H[i],  i < n/2,
//   G = DCT-III_{n/2}(x_e),  H[i] = DCT-III_{n/2}(y)[i] / (2 cos(pi (2i + 1) / (2n))).
// The recursion is unrolled into log2 n top-down splitting levels and log2 n
// bottom-up butterfly levels, O(n log n) FP64 operations per transform
// instead of O(n Km).  One warp per transform (warp-synchronous); a block
// handles 16 transforms so that its input and output rows are contiguous
// (128-byte rows), and three blocks fit an SM.
// Stage 1 (along x, one transform per y-mode l) writes T^T[i][l]; stage 2
// (along y, one transform per column i) writes U[j][i].
// ------------------------------------------------------------------------
// FCT_T (transforms per block) and FCT_WARPS, and the block's shared memory, are in
// smcgm_internal.cuh (the grid-size limit of the configuration follows from them).

// Arithmetic of the transforms: FP64, or df32 on the FP32 pipes for the
// mixed-precision forward solve (u to ~1e-13 absolute; the coefficients need
// FP64 accuracy only to ~1e-13 relative, far below the solver tolerance).
struct F64Ops {
    using V = double;
    using W = double;    // twiddle
    static __device__ V zero() { return 0.0; }
    static __device__ V add(V a, V b) { return a + b; }
    static __device__ V sub(V a, V b) { return a - b; }
    static __device__ V mul(V a, W t) { return a * t; }
    static __device__ V from_input(double x) { return x; }
    static __device__ double to_double(V v) { return v; }
    // the pair (v[0], v[1]) of a 16-byte aligned address, in one load
    static __device__ void load_pair(const V* v, V& a, V& b) {
        const double2 t = *reinterpret_cast<const double2*>(v);
        a = t.x;
        b = t.y;
    }
    static __device__ void store_pair(V* v, V a, V b) { *reinterpret_cast<double2*>(v) = make_double2(a, b); }
    static __device__ V shfl_up(V v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
    static __device__ V shfl(V v, int src) { return __shfl_sync(0xffffffffu, v, src); }
};
struct DfOps {
    using V = df32;
    using W = float2;
    static __device__ V zero() { return df32{0.f, 0.f}; }
    static __device__ V add(V a, V b) { return df_add(a, b); }
    static __device__ V sub(V a, V b) { return df_add(a, df_neg(b)); }
    static __device__ V mul(V a, W t) { return df_mul(a, df32{t.x, t.y}); }
    static __device__ V from_input(double x) { return df_from_double_bits(x); }
    static __device__ double to_double(V v) { return (double)v.hi + (double)v.lo; }
    static __device__ void load_pair(const V* v, V& a, V& b) {
        const float4 t = *reinterpret_cast<const float4*>(v);
        a = df32{t.x, t.y};
        b = df32{t.z, t.w};
    }
    static __device__ void store_pair(V* v, V a, V b) { *reinterpret_cast<float4*>(v) = make_float4(a.hi, a.lo, b.hi, b.lo); }
    static __device__ V shfl_up(V v, int d) {
        return df32{__shfl_up_sync(0xffffffffu, v.hi, d), __shfl_up_sync(0xffffffffu, v.lo, d)};
    }
    static __device__ V shfl(V v, int src) { return df32{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)}; }
};

template <class O> __device__ inline typename O::W sqrt2_of();
template <> __device__ inline double sqrt2_of<F64Ops>() { return M_SQRT2; }
template <> __device__ inline float2 sqrt2_of<DfOps>() {   // df32 split of sqrt(2): hi = round(sqrt 2), lo = round(sqrt 2 - hi)
    return make_float2(1.41421353816986083984375f, 2.42032343e-8f);
}

// fct_swz (smcgm_internal.cuh) places the elements of the two buffers around the
// register passes below.
template <bool SWZ>
__device__ __forceinline__ int fct_ix(int i) { return SWZ ? fct_swz(i) : i; }

// One butterfly level lm: G = src[o + i], H = src[o + h + i] (i < h = M/2) to
// X[o + i] = G + t_i H, X[o + M - 1 - i] = G - t_i H.
template <class O, bool SWZ>
__device__ __forceinline__ void fct_level(const typename O::V* src, typename O::V* dst, int N, int lm,
                                 const typename O::W* __restrict__ tw, int lane) {
    using V = typename O::V;
    const int M = 1 << lm, h = M >> 1, lh = lm - 1;
    const typename O::W* twa = tw + (h - 1);
    for (int g = lane; g < (N >> 1); g += 32) {
        const int o = (g >> lh) << lm, i = g & (h - 1);
        const V G = src[fct_ix<SWZ>(o + i)];
        const V ht = O::mul(src[fct_ix<SWZ>(o + h + i)], twa[i]);
        dst[o + i] = O::add(G, ht);
        dst[o + M - 1 - i] = O::sub(G, ht);
    }
}

// Butterfly levels lm and lm + 1 in one pass: the four values src[o2 + i],
// src[o2 + h + i], src[o2 + M + i], src[o2 + M + h + i] of level lm give, through
// it, the G and H of two output pairs (i and M - 1 - i) of level lm + 1, so a group
// of four is closed under both and shared memory is read and written once for the two.
template <class O, bool SWZ>
__device__ __forceinline__ void fct_level_pair(const typename O::V* src, typename O::V* dst, int N, int lm,
                                      const typename O::W* __restrict__ tw, int lane) {
    using V = typename O::V;
    const int M = 1 << lm, h = M >> 1, lh = lm - 1;
    const typename O::W* twa = tw + (h - 1);             // level lm
    const typename O::W* twb = tw + (M - 1);             // level lm + 1 (half size M)
    for (int g = lane; g < (N >> 2); g += 32) {
        const int o2 = (g >> lh) << (lm + 1), i = g & (h - 1);
        const typename O::W ta = twa[i];
        const V a = src[fct_ix<SWZ>(o2 + i)];
        const V bt = O::mul(src[fct_ix<SWZ>(o2 + h + i)], ta);
        const V c = src[fct_ix<SWZ>(o2 + M + i)];
        const V dt = O::mul(src[fct_ix<SWZ>(o2 + M + h + i)], ta);
        const V x0 = O::add(a, bt), x1 = O::sub(a, bt);   // level lm: o2 + i, o2 + M - 1 - i
        const V y0 = O::add(c, dt), y1 = O::sub(c, dt);   // o2 + M + i, o2 + 2M - 1 - i
        const V p = O::mul(y0, twb[i]);
        const V q = O::mul(y1, twb[M - 1 - i]);
        dst[o2 + i] = O::add(x0, p);
        dst[o2 + 2 * M - 1 - i] = O::sub(x0, p);
        dst[o2 + M - 1 - i] = O::add(x1, q);
        dst[o2 + M + i] = O::sub(x1, q);
    }
}

// The DCT-III of one row (N = 2^lgN >= 64 values) by one warp, ping-ponging between
// b0 and b1; returns the buffer holding the result.  Lee's network: splitting levels
// lgN .. 1, then butterfly levels 1 .. lgN.  Splitting levels down to segment size 16
// run one per shared-memory pass; the splitting levels of segment sizes 8 and 4 (that
// of size 2 is the identity) and the butterfly levels 1 .. 3 act within segments of 8
// consecutive values, so each lane takes whole segments through them in registers
// (one pass); the remaining butterfly levels run two per pass.  Every value goes
// through the same operations, in the same order, as one level at a time.
template <class O>
__device__ inline typename O::V* fct_warp(typename O::V* b0, typename O::V* b1, int N, int lgN,
                                          const typename O::W* __restrict__ tw, int lane) {
    using V = typename O::V;
    V* src = b0;
    V* dst = b1;
    const int half = N >> 1;
    // top-down splitting: segment size M -> [even | odd sums].  Thread idx reads
    // its pair (2m, 2m+1) in one 16-byte load and takes element 2m-1 from the
    // thread before it (a shuffle, or the last lane of the previous round).
    for (int lm = lgN; lm >= 4; --lm) {
        const int M = 1 << lm, h = M >> 1, lh = lm - 1;
        const bool last = lm == 4;                          // writes the register pass's input
        V carry = O::zero();
        for (int idx = lane; idx < half; idx += 32) {        // half is a multiple of 32: all lanes take part
            const int o = (idx >> lh) << lm, m = idx & (h - 1);
            V a0, a1;
            O::load_pair(src + o + 2 * m, a0, a1);
            V prev = O::shfl_up(a1, 1);
            if (lane == 0) prev = carry;
            carry = O::shfl(a1, 31);
            const V odd = m > 0 ? O::add(a1, prev) : a1;
            dst[last ? fct_swz(o + m) : o + m] = a0;
            dst[last ? fct_swz(o + h + m) : o + h + m] = odd;
        }
        __syncwarp();
        V* t = src; src = dst; dst = t;
    }
    // segments of 8 in registers: splitting (sizes 8, 4), butterflies 1, 2, 3
    {
        const typename O::W t1 = tw[0], t2a = tw[1], t2b = tw[2];
        for (int sg = lane; sg < (N >> 3); sg += 32) {
            const int o = sg << 3;
            V x[8];
#pragma unroll
            for (int j = 0; j < 4; ++j) O::load_pair(src + fct_swz(o + 2 * j), x[2 * j], x[2 * j + 1]);
            // splitting, segment size 8: [x0 x2 x4 x6 | x1, x3+x1, x5+x3, x7+x5]
            const V a4 = x[1], a5 = O::add(x[3], x[1]), a6 = O::add(x[5], x[3]), a7 = O::add(x[7], x[5]);
            // splitting, segment size 4, of [x0 x2 x4 x6] and [a4 a5 a6 a7]
            V b[8] = {x[0], x[4], x[2], O::add(x[6], x[2]), a4, a6, a5, O::add(a7, a5)};
            // butterfly level 1 (pairs)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const V ht = O::mul(b[2 * j + 1], t1);
                const V g = b[2 * j];
                b[2 * j] = O::add(g, ht);
                b[2 * j + 1] = O::sub(g, ht);
            }
            // butterfly level 2 (quads): i = 0, 1 with t = tw[1 + i]
            V d[8];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const V h0 = O::mul(b[4 * q + 2], t2a), h1 = O::mul(b[4 * q + 3], t2b);
                d[4 * q + 0] = O::add(b[4 * q + 0], h0);
                d[4 * q + 3] = O::sub(b[4 * q + 0], h0);
                d[4 * q + 1] = O::add(b[4 * q + 1], h1);
                d[4 * q + 2] = O::sub(b[4 * q + 1], h1);
            }
            // butterfly level 3 (the segment): i < 4 with t = tw[3 + i]
            V e[8];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const V ht = O::mul(d[4 + i], tw[3 + i]);
                e[i] = O::add(d[i], ht);
                e[7 - i] = O::sub(d[i], ht);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) O::store_pair(dst + fct_swz(o + 2 * j), e[2 * j], e[2 * j + 1]);
        }
        __syncwarp();
        V* t = src; src = dst; dst = t;
    }
    // bottom-up butterflies 4 .. lgN: one level alone first when their number is odd,
    // then two per pass; the first pass reads the register pass's rotated chunks
    int lm = 4;
    bool first = true;
    if ((lgN - 3) & 1) {
        fct_level<O, true>(src, dst, N, 4, tw, lane);
        __syncwarp();
        V* t = src; src = dst; dst = t;
        lm = 5;
        first = false;
    }
    for (; lm < lgN; lm += 2) {
        if (first) fct_level_pair<O, true>(src, dst, N, lm, tw, lane);
        else fct_level_pair<O, false>(src, dst, N, lm, tw, lane);
        first = false;
        __syncwarp();
        V* t = src; src = dst; dst = t;
    }
    return src;
}

// stage: 0 = along x (input V[k][l], FP64, one transform per l, output T^T[i][l]),
//        1 = along y (input T^T[i][l], one transform per i, output U[j][i]).
// The FP64 input of stage 0 is scaled by c_k in FP64 and then converted.
template <class O>
__global__ void __launch_bounds__(32 * FCT_WARPS, 3) k_fct(int stage, int n, int lgn, int Km, const double* __restrict__ in64,
                                                      const typename O::V* __restrict__ in, typename O::V* __restrict__ out,
                                                      const typename O::W* __restrict__ tw) {
    using V = typename O::V;
    extern __shared__ __align__(16) unsigned char fsm_raw[];
    V* fsm = reinterpret_cast<V*>(fsm_raw);
    const int SP = n + 1;                               // padded staging row
    V* stg = fsm;                                       // FCT_T x SP
    V* work = fsm + FCT_T * SP;                         // FCT_WARPS x 2n
    const int p = blockIdx.y;
    const int t0 = blockIdx.x * FCT_T;                  // first transform of the block
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t inb = stage == 0 ? (size_t)p * Km * Km : (size_t)p * n * Km;
    const size_t outb = stage == 0 ? (size_t)p * n * Km : (size_t)p * n * n;
    // stage 0: the inputs V[k][t0 .. t0 + 15] (a column per transform) go through the
    // staging rows, read coalesced along t; stage 1 reads each row T^T[t0 + t][0 .. Km)
    // straight into the transform's buffer
    if (stage == 0) {
        for (int idx = threadIdx.x; idx < FCT_T * Km; idx += blockDim.x) {
            const int k = idx / FCT_T, t = idx % FCT_T;
            stg[t * SP + k] = t0 + t < Km ? O::from_input(in64[inb + (size_t)k * Km + t0 + t] * (k == 0 ? 1.0 : M_SQRT2)) : O::zero();
        }
        __syncthreads();
    }
    V* b0 = work + warp * 2 * n;
    V* b1 = b0 + n;
    for (int t = warp; t < FCT_T; t += FCT_WARPS) {
        if (stage == 0) {
            for (int k = lane; k < n; k += 32) b0[k] = k < Km ? stg[t * SP + k] : O::zero();
        } else {
            const V* row = in + inb + (size_t)(t0 + t) * Km;
            for (int k = lane; k < n; k += 32) {
                const V v = k < Km ? row[k] : O::zero();
                b0[k] = (k == 0 || k >= Km) ? v : O::mul(v, sqrt2_of<O>());
            }
        }
        __syncwarp();
        const V* res = fct_warp<O>(b0, b1, n, lgn, tw, lane);
        for (int k = lane; k < n; k += 32) stg[t * SP + k] = res[k];
        __syncwarp();
    }
    __syncthreads();
    // write: stage 0 -> T^T[i][t0 + t]; stage 1 -> U[j][t0 + t]
    const int rowlen = stage == 0 ? Km : n;
    for (int idx = threadIdx.x; idx < FCT_T * n; idx += blockDim.x) {
        const int i = idx / FCT_T, t = idx % FCT_T;
        if (t0 + t < rowlen) out[outb + (size_t)i * rowlen + t0 + t] = stg[t * SP + i];
    }
}

template <class O>
static void launch_fct(Ctx& c, const double* X, int count, typename O::V* tmp, typename O::V* U, const typename O::W* tw) {
    const int n = c.n, Km = c.Km;
    int lgn = 0;
    while ((1 << lgn) < n) ++lgn;
    const size_t smem = fct_smem_bytes(n);
    static size_t attr = 0;
    if (attr < smem) {
        check(cudaFuncSetAttribute(k_fct<O>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "attr");
        attr = smem;
    }
    // stage 1: ceil(Km / 32) blocks per particle (transforms past Km are masked); stage 2: n / 32
    const int b1 = (Km + FCT_T - 1) / FCT_T, b2 = n / FCT_T;
    k_fct<O><<<dim3(b1, count), 32 * FCT_WARPS, smem, c.stream>>>(0, n, lgn, Km, X, nullptr, tmp, tw); ++c.pc.launches;
    k_fct<O><<<dim3(b2, count), 32 * FCT_WARPS, smem, c.stream>>>(1, n, lgn, Km, nullptr, tmp, U, tw); ++c.pc.launches;
    check(cudaGetLastError(), "synth2d");
}

void launch_synth2d(Ctx& c, const double* X, int count, double* U) {
    launch_fct<F64Ops>(c, X, count, c.fct_tmp, U, c.fct_tw);
}

// The field of the mixed-precision forward solve, as df32 pairs.
void launch_synth2d_df(Ctx& c, const double* X, int count, float2* U) {
    launch_fct<DfOps>(c, X, count, reinterpret_cast<df32*>(c.fct_tmp), reinterpret_cast<df32*>(U),
                      reinterpret_cast<const float2*>(c.fct_tw_df));
}

// ------------------------------------------------------------------------
// Analysis G = S^T g, the transpose of the synthesis (the last step of the
// potential gradient): G[k][l] = c_k c_l sum_{i,j} g[j][i] cos(k pi x_i)
// cos(l pi y_j), a DCT-II along each axis keeping the Km lowest outputs.  The
// network is the transpose of fct_warp's: the butterfly levels first, in
// reverse order (two per shared-memory pass), each mapping the pair
// (X[o + i], X[o + M - 1 - i]) to G = X[o + i] + X[o + M - 1 - i],
// H = t_i (X[o + i] - X[o + M - 1 - i]); then
// the splitting levels, in reverse order, x[2m] = e[m], x[2m + 1] =
// y[m] + y[m + 1] (y[h] = 0).
// ------------------------------------------------------------------------
// One transposed butterfly level lm: the pair (X[o + i], X[o + M - 1 - i]), i < h,
// to G = X[o + i] + X[o + M - 1 - i] at o + i and H = t_i (X[o + i] - X[o + M - 1 - i])
// at o + h + i; SWZ: the outputs go to the rotated chunks of fct_swz.
template <class O, bool SWZ>
__device__ __forceinline__ void fct_level_t(const typename O::V* src, typename O::V* dst, int N, int lm,
                                            const typename O::W* __restrict__ tw, int lane) {
    using V = typename O::V;
    const int M = 1 << lm, h = M >> 1, lh = lm - 1;
    const typename O::W* twa = tw + (h - 1);
    for (int g = lane; g < (N >> 1); g += 32) {
        const int o = (g >> lh) << lm, i = g & (h - 1);
        const V a = src[o + i], b = src[o + M - 1 - i];
        dst[fct_ix<SWZ>(o + i)] = O::add(a, b);
        dst[fct_ix<SWZ>(o + h + i)] = O::mul(O::sub(a, b), twa[i]);
    }
}

// Transposed butterfly levels lm + 1 and lm in one pass (the transpose of fct_level_pair):
// the four values at o2 + i, o2 + 2M - 1 - i, o2 + M - 1 - i, o2 + M + i map to o2 + i,
// o2 + h + i, o2 + M + i, o2 + M + h + i.
template <class O, bool SWZ>
__device__ __forceinline__ void fct_level_pair_t(const typename O::V* src, typename O::V* dst, int N, int lm,
                                                 const typename O::W* __restrict__ tw, int lane) {
    using V = typename O::V;
    const int M = 1 << lm, h = M >> 1, lh = lm - 1;
    const typename O::W* twa = tw + (h - 1);
    const typename O::W* twb = tw + (M - 1);
    for (int g = lane; g < (N >> 2); g += 32) {
        const int o2 = (g >> lh) << (lm + 1), i = g & (h - 1);
        const V A = src[o2 + i], B = src[o2 + 2 * M - 1 - i], C = src[o2 + M - 1 - i], D = src[o2 + M + i];
        const V x0 = O::add(A, B), x1 = O::add(C, D);
        const V y0 = O::mul(O::sub(A, B), twb[i]);
        const V y1 = O::mul(O::sub(C, D), twb[M - 1 - i]);
        const typename O::W ta = twa[i];
        dst[fct_ix<SWZ>(o2 + i)] = O::add(x0, x1);
        dst[fct_ix<SWZ>(o2 + h + i)] = O::mul(O::sub(x0, x1), ta);
        dst[fct_ix<SWZ>(o2 + M + i)] = O::add(y0, y1);
        dst[fct_ix<SWZ>(o2 + M + h + i)] = O::mul(O::sub(y0, y1), ta);
    }
}

// The transpose of fct_warp (N = 2^lgN >= 64): the butterfly levels lgN .. 4 two per
// shared-memory pass from the top (a last one alone when their number is odd; the last
// pass writes the rotated chunks of fct_swz), then each lane takes segments of 8 through
// the transposed butterfly levels 3, 2, 1 and the splitting levels of sizes 4 and 8 in
// registers, then the splitting levels 16 .. N (the level of size 2 is the identity);
// splitting maps x[2m] = e[m], x[2m + 1] = y[m] + y[m + 1] (y[h] = 0).  Every value goes
// through the same operations, in the same order, as one level at a time.
template <class O>
__device__ inline typename O::V* fct_warp_t(typename O::V* b0, typename O::V* b1, int N, int lgN,
                                            const typename O::W* __restrict__ tw, int lane) {
    using V = typename O::V;
    V* src = b0;
    V* dst = b1;
    const int half = N >> 1;
    const int c = lgN - 3;                              // butterfly levels lgN .. 4
    int lm = lgN - 1;
    for (int k = 0; k < c / 2; ++k, lm -= 2) {
        if (k == c / 2 - 1 && !(c & 1)) fct_level_pair_t<O, true>(src, dst, N, lm, tw, lane);
        else fct_level_pair_t<O, false>(src, dst, N, lm, tw, lane);
        __syncwarp();
        V* t = src; src = dst; dst = t;
    }
    if (c & 1) {
        fct_level_t<O, true>(src, dst, N, 4, tw, lane);
        __syncwarp();
        V* t = src; src = dst; dst = t;
    }
    {
        const typename O::W t1 = tw[0], t2a = tw[1], t2b = tw[2];
        for (int sg = lane; sg < (N >> 3); sg += 32) {
            const int o = sg << 3;
            V x[8];
#pragma unroll
            for (int j = 0; j < 4; ++j) O::load_pair(src + fct_swz(o + 2 * j), x[2 * j], x[2 * j + 1]);
            V d[8];                                      // transposed butterfly level 3
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                d[i] = O::add(x[i], x[7 - i]);
                d[4 + i] = O::mul(O::sub(x[i], x[7 - i]), tw[3 + i]);
            }
            V b[8];                                      // level 2 on each half
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                b[4 * q + 0] = O::add(d[4 * q + 0], d[4 * q + 3]);
                b[4 * q + 2] = O::mul(O::sub(d[4 * q + 0], d[4 * q + 3]), t2a);
                b[4 * q + 1] = O::add(d[4 * q + 1], d[4 * q + 2]);
                b[4 * q + 3] = O::mul(O::sub(d[4 * q + 1], d[4 * q + 2]), t2b);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {                 // level 1 on pairs
                const V a = b[2 * j], bb = b[2 * j + 1];
                b[2 * j] = O::add(a, bb);
                b[2 * j + 1] = O::mul(O::sub(a, bb), t1);
            }
            // splitting, size 4 on each half: [a0, a2 + a3, a1, a3]
            const V e0 = b[0], e1 = O::add(b[2], b[3]), e2 = b[1], e3 = b[3];
            const V e4 = b[4], e5 = O::add(b[6], b[7]), e6 = b[5], e7 = b[7];
            // splitting, size 8: [e0, e4 + e5, e1, e5 + e6, e2, e6 + e7, e3, e7]
            O::store_pair(dst + fct_swz(o + 0), e0, O::add(e4, e5));
            O::store_pair(dst + fct_swz(o + 2), e1, O::add(e5, e6));
            O::store_pair(dst + fct_swz(o + 4), e2, O::add(e6, e7));
            O::store_pair(dst + fct_swz(o + 6), e3, e7);
        }
        __syncwarp();
        V* t = src; src = dst; dst = t;
    }
    for (int ls = 4; ls <= lgN; ++ls) {
        const int M = 1 << ls, h = M >> 1, lh = ls - 1;
        const bool first = ls == 4;                      // reads the register pass's rotated chunks
        for (int idx = lane; idx < half; idx += 32) {
            const int o = (idx >> lh) << ls, m = idx & (h - 1);
            const V ev = src[first ? fct_swz(o + m) : o + m];
            const V y0 = src[first ? fct_swz(o + h + m) : o + h + m];
            dst[o + 2 * m] = ev;
            dst[o + 2 * m + 1] = m + 1 < h ? O::add(y0, src[first ? fct_swz(o + h + m + 1) : o + h + m + 1]) : y0;
        }
        __syncwarp();
        V* t = src; src = dst; dst = t;
    }
    return src;
}

// stage: 0 = along y (input g[j][i], FP64, one transform per column i, output
//            T^T[i][l] = c_l (DCT-II over j)[l] for l < Km),
//        1 = along x (input T^T[i][l], one transform per l, output G[k][l] =
//            c_k (DCT-II over i)[k] for k < Km, FP64).
template <class O>
__global__ void __launch_bounds__(32 * FCT_WARPS, 3) k_fct_t(int stage, int n, int lgn, int Km, const double* __restrict__ in64,
                                                        const typename O::V* __restrict__ in, typename O::V* __restrict__ out,
                                                        double* __restrict__ out64, const typename O::W* __restrict__ tw) {
    using V = typename O::V;
    extern __shared__ __align__(16) unsigned char fsm_raw[];
    V* fsm = reinterpret_cast<V*>(fsm_raw);
    const int SP = n + 1;
    V* stg = fsm;                                       // FCT_T x SP
    V* work = fsm + FCT_T * SP;                         // FCT_WARPS x 2n
    const int p = blockIdx.y;
    const int t0 = blockIdx.x * FCT_T;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntr = stage == 0 ? n : Km;                // transforms of this stage
    // load: stage 0 rows g[j][t0 .. t0+15]; stage 1 rows T^T[i][t0 .. t0+15]
    for (int idx = threadIdx.x; idx < FCT_T * n; idx += blockDim.x) {
        const int j = idx / FCT_T, t = idx % FCT_T;
        V v = O::zero();
        if (t0 + t < ntr)
            v = stage == 0 ? O::from_input(in64[(size_t)p * n * n + (size_t)j * n + t0 + t])
                           : in[(size_t)p * n * Km + (size_t)j * Km + t0 + t];
        stg[t * SP + j] = v;
    }
    __syncthreads();
    V* b0 = work + warp * 2 * n;
    V* b1 = b0 + n;
    for (int t = warp; t < FCT_T; t += FCT_WARPS) {
        for (int k = lane; k < n; k += 32) b0[k] = stg[t * SP + k];
        __syncwarp();
        const V* res = fct_warp_t<O>(b0, b1, n, lgn, tw, lane);
        for (int k = lane; k < Km; k += 32) stg[t * SP + k] = k == 0 ? res[k] : O::mul(res[k], sqrt2_of<O>());
        __syncwarp();
    }
    __syncthreads();
    if (stage == 0) {   // T^T[t0 + t][l], l < Km: one contiguous row per transform
        for (int idx = threadIdx.x; idx < FCT_T * Km; idx += blockDim.x) {
            const int t = idx / Km, l = idx % Km;
            out[(size_t)p * n * Km + (size_t)(t0 + t) * Km + l] = stg[t * SP + l];
        }
    } else {            // G[k][t0 + t] in FP64
        for (int idx = threadIdx.x; idx < FCT_T * Km; idx += blockDim.x) {
            const int k = idx / FCT_T, t = idx % FCT_T;
            if (t0 + t < Km) out64[(size_t)p * Km * Km + (size_t)k * Km + t0 + t] = O::to_double(stg[t * SP + k]);
        }
    }
}

template <class O>
static void launch_fct_t(Ctx& c, const double* g, int count, typename O::V* tmp, double* G, const typename O::W* tw) {
    const int n = c.n, Km = c.Km;
    int lgn = 0;
    while ((1 << lgn) < n) ++lgn;
    const size_t smem = fct_smem_bytes(n);
    static size_t attr = 0;
    if (attr < smem) {
        check(cudaFuncSetAttribute(k_fct_t<O>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "attr");
        attr = smem;
    }
    k_fct_t<O><<<dim3(n / FCT_T, count), 32 * FCT_WARPS, smem, c.stream>>>(0, n, lgn, Km, g, nullptr, tmp, nullptr, tw); ++c.pc.launches;
    k_fct_t<O><<<dim3((Km + FCT_T - 1) / FCT_T, count), 32 * FCT_WARPS, smem, c.stream>>>(1, n, lgn, Km, nullptr, tmp, nullptr, G,
                                                                                        tw); ++c.pc.launches;
    check(cudaGetLastError(), "analysis2d");
}

// G = S^T g for `count` grids (FP64 in and out), in df32 for the mixed-precision
// context (inputs and outputs FP64, ~1e-13 relative) and FP64 otherwise.
void launch_analysis2d(Ctx& c, const double* g, int count, double* G) {
    if (mixed_precision(c.cfg))
        launch_fct_t<DfOps>(c, g, count, reinterpret_cast<df32*>(c.fct_tmp), G, reinterpret_cast<const float2*>(c.fct_tw_df));
    else
        launch_fct_t<F64Ops>(c, g, count, c.fct_tmp, G, c.fct_tw);
}

// ------------------------------------------------------------------------
// Observation of the cell-centred solution (bilinear, odd reflection across
// the walls so the interpolant vanishes there) and the potential
// Phi = |F(u) - d|^2 / (2 sigma^2) (Sec. 2.1, eq. Phi).  One warp per particle.
// ------------------------------------------------------------------------
// Cell-centred FP64 solution of one particle.
struct DoubleGrid {
    const double* w;
    __device__ double at(size_t i) const { return w[i]; }
    __device__ DoubleGrid particle(size_t off) const { return DoubleGrid{w + off}; }
};

// w at cell (i, j), extended past the walls by odd reflection (w = 0 on the wall).
template <class W>
__device__ inline double wghost(const W& w, int n, int i, int j) {
    double s = 1.0;
    if (i < 0) { i = 0; s = -s; }
    if (i > n - 1) { i = n - 1; s = -s; }
    if (j < 0) { j = 0; s = -s; }
    if (j > n - 1) { j = n - 1; s = -s; }
    return s * w.at((size_t)j * n + i);
}

// One warp per particle: bilinear interpolation at the observation points and Phi.
template <class W>
__device__ inline void observe2d_body(int n, int count, int nobs, const W& w, const double* __restrict__ obs,
                                      const double* __restrict__ data, double inv2s2, double* __restrict__ Phi) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= count) return;
    const W wp = w.particle((size_t)warp * n * n);
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

__global__ void k_observe2d(int n, int count, int nobs, const double* __restrict__ w, const double* __restrict__ obs,
                            const double* __restrict__ data, double inv2s2, double* __restrict__ Phi) {
    observe2d_body(n, count, nobs, DoubleGrid{w}, obs, data, inv2s2, Phi);
}
void launch_observe(Ctx& c, const double* w, int count, double* Phi) {
    const double inv2s2 = 1.0 / (2.0 * c.cfg.sigma * c.cfg.sigma);
    const int threads = 256;
    const int blocks = (count * 32 + threads - 1) / threads;
    k_observe2d<<<blocks, threads, 0, c.stream>>>(c.n, count, c.nobs, w, c.obs, c.data, inv2s2, Phi); ++c.pc.launches;
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
                                                          c.u64); ++c.pc.launches;
    }
    check(cudaGetLastError(), "forward1d");
}

}  // namespace smcgm
