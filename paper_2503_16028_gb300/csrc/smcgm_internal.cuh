// Internal declarations shared by the CUDA translation units of libsmcgm.so.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/smcgm.h"
#include "df32.cuh"
#include "dfnormal.cuh"

namespace smcgm {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the
// published definition: ten rounds of two 32x32->64-bit products with the
// published multipliers; the key is bumped by the published Weyl constants.
// ---------------------------------------------------------------------------
enum Purpose : uint32_t { P_INIT = 1, P_COMP = 2, P_NORMAL = 3, P_ACCEPT = 4, P_RESAMPLE = 5, P_EMINIT = 6 };

struct U4 { uint32_t x, y, z, w; };

__host__ __device__ inline U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int rnd = 0; rnd < 10; ++rnd) {
        if (rnd > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

// U = (u53 + 1/2) 2^-53, u53 = top 27 bits of a, top 26 bits of b.  Exact in binary64.
__host__ __device__ inline double open53(uint32_t a, uint32_t b) {
    uint64_t u = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return ((double)u + 0.5) * 0x1.0p-53;
}

struct Key { uint32_t k0, k1; };
// Cosine-transform blocks (synthesis and its transpose): FCT_T transforms per
// block (16 x 8 bytes: whole 128-byte rows), FCT_WARPS warps.  A block stages
// FCT_T transforms of n + 1 values and gives each warp two n-value work rows,
// all in doubles (a df32 pair is 8 bytes too).
constexpr int FCT_T = 16;
constexpr int FCT_WARPS = 8;
constexpr size_t fct_smem_bytes(int n) { return 8 * ((size_t)FCT_T * (n + 1) + (size_t)FCT_WARPS * 2 * n); }
// Slot of element i (8 bytes) in the two work buffers around a transform's register
// pass, in which each lane takes a segment of 8 consecutive elements: each segment's
// four 16-byte chunks are rotated by ((i / 16) mod 4), so that the 8 lanes of a quarter
// warp, each reading or writing the j-th chunk of its own segment, hit 8 different
// 16-byte bank groups.  Pairs (2m, 2m + 1) stay together and in order.
__host__ __device__ inline int fct_swz(int i) { return (i & ~7) | ((((i >> 1) + (i >> 4)) & 3) << 1) | (i & 1); }
// Largest 2D grid: the transform block of a 1024-point grid would need 256 KB of
// shared memory, above the 227 KB a block can have.
constexpr int MAX_N2D = 512;

// False when CUDA reports `p` as host memory it does not know (an ordinary
// malloc or stack address), which a kernel must not dereference, or as device
// memory of another GPU than the current one (a kernel here would read it as a
// peer access, which faults unless peer access was enabled).  Device memory of
// the current GPU, managed and registered (mapped) host memory pass; so does a
// pointer whose query fails, which leaves the decision to the caller's contract
// rather than rejecting valid memory.
inline bool device_visible(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return true;
    }
    if (a.type == cudaMemoryTypeUnregistered) return false;
    if (a.type == cudaMemoryTypeDevice) {
        int dev = -1;
        if (cudaGetDevice(&dev) != cudaSuccess) {
            (void)cudaGetLastError();
            return true;
        }
        return a.device == dev;
    }
    return true;
}

inline Key key_of(unsigned long long seed) { return Key{(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)}; }

// ---------------------------------------------------------------------------
// Device arrays of one multigrid level for a batch of B particles.
// Kw[p][j][i]: coefficient of the west face of cell (i, j) (wall face for i = 0);
// Ks[p][j][i]: south face (wall face for j = 0); E[p][j]: east wall face of
// row j; Nn[p][i]: north wall face of column i.  Couplings across wall faces
// are zero; the wall faces only enter the diagonal.
// ---------------------------------------------------------------------------
template <typename T>
struct LevelArrays {
    int n = 0;
    T* Kw = nullptr; T* Ks = nullptr; T* E = nullptr; T* Nn = nullptr;
    T* r = nullptr;   // right-hand side at this level (levels >= 1)
    T* e = nullptr;   // pre-smoothed correction
    T* e2 = nullptr;  // post-smoothed correction (levels >= 1)
    // SMC_P_BF16SMOOTH_REFINE: BF16 copies of Kw and Ks for the smoother (tiled levels)
    __nv_bfloat16* Kwb = nullptr;
    __nv_bfloat16* Ksb = nullptr;
};

// The mixed-precision solver (FP32 inner solves, FP64-accurate refinement),
// with FP32 or BF16 smoother faces.
inline bool mixed_precision(const smc_config& cfg) {
    return cfg.precision == SMC_P_FP32_REFINE || cfg.precision == SMC_P_BF16SMOOTH_REFINE;
}
inline bool bf16_smoother(const smc_config& cfg) { return cfg.precision == SMC_P_BF16SMOOTH_REFINE; }

struct SolverScalars {       // per particle, device
    double *rz, *rr0, *rr, *pq, *alpha, *betac, *res2, *b2;
    int *act_in, *act_out, *iters, *flags;
    int *count;              // [0] active inner count, [1] active outer count, [2] max iters
};

// TMA descriptors of the tiled levels (boxes described in tiles.cuh).
// Tensor maps of the TMA-staged smoothing kernels (FP32 inner solver).
struct TmaMaps {
    CUtensorMap kw[12], ks[12], r[12], e[12], ec[12];   // per tiled level
    CUtensorMap kwb[12], ksb[12];                        // BF16 smoother faces (SMC_P_BF16SMOOTH_REFINE)
    CUtensorMap r0[2], q, x, p[2];                       // finest level, CG vectors
};

template <typename T>
struct InnerSolver {
    TmaMaps* maps = nullptr;
    int* list = nullptr;     // active particle indices (device)
    int* nact = nullptr;     // their count (device)
    int nlev = 0;            // number of levels down to 1 x 1
    int ntile_levels = 0;    // levels handled by the tiled kernels (n_l > coarse_top)
    int coarse_top = 0;      // first level handled by the one-block coarse kernel
    std::vector<LevelArrays<T>> lv;
    T *r[2] = {nullptr, nullptr}, *p[2] = {nullptr, nullptr};
    T *x = nullptr, *q = nullptr, *z = nullptr;
};

struct Partials { double *rr, *rz, *pq, *res; int ntiles; };

// Counters of the solves run inside a CUDA graph (device; the host reads them afterwards).
struct GraphCounters {
    unsigned long long cg_iterations, inner_solves, residuals, nonconv;
    int itmax, pad;
};

struct Ctx;

// kernels / launchers (defined in the .cu files)
void launch_prior_draw(Ctx& c, double* X, int N, uint32_t counter2, uint32_t purpose);
void launch_synth2d(Ctx& c, const double* X, int count, double* U);
void launch_synth2d_df(Ctx& c, const double* X, int count, float2* U);
void launch_analysis2d(Ctx& c, const double* g, int count, double* G);
void launch_setup_coeffs(Ctx& c, int count);
template <typename T> void launch_coarsen_all(Ctx& c, InnerSolver<T>& s, int count);
template <typename T> void build_tma_maps(Ctx& c, InnerSolver<T>& s);
int forward_solve(Ctx& c, const double* X, int count, double* Phi_out, double* w_out);
// Right-hand side of a batch of solves: one shared by every particle (stride 0)
// or one per particle (stride n*n); FP64 (b64) and, for the mixed-precision
// solver, as df32 pairs (bdf); |b|^2 per particle (b2pp) or common (b2const).
struct Rhs {
    const double* b64;
    const float2* bdf;
    size_t stride;
    const double* b2pp;
    double b2const;
};
Rhs shared_rhs(const Ctx& c);
int solve_batch(Ctx& c, int count, const Rhs& R, double* W);   // W: the FP64 solutions (count x n x n)
void forward_solve_graph(Ctx& c, const double* X, int count, double* Phi_out);   // into the graph being captured
void capture_move_steps(Ctx& c, int steps, int* acc_count);                      // into the graph being captured
void launch_mark_out_of_range(Ctx& c, int count, double* Phi);
void launch_observe(Ctx& c, const double* w, int count, double* Phi);
void launch_forward1d(Ctx& c, const double* X, int count, double* Phi, double* w_out);
// Schedule of a move read from device memory by the move kernels of a CUDA graph
// (t, beta, gamma and the Philox step of its first step); null: the host's values.
struct MoveSched {
    double t, beta, gamma;
    unsigned int step, pad;
};
void launch_move_tables(Ctx& c, const MoveSched* ms = nullptr);
void launch_propose(Ctx& c, const MoveSched* ms = nullptr, uint32_t step_off = 0);
void launch_accept(Ctx& c, int* acc_count, const MoveSched* ms = nullptr, uint32_t step_off = 0);
void launch_propose_pcnl(Ctx& c);
void launch_gmpcnl_terms(Ctx& c);
void launch_copy_accepted_gradients(Ctx& c);
void launch_accept_pcnl(Ctx& c, int* acc_count);
void launch_temper(Ctx& c, double* out5);
void launch_resample(Ctx& c);
double gm_fit_device(Ctx& c);
void factor_mixture(Ctx& c, const double* cov_host);   // Cholesky, inverse and log det of every C_j (device); waits
size_t cov_partial_doubles(int K, int r);               // scratch of the full-covariance contraction
void launch_propose_full(Ctx& c, const MoveSched* ms = nullptr, uint32_t step_off = 0);
void launch_moments(Ctx& c, double* mean, double* var);
void launch_grid_moments(Ctx& c, const double* mean_kl, double* mean_grid, double* var_grid);
int gradient_batch(Ctx& c, const double* X, int count, double* Phi_out, double* grad_out);   // largest CG iteration count

struct Ctx {
    smc_config cfg;
    std::vector<double> obs_h, data_h;
    cudaStream_t stream = nullptr;
    int dim = 2, n = 0, Km = 0, d = 0, N = 0, K = 1, r = 1, nobs = 0, B = 0;
    Key key{0, 0};
    // prior, basis and problem tables
    double *lam = nullptr, *sqrtlam = nullptr, *basis = nullptr, *b64 = nullptr, *obs = nullptr, *data = nullptr;
    int *S = nullptr, *slot = nullptr;
    // particle state
    double *X = nullptr, *X2 = nullptr, *V = nullptr, *Phi = nullptr, *Phi2 = nullptr, *PhiV = nullptr;
    double *logw = nullptr, *logalpha = nullptr, *lfwd = nullptr, *lrev = nullptr;
    unsigned char* acc = nullptr;
    int* idx = nullptr;
    int* icount = nullptr;     // small device integer scratch
    double* dscal = nullptr;   // small device double scratch (temper outputs etc.)
    // mixture and proposal tables
    double *gw = nullptr, *gmu = nullptr, *glam = nullptr;
    // full covariances on the mixture modes (cfg.full_cov): C_j, its Cholesky
    // factor L_j (lower), L_j^{-1} and log det L_j; glam holds diag(C_j)
    double *gcov = nullptr, *gL = nullptr, *gLi = nullptr, *glogdet = nullptr;
    double* covpart = nullptr;  // chunk partials of the covariance contraction (full_cov)
    double *tab = nullptr;     // per (j, s): c0, a, mu, sq; then per s: b; then per j: log w, cumulative w
    // EM scratch
    double *xsT = nullptr, *resp = nullptr, *nj = nullptr, *pooled = nullptr, *lse = nullptr, *gmax = nullptr;
    // forward-solve batch arrays
    double *u64 = nullptr, *Kw64 = nullptr, *Ks64 = nullptr, *E64 = nullptr, *N64 = nullptr, *w64 = nullptr;
    // mixed precision: FP64-accurate faces and right-hand side as df32 pairs (the
    // high parts of the faces are the inner solver's FP32 faces); the solution stays FP64
    float *Kwlo = nullptr, *Kslo = nullptr, *Elo = nullptr, *Nlo = nullptr;
    float2* bdf = nullptr;     // the shared right-hand side h^2 f as df32 pairs
    // gradient (cfg.gradient): the adjoint solution and a per-particle right-hand
    // side (FP64, or df32 pairs in the same storage), reused for dPhi/du
    double *lam64 = nullptr, *rhs = nullptr, *rhs_b2 = nullptr;
    double *G = nullptr, *GV = nullptr;   // pCN-Langevin: DPhi of the particles and of the proposals (N x d)
    float* exptab = nullptr;   // 2^(j/64), j < 64, as df32 pairs (the df32 exponential)
    ExpConsts expc{};
    float* normtab = nullptr;  // logarithm table of the df32 Box-Muller normals (NORMAL_TAB pairs)
    NormalConsts normc{};
    InnerSolver<float> s32;
    InnerSolver<double> s64;
    Partials part{};
    SolverScalars sc{};
    // moments scratch
    double* gridtmp = nullptr;
    // fast cosine synthesis: twiddles 1/(2 cos(pi (2i+1) / (2M))) for M = 2, 4, .., n and the stage-1 output
    double *fct_tw = nullptr, *fct_tmp = nullptr;
    float* fct_tw_df = nullptr;   // the twiddles as df32 pairs (mixed precision)
    double b2 = 0.0;           // |h^2 f|^2 on the grid (the initial FP64 residual of w = 0)
    // host state
    double t = 0.0, beta = 0.2;
    int layer = 0;
    unsigned int step = 0;
    int stage = 0;             // 0 uninitialised, 1 ready for temper, 2 tempered, 3 resampled
    bool fitted = false;
    int last_iters = 0;
    long long nonconv = 0;
    // profiling counters (see smc_profile in smcgm.h)
    bool prof = false;
    smc_profile pc{};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int* dev_err = nullptr;    // device flag set by kernels whose bounded waits time out
    int* badp = nullptr;       // per batch particle: field outside the mixed-precision range
    bool lenient = false;      // in a move: such proposals are rejected instead of failing the call
    int sm_count = 0;
    std::string err;
    // CUDA-graph capture of the solver and the move (smc_batch_*): launches are sized
    // before the active counts are known and read them from device memory; the loops
    // become conditional nodes whose bodies are captured on the auxiliary streams.
    bool graph = false;
    int gdepth = 0;                   // nesting depth of the body being captured
    cudaStream_t gaux[4] = {nullptr, nullptr, nullptr, nullptr};
    GraphCounters* gcnt = nullptr;    // device counters of graph-mode solves
    int* gouter = nullptr;            // device: [0] refinement phase, [1] particles entering it
    MoveSched* msched = nullptr;      // device schedule of a graph-mode move
    int* gsteps = nullptr;            // device: steps left in a graph-mode move
};

// status helper
struct CudaError { cudaError_t e; const char* what; };
struct InputError { const char* what; };   // input the solver cannot take (reported as SMC_EINVAL)
void set_global_error(const char* msg);
std::string& global_error();
void check(cudaError_t e, const char* what);   // throws CudaError
// Waits for the context's stream (counted in smc_profile::host_syncs).
void sync_stream(Ctx& c);
// An NVTX range named after a kernel family (set-up, solve, proposal, ...) for the
// duration of a scope, so that profiler timelines group the library's launches.
struct NvtxRange {
    explicit NvtxRange(const char* name);
    ~NvtxRange();
};

constexpr int TILE = 32;          // inner tile edge of the tiled multigrid kernels
constexpr int MAXK = 16;          // max mixture components
constexpr int MAXR = 256;         // max mixture modes

}  // namespace smcgm

struct smc_ctx { smcgm::Ctx c; };
