// C ABI of libsmcgm.so (declared in include/smcgm.h): configuration checks,
// workspace planning, and the SMC driver steps of Alg. 1 / Alg. 2 / Alg. 3
// issued on the caller's stream.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <algorithm>
#include <numeric>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>
#include "smcgm_internal.cuh"

namespace smcgm {

void check(cudaError_t e, const char* what) {
    if (e != cudaSuccess) throw CudaError{e, what};
}

void sync_stream(Ctx& c) {
    ++c.pc.host_syncs;
    check(cudaStreamSynchronize(c.stream), "sync");
}

NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

struct Planner {
    char* base;
    size_t off = 0;
    explicit Planner(char* b) : base(b) {}
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

static int ilog2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

static const char* validate(const smc_config& c) {
    if (c.dim != 1 && c.dim != 2) return "dim must be 1 or 2";
    if (c.dim == 2) {
        if (c.n < 64 || (c.n & (c.n - 1))) return "2D grid size n must be a power of two >= 64";
        if (c.n > MAX_N2D) return "2D grid size n must be <= 512 (shared memory of the cosine-transform block)";
        if (c.kl_modes < 2 || c.kl_modes > c.n / 2 || (c.kl_modes & 1)) return "2D kl_modes must be even and in [2, n/2]";
        if (c.kl_modes > 256) return "2D kl_modes must be <= 256";
    } else {
        if (c.n < 4 || c.n > 65536) return "1D n must be in [4, 65536]";
        if (c.kl_modes < 2 || (c.kl_modes & 1)) return "1D kl_modes must be even and >= 2";
    }
    if (!(c.alpha > 0)) return "alpha must be > 0";
    if (c.n_obs < 1 || !c.obs || !c.data) return "observations required";
    if (!(c.sigma > 0)) return "sigma must be > 0";
    if (c.n_particles < 2 || c.n_particles > 32768) return "n_particles must be in [2, 32768]";
    if (c.n_components < 1 || c.n_components > MAXK) return "n_components must be in [1, 16]";
    if (c.gm_rank < 1 || c.gm_rank > MAXR) return "gm_rank must be in [1, 256]";
    if (c.em_iters < 0) return "em_iters must be >= 0";
    if (!(c.beta0 > 0 && c.beta0 <= 1)) return "beta0 must be in (0, 1]";
    if (!(c.ess_frac > 0 && c.ess_frac <= 1)) return "ess_frac must be in (0, 1]";
    if (c.kernel < 0 || c.kernel > 4) return "unknown kernel";
    if ((c.kernel == SMC_K_PCNL || c.kernel == SMC_K_GMPCNL) && (!c.gradient || c.dim != 2))
        return "the Langevin kernels need gradient = 1 and dim = 2";
    if (c.precision < 0 || c.precision > 2) return "unknown precision";
    if (!(c.tol_inner > 0 && c.tol_inner < 1) || !(c.tol_outer > 0 && c.tol_outer < 1)) return "tolerances must be in (0, 1)";
    if (c.max_iter < 1 || c.max_refine < 1) return "max_iter and max_refine must be >= 1";
    if (c.smooth_sweeps != 1 && c.smooth_sweeps != 2) return "smooth_sweeps must be 1 or 2";
    if (c.fine_sweeps != 1 && c.fine_sweeps != 2) return "fine_sweeps must be 1 or 2";
    if (!(c.coarse_scale > 0 && c.coarse_scale <= 2.5)) return "coarse_scale must be in (0, 2.5]";
    if (c.solve_batch < 0) return "solve_batch must be >= 0";
    if (c.gradient != 0 && c.gradient != 1) return "gradient must be 0 or 1";
    if (c.full_cov != 0 && c.full_cov != 1) return "full_cov must be 0 or 1";
    if (c.tile_kernel < 0 || c.tile_kernel > 4) return "tile_kernel must be 0, 1, 2, 3 or 4";
    if (c.full_cov && c.kernel != SMC_K_PCN_GM && c.kernel != SMC_K_GM_INDEP)
        return "full_cov needs the pCN-GM or the mixture independence kernel";
    if (c.full_cov && !(c.var_floor > 0)) return "full_cov needs var_floor > 0 (the covariance ridge)";
    if (c.gradient && c.dim != 2) return "gradients are built for dim = 2 only";
    for (int i = 0; i < c.n_obs * c.dim; ++i)
        if (!(c.obs[i] > 0.0 && c.obs[i] < 1.0)) return "observation points must lie inside the domain";
    return nullptr;
}

template <typename T>
static void plan_inner(Planner& P, InnerSolver<T>& s, int n, int B, int coarse_top, bool alias0, double* Kw64, double* Ks64,
                       double* E64, double* N64, bool bf16_faces = false) {
    s.nlev = ilog2(n) + 1;
    int nt = 0;
    for (int l = 0; l < s.nlev; ++l) if ((n >> l) > coarse_top) ++nt;
    s.ntile_levels = std::max(1, nt);
    s.coarse_top = n >> s.ntile_levels;
    s.lv.assign(s.nlev, LevelArrays<T>());
    const size_t nn = (size_t)n * n * B;
    for (int l = 0; l < s.nlev; ++l) {
        LevelArrays<T>& L = s.lv[l];
        L.n = n >> l;
        const size_t cells = (size_t)L.n * L.n * B;
        if (l == 0 && alias0) {
            L.Kw = reinterpret_cast<T*>(Kw64); L.Ks = reinterpret_cast<T*>(Ks64);
            L.E = reinterpret_cast<T*>(E64); L.Nn = reinterpret_cast<T*>(N64);
        } else {
            L.Kw = P.take<T>(cells); L.Ks = P.take<T>(cells);
            L.E = P.take<T>((size_t)L.n * B); L.Nn = P.take<T>((size_t)L.n * B);
        }
        L.e = P.take<T>(cells);
        if (l > 0) { L.r = P.take<T>(cells); L.e2 = P.take<T>(cells); }
        if (bf16_faces && l == 0) { L.Kwb = P.take<__nv_bfloat16>(cells); L.Ksb = P.take<__nv_bfloat16>(cells); }
    }
    s.list = P.take<int>(B); s.nact = P.take<int>(4);
    s.r[0] = P.take<T>(nn); s.r[1] = P.take<T>(nn);
    s.p[0] = P.take<T>(nn); s.p[1] = P.take<T>(nn);
    s.x = P.take<T>(nn); s.q = P.take<T>(nn); s.z = P.take<T>(nn);
}

// Lays out every device array; with base == nullptr only sizes them.
// Particles per solve batch when the configuration leaves it to the library: all of them,
// up to 2^28 cells per batch.  Measured (256^2, BF16 smoother): 4096 particles per batch
// 38.6k solves/s, 8192 37.8k, 16384 35.2k (the same 16384 in batches of 4096: 38.3k; of
// 2048: 37.1k); 512^2: batches of 1024 beat 2048 and 512; 128^2: 16384 beat 8192.
static int default_solve_batch(size_t cells) {
    const size_t b = ((size_t)1 << 28) / std::max<size_t>(cells, 1);
    return (int)std::max<size_t>(1, std::min<size_t>(b, 1 << 30));
}

static size_t plan(const smc_config& cfg, Ctx* c, char* base) {
    Ctx tmp;
    Ctx& C = c ? *c : tmp;
    Planner P(base);
    const int dim = cfg.dim, n = cfg.n, Km = cfg.kl_modes;
    const int d = dim == 2 ? Km * Km : Km;
    const int N = cfg.n_particles;
    const int K = (cfg.kernel == SMC_K_PCN || cfg.kernel == SMC_K_PCNL) ? 1 : cfg.n_components;
    const int r = std::min(cfg.gm_rank, d);
    const size_t cells = dim == 2 ? (size_t)n * n : (size_t)n;
    const int B = cfg.solve_batch > 0 ? std::min(cfg.solve_batch, N) : std::min(N, default_solve_batch(cells));
    C.dim = dim; C.n = n; C.Km = Km; C.d = d; C.N = N; C.K = K; C.r = r; C.B = B; C.nobs = cfg.n_obs;
    C.lam = P.take<double>(d); C.sqrtlam = P.take<double>(d);
    C.basis = P.take<double>((size_t)n * Km);
    C.b64 = P.take<double>(dim == 2 ? cells : (size_t)(n - 1));
    C.obs = P.take<double>((size_t)cfg.n_obs * dim); C.data = P.take<double>(cfg.n_obs);
    C.S = P.take<int>(r); C.slot = P.take<int>(d);
    C.X = P.take<double>((size_t)N * d); C.X2 = P.take<double>((size_t)N * d); C.V = P.take<double>((size_t)N * d);
    C.Phi = P.take<double>(N); C.Phi2 = P.take<double>(N); C.PhiV = P.take<double>(N);
    C.logw = P.take<double>(N); C.logalpha = P.take<double>(N);
    C.lfwd = P.take<double>((size_t)N * K); C.lrev = P.take<double>((size_t)N * K);
    C.acc = P.take<unsigned char>(N); C.idx = P.take<int>(N);
    C.icount = P.take<int>(64); C.dscal = P.take<double>(64); C.dev_err = P.take<int>(4);
    C.gcnt = P.take<GraphCounters>(1); C.gouter = P.take<int>(2); C.msched = P.take<MoveSched>(1); C.gsteps = P.take<int>(1);
    C.normtab = P.take<float>(2 * NORMAL_TAB);
    C.gw = P.take<double>(K); C.gmu = P.take<double>((size_t)K * r); C.glam = P.take<double>((size_t)K * r);
    if (cfg.full_cov) {
        C.gcov = P.take<double>((size_t)K * r * r); C.gL = P.take<double>((size_t)K * r * r);
        C.gLi = P.take<double>((size_t)K * r * r); C.glogdet = P.take<double>(K);
        C.covpart = P.take<double>(cov_partial_doubles(K, r));
    }
    C.tab = P.take<double>(4 * (size_t)K * r + r + 2 * K);
    C.xsT = P.take<double>((size_t)r * N); C.resp = P.take<double>((size_t)K * N); C.nj = P.take<double>(K);
    C.pooled = P.take<double>(2 * (size_t)r); C.lse = P.take<double>(N); C.gmax = P.take<double>(N);
    C.gridtmp = P.take<double>(std::max<size_t>(N, 2 * cells));
    if (dim == 2) {
        const size_t bn = (size_t)B * n * n;
        C.u64 = P.take<double>(bn);
        C.fct_tw = P.take<double>(n);
        C.fct_tmp = P.take<double>((size_t)B * n * Km);
        if (mixed_precision(cfg)) {
            C.Kwlo = P.take<float>(bn); C.Kslo = P.take<float>(bn);
            C.Elo = P.take<float>((size_t)B * n); C.Nlo = P.take<float>((size_t)B * n);
            C.w64 = P.take<double>(bn);
            C.bdf = P.take<float2>(cells);
            C.badp = P.take<int>(B);
            C.exptab = P.take<float>(128);
            C.fct_tw_df = P.take<float>(2 * (size_t)n);
        } else {
            C.Kw64 = P.take<double>(bn); C.Ks64 = P.take<double>(bn);
            C.E64 = P.take<double>((size_t)B * n); C.N64 = P.take<double>((size_t)B * n);
            C.w64 = P.take<double>(bn);
        }
        if (cfg.gradient) {
            C.lam64 = P.take<double>(bn);
            C.rhs = P.take<double>(bn);
            C.rhs_b2 = P.take<double>(B);
        }
        if (cfg.kernel == SMC_K_PCNL || cfg.kernel == SMC_K_GMPCNL) {
            C.G = P.take<double>((size_t)N * d);
            C.GV = P.take<double>((size_t)N * d);
        }
        const int ntiles = (n / 16) * (n / 16);   // the finest tiled level's tiles (16 x 16 warp tiles or fewer)
        C.part.ntiles = ntiles;
        C.part.rr = P.take<double>((size_t)B * ntiles); C.part.rz = P.take<double>((size_t)B * ntiles);
        C.part.pq = P.take<double>((size_t)B * ntiles); C.part.res = P.take<double>((size_t)B * ntiles);
        SolverScalars& s = C.sc;
        s.rz = P.take<double>(B); s.rr0 = P.take<double>(B); s.rr = P.take<double>(B); s.pq = P.take<double>(B);
        s.alpha = P.take<double>(B); s.betac = P.take<double>(B); s.res2 = P.take<double>(B); s.b2 = P.take<double>(B);
        s.act_in = P.take<int>(B); s.act_out = P.take<int>(B); s.iters = P.take<int>(B); s.flags = P.take<int>(B);
        s.count = P.take<int>(4);
        // levels with n_l <= coarse_top run in the one-block-per-particle coarse kernel
        const int ctop = 32;
        if (mixed_precision(cfg))
            plan_inner<float>(P, C.s32, n, B, ctop, false, nullptr, nullptr, nullptr, nullptr, bf16_smoother(cfg));
        else
            plan_inner<double>(P, C.s64, n, B, 32, true, C.Kw64, C.Ks64, C.E64, C.N64);
    } else {
        C.u64 = P.take<double>((size_t)B * (3 * n + 2));
    }
    return P.off + 256;
}

static void host_tables(Ctx& c, std::vector<double>& lam, std::vector<double>& basis, std::vector<double>& b,
                        std::vector<int>& S, std::vector<int>& slot) {
    const smc_config& cfg = c.cfg;
    const int n = c.n, Km = c.Km, d = c.d;
    lam.resize(d);
    basis.resize((size_t)n * Km);
    if (c.dim == 2) {
        for (int k = 0; k < Km; ++k)
            for (int l = 0; l < Km; ++l)
                lam[k * Km + l] = std::pow(1.0 + cfg.alpha * M_PI * M_PI * ((double)k * k + (double)l * l), -2.0);
        for (int i = 0; i < n; ++i) {
            const double x = (i + 0.5) / n;
            for (int k = 0; k < Km; ++k) basis[(size_t)i * Km + k] = std::cos(M_PI * (x * k)) * (k == 0 ? 1.0 : std::sqrt(2.0));
        }
        b.resize((size_t)n * n);
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                const double x = (i + 0.5) / n, y = (j + 0.5) / n;
                double f = cfg.src_amp;
                if (cfg.source_kind == 1) f = cfg.src_amp * std::exp(-cfg.src_width * ((x - 0.5) * (x - 0.5) + (y - 0.5) * (y - 0.5)));
                b[(size_t)j * n + i] = f / ((double)n * n);
            }
        std::vector<int> order(d);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int bb) {
            const int ka = a / Km, la = a % Km, kb = bb / Km, lb = bb % Km;
            const int qa = ka * ka + la * la, qb = kb * kb + lb * lb;
            if (qa != qb) return qa < qb;
            if (ka != kb) return ka < kb;
            return la < lb;
        });
        S.assign(order.begin(), order.begin() + c.r);
    } else {
        for (int k = 1; k <= Km; ++k) lam[k - 1] = std::pow(1.0 + cfg.alpha * M_PI * M_PI * (double)k * k, -2.0);
        for (int i = 0; i < n; ++i) {
            const double x = (i + 0.5) / n;
            for (int k = 1; k <= Km; ++k) basis[(size_t)i * Km + (k - 1)] = std::sqrt(2.0) * std::sin(M_PI * (x * k));
        }
        b.resize(n - 1);
        for (int i = 1; i < n; ++i) {
            const double x = (double)i / n;
            double f = cfg.src_amp;
            if (cfg.source_kind == 1) f = cfg.src_amp * std::exp(-cfg.src_width * (x - 0.5) * (x - 0.5));
            b[i - 1] = f / ((double)n * n);
        }
        S.resize(c.r);
        std::iota(S.begin(), S.end(), 0);
    }
    std::sort(S.begin(), S.end());
    slot.assign(d, -1);
    for (int s = 0; s < (int)S.size(); ++s) slot[S[s]] = s;
}

static void set_prior_mixture(Ctx& c) {
    std::vector<double> lam(c.d);
    check(cudaMemcpyAsync(lam.data(), c.lam, c.d * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "lam");
    std::vector<int> S(c.r);
    check(cudaMemcpyAsync(S.data(), c.S, c.r * sizeof(int), cudaMemcpyDeviceToHost, c.stream), "S");
    sync_stream(c);
    std::vector<double> w(c.K, 1.0 / c.K), m((size_t)c.K * c.r, 0.0), l((size_t)c.K * c.r);
    for (int j = 0; j < c.K; ++j)
        for (int s = 0; s < c.r; ++s) l[(size_t)j * c.r + s] = lam[S[s]];
    check(cudaMemcpyAsync(c.gw, w.data(), c.K * sizeof(double), cudaMemcpyHostToDevice, c.stream), "w");
    check(cudaMemcpyAsync(c.gmu, m.data(), m.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream), "m");
    check(cudaMemcpyAsync(c.glam, l.data(), l.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream), "lam");
    sync_stream(c);
}

}  // namespace smcgm

using namespace smcgm;

#define API_BEGIN try {
#define API_END(ctxp)                                                                           \
    }                                                                                           \
    catch (const InputError& ie) {                                                              \
        if (ctxp) (ctxp)->c.err = ie.what;                                                      \
        return SMC_EINVAL;                                                                      \
    }                                                                                           \
    catch (const CudaError& ce) {                                                               \
        if (ctxp) (ctxp)->c.err = std::string(ce.what) + ": " + cudaGetErrorString(ce.e);     \
        return SMC_ECUDA;                                                                       \
    }                                                                                           \
    catch (const std::bad_alloc&) {                                                             \
        if (ctxp) (ctxp)->c.err = "host allocation failed";                                   \
        return SMC_ENOMEM;                                                                      \
    }

namespace smcgm {
// Message for smc_last_error(NULL), set by entry points that have no context.
std::string& global_error() {
    static thread_local std::string msg;
    return msg;
}
void set_global_error(const char* msg) { global_error() = msg; }
}  // namespace smcgm

static smc_status fail(smc_ctx* ctx, smc_status s, const std::string& msg) {
    if (ctx) ctx->c.err = msg;
    return s;
}

extern "C" {

const char* smc_version(void) { return "smcgm 0.1 (sm_103a)"; }

size_t smc_config_size(void) { return sizeof(smc_config); }

smc_status smc_profile_query(smc_ctx* ctx, int enable, smc_profile* out, int reset) {
    if (!ctx) return SMC_EINVAL;
    Ctx& c = ctx->c;
    API_BEGIN
    if (enable == 1 && !c.ev0) {
        check(cudaEventCreate(&c.ev0), "event");
        check(cudaEventCreate(&c.ev1), "event");
    }
    if (enable == 0 || enable == 1) c.prof = enable == 1;
    if (out) *out = c.pc;
    if (reset) { const int cells = c.pc.cells, wb = c.pc.word_bytes; c.pc = smc_profile{}; c.pc.cells = cells; c.pc.word_bytes = wb; }
    return SMC_OK;
    API_END(ctx)
}

smc_status smc_copy_to_host(smc_ctx* ctx, void* dst, const void* src, size_t bytes) {
    if (!ctx || (!dst && bytes) || (!src && bytes)) return SMC_EINVAL;
    Ctx& c = ctx->c;
    API_BEGIN
    if (bytes) check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c.stream), "copy to host");
    sync_stream(c);
    return SMC_OK;
    API_END(ctx)
}

smc_status smc_config_init(smc_config* cfg) {
    if (!cfg) return SMC_EINVAL;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->dim = 2; cfg->n = 64; cfg->kl_modes = 32; cfg->alpha = 0.02;
    cfg->sigma = 0.01; cfg->source_kind = 1; cfg->src_amp = 10.0; cfg->src_width = 50.0;
    cfg->n_particles = 1024; cfg->n_components = 4; cfg->gm_rank = 64; cfg->em_iters = 50; cfg->var_floor = 1e-3;
    cfg->beta0 = 0.2; cfg->ess_frac = 0.5; cfg->kernel = SMC_K_PCN_GM; cfg->precision = SMC_P_FP32_REFINE;
    cfg->tol_inner = 5e-4; cfg->tol_outer = 1e-10; cfg->max_iter = 60; cfg->max_refine = 6;
    cfg->smooth_sweeps = 2; cfg->fine_sweeps = 1; cfg->coarse_scale = 2.0; cfg->solve_batch = 0; cfg->seed = 2503016028ull;
    return SMC_OK;
}

smc_status smc_workspace_size(const smc_config* cfg, size_t* bytes) {
    if (!cfg || !bytes) return SMC_EINVAL;
    if (const char* why = validate(*cfg)) {
        set_global_error(why);
        return SMC_EINVAL;
    }
    *bytes = plan(*cfg, nullptr, nullptr);
    return SMC_OK;
}

static thread_local std::string& g_init_error = smcgm::global_error();

smc_status smc_init(const smc_config* cfg, void* d_ws, size_t bytes, void* stream, smc_ctx** out) {
    if (!cfg || !out) return SMC_EINVAL;
    *out = nullptr;
    if (const char* why = validate(*cfg)) { g_init_error = why; return SMC_EINVAL; }
    const size_t need = plan(*cfg, nullptr, nullptr);
    if (!d_ws || bytes < need) { g_init_error = "workspace smaller than smc_workspace_size()"; return SMC_ENOMEM; }
    if (reinterpret_cast<uintptr_t>(d_ws) % 256 != 0) { g_init_error = "workspace must be 256-byte aligned"; return SMC_EINVAL; }
    smc_ctx* ctx = new (std::nothrow) smc_ctx();
    if (!ctx) return SMC_ENOMEM;
    Ctx& c = ctx->c;
    c.cfg = *cfg;
    c.obs_h.assign(cfg->obs, cfg->obs + (size_t)cfg->n_obs * cfg->dim);
    c.data_h.assign(cfg->data, cfg->data + cfg->n_obs);
    c.cfg.obs = nullptr;
    c.cfg.data = nullptr;
    c.stream = reinterpret_cast<cudaStream_t>(stream);
    c.key = key_of(cfg->seed);
    // align the carve base to 256 bytes (the planner's offsets start at 0)
    plan(*cfg, &c, reinterpret_cast<char*>(d_ws));
    API_BEGIN
    std::vector<double> lam, basis, b;
    std::vector<int> S, slot;
    host_tables(c, lam, basis, b, S, slot);
    c.b2 = 0.0;
    for (double v : b) c.b2 += v * v;
    std::vector<double> sq(lam.size());
    for (size_t i = 0; i < lam.size(); ++i) sq[i] = std::sqrt(lam[i]);
    check(cudaMemcpyAsync(c.lam, lam.data(), lam.size() * 8, cudaMemcpyHostToDevice, c.stream), "h2d");
    check(cudaMemcpyAsync(c.sqrtlam, sq.data(), sq.size() * 8, cudaMemcpyHostToDevice, c.stream), "h2d");
    check(cudaMemcpyAsync(c.basis, basis.data(), basis.size() * 8, cudaMemcpyHostToDevice, c.stream), "h2d");
    check(cudaMemcpyAsync(c.b64, b.data(), b.size() * 8, cudaMemcpyHostToDevice, c.stream), "h2d");
    std::vector<float2> bdf;
    if (c.bdf) {   // df32 split of the right-hand side: hi = round(b), lo = round(b - hi)
        bdf.resize(b.size());
        for (size_t i = 0; i < b.size(); ++i) {
            const float h = (float)b[i];
            bdf[i] = float2{h, (float)(b[i] - (double)h)};
        }
        check(cudaMemcpyAsync(c.bdf, bdf.data(), bdf.size() * 8, cudaMemcpyHostToDevice, c.stream), "h2d");
    }
    // df32 Box-Muller: logarithm table and constants (df32 pairs hi = round(v), lo = round(v - hi))
    auto split = [](double v) { const float h = (float)v; return float2{h, (float)(v - (double)h)}; };
    std::vector<float2> ntab(NORMAL_TAB);
    for (int j = 0; j <= 64; ++j) {
        const double F = 1.0 + j / 64.0;
        ntab[j] = split(j < 32 ? std::log(F) : std::log(F / 2.0));
        ntab[65 + j] = split(1.0 / F);
    }
    {
        const double ln2 = std::log(2.0);
        int ex = 0;
        const double f = std::frexp(ln2, &ex);
        const double a = std::ldexp(std::nearbyint(std::ldexp(f, 16)), ex - 16);   // 16 significant bits
        c.normc.ln2a = (float)a;
        c.normc.ln2b = (float)(ln2 - a);
        c.normc.ln2c = (float)(ln2 - a - (double)c.normc.ln2b);
        c.normc.pi = split(M_PI);
        c.normc.s3 = split(1.0 / 6.0); c.normc.s5 = split(1.0 / 120.0); c.normc.s7 = split(1.0 / 5040.0); c.normc.s9 = split(1.0 / 362880.0);
        c.normc.c2 = split(0.5); c.normc.c4 = split(1.0 / 24.0); c.normc.c6 = split(1.0 / 720.0); c.normc.c8 = split(1.0 / 40320.0);
        c.normc.third = split(1.0 / 3.0);
    }
    check(cudaMemcpyAsync(c.normtab, ntab.data(), ntab.size() * sizeof(float2), cudaMemcpyHostToDevice, c.stream), "h2d");
    std::vector<float> etab;
    if (c.exptab) {   // df32 exponential: 2^(j/64) split into pairs, ln2/64 in three parts
        etab.resize(128);
        for (int j = 0; j < 64; ++j) {
            const double v = std::exp2(j / 64.0);
            etab[2 * j] = (float)v;
            etab[2 * j + 1] = (float)(v - (double)etab[2 * j]);
        }
        const double C = std::log(2.0) / 64.0;
        int ex = 0;
        const double f = std::frexp(C, &ex);
        const double c1 = std::ldexp(std::nearbyint(std::ldexp(f, 11)), ex - 11);   // 11 significant bits
        c.expc.c1 = (float)c1;
        c.expc.c2 = (float)(C - c1);
        c.expc.c3 = (float)(C - c1 - (double)c.expc.c2);
        check(cudaMemcpyAsync(c.exptab, etab.data(), etab.size() * 4, cudaMemcpyHostToDevice, c.stream), "h2d");
    }
    check(cudaMemcpyAsync(c.obs, c.obs_h.data(), c.obs_h.size() * 8, cudaMemcpyHostToDevice, c.stream), "h2d");
    check(cudaMemcpyAsync(c.data, c.data_h.data(), c.data_h.size() * 8, cudaMemcpyHostToDevice, c.stream), "h2d");
    check(cudaMemcpyAsync(c.S, S.data(), S.size() * 4, cudaMemcpyHostToDevice, c.stream), "h2d");
    std::vector<double> tw;
    std::vector<float> twdf;
    if (c.dim == 2) {
        // twiddles of the fast cosine synthesis, block M/2 - 1 .. M - 2 for M = 2, 4, ..., n
        tw.assign(c.n, 0.0);
        for (int M = 2; M <= c.n; M *= 2)
            for (int i = 0; i < M / 2; ++i) tw[M / 2 - 1 + i] = 1.0 / (2.0 * std::cos(M_PI * (2.0 * i + 1.0) / (2.0 * M)));
        check(cudaMemcpyAsync(c.fct_tw, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice, c.stream), "h2d");
        if (c.fct_tw_df) {
            twdf.resize(2 * tw.size());
            for (size_t i = 0; i < tw.size(); ++i) {
                twdf[2 * i] = (float)tw[i];
                twdf[2 * i + 1] = (float)(tw[i] - (double)twdf[2 * i]);
            }
            check(cudaMemcpyAsync(c.fct_tw_df, twdf.data(), twdf.size() * 4, cudaMemcpyHostToDevice, c.stream), "h2d");
        }
    }
    check(cudaMemcpyAsync(c.slot, slot.data(), slot.size() * 4, cudaMemcpyHostToDevice, c.stream), "h2d");
    check(cudaMemsetAsync(c.dev_err, 0, 4 * sizeof(int), c.stream), "memset err");
    sync_stream(c);
    {
        int dev = 0;
        check(cudaGetDevice(&dev), "device");
        check(cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, dev), "sm count");
    }
    if (c.dim == 2) {
        if (mixed_precision(c.cfg)) build_tma_maps<float>(c, c.s32);
        else build_tma_maps<double>(c, c.s64);
    }
    set_prior_mixture(c);
    c.fitted = (c.cfg.kernel == SMC_K_PCN || c.cfg.kernel == SMC_K_PCNL);
    c.t = 0.0;
    c.beta = c.cfg.kernel == SMC_K_GM_INDEP ? 1.0 : c.cfg.beta0;
    c.layer = 0;
    c.step = 0;
    launch_prior_draw(c, c.X, c.N, 0u, P_INIT);
    forward_solve(c, c.X, c.N, c.Phi, nullptr);
    sync_stream(c);
    c.stage = 1;
    *out = ctx;
    return SMC_OK;
    }
    catch (const CudaError& ce) {
        g_init_error = std::string(ce.what) + ": " + cudaGetErrorString(ce.e);
        delete ctx;
        return SMC_ECUDA;
    }
}

const char* smc_last_error(const smc_ctx* ctx) {
    if (!ctx) return g_init_error.c_str();
    return ctx->c.err.c_str();
}

void smc_destroy(smc_ctx* ctx) {
    if (!ctx) return;
    if (ctx->c.ev0) cudaEventDestroy(ctx->c.ev0);
    if (ctx->c.ev1) cudaEventDestroy(ctx->c.ev1);
    delete ctx->c.s32.maps;
    delete ctx->c.s64.maps;
    delete ctx;
}

smc_status smc_temper_step(smc_ctx* ctx, double* h, double* ess, double* logZ_inc, int* done) {
    if (!ctx) return SMC_EINVAL;
    NvtxRange nvtx("smc_temper_step");
    Ctx& c = ctx->c;
    if (c.stage != 1) return fail(ctx, SMC_ESTATE, "smc_temper_step: expected after init or move");
    if (c.t >= 1.0) return fail(ctx, SMC_ESTATE, "smc_temper_step: t already 1");
    API_BEGIN
    double out[4];
    launch_temper(c, c.dscal);
    check(cudaMemcpyAsync(out, c.dscal, 4 * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "d2h");
    sync_stream(c);
    if (h) *h = out[0];
    if (ess) *ess = out[1];
    if (logZ_inc) *logZ_inc = out[2];
    if (!(out[0] > 0.0)) return fail(ctx, SMC_EDEGENERATE, "tempering step h = 0");
    c.t = out[3];
    if (done) *done = c.t >= 1.0 ? 1 : 0;
    c.stage = 2;
    return SMC_OK;
    API_END(ctx)
}

smc_status smc_resample(smc_ctx* ctx) {
    if (!ctx) return SMC_EINVAL;
    NvtxRange nvtx("smc_resample");
    Ctx& c = ctx->c;
    if (c.stage != 2) return fail(ctx, SMC_ESTATE, "smc_resample: expected after smc_temper_step");
    API_BEGIN
    launch_resample(c);
    sync_stream(c);
    c.stage = 3;
    return SMC_OK;
    API_END(ctx)
}

smc_status gm_fit(smc_ctx* ctx, double* loglik) {
    if (!ctx) return SMC_EINVAL;
    NvtxRange nvtx("gm_fit");
    Ctx& c = ctx->c;
    if (c.stage < 1) return fail(ctx, SMC_ESTATE, "gm_fit: context not initialised");
    if (c.cfg.kernel == SMC_K_PCN || c.cfg.kernel == SMC_K_PCNL) { if (loglik) *loglik = 0.0; return SMC_OK; }
    API_BEGIN
    const double ll = gm_fit_device(c);
    if (loglik) *loglik = ll;
    c.fitted = true;
    return SMC_OK;
    API_END(ctx)
}

smc_status smc_move(smc_ctx* ctx, int steps, double* accept_rate, int* iters_max) {
    if (!ctx || steps < 1) return SMC_EINVAL;
    NvtxRange nvtx("smc_move");
    Ctx& c = ctx->c;
    if (c.stage < 1) return fail(ctx, SMC_ESTATE, "smc_move: context not initialised");
    if (!c.fitted) return fail(ctx, SMC_ESTATE, "smc_move: the pCN-GM kernels need gm_fit or smc_set_mixture first");
    API_BEGIN
    struct Lenient {   // proposals outside the mixed-precision field range are rejected, not fatal
        Ctx& c;
        explicit Lenient(Ctx& cc) : c(cc) { c.lenient = true; }
        ~Lenient() { c.lenient = false; }
    } lenient_guard(c);
    int* accn = c.icount;
    check(cudaMemsetAsync(accn, 0, sizeof(int), c.stream), "memset");
    const long long nc0 = c.nonconv;
    int itmax = 0;
    long long solves = (long long)c.N * steps;
    if (c.cfg.kernel == SMC_K_PCNL) {
        itmax = gradient_batch(c, c.X, c.N, c.Phi2, c.G);   // DPhi of the current particles (Phi2: scratch)
        for (int s = 0; s < steps; ++s) {
            launch_propose_pcnl(c);
            itmax = std::max(itmax, gradient_batch(c, c.V, c.N, c.PhiV, c.GV));
            launch_accept_pcnl(c, accn);
            ++c.step;
        }
        solves = 2LL * c.N * (steps + 1);
    } else if (c.cfg.kernel == SMC_K_GMPCNL) {
        launch_move_tables(c);
        itmax = gradient_batch(c, c.X, c.N, c.Phi2, c.G);
        for (int s = 0; s < steps; ++s) {
            launch_propose(c);                               // with the drift; the terms wait for DPhi(v)
            itmax = std::max(itmax, gradient_batch(c, c.V, c.N, c.PhiV, c.GV));
            launch_gmpcnl_terms(c);
            launch_accept(c, accn);
            launch_copy_accepted_gradients(c);
            ++c.step;
        }
        solves = 2LL * c.N * (steps + 1);
    } else {
        launch_move_tables(c);
        for (int s = 0; s < steps; ++s) {
            if (c.cfg.full_cov) launch_propose_full(c);
            else launch_propose(c);
            itmax = std::max(itmax, forward_solve(c, c.V, c.N, c.PhiV, nullptr));
            launch_accept(c, accn);
            ++c.step;
        }
    }
    int hacc = 0;
    check(cudaMemcpyAsync(&hacc, accn, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "d2h");
    sync_stream(c);
    const double rate = (double)hacc / ((double)c.N * steps);
    if (accept_rate) *accept_rate = rate;
    if (iters_max) *iters_max = itmax;
    if (c.cfg.kernel != SMC_K_GM_INDEP) {
        double b = c.beta;
        if (rate > 0.3) b = 2.0 * b;
        else if (rate < 0.15) b = 0.5 * b;
        c.beta = std::min(b, 1.0);
    }
    ++c.layer;
    c.stage = 1;
    if ((c.nonconv - nc0) * 100 > solves)
        return fail(ctx, SMC_ENOCONV, "more than 1% of forward solves missed the tolerance");
    return SMC_OK;
    API_END(ctx)
}

smc_status smc_move_host(smc_ctx* ctx, const double* X_in, const double* Phi_in, double* X_out, double* Phi_out, double* accept_rate) {
    if (!ctx || !X_in || !Phi_in) return SMC_EINVAL;
    Ctx& c = ctx->c;
    API_BEGIN
    check(cudaMemcpyAsync(c.X, X_in, (size_t)c.N * c.d * sizeof(double), cudaMemcpyHostToDevice, c.stream), "h2d X");
    check(cudaMemcpyAsync(c.Phi, Phi_in, (size_t)c.N * sizeof(double), cudaMemcpyHostToDevice, c.stream), "h2d Phi");
    smc_status st = smc_move(ctx, 1, accept_rate, nullptr);
    if (st != SMC_OK && st != SMC_ENOCONV) return st;
    if (X_out) check(cudaMemcpyAsync(X_out, c.X, (size_t)c.N * c.d * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "d2h X");
    if (Phi_out) check(cudaMemcpyAsync(Phi_out, c.Phi, (size_t)c.N * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "d2h Phi");
    sync_stream(c);
    return st;
    API_END(ctx)
}

smc_status smc_posterior_moments(smc_ctx* ctx, double* mean_kl, double* var_kl, double* mean_grid, double* var_grid) {
    if (!ctx) return SMC_EINVAL;
    Ctx& c = ctx->c;
    if (c.stage < 1) return fail(ctx, SMC_ESTATE, "smc_posterior_moments: context not initialised");
    API_BEGIN
    double* dm = c.V;
    double* dv = c.V + c.d;
    launch_moments(c, dm, dv);
    if (mean_kl) check(cudaMemcpyAsync(mean_kl, dm, c.d * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "d2h");
    if (var_kl) check(cudaMemcpyAsync(var_kl, dv, c.d * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "d2h");
    if (mean_grid || var_grid) {
        const size_t cells = c.dim == 2 ? (size_t)c.n * c.n : (size_t)c.n;
        launch_grid_moments(c, dm, c.gridtmp, c.gridtmp + cells);
        if (mean_grid) check(cudaMemcpyAsync(mean_grid, c.gridtmp, cells * 8, cudaMemcpyDeviceToHost, c.stream), "d2h");
        if (var_grid) check(cudaMemcpyAsync(var_grid, c.gridtmp + cells, cells * 8, cudaMemcpyDeviceToHost, c.stream), "d2h");
    }
    sync_stream(c);
    return SMC_OK;
    API_END(ctx)
}

smc_status smc_gradient(smc_ctx* ctx, const double* d_X, int count, double* d_Phi, double* d_grad) {
    if (!ctx || !d_X || !d_Phi || !d_grad || count < 1) return SMC_EINVAL;
    Ctx& c = ctx->c;
    if (!device_visible(d_X) || !device_visible(d_Phi) || !device_visible(d_grad))
        return fail(ctx, SMC_EINVAL, "smc_gradient: d_X, d_Phi and d_grad must be device memory");
    if (c.stage < 1) return fail(ctx, SMC_ESTATE, "smc_gradient: context not initialised");
    if (!c.lam64) return fail(ctx, SMC_ESTATE, "smc_gradient: the context was set up without cfg.gradient = 1");
    API_BEGIN
    const long long nc0 = c.nonconv;
    gradient_batch(c, d_X, count, d_Phi, d_grad);
    sync_stream(c);
    if ((c.nonconv - nc0) * 100 > 2LL * count) return fail(ctx, SMC_ENOCONV, "more than 1% of forward or adjoint solves missed the tolerance");
    return SMC_OK;
    API_END(ctx)
}

smc_status smc_forward(smc_ctx* ctx, const double* d_X, int count, double* d_Phi, double* d_w, int* iters) {
    if (!ctx || !d_X || !d_Phi || count < 1) return SMC_EINVAL;
    Ctx& c = ctx->c;
    if (!device_visible(d_X) || !device_visible(d_Phi) || (d_w && !device_visible(d_w)))
        return fail(ctx, SMC_EINVAL, "smc_forward: d_X, d_Phi and d_w must be device memory");
    if (c.stage < 1) return fail(ctx, SMC_ESTATE, "smc_forward: context not initialised");
    API_BEGIN
    const long long nc0 = c.nonconv;
    int it = forward_solve(c, d_X, count, d_Phi, d_w);
    sync_stream(c);
    if (iters) *iters = it;
    if ((c.nonconv - nc0) * 100 > count) return fail(ctx, SMC_ENOCONV, "more than 1% of forward solves missed the tolerance");
    return SMC_OK;
    API_END(ctx)
}

smc_status smc_get_particles(smc_ctx* ctx, const double** d_X, const double** d_Phi) {
    if (!ctx) return SMC_EINVAL;
    if (d_X) *d_X = ctx->c.X;
    if (d_Phi) *d_Phi = ctx->c.Phi;
    return SMC_OK;
}

smc_status smc_set_particles(smc_ctx* ctx, const double* X, const double* Phi, int on_device) {
    if (!ctx || !X) return SMC_EINVAL;
    Ctx& c = ctx->c;
    API_BEGIN
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    check(cudaMemcpyAsync(c.X, X, (size_t)c.N * c.d * sizeof(double), kind, c.stream), "set X");
    if (Phi) check(cudaMemcpyAsync(c.Phi, Phi, (size_t)c.N * sizeof(double), kind, c.stream), "set Phi");
    else forward_solve(c, c.X, c.N, c.Phi, nullptr);
    sync_stream(c);
    if (c.stage < 1) c.stage = 1;
    return SMC_OK;
    API_END(ctx)
}

smc_status smc_set_schedule(smc_ctx* ctx, double t, double beta, int layer, unsigned int step) {
    if (!ctx || !(t >= 0.0 && t <= 1.0) || !(beta > 0.0 && beta <= 1.0) || layer < 0) return SMC_EINVAL;
    Ctx& c = ctx->c;
    c.t = t; c.beta = beta; c.layer = layer; c.step = step;
    c.stage = 1;
    return SMC_OK;
}

smc_status smc_get_schedule(smc_ctx* ctx, double* t, double* beta, int* layer, unsigned int* step) {
    if (!ctx) return SMC_EINVAL;
    Ctx& c = ctx->c;
    if (t) *t = c.t;
    if (beta) *beta = c.beta;
    if (layer) *layer = c.layer;
    if (step) *step = c.step;
    return SMC_OK;
}

smc_status smc_set_mixture(smc_ctx* ctx, const double* w, const double* m, const double* lam) {
    if (!ctx || !w || !m || !lam) return SMC_EINVAL;
    Ctx& c = ctx->c;
    for (int j = 0; j < c.K; ++j) if (!(w[j] > 0.0)) return fail(ctx, SMC_EINVAL, "mixture weights must be > 0");
    for (int t = 0; t < c.K * c.r; ++t) if (!(lam[t] > 0.0)) return fail(ctx, SMC_EINVAL, "mixture variances must be > 0");
    API_BEGIN
    check(cudaMemcpyAsync(c.gw, w, c.K * sizeof(double), cudaMemcpyHostToDevice, c.stream), "w");
    check(cudaMemcpyAsync(c.gmu, m, (size_t)c.K * c.r * sizeof(double), cudaMemcpyHostToDevice, c.stream), "m");
    check(cudaMemcpyAsync(c.glam, lam, (size_t)c.K * c.r * sizeof(double), cudaMemcpyHostToDevice, c.stream), "lam");
    if (c.cfg.full_cov) {                                  // diagonal covariances in the full form
        std::vector<double> cov((size_t)c.K * c.r * c.r, 0.0);
        for (int j = 0; j < c.K; ++j)
            for (int a = 0; a < c.r; ++a) cov[((size_t)j * c.r + a) * c.r + a] = lam[(size_t)j * c.r + a];
        factor_mixture(c, cov.data());
    }
    sync_stream(c);
    c.fitted = true;
    return SMC_OK;
    API_END(ctx)
}

smc_status smc_set_mixture_cov(smc_ctx* ctx, const double* w, const double* m, const double* cov) {
    if (!ctx || !w || !m || !cov) return SMC_EINVAL;
    Ctx& c = ctx->c;
    if (!c.cfg.full_cov) return fail(ctx, SMC_ESTATE, "smc_set_mixture_cov: the context was set up without cfg.full_cov = 1");
    for (int j = 0; j < c.K; ++j) if (!(w[j] > 0.0)) return fail(ctx, SMC_EINVAL, "mixture weights must be > 0");
    API_BEGIN
    const size_t Kr = (size_t)c.K * c.r;
    std::vector<double> lam(Kr);
    for (size_t t = 0; t < Kr; ++t) lam[t] = cov[(t / c.r * c.r + t % c.r) * c.r + t % c.r];
    factor_mixture(c, cov);                                // fails for a covariance that is not positive definite
    check(cudaMemcpyAsync(c.gw, w, c.K * sizeof(double), cudaMemcpyHostToDevice, c.stream), "w");
    check(cudaMemcpyAsync(c.gmu, m, Kr * sizeof(double), cudaMemcpyHostToDevice, c.stream), "m");
    check(cudaMemcpyAsync(c.glam, lam.data(), Kr * sizeof(double), cudaMemcpyHostToDevice, c.stream), "lam");
    sync_stream(c);
    c.fitted = true;
    return SMC_OK;
    API_END(ctx)
}

smc_status smc_get_mixture_cov(smc_ctx* ctx, double* cov) {
    if (!ctx || !cov) return SMC_EINVAL;
    Ctx& c = ctx->c;
    if (!c.cfg.full_cov) return fail(ctx, SMC_ESTATE, "smc_get_mixture_cov: the context was set up without cfg.full_cov = 1");
    API_BEGIN
    check(cudaMemcpyAsync(cov, c.gcov, (size_t)c.K * c.r * c.r * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "cov");
    sync_stream(c);
    return SMC_OK;
    API_END(ctx)
}

smc_status smc_get_mixture(smc_ctx* ctx, double* w, double* m, double* lam, int* modes) {
    if (!ctx) return SMC_EINVAL;
    Ctx& c = ctx->c;
    API_BEGIN
    if (w) check(cudaMemcpyAsync(w, c.gw, c.K * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "w");
    if (m) check(cudaMemcpyAsync(m, c.gmu, (size_t)c.K * c.r * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "m");
    if (lam) check(cudaMemcpyAsync(lam, c.glam, (size_t)c.K * c.r * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "lam");
    if (modes) check(cudaMemcpyAsync(modes, c.S, c.r * sizeof(int), cudaMemcpyDeviceToHost, c.stream), "S");
    sync_stream(c);
    return SMC_OK;
    API_END(ctx)
}

smc_status smc_get_diagnostics(smc_ctx* ctx, const double** d_log_alpha, const unsigned char** d_accepted, const double** d_phi_proposed,
                               const double** d_logw, const int** d_indices) {
    if (!ctx) return SMC_EINVAL;
    Ctx& c = ctx->c;
    if (d_log_alpha) *d_log_alpha = c.logalpha;
    if (d_accepted) *d_accepted = c.acc;
    if (d_phi_proposed) *d_phi_proposed = c.PhiV;
    if (d_logw) *d_logw = c.logw;
    if (d_indices) *d_indices = c.idx;
    return SMC_OK;
}

struct SaveHeader {
    char magic[8];
    int N, d, K, r, layer, stage, fitted, pad;
    unsigned int step, pad2;
    double t, beta;
};

smc_status smc_save(smc_ctx* ctx, void* host_buf, size_t* bytes) {
    if (!ctx || !bytes) return SMC_EINVAL;
    Ctx& c = ctx->c;
    const size_t covn = c.cfg.full_cov ? (size_t)c.K * c.r * c.r : 0;
    const size_t need = sizeof(SaveHeader) + sizeof(double) * ((size_t)c.N * c.d + c.N + c.K + 2 * (size_t)c.K * c.r + covn);
    if (!host_buf) { *bytes = need; return SMC_OK; }
    if (*bytes < need) return fail(ctx, SMC_EINVAL, "smc_save: buffer too small");
    API_BEGIN
    SaveHeader h{};
    std::memcpy(h.magic, "SMCGMv1", 8);
    h.N = c.N; h.d = c.d; h.K = c.K; h.r = c.r; h.layer = c.layer; h.stage = c.stage; h.fitted = c.fitted ? 1 : 0;
    h.step = c.step; h.t = c.t; h.beta = c.beta;
    char* p = reinterpret_cast<char*>(host_buf);
    std::memcpy(p, &h, sizeof(h));
    double* q = reinterpret_cast<double*>(p + sizeof(h));
    check(cudaMemcpyAsync(q, c.X, (size_t)c.N * c.d * 8, cudaMemcpyDeviceToHost, c.stream), "save");
    q += (size_t)c.N * c.d;
    check(cudaMemcpyAsync(q, c.Phi, (size_t)c.N * 8, cudaMemcpyDeviceToHost, c.stream), "save");
    q += c.N;
    check(cudaMemcpyAsync(q, c.gw, (size_t)c.K * 8, cudaMemcpyDeviceToHost, c.stream), "save");
    q += c.K;
    check(cudaMemcpyAsync(q, c.gmu, (size_t)c.K * c.r * 8, cudaMemcpyDeviceToHost, c.stream), "save");
    q += (size_t)c.K * c.r;
    check(cudaMemcpyAsync(q, c.glam, (size_t)c.K * c.r * 8, cudaMemcpyDeviceToHost, c.stream), "save");
    q += (size_t)c.K * c.r;
    if (covn) check(cudaMemcpyAsync(q, c.gcov, covn * 8, cudaMemcpyDeviceToHost, c.stream), "save");
    sync_stream(c);
    *bytes = need;
    return SMC_OK;
    API_END(ctx)
}

smc_status smc_load(smc_ctx* ctx, const void* host_buf, size_t bytes) {
    if (!ctx || !host_buf || bytes < sizeof(SaveHeader)) return SMC_EINVAL;
    Ctx& c = ctx->c;
    SaveHeader h;
    std::memcpy(&h, host_buf, sizeof(h));
    if (std::memcmp(h.magic, "SMCGMv1", 8) != 0 || h.N != c.N || h.d != c.d || h.K != c.K || h.r != c.r)
        return fail(ctx, SMC_EINVAL, "smc_load: checkpoint does not match this configuration");
    const size_t covn = c.cfg.full_cov ? (size_t)c.K * c.r * c.r : 0;
    const size_t need = sizeof(SaveHeader) + sizeof(double) * ((size_t)c.N * c.d + c.N + c.K + 2 * (size_t)c.K * c.r + covn);
    if (bytes < need) return fail(ctx, SMC_EINVAL, "smc_load: truncated checkpoint");
    API_BEGIN
    const double* q = reinterpret_cast<const double*>(reinterpret_cast<const char*>(host_buf) + sizeof(h));
    check(cudaMemcpyAsync(c.X, q, (size_t)c.N * c.d * 8, cudaMemcpyHostToDevice, c.stream), "load");
    q += (size_t)c.N * c.d;
    check(cudaMemcpyAsync(c.Phi, q, (size_t)c.N * 8, cudaMemcpyHostToDevice, c.stream), "load");
    q += c.N;
    check(cudaMemcpyAsync(c.gw, q, (size_t)c.K * 8, cudaMemcpyHostToDevice, c.stream), "load");
    q += c.K;
    check(cudaMemcpyAsync(c.gmu, q, (size_t)c.K * c.r * 8, cudaMemcpyHostToDevice, c.stream), "load");
    q += (size_t)c.K * c.r;
    check(cudaMemcpyAsync(c.glam, q, (size_t)c.K * c.r * 8, cudaMemcpyHostToDevice, c.stream), "load");
    q += (size_t)c.K * c.r;
    if (covn && h.fitted) factor_mixture(c, q);            // uploads C_j and its factors
    sync_stream(c);
    c.layer = h.layer; c.stage = h.stage; c.fitted = h.fitted != 0; c.step = h.step; c.t = h.t; c.beta = h.beta;
    return SMC_OK;
    API_END(ctx)
}

// ---------------------------------------------------------------------------
// Batched moves in one CUDA graph
// ---------------------------------------------------------------------------
struct smc_batch {
    std::vector<smc_ctx*> ctxs;
    int steps = 0;
    cudaStream_t origin = nullptr;
    std::vector<cudaStream_t> streams;   // one capture stream per context
    cudaStream_t aux[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> done;       // per context: its branch / its stream
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static void batch_free(smc_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaStream_t st : b->streams) if (st) cudaStreamDestroy(st);
    for (cudaStream_t st : b->aux) if (st) cudaStreamDestroy(st);
    if (b->origin) cudaStreamDestroy(b->origin);
    if (b->fork) cudaEventDestroy(b->fork);
    for (cudaEvent_t e : b->done) if (e) cudaEventDestroy(e);
    delete b;
}

smc_status smc_batch_create(smc_ctx* const* ctxs, int count, int steps, smc_batch** out) {
    if (!ctxs || !out || count < 1 || steps < 1) {
        set_global_error("smc_batch_create: null pointer, count < 1 or steps < 1");
        return SMC_EINVAL;
    }
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { set_global_error("smc_batch_create: no CUDA device"); return SMC_ECUDA; }
    for (int i = 0; i < count; ++i) {
        if (!ctxs[i]) { set_global_error("smc_batch_create: null context"); return SMC_EINVAL; }
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == ctxs[i]) { set_global_error("smc_batch_create: a context appears twice"); return SMC_EINVAL; }
        const Ctx& c = ctxs[i]->c;
        if (c.dim != 2) { set_global_error("smc_batch_create: graph capture is built for the 2D problem"); return SMC_EINVAL; }
        if (c.cfg.kernel != SMC_K_PCN && c.cfg.kernel != SMC_K_PCN_GM && c.cfg.kernel != SMC_K_GM_INDEP) {
            set_global_error("smc_batch_create: the pCN, pCN-GM and SMC-GM kernels only");
            return SMC_EINVAL;
        }
        if (!device_visible(c.X)) { set_global_error("smc_batch_create: a context lives on another device"); return SMC_EINVAL; }
        if (c.cfg.tile_kernel == 1) {
            set_global_error("smc_batch_create: graph capture needs the warp-tile kernels on the finest level (tile_kernel 0, 2, 3 or 4)");
            return SMC_EINVAL;
        }
    }
    smc_batch* b = new smc_batch();
    b->steps = steps;
    b->ctxs.assign(ctxs, ctxs + count);
    std::vector<cudaStream_t> saved(count, nullptr);
    int captured = -1;
    try {
        check(cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking), "stream");
        for (auto& st : b->aux) check(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream");
        b->streams.assign(count, nullptr);
        b->done.assign(count, nullptr);
        for (int i = 0; i < count; ++i) {
            check(cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking), "stream");
            check(cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming), "event");
            check(cudaStreamSynchronize(ctxs[i]->c.stream), "sync");   // the context's own work is done
        }
        check(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event");
        check(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed), "begin capture");
        check(cudaEventRecord(b->fork, b->origin), "fork");
        for (int i = 0; i < count; ++i) {
            Ctx& c = ctxs[i]->c;
            captured = i;
            saved[i] = c.stream;
            const smc_profile pc = c.pc;
            const bool prof = c.prof;
            c.stream = b->streams[i];
            c.graph = true; c.lenient = true; c.prof = false; c.gdepth = 0;
            for (int k = 0; k < 4; ++k) c.gaux[k] = b->aux[k];
            check(cudaStreamWaitEvent(c.stream, b->fork, 0), "fork wait");
            check(cudaMemsetAsync(c.icount, 0, sizeof(int), c.stream), "memset");
            check(cudaMemsetAsync(c.gcnt, 0, sizeof(GraphCounters), c.stream), "memset");
            capture_move_steps(c, steps, c.icount);
            check(cudaEventRecord(b->done[i], c.stream), "join");
            check(cudaStreamWaitEvent(b->origin, b->done[i], 0), "join wait");
            c.stream = saved[i]; c.graph = false; c.lenient = false; c.prof = prof; c.pc = pc;
            captured = -1;
        }
        check(cudaStreamEndCapture(b->origin, &b->graph), "end capture");
        check(cudaGraphInstantiate(&b->exec, b->graph, 0), "instantiate");
    } catch (const CudaError& ce) {
        if (captured >= 0) {
            Ctx& c = ctxs[captured]->c;
            c.stream = saved[captured]; c.graph = false; c.lenient = false;
        }
        cudaGraph_t tmp = nullptr;
        cudaStreamCaptureStatus cs;
        if (b->origin && cudaStreamIsCapturing(b->origin, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            (void)cudaStreamEndCapture(b->origin, &tmp);
        if (tmp) cudaGraphDestroy(tmp);
        (void)cudaGetLastError();
        set_global_error((std::string("smc_batch_create: ") + ce.what + ": " + cudaGetErrorString(ce.e)).c_str());
        batch_free(b);
        return SMC_ECUDA;
    } catch (const InputError& ie) {
        if (captured >= 0) {
            Ctx& c = ctxs[captured]->c;
            c.stream = saved[captured]; c.graph = false; c.lenient = false;
        }
        cudaGraph_t tmp = nullptr;
        cudaStreamCaptureStatus cs;
        if (b->origin && cudaStreamIsCapturing(b->origin, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            (void)cudaStreamEndCapture(b->origin, &tmp);
        if (tmp) cudaGraphDestroy(tmp);
        (void)cudaGetLastError();
        set_global_error((std::string("smc_batch_create: ") + ie.what).c_str());
        batch_free(b);
        return SMC_EINVAL;
    }
    *out = b;
    return SMC_OK;
}

// The batched move; with host arrays, each context's particles and potentials are
// copied in before the launch and out after it, on the graph's stream.
static smc_status batch_move(smc_batch* b, double* accept_rates, const double* const* X_in, const double* const* Phi_in,
                             double* const* X_out, double* const* Phi_out) {
    if (!b) return SMC_EINVAL;
    const int count = (int)b->ctxs.size();
    for (int i = 0; i < count; ++i) {
        const Ctx& c = b->ctxs[i]->c;
        if (c.stage < 1 || !c.fitted) {
            set_global_error("smc_batch_move: every context needs an initialised state and a fitted mixture");
            return SMC_ESTATE;
        }
    }
    std::vector<MoveSched> ms(count);
    std::vector<int> acc(count, 0);
    std::vector<GraphCounters> gc(count);
    std::vector<int> err(2 * count, 0);
    try {
        for (int i = 0; i < count; ++i) {
            Ctx& c = b->ctxs[i]->c;
            ms[i].t = c.t; ms[i].beta = c.beta; ms[i].gamma = std::sqrt(1.0 - c.beta * c.beta); ms[i].step = c.step; ms[i].pad = 0;
            check(cudaEventRecord(b->done[i], c.stream), "record");          // earlier work on the context's stream first
            check(cudaStreamWaitEvent(b->origin, b->done[i], 0), "wait");
            check(cudaMemcpyAsync(c.msched, &ms[i], sizeof(MoveSched), cudaMemcpyHostToDevice, b->origin), "schedule");
            if (X_in) {
                check(cudaMemcpyAsync(c.X, X_in[i], (size_t)c.N * c.d * sizeof(double), cudaMemcpyHostToDevice, b->origin), "h2d X");
                check(cudaMemcpyAsync(c.Phi, Phi_in[i], (size_t)c.N * sizeof(double), cudaMemcpyHostToDevice, b->origin), "h2d Phi");
            }
        }
        check(cudaGraphLaunch(b->exec, b->origin), "graph launch");
        for (int i = 0; i < count; ++i) {
            Ctx& c = b->ctxs[i]->c;
            if (X_out && X_out[i])
                check(cudaMemcpyAsync(X_out[i], c.X, (size_t)c.N * c.d * sizeof(double), cudaMemcpyDeviceToHost, b->origin), "d2h X");
            if (Phi_out && Phi_out[i])
                check(cudaMemcpyAsync(Phi_out[i], c.Phi, (size_t)c.N * sizeof(double), cudaMemcpyDeviceToHost, b->origin), "d2h Phi");
            check(cudaMemcpyAsync(&acc[i], c.icount, sizeof(int), cudaMemcpyDeviceToHost, b->origin), "d2h");
            check(cudaMemcpyAsync(&gc[i], c.gcnt, sizeof(GraphCounters), cudaMemcpyDeviceToHost, b->origin), "d2h");
            check(cudaMemcpyAsync(&err[2 * i], c.dev_err, 2 * sizeof(int), cudaMemcpyDeviceToHost, b->origin), "d2h");
            check(cudaMemsetAsync(c.dev_err, 0, 2 * sizeof(int), b->origin), "memset");
        }
        check(cudaStreamSynchronize(b->origin), "sync");
    } catch (const CudaError& ce) {
        set_global_error((std::string("smc_batch_move: ") + ce.what + ": " + cudaGetErrorString(ce.e)).c_str());
        return SMC_ECUDA;
    }
    smc_status st = SMC_OK;
    for (int i = 0; i < count; ++i) {
        Ctx& c = b->ctxs[i]->c;
        if (err[2 * i]) {
            set_global_error("smc_batch_move: a kernel's bounded mbarrier wait timed out");
            st = SMC_ECUDA;
        }
        const long long solves = (long long)c.N * b->steps;
        const double rate = (double)acc[i] / (double)solves;
        if (accept_rates) accept_rates[i] = rate;
        if (c.cfg.kernel != SMC_K_GM_INDEP) {
            double be = c.beta;
            if (rate > 0.3) be = 2.0 * be;
            else if (rate < 0.15) be = 0.5 * be;
            c.beta = std::min(be, 1.0);
        }
        c.step += (unsigned int)b->steps;
        ++c.layer;
        c.stage = 1;
        c.last_iters = gc[i].itmax;
        c.nonconv += (long long)gc[i].nonconv;
        c.pc.solves += solves;
        c.pc.cg_iterations += (long long)gc[i].cg_iterations;
        c.pc.inner_solves += (long long)gc[i].inner_solves;
        c.pc.residuals += (long long)gc[i].residuals;
        c.pc.graph_launches += 1;
        c.pc.host_syncs += 1;                        // the one wait after the launch
        c.pc.cells = c.n * c.n;
        c.pc.word_bytes = mixed_precision(c.cfg) ? 4 : 8;
        if (st == SMC_OK && (long long)gc[i].nonconv * 100 > solves) {
            set_global_error("smc_batch_move: more than 1% of a context's forward solves missed the tolerance");
            st = SMC_ENOCONV;
        }
    }
    return st;
}

smc_status smc_batch_move(smc_batch* b, double* accept_rates) {
    NvtxRange nvtx("smc_batch_move");
    return batch_move(b, accept_rates, nullptr, nullptr, nullptr, nullptr);
}

smc_status smc_batch_move_host(smc_batch* b, const double* const* X_in, const double* const* Phi_in, double* const* X_out,
                               double* const* Phi_out, double* accept_rates) {
    if (!b || !X_in || !Phi_in) return SMC_EINVAL;
    for (size_t i = 0; i < b->ctxs.size(); ++i)
        if (!X_in[i] || !Phi_in[i]) {
            set_global_error("smc_batch_move_host: every context needs X_in and Phi_in");
            return SMC_EINVAL;
        }
    NvtxRange nvtx("smc_batch_move_host");
    return batch_move(b, accept_rates, X_in, Phi_in, X_out, Phi_out);
}

void smc_batch_destroy(smc_batch* b) { batch_free(b); }

}  // extern "C"

