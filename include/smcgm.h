/*
 * smcgm.h -- C ABI of libsmcgm.so: the per-tempering-step particle move of
 * SMC with the Gaussian-mixture preconditioned Crank-Nicolson kernel
 * (SMC-pCN-GM) for the Darcy-flow inverse problem, on one sm_103a GPU.
 *
 * Paper: Lu, Jia, Meng, "Sequential Monte Carlo with Gaussian Mixture
 * Approximation for Infinite-Dimensional Statistical Inverse Problems",
 * arXiv 2503.16028.  Citations below name the paper's sections, equations and
 * algorithms.
 *
 * Conventions shared by every entry point
 *   - Return a smc_status; no C++ exception crosses the ABI, nothing exits or
 *     traps.  After an error, smc_last_error(ctx) describes it.
 *   - Device memory is owned by the caller: smc_init() receives one device
 *     buffer (smc_workspace_size() bytes, 256-byte aligned) and carves every
 *     device array from it; the buffer must outlive the context.
 *   - Host input arrays are copied during the call; host output pointers are
 *     caller-owned and may be NULL where stated.
 *   - Work is issued on the CUDA stream given to smc_init().  Calls that
 *     return host scalars synchronise that stream; smc_move() and
 *     smc_forward() also synchronise once per solver iteration to stop as
 *     soon as every particle has converged.
 *   - Calls must follow the SMC order (init -> [temper -> resample -> fit ->
 *     move]* -> moments); out-of-order calls return SMC_ESTATE.
 *   - All random numbers come from Philox4x32-10 (Salmon et al., SC'11) with
 *     key = seed and counter = (word group, particle, step counter, purpose),
 *     so a run is reproducible bit for bit on the same GPU.
 */
#ifndef SMCGM_H
#define SMCGM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct smc_ctx smc_ctx;

typedef enum {
    SMC_OK = 0,
    SMC_EINVAL = 1,      /* invalid argument or configuration */
    SMC_ENOMEM = 2,      /* workspace smaller than smc_workspace_size() */
    SMC_ECUDA = 3,       /* a CUDA runtime call failed (message in smc_last_error) */
    SMC_ENOCONV = 4,     /* more than 1% of forward solves missed the tolerance */
    SMC_EDEGENERATE = 5, /* tempering step collapsed to h = 0 */
    SMC_ESTATE = 6       /* call out of order */
} smc_status;

/* Mutation kernels (App. A).  SMC_K_PCN: pCN (eq. pCNproposal, a_pCN);
 * SMC_K_PCN_GM: pCN-GM (Alg. 2); SMC_K_GM_INDEP: the mixture independence
 * sampler with every proposal accepted (Alg. 3, SMC-GM); SMC_K_PCNL:
 * pCN-Langevin, the Langevin equation of App. B with its drift kept
 * (Crank-Nicolson in the linear part, explicit drift, tempered target
 * exp(-t Phi) mu0): v = gamma u - (1 - gamma) t C DPhi(u) + beta C^{1/2} z,
 * log alpha = t (Phi(u) - Phi(v)) + rho(v, u) - rho(u, v) with
 * rho(a, b) = -(1-gamma) t <DPhi(a), b - gamma a>/beta^2
 *             - (1-gamma)^2 t^2 <DPhi(a), C DPhi(a)>/(2 beta^2);
 * each step evaluates Phi and DPhi at the proposal (smc_gradient's forward
 * and adjoint solves), and smc_move starts from DPhi of the current
 * particles (one extra gradient per call).  Needs cfg.gradient = 1.
 * SMC_K_GMPCNL: GMpCN-Langevin (a definition; the paper gives no Langevin
 * kernel): the pCN-GM proposal with the drift preconditioned by the drawn
 * component, v = gamma u + (1-gamma) m_j - (1-gamma) t C_j DPhi(u) +
 * beta C_j^{1/2} z, and log alpha = t (Phi(u) - Phi(v)) + log sum_j w_j
 * R_j(v, u) - log sum_j w_j R_j(u, v), R_j(a, b) the ratio of the drawn
 * component's proposal density to the pCN one; needs cfg.gradient = 1 and a
 * mixture (gm_fit or smc_set_mixture). */
typedef enum { SMC_K_PCN = 0, SMC_K_PCN_GM = 1, SMC_K_GM_INDEP = 2, SMC_K_PCNL = 3, SMC_K_GMPCNL = 4 } smc_kernel;

/* Arithmetic of the forward solve.  SMC_P_FP64: FP64 multigrid-preconditioned
 * CG to tol_outer.  SMC_P_FP32_REFINE: FP32 multigrid-preconditioned CG inner
 * solves to tol_inner, corrected by iterative refinement on the FP64 solution
 * with an FP64-accurate residual until its relative residual is <= tol_outer
 * (an inner solve stops once its residual has fallen by tol_inner or below
 * tol_outer / 2 of the right-hand side, whichever comes first);
 * the coefficients (e^u and the harmonic faces) and the residual's products
 * are formed in double-float (pairs of FP32) arithmetic, ~1e-14 relative, and
 * need |u| < 64 (else the call fails; use SMC_P_FP64).
 * SMC_P_BF16SMOOTH_REFINE: SMC_P_FP32_REFINE with the multigrid smoother's
 * face coefficients stored in BF16 on every tiled level (n_l > 32): the
 * red-black Gauss-Seidel sweeps, the V-cycle residuals and the restriction
 * read the interior west / south faces as BF16 (8-bit significand, converted
 * to FP32 as they are read; FP32 arithmetic throughout), the wall faces,
 * right-hand sides and corrections stay FP32.  The faces are fixed during a
 * solve, so the V-cycle stays a fixed symmetric positive definite
 * preconditioner of the FP32 CG operator, which keeps its FP32 faces; the
 * coarse levels (n_l <= 32) keep FP32 faces; the FP64-accurate refinement
 * is unchanged, so w and Phi meet the same tol_outer.  The paper specifies
 * no solver: this is a storage precision choice of the preconditioner. */
typedef enum { SMC_P_FP64 = 0, SMC_P_FP32_REFINE = 1, SMC_P_BF16SMOOTH_REFINE = 2 } smc_precision;

typedef struct smc_config {
    int dim;            /* 1: -(e^u w')' = f on [0,1]; 2: -div(e^u grad w) = f on (0,1)^2 (Sec. 3.2) */
    int n;              /* 2D: cells per side (power of two, 64..512); 1D: FD intervals (>= 4) */
    int kl_modes;       /* 2D: cosine modes per side, d = kl_modes^2 (<= n/2); 1D: sine modes, d = kl_modes */
    double alpha;       /* prior covariance C = (I - alpha Lap)^-2 (Sec. 2.1, Sec. 3) */
    int n_obs;          /* number of point observations N_d */
    const double* obs;  /* host: 2D n_obs x (x, y) in (0,1)^2; 1D n_obs abscissae */
    const double* data; /* host: n_obs observed values d (Sec. 2.1, eq. forward model) */
    double sigma;       /* noise standard deviation, Phi = |F(u) - d|^2 / (2 sigma^2) */
    int source_kind;    /* 0: f = src_amp; 1: f = src_amp exp(-src_width |x - centre|^2) */
    double src_amp, src_width;
    int n_particles;    /* N (<= 32768) */
    int n_components;   /* mixture components K (1..16) */
    int gm_rank;        /* leading KL modes r carrying the mixture (1..min(d, 256)) */
    int em_iters;       /* EM iterations per fit */
    double var_floor;   /* EM variance floor, as a fraction of the prior eigenvalue */
    double beta0;       /* initial pCN step beta (App. C) */
    double ess_frac;    /* ESS target as a fraction of N (App. C) */
    int kernel;         /* smc_kernel */
    int precision;      /* smc_precision */
    double tol_inner;   /* FP32 inner solve: relative residual reduction per refinement step (default 5e-4) */
    double tol_outer;   /* final FP64 relative residual |b - A w| / |b| */
    int max_iter;       /* CG iterations per inner solve */
    int max_refine;     /* refinement (outer) iterations */
    int smooth_sweeps;  /* red-black Gauss-Seidel sweeps per pre/post smoothing on coarse levels (1 or 2) */
    int fine_sweeps;    /* the same on the finest level (1 or 2) */
    double coarse_scale;/* multigrid coarse-correction factor */
    int solve_batch;    /* particles per forward-solve batch (0: the library's choice, all N up
                           to 2^28 grid cells per batch, e.g. 4096 particles at 256^2; larger
                           batches measured slower).  Results do not depend on it */
    unsigned long long seed;
    int gradient;       /* 1: also lay out the arrays of smc_gradient (2D only; two more
                           solution-sized FP64 arrays per batch particle); 0: no gradients */
    int full_cov;       /* 1: mixture components with full r x r covariances on the mixture
                           modes (EM with the ridge var_floor * diag(lambda_S)); 0: diagonal
                           lambda_j as in Sec. 2.3.  pCN-GM and independence kernels only */
    int tile_kernel;    /* stencil tiles of the multigrid / CG passes on the tiled levels:
                           0 = the default (2); 1 = 32 x 32 tiles, one thread block each;
                           2 = 16 x 16 tiles, one warp each, the finest level's inputs staged
                           by TMA (FP32; the FP64 solver uses 3); 3 = 16 x 16 tiles, one warp
                           each, loading from global memory; 4 = the finest level as 2, the
                           coarser tiled levels as 1.  Same results to the solver tolerance; a
                           speed choice (batch.autotune times them).  smc_batch_* needs 0, 2,
                           3 or 4 */
} smc_config;

/* Fills cfg with the defaults (2D, n = 64, 32 x 32 modes, alpha = 0.02, ...). */
smc_status smc_config_init(smc_config* cfg);

/* Device bytes smc_init() needs for cfg; SMC_EINVAL for an invalid cfg, with the
 * reason in smc_last_error(NULL). */
smc_status smc_workspace_size(const smc_config* cfg, size_t* bytes);

/* Sets up a context on `stream` (a cudaStream_t, NULL = default stream):
 * copies the host inputs, draws v_n ~ mu_0 = N(0, C) (the input step of
 * Alg. 1), solves the N forward problems and stores Phi(v_n).  t = 0,
 * beta = beta0.  d_workspace: the caller's device buffer of `bytes` >=
 * smc_workspace_size() bytes, 256-byte aligned, kept until smc_destroy().
 * On success *out is the new context (release it with smc_destroy()).
 * SMC_EINVAL for an invalid cfg (reason in smc_last_error(NULL)), SMC_ENOMEM
 * when bytes is too small (checked before the GPU is touched), SMC_ECUDA if a
 * CUDA call fails. */
smc_status smc_init(const smc_config* cfg, void* d_workspace, size_t bytes, void* stream, smc_ctx** out);

/* Reweighting step of Alg. 1 with the tempering rule of App. C: finds
 * h = h_{j+1} by 64-step bisection so that ESS(h) >= ess_frac N (or
 * h = 1 - t when that already satisfies it), stores the normalised log
 * weights -h Phi_n - LSE, advances t.  Outputs (host, may be NULL): h, the
 * ESS, the log-evidence increment log((1/N) sum exp(-h Phi_n)), and done = (t == 1). */
smc_status smc_temper_step(smc_ctx* ctx, double* h, double* ess, double* logZ_inc, int* done);

/* Resampling step of Alg. 1: systematic resampling from the stored weights
 * on a 2^48 fixed-point CDF (order-independent, bit-exact), then a particle gather. */
smc_status smc_resample(smc_ctx* ctx);

/* Mixture estimation of Alg. 3 / Sec. 2.4: EM for K diagonal Gaussians (or,
 * with cfg.full_cov, Gaussians with full covariances) on the gm_rank leading
 * KL coordinates of the particles; prior elsewhere.  loglik (host, may be
 * NULL) receives the final log-likelihood. */
smc_status gm_fit(smc_ctx* ctx, double* loglik);

/* Mutation step: `steps` steps of cfg.kernel (pCN-GM: Alg. 2, proposal eq.
 * pCN-GM proposal, acceptance eqs. auv of pCN-GMM..GMM4; the other kernels
 * as described at smc_kernel) for all particles at the current t, each step
 * solving N forward problems (2N with the Langevin kernels); then the beta
 * rule of App. C (not for SMC_K_GM_INDEP).  A proposal whose field leaves
 * the mixed-precision range (|u| >= 64) is not solved and is rejected.
 * accept_rate: mean acceptance over the steps; iters_max: the largest
 * number of CG iterations any solve used (both host, may be NULL). */
smc_status smc_move(smc_ctx* ctx, int steps, double* accept_rate, int* iters_max);

/* Same as smc_move() for steps = 1, but the particle state comes from and
 * returns to HOST buffers (X: N x d, Phi: N), with the copies on the
 * context's stream: the end-to-end form of one move. */
smc_status smc_move_host(smc_ctx* ctx, const double* X_in, const double* Phi_in,
                         double* X_out, double* Phi_out, double* accept_rate);

/* Posterior moments of the particles (output of Alg. 1): KL mean and
 * population variance (d each) and, when the grid pointers are non-NULL,
 * the pointwise mean and variance of u on the grid (2D: n x n, 1D: n
 * midpoints).  Host outputs; any may be NULL. */
smc_status smc_posterior_moments(smc_ctx* ctx, double* mean_kl, double* var_kl,
                                 double* mean_grid, double* var_grid);

/* Forward map F for `count` coefficient vectors already on the device
 * (d_X: count x d, FP64): synthesis, Darcy solve, observation, Phi.
 * d_Phi (count) and d_w (count x grid, FP64, may be NULL; grid = n x n
 * cells in 2D, the n - 1 interior nodes in 1D) are device
 * outputs; iters (host, may be NULL) gets the largest CG iteration count.
 * SMC_EINVAL if a device argument is host memory CUDA does not know (an
 * ordinary malloc or stack address) or memory of another GPU than the
 * current one, checked before any kernel runs. */
smc_status smc_forward(smc_ctx* ctx, const double* d_X, int count, double* d_Phi, double* d_w, int* iters);

/* Potential and its gradient for `count` coefficient vectors on the device
 * (d_X: count x d, FP64): d_Phi (count) and d_grad (count x d, FP64), device
 * outputs, get Phi(x) and dPhi/dx.  The gradient is that of the discrete
 * model by its adjoint: w solves A(u) w = b; lam solves A lam = O^T (O w - d)
 * / sigma^2 (A is symmetric, so the same multigrid-preconditioned solver and
 * precision serve both); dPhi/du_c = -sum over the faces f of cell c of
 * (dK_f/du_c)(lam_c - lam_nb)(w_c - w_nb) with dK_f/du_c = K_f^2 e^{-u_c} / 2
 * for a harmonic face and K_f for a wall face; dPhi/dx is the transpose of the
 * synthesis applied to it.  The drift of the Langevin equation of App. B.
 * Needs cfg.gradient = 1 and dim = 2 (else SMC_ESTATE / SMC_EINVAL); device
 * arguments are checked as in smc_forward. */
smc_status smc_gradient(smc_ctx* ctx, const double* d_X, int count, double* d_Phi, double* d_grad);

/* Full-covariance mixtures (cfg.full_cov = 1): set or read the components'
 * r x r covariances C_j on the mixture modes (host, K x r x r, row-major,
 * symmetric positive definite; w and m as in smc_set_mixture).  The library
 * keeps C_j = L_j L_j^T, L_j^{-1} and log det L_j; the pCN-GM proposal draws
 * beta L_j z on the mixture modes and the acceptance ratio uses
 * N(e; (1-gamma) m_j, beta^2 C_j) / N(e; 0, beta^2 diag(lambda)).  gm_fit
 * then fits full covariances (EM, ridge var_floor * diag(lambda)).  The
 * factors are formed on the device (FP64 Cholesky, one block per component).
 * SMC_ESTATE without cfg.full_cov; SMC_EINVAL for a C_j that is not positive
 * definite, after which the context holds no usable mixture (smc_move returns
 * SMC_ESTATE until smc_set_mixture, smc_set_mixture_cov or gm_fit succeeds). */
smc_status smc_set_mixture_cov(smc_ctx* ctx, const double* w, const double* m, const double* cov);
smc_status smc_get_mixture_cov(smc_ctx* ctx, double* cov);

/* Device views of the particle state (borrowed; valid until the next call). */
smc_status smc_get_particles(smc_ctx* ctx, const double** d_X, const double** d_Phi);

/* Replaces the particle state.  on_device = 1: X, Phi are device pointers;
 * 0: host pointers.  Phi may be NULL to recompute it with the forward map. */
smc_status smc_set_particles(smc_ctx* ctx, const double* X, const double* Phi, int on_device);

/* Temperature t, pCN step beta, layer index and Philox step counter. */
smc_status smc_set_schedule(smc_ctx* ctx, double t, double beta, int layer, unsigned int step);
smc_status smc_get_schedule(smc_ctx* ctx, double* t, double* beta, int* layer, unsigned int* step);

/* Mixture tables (host): w (K), m (K x r), lam (K x r) on the modes returned
 * in `modes` (r ints, storage indices).  smc_set_mixture marks the mixture fitted. */
smc_status smc_set_mixture(smc_ctx* ctx, const double* w, const double* m, const double* lam);
smc_status smc_get_mixture(smc_ctx* ctx, double* w, double* m, double* lam, int* modes);

/* Device views of the last move step: log alpha, accept flags and the
 * proposals' Phi (N each); normalised log weights and resampling indices of
 * the last temper/resample call (N each). */
smc_status smc_get_diagnostics(smc_ctx* ctx, const double** d_log_alpha, const unsigned char** d_accepted,
                               const double** d_phi_proposed, const double** d_logw, const int** d_indices);

/* Checkpoint: particles, Phi, schedule, mixture and counters to a host
 * buffer (call with buf = NULL to get the size), and back. */
smc_status smc_save(smc_ctx* ctx, void* host_buf, size_t* bytes);
smc_status smc_load(smc_ctx* ctx, const void* host_buf, size_t bytes);

/* Last error message of ctx ("" if none; a static message for ctx == NULL). */
const char* smc_last_error(const smc_ctx* ctx);

/* Frees the context's host memory; the device workspace stays the caller's. */
void smc_destroy(smc_ctx* ctx);

/* Solver counters for throughput and roofline accounting (host-side
 * bookkeeping; the CUDA-event timing of the dominant kernel is taken only
 * while profiling is enabled).  The dominant kernel is the finest-level
 * pass that applies the CG update and runs the multigrid pre-smoothing,
 * residual and restriction. */
typedef struct smc_profile {
    long long solves;          /* forward solves (particle-solves) */
    long long cg_iterations;   /* inner CG iterations summed over particles */
    long long inner_solves;    /* inner solves (refinement steps) summed over particles */
    long long residuals;       /* FP64 residual evaluations summed over particles */
    long long dom_launches;    /* launches of the dominant kernel */
    long long dom_particles;   /* particles processed by those launches */
    double dom_ms;             /* summed CUDA-event durations of those launches */
    double dom_bytes;          /* their algorithmic DRAM bytes (inputs read once, outputs written once) */
    long long launches;        /* kernel launches issued by the library (outside CUDA graphs) */
    int cells;                 /* grid cells per solve */
    int word_bytes;            /* bytes per word of the inner solver (4: FP32, 8: FP64) */
    long long graph_launches;  /* launches of batch graphs (smc_batch_move) that moved this context */
    long long host_syncs;      /* waits of the host for the context's stream (the host-driven solver
                                  reads its active counts after every CG step; a graph launch: one) */
} smc_profile;

/* enable: 1 turns event timing of the dominant kernel on, 0 off, any other
 * value (-1) leaves it as is.  If out is non-NULL (host, caller-owned) the
 * counters accumulated since the last reset are copied there and, when reset
 * is non-zero, cleared.  SMC_EINVAL for a NULL ctx, SMC_ECUDA if the timing
 * events cannot be created. */
smc_status smc_profile_query(smc_ctx* ctx, int enable, smc_profile* out, int reset);

/* Copies `bytes` from device address `src` (e.g. a view returned above) to
 * host memory `dst` on the context's stream and waits for it: a helper for
 * bindings that have no CUDA runtime of their own.  Both buffers stay the
 * caller's.  SMC_EINVAL for a NULL ctx or a NULL pointer with bytes > 0,
 * SMC_ECUDA if the copy fails (message in smc_last_error(ctx)). */
smc_status smc_copy_to_host(smc_ctx* ctx, void* dst, const void* src, size_t bytes);

/* Largest particle count smc_resample_indices_static() accepts: its scratch is
 * a fixed device array of this many 64-bit words (256 KiB). */
#define SMC_STATIC_RESAMPLE_MAX 32768

/* Systematic-resampling indices without any allocation.  The paper has no
 * counterpart: this is an interface for callers that cannot give the library
 * device memory (an application whose own pool owns all device memory and
 * forbids other allocations, or a loop that must not risk the implicit
 * synchronisation of cudaMalloc).  It computes exactly what smc_resample()
 * computes for one layer: d_logw (device, n_particles log weights), the key
 * `seed` and the layer index select the Philox draw; d_indices (device,
 * n_particles ints) receives the indices.  Scratch is a file-scope device
 * array of SMC_STATIC_RESAMPLE_MAX words that each GPU loading the library
 * keeps until the process exits; the library calls no cudaMalloc, cudaFree or
 * allocating routine.  Every call looks up the array's device address on the
 * current device (so a device reset in between does no harm); the first call
 * on a device also loads the array there, so make it before capturing work
 * into a stream graph.  All calls share the array: calls that overlap on the
 * GPU race and must be serialised by the caller (e.g. one stream).  Returns
 * SMC_EINVAL for n_particles outside [1, SMC_STATIC_RESAMPLE_MAX] or a
 * d_logw / d_indices that CUDA reports as unregistered host memory or as
 * memory of another GPU than the current one (message in
 * smc_last_error(NULL)), SMC_ECUDA if a CUDA call fails.  Asynchronous on
 * `stream` (a cudaStream_t, NULL = default stream). */
smc_status smc_resample_indices_static(const double* d_logw, int n_particles, unsigned long long seed, int layer,
                                       int* d_indices, void* stream);

/* Batched moves in one CUDA graph (many independent problems, one launch).
 *
 * smc_batch_create captures `steps` moves of every context in ctxs (count >= 1
 * distinct contexts, on the current device, dim = 2, kernel SMC_K_PCN,
 * SMC_K_PCN_GM or SMC_K_GM_INDEP; any grid size, particle count and precision)
 * into one CUDA graph and instantiates it.  The whole move runs on the device:
 * the steps, the refinement phases and the CG iterations are conditional
 * 'while' nodes whose conditions kernels set from the device's counts, and the
 * launches between two compactions of the active particles are 'switch' nodes
 * over launch sizes (all, 1/2, 1/4, ... of the particles); the contexts' moves are
 * parallel branches of the graph.  smc_batch_move launches it once: the same
 * moves, with the same random streams and results, as smc_move(ctx, steps) on
 * every context in turn (each context's t, beta and Philox step are read at the
 * launch; afterwards beta follows the acceptance rule, the layer and step
 * advance, and the counters grow as after smc_move).  accept_rates (host,
 * count doubles, may be NULL) receives each context's acceptance rate.  The
 * batch keeps pointers into the contexts' workspaces: destroy it before any of
 * its contexts, and do not use a context while its batch's move runs.
 * smc_batch_create: SMC_EINVAL for invalid arguments or an unsupported context,
 * SMC_ECUDA if the capture or instantiation fails (messages in
 * smc_last_error(NULL)).  smc_batch_move: SMC_ESTATE if a context has no mixture
 * fitted, SMC_ECUDA if a kernel's bounded wait timed out, SMC_ENOCONV if more
 * than 1% of a context's solves missed the tolerance (after all contexts have
 * moved).  The paper moves one problem at a time; this is its batched form on
 * one GPU. */
typedef struct smc_batch smc_batch;
smc_status smc_batch_create(smc_ctx* const* ctxs, int count, int steps, smc_batch** out);
smc_status smc_batch_move(smc_batch* batch, double* accept_rates);

/* smc_batch_move with the particles in host memory: context i's state is first
 * replaced by X_in[i] (N x d doubles, row-major) and Phi_in[i] (N doubles), the
 * graph moves every context, and the moved state is copied to X_out[i] and
 * Phi_out[i] (the arrays X_out, Phi_out, or an entry of them, may be NULL to skip
 * that copy).  All arrays have one entry per context, in the order given to
 * smc_batch_create; the buffers belong to the caller (page-locked ones make the
 * copies asynchronous).  The copies run on the graph's stream around the launch,
 * and the call returns after the last one, with one wait.  Errors as
 * smc_batch_move, and SMC_EINVAL for a NULL X_in, Phi_in or entry of them. */
smc_status smc_batch_move_host(smc_batch* batch, const double* const* X_in, const double* const* Phi_in,
                               double* const* X_out, double* const* Phi_out, double* accept_rates);
void smc_batch_destroy(smc_batch* batch);

/* Library version string (static storage owned by the library; never NULL). */
const char* smc_version(void);

/* sizeof(smc_config) as compiled into the library (lets bindings check their
 * layout before passing a config; a mismatch means the binding is stale). */
size_t smc_config_size(void);

#ifdef __cplusplus
}
#endif

#endif /* SMCGM_H */
