"""Thin ctypes binding of libsmcgm.so (include/smcgm.h): argument marshalling
only -- every step of the particle move runs in the library's CUDA kernels.

The library must have been built (``paper_2503_16028_gb300.build.build()``);
loading fails loudly otherwise -- there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsmcgm.so")

SMC_STATIC_RESAMPLE_MAX = 32768
SMC_OK, SMC_EINVAL, SMC_ENOMEM, SMC_ECUDA, SMC_ENOCONV, SMC_EDEGENERATE, SMC_ESTATE = range(7)
SMC_K_PCN, SMC_K_PCN_GM, SMC_K_GM_INDEP, SMC_K_PCNL, SMC_K_GMPCNL = range(5)
SMC_P_FP64, SMC_P_FP32_REFINE, SMC_P_BF16SMOOTH_REFINE = range(3)
STATUS_NAMES = ["SMC_OK", "SMC_EINVAL", "SMC_ENOMEM", "SMC_ECUDA", "SMC_ENOCONV", "SMC_EDEGENERATE", "SMC_ESTATE"]

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p


class smc_config(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n", ctypes.c_int), ("kl_modes", ctypes.c_int), ("alpha", ctypes.c_double),
        ("n_obs", ctypes.c_int), ("obs", _dp), ("data", _dp), ("sigma", ctypes.c_double),
        ("source_kind", ctypes.c_int), ("src_amp", ctypes.c_double), ("src_width", ctypes.c_double),
        ("n_particles", ctypes.c_int), ("n_components", ctypes.c_int), ("gm_rank", ctypes.c_int), ("em_iters", ctypes.c_int),
        ("var_floor", ctypes.c_double), ("beta0", ctypes.c_double), ("ess_frac", ctypes.c_double),
        ("kernel", ctypes.c_int), ("precision", ctypes.c_int), ("tol_inner", ctypes.c_double), ("tol_outer", ctypes.c_double),
        ("max_iter", ctypes.c_int), ("max_refine", ctypes.c_int), ("smooth_sweeps", ctypes.c_int), ("fine_sweeps", ctypes.c_int),
        ("coarse_scale", ctypes.c_double), ("solve_batch", ctypes.c_int), ("seed", ctypes.c_ulonglong),
        ("gradient", ctypes.c_int), ("full_cov", ctypes.c_int), ("tile_kernel", ctypes.c_int),
    ]


class smc_profile(ctypes.Structure):
    _fields_ = [("solves", ctypes.c_longlong), ("cg_iterations", ctypes.c_longlong), ("inner_solves", ctypes.c_longlong),
                ("residuals", ctypes.c_longlong), ("dom_launches", ctypes.c_longlong), ("dom_particles", ctypes.c_longlong),
                ("dom_ms", ctypes.c_double), ("dom_bytes", ctypes.c_double), ("launches", ctypes.c_longlong), ("cells", ctypes.c_int),
                ("word_bytes", ctypes.c_int), ("graph_launches", ctypes.c_longlong),
                ("host_syncs", ctypes.c_longlong)]


EXPORTS = {
    "smc_config_init": (ctypes.c_int, [ctypes.POINTER(smc_config)]),
    "smc_workspace_size": (ctypes.c_int, [ctypes.POINTER(smc_config), ctypes.POINTER(ctypes.c_size_t)]),
    "smc_init": (ctypes.c_int, [ctypes.POINTER(smc_config), _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]),
    "smc_temper_step": (ctypes.c_int, [_vp, _dp, _dp, _dp, _ip]),
    "smc_resample": (ctypes.c_int, [_vp]),
    "gm_fit": (ctypes.c_int, [_vp, _dp]),
    "smc_move": (ctypes.c_int, [_vp, ctypes.c_int, _dp, _ip]),
    "smc_move_host": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _dp]),
    "smc_posterior_moments": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "smc_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp, _ip]),
    "smc_gradient": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp]),
    "smc_get_particles": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    "smc_set_particles": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int]),
    "smc_set_schedule": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_uint]),
    "smc_get_schedule": (ctypes.c_int, [_vp, _dp, _dp, _ip, ctypes.POINTER(ctypes.c_uint)]),
    "smc_set_mixture": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "smc_get_mixture": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "smc_set_mixture_cov": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "smc_get_mixture_cov": (ctypes.c_int, [_vp, _vp]),
    "smc_get_diagnostics": (ctypes.c_int, [_vp] + [ctypes.POINTER(_vp)] * 5),
    "smc_save": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_size_t)]),
    "smc_load": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "smc_last_error": (ctypes.c_char_p, [_vp]),
    "smc_destroy": (None, [_vp]),
    "smc_version": (ctypes.c_char_p, []),
    "smc_config_size": (ctypes.c_size_t, []),
    "smc_profile_query": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(smc_profile), ctypes.c_int]),
    "smc_copy_to_host": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_size_t]),
    "smc_resample_indices_static": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_ulonglong, ctypes.c_int, _vp, _vp]),
    "smc_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)]),
    "smc_batch_move": (ctypes.c_int, [_vp, _vp]),
    "smc_batch_move_host": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "smc_batch_destroy": (None, [_vp]),
}

_LIB = None


def load_library(path=LIB_PATH):
    """Load libsmcgm.so and declare every export; raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise ImportError("libsmcgm.so not found at %s: build it with paper_2503_16028_gb300.build.build() "
                          "(there is no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.smc_config_size() != ctypes.sizeof(smc_config):
        raise ImportError("smc_config layout mismatch between libsmcgm.so and the binding")
    _LIB = lib
    return lib


class SMCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 7 else status, msg))
        self.status = status


def _ptr(a):
    """Device pointer of a torch tensor, address of a numpy array, or None."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _device_f64(t, count, name):
    """Check that `t` is a contiguous float64 CUDA tensor with at least `count` elements (the
    library's kernels read it as device memory)."""
    if not getattr(t, "is_cuda", False):
        raise ValueError("%s must be a CUDA tensor" % name)
    if str(t.dtype) != "torch.float64":
        raise ValueError("%s must be float64, got %s" % (name, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.numel() < count:
        raise ValueError("%s holds %d elements, %d needed" % (name, t.numel(), count))
    return t


def _host_f64(a, count, name):
    """Check that `a` is a contiguous float64 host array (numpy or CPU tensor) with at least
    `count` elements (the library copies it with cudaMemcpyAsync)."""
    if getattr(a, "is_cuda", False):
        raise ValueError("%s must be host memory" % name)
    dt = str(a.dtype)
    if dt not in ("float64", "torch.float64"):
        raise ValueError("%s must be float64, got %s" % (name, dt))
    contiguous = a.is_contiguous() if hasattr(a, "is_contiguous") else a.flags["C_CONTIGUOUS"]
    if not contiguous:
        raise ValueError("%s must be contiguous" % name)
    n = a.numel() if hasattr(a, "numel") else a.size
    if n < count:
        raise ValueError("%s holds %d elements, %d needed" % (name, n, count))
    return a


def make_config(preset, **overrides):
    """smc_config from a dict (inputs.PRESETS entry merged with obs/data arrays); keeps the arrays alive."""
    lib = load_library()
    cfg = smc_config()
    lib.smc_config_init(ctypes.byref(cfg))
    p = dict(preset)
    p.update(overrides)
    obs = np.ascontiguousarray(np.asarray(p["obs"], dtype=np.float64).reshape(-1))
    data = np.ascontiguousarray(np.asarray(p["data"], dtype=np.float64))
    cfg.dim = p["dim"]; cfg.n = p["n"]; cfg.kl_modes = p["kl_modes"]; cfg.alpha = p["alpha"]
    cfg.n_obs = data.shape[0]
    cfg.obs = obs.ctypes.data_as(_dp); cfg.data = data.ctypes.data_as(_dp); cfg.sigma = p["sigma"]
    cfg.source_kind = p["source_kind"]; cfg.src_amp = p["src_amp"]; cfg.src_width = p["src_width"]
    cfg.n_particles = p["n_particles"]; cfg.n_components = p["n_components"]; cfg.gm_rank = p["gm_rank"]
    cfg.beta0 = p["beta0"]; cfg.ess_frac = p["ess_frac"]; cfg.seed = p["seed"]
    for key in ("em_iters", "var_floor", "kernel", "precision", "tol_inner", "tol_outer", "max_iter", "max_refine",
                "smooth_sweeps", "fine_sweeps", "coarse_scale", "solve_batch", "gradient", "full_cov", "tile_kernel"):
        if key in p:
            setattr(cfg, key, p[key])
    cfg._keep = (obs, data)
    return cfg


def choose_solve_batch(workspace_size, n_particles, budget):
    """Largest solve batch B in [1, N] whose workspace (workspace_size(B) bytes) fits `budget`
    bytes; N itself when it fits.  The results do not depend on B (each particle's solve is
    its own), only the memory and the number of batches do.  Raises MemoryError when even
    B = 1 does not fit (the particle arrays alone exceed the budget)."""
    if workspace_size(n_particles) <= budget:
        return n_particles
    if workspace_size(1) > budget:
        raise MemoryError("the workspace needs %d bytes even with one particle per solve batch; %d available"
                          % (workspace_size(1), budget))
    lo, hi = 1, n_particles          # workspace_size(lo) fits, workspace_size(hi) does not
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if workspace_size(mid) <= budget:
            lo = mid
        else:
            hi = mid
    return lo


class Sampler:
    """One smc_ctx with its caller-owned device workspace (a torch uint8 tensor).

    With cfg.solve_batch = 0 (the library's choice: all particles, up to 2^28 grid cells per
    solve batch) and a workspace larger than 90 % of the device's free memory, the batch is
    reduced to the largest that fits (choose_solve_batch); cfg.solve_batch is updated to the
    value used."""

    def __init__(self, cfg, device="cuda:0", stream=None):
        import torch
        self.lib = load_library()
        self.cfg = cfg
        size = ctypes.c_size_t()
        self._check(self.lib.smc_workspace_size(ctypes.byref(cfg), ctypes.byref(size)), None)
        budget = None
        if cfg.solve_batch == 0:
            try:
                budget = int(0.9 * torch.cuda.mem_get_info(torch.device(device))[0])
            except Exception:          # no memory figure: one batch of all particles, as configured
                budget = None
        if budget is not None and size.value + 256 > budget:
            def ws(b):
                cfg.solve_batch = int(b)
                self._check(self.lib.smc_workspace_size(ctypes.byref(cfg), ctypes.byref(size)), None)
                return size.value + 256
            try:
                cfg.solve_batch = choose_solve_batch(ws, cfg.n_particles, budget)
            except MemoryError:
                cfg.solve_batch = 0
                raise
            ws(cfg.solve_batch)                 # size.value: the workspace of the batch chosen
        self.ws = torch.empty(size.value + 256, dtype=torch.uint8, device=device)
        base = self.ws.data_ptr()
        aligned = (base + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        ctx = ctypes.c_void_p()
        st = self.lib.smc_init(ctypes.byref(cfg), ctypes.c_void_p(aligned), size.value,
                               ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx))
        if st != SMC_OK:
            raise SMCError(st, self.lib.smc_last_error(None).decode())
        self.ctx = ctx
        self.d = cfg.kl_modes ** 2 if cfg.dim == 2 else cfg.kl_modes
        self.N = cfg.n_particles
        self.K = 1 if cfg.kernel in (SMC_K_PCN, SMC_K_PCNL) else cfg.n_components
        self.r = min(cfg.gm_rank, self.d)

    def _check(self, st, ctx, allow=()):
        if st != SMC_OK and st not in allow:
            msg = self.lib.smc_last_error(ctx).decode()
            raise SMCError(st, msg)
        return st

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.smc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- SMC steps -------------------------------------------------------
    def smc_temper_step(self):
        h, ess, lz = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        done = ctypes.c_int()
        self._check(self.lib.smc_temper_step(self.ctx, ctypes.byref(h), ctypes.byref(ess), ctypes.byref(lz),
                                             ctypes.byref(done)), self.ctx)
        return h.value, ess.value, lz.value, bool(done.value)

    def smc_resample(self):
        self._check(self.lib.smc_resample(self.ctx), self.ctx)

    def gm_fit(self):
        ll = ctypes.c_double()
        self._check(self.lib.gm_fit(self.ctx, ctypes.byref(ll)), self.ctx)
        return ll.value

    def smc_move(self, steps=1, allow_noconv=False):
        acc, it = ctypes.c_double(), ctypes.c_int()
        st = self._check(self.lib.smc_move(self.ctx, steps, ctypes.byref(acc), ctypes.byref(it)), self.ctx,
                         allow=(SMC_ENOCONV,) if allow_noconv else ())
        return acc.value, it.value

    def smc_move_host(self, X_in, Phi_in, X_out, Phi_out):
        for a, cnt, nm in ((X_in, self.N * self.d, "X_in"), (Phi_in, self.N, "Phi_in"),
                           (X_out, self.N * self.d, "X_out"), (Phi_out, self.N, "Phi_out")):
            _host_f64(a, cnt, nm)
        acc = ctypes.c_double()
        self._check(self.lib.smc_move_host(self.ctx, _ptr(X_in), _ptr(Phi_in), _ptr(X_out), _ptr(Phi_out),
                                           ctypes.byref(acc)), self.ctx)
        return acc.value

    def smc_posterior_moments(self, grid=False):
        mean = np.empty(self.d); var = np.empty(self.d)
        cells = (self.cfg.n ** 2) if self.cfg.dim == 2 else self.cfg.n
        mg = np.empty(cells) if grid else None
        vg = np.empty(cells) if grid else None
        self._check(self.lib.smc_posterior_moments(self.ctx, _ptr(mean), _ptr(var), _ptr(mg), _ptr(vg)), self.ctx)
        return (mean, var, mg, vg) if grid else (mean, var)

    def smc_forward(self, X_dev, Phi_dev, w_dev=None):
        count = int(X_dev.shape[0])
        _device_f64(X_dev, count * self.d, "X_dev")
        _device_f64(Phi_dev, count, "Phi_dev")
        if w_dev is not None:
            cells = (self.cfg.n ** 2) if self.cfg.dim == 2 else self.cfg.n - 1
            _device_f64(w_dev, count * cells, "w_dev")
        it = ctypes.c_int()
        self._check(self.lib.smc_forward(self.ctx, _ptr(X_dev), int(X_dev.shape[0]), _ptr(Phi_dev), _ptr(w_dev),
                                         ctypes.byref(it)), self.ctx)
        return it.value

    def smc_gradient(self, X_dev, Phi_dev, G_dev):
        """Phi(x) and dPhi/dx of the rows of X_dev (device tensors, FP64) into Phi_dev and G_dev."""
        count = int(X_dev.shape[0])
        _device_f64(X_dev, count * self.d, "X_dev")
        _device_f64(Phi_dev, count, "Phi_dev")
        _device_f64(G_dev, count * self.d, "G_dev")
        self._check(self.lib.smc_gradient(self.ctx, _ptr(X_dev), int(X_dev.shape[0]), _ptr(Phi_dev), _ptr(G_dev)), self.ctx)

    # --- state access ----------------------------------------------------
    def particles(self):
        """(X, Phi) copied to host numpy arrays."""
        xp, pp = ctypes.c_void_p(), ctypes.c_void_p()
        self._check(self.lib.smc_get_particles(self.ctx, ctypes.byref(xp), ctypes.byref(pp)), self.ctx)
        return self.to_host(xp.value, self.N * self.d).reshape(self.N, self.d), self.to_host(pp.value, self.N)

    def smc_set_particles(self, X, Phi=None):
        X = np.ascontiguousarray(X, dtype=np.float64)
        Phi = None if Phi is None else np.ascontiguousarray(Phi, dtype=np.float64)
        self._check(self.lib.smc_set_particles(self.ctx, _ptr(X), _ptr(Phi), 0), self.ctx)

    def smc_set_schedule(self, t, beta, layer, step):
        self._check(self.lib.smc_set_schedule(self.ctx, t, beta, layer, step), self.ctx)

    def smc_get_schedule(self):
        t, b, l, s = ctypes.c_double(), ctypes.c_double(), ctypes.c_int(), ctypes.c_uint()
        self._check(self.lib.smc_get_schedule(self.ctx, ctypes.byref(t), ctypes.byref(b), ctypes.byref(l), ctypes.byref(s)), self.ctx)
        return t.value, b.value, l.value, s.value

    def smc_set_mixture(self, w, m, lam):
        w = np.ascontiguousarray(w, dtype=np.float64); m = np.ascontiguousarray(m, dtype=np.float64)
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        self._check(self.lib.smc_set_mixture(self.ctx, _ptr(w), _ptr(m), _ptr(lam)), self.ctx)

    def smc_set_mixture_cov(self, w, m, cov):
        w = np.ascontiguousarray(w, dtype=np.float64); m = np.ascontiguousarray(m, dtype=np.float64)
        cov = np.ascontiguousarray(cov, dtype=np.float64)
        self._check(self.lib.smc_set_mixture_cov(self.ctx, _ptr(w), _ptr(m), _ptr(cov)), self.ctx)

    def smc_get_mixture_cov(self):
        cov = np.empty((self.K, self.r, self.r))
        self._check(self.lib.smc_get_mixture_cov(self.ctx, _ptr(cov)), self.ctx)
        return cov

    def smc_get_mixture(self):
        w = np.empty(self.K); m = np.empty((self.K, self.r)); lam = np.empty((self.K, self.r))
        modes = np.empty(self.r, dtype=np.int32)
        self._check(self.lib.smc_get_mixture(self.ctx, _ptr(w), _ptr(m), _ptr(lam), _ptr(modes)), self.ctx)
        return w, m, lam, modes

    def diagnostics(self):
        ptrs = [ctypes.c_void_p() for _ in range(5)]
        self._check(self.lib.smc_get_diagnostics(self.ctx, *[ctypes.byref(p) for p in ptrs]), self.ctx)
        la = self.to_host(ptrs[0].value, self.N)
        acc = self.to_host(ptrs[1].value, self.N, np.uint8)
        pv = self.to_host(ptrs[2].value, self.N)
        lw = self.to_host(ptrs[3].value, self.N)
        idx = self.to_host(ptrs[4].value, self.N, np.int32)
        return dict(log_alpha=la, accepted=acc.astype(bool), phi_proposed=pv, logw=lw, indices=idx)

    def smc_profile_query(self, enable=-1, reset=False):
        out = smc_profile()
        self._check(self.lib.smc_profile_query(self.ctx, enable, ctypes.byref(out), int(reset)), self.ctx)
        return {k: getattr(out, k) for k, _ in smc_profile._fields_}

    def diagnostics_pointers(self):
        """Device addresses of (log alpha, accepted, phi proposed, logw, indices)."""
        ptrs = [ctypes.c_void_p() for _ in range(5)]
        self._check(self.lib.smc_get_diagnostics(self.ctx, *[ctypes.byref(p) for p in ptrs]), self.ctx)
        return [p.value for p in ptrs]

    def smc_save(self):
        size = ctypes.c_size_t()
        self._check(self.lib.smc_save(self.ctx, None, ctypes.byref(size)), self.ctx)
        buf = np.empty(size.value, dtype=np.uint8)
        self._check(self.lib.smc_save(self.ctx, _ptr(buf), ctypes.byref(size)), self.ctx)
        return buf

    def smc_load(self, buf):
        self._check(self.lib.smc_load(self.ctx, _ptr(buf), buf.nbytes), self.ctx)

    def to_host(self, ptr, count, dtype=np.float64):
        """Copy `count` elements at a device address into a new numpy array (smc_copy_to_host)."""
        out = np.empty(count, dtype=dtype)
        self._check(self.lib.smc_copy_to_host(self.ctx, _ptr(out), ctypes.c_void_p(ptr), out.nbytes), self.ctx)
        return out


class Batch:
    """smc_batch: `steps` moves of several samplers (any grid size, particle count and
    precision; pCN, pCN-GM or SMC-GM kernels) captured in one CUDA graph and run with one
    launch per move() -- the same results as smc_move(steps) on each sampler in turn.
    Keeps the samplers alive; close it before closing them."""

    def __init__(self, samplers, steps):
        self.lib = load_library()
        self.samplers = list(samplers)
        arr = (_vp * len(self.samplers))(*[s.ctx.value for s in self.samplers])
        out = _vp()
        st = self.lib.smc_batch_create(arr, len(self.samplers), int(steps), ctypes.byref(out))
        if st != SMC_OK:
            raise SMCError(st, self.lib.smc_last_error(None).decode())
        self.handle = out
        self.steps = int(steps)

    def move(self, allow_noconv=False):
        """One launch of the graph; returns the acceptance rate of every sampler."""
        rates = np.empty(len(self.samplers))
        st = self.lib.smc_batch_move(self.handle, _ptr(rates))
        if st != SMC_OK and not (allow_noconv and st == SMC_ENOCONV):
            raise SMCError(st, self.lib.smc_last_error(None).decode())
        return rates

    def move_host(self, X_in, Phi_in, X_out=None, Phi_out=None, allow_noconv=False):
        """move() with every sampler's particles taken from and returned to host arrays
        (lists with one float64 array per sampler: X as N x d, Phi as N); returns the
        acceptance rates."""
        k = len(self.samplers)
        for name, arrs in (("X_in", X_in), ("Phi_in", Phi_in), ("X_out", X_out), ("Phi_out", Phi_out)):
            if arrs is not None and len(arrs) != k:
                raise ValueError("%s needs one array per sampler" % name)
        for i, s in enumerate(self.samplers):
            _host_f64(X_in[i], s.N * s.d, "X_in[%d]" % i)
            _host_f64(Phi_in[i], s.N, "Phi_in[%d]" % i)
            if X_out is not None:
                _host_f64(X_out[i], s.N * s.d, "X_out[%d]" % i)
            if Phi_out is not None:
                _host_f64(Phi_out[i], s.N, "Phi_out[%d]" % i)

        def table(arrs):
            return None if arrs is None else (_vp * k)(*[_ptr(a).value for a in arrs])
        rates = np.empty(k)
        st = self.lib.smc_batch_move_host(self.handle, table(X_in), table(Phi_in), table(X_out), table(Phi_out), _ptr(rates))
        if st != SMC_OK and not (allow_noconv and st == SMC_ENOCONV):
            raise SMCError(st, self.lib.smc_last_error(None).decode())
        return rates

    def close(self):
        if getattr(self, "handle", None):
            self.lib.smc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
