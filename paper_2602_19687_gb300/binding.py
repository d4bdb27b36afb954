"""Thin ctypes binding of libexoskry.so (include/exoskry.h).

Argument marshalling only: every step of the forward model, likelihood and
adjoint runs in the library's CUDA kernels. Device buffers are torch CUDA
tensors (PyTorch provides device memory and streams); host buffers are numpy
arrays. If the library is missing this module raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libexoskry.so")

ES_OK, ES_EINVAL, ES_ENOMEM, ES_ECUDA, ES_ESTATE, ES_ETIMEOUT = range(6)
ES_MEM_HOST, ES_MEM_DEVICE = 0, 1
ES_TABLE_F32, ES_TABLE_BF16 = 0, 1
ES_FLAG_INVALID, ES_FLAG_TIMEOUT = 1, 2
ES_TEST_WAIT_TIMEOUT = 1
ES_MAX_SPECIES = 16
ES_P_N_EXTRA = 28
ES_MAX_PARAMS = ES_MAX_SPECIES + ES_P_N_EXTRA
ES_MAX_LAYERS = 112
STATUS_NAMES = {0: "ES_OK", 1: "ES_EINVAL", 2: "ES_ENOMEM", 3: "ES_ECUDA", 4: "ES_ESTATE", 5: "ES_ETIMEOUT"}

EXPORTS = ["es_create", "es_load_tables", "es_set_grid", "es_set_data", "es_set_batch", "es_forward",
           "es_loglike", "es_forward_backward", "es_loglike_noalloc", "es_autotune", "es_set_graphs",
           "es_get_flags", "es_query", "es_set_profiling", "es_probe_rates",
           "es_set_memory_limit", "es_set_test_hooks",
           "es_get_profile", "es_last_error", "es_destroy"]


class es_model_desc(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int),
                ("p_top_bar", ctypes.c_double), ("p_bot_bar", ctypes.c_double), ("p_ref_bar", ctypes.c_double),
                ("tp_kind", ctypes.c_int), ("cloud_kind", ctypes.c_int), ("n_species", ctypes.c_int),
                ("species_mass_amu", ctypes.c_double * ES_MAX_SPECIES),
                ("r_star_cm", ctypes.c_double), ("t_star_k", ctypes.c_double),
                ("ray_h2_cm2", ctypes.c_double), ("ray_he_cm2", ctypes.c_double), ("ray_nu_ref", ctypes.c_double),
                ("theta_fixed", ctypes.c_double * ES_MAX_PARAMS),
                ("n_free", ctypes.c_int), ("free_idx", ctypes.c_int * ES_MAX_PARAMS),
                ("emission_flux", ctypes.c_int), ("distance_cm", ctypes.c_double),
                ("cloud_profile", ctypes.c_int), ("cloud_feature", ctypes.c_int),
                ("emission_quadrature", ctypes.c_int), ("emission_solver", ctypes.c_int),
                ("cloud_ssa", ctypes.c_double), ("cloud_g", ctypes.c_double)]


class es_tables_desc(ctypes.Structure):
    _fields_ = [("n_nu", ctypes.c_int), ("nu", ctypes.POINTER(ctypes.c_double)),
                ("n_t", ctypes.c_int), ("t_grid", ctypes.POINTER(ctypes.c_double)),
                ("n_p", ctypes.c_int), ("p_grid_bar", ctypes.POINTER(ctypes.c_double)),
                ("log10_sigma", ctypes.POINTER(ctypes.c_float)),
                ("n_t_cia", ctypes.c_int), ("cia_t_grid", ctypes.POINTER(ctypes.c_double)),
                ("cia_h2h2", ctypes.POINTER(ctypes.c_float)), ("cia_h2he", ctypes.POINTER(ctypes.c_float)),
                ("storage", ctypes.c_int)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libexoskry.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libexoskry.so is not built (run __graft_entry__.build()); "
                           "there is no CPU fallback")
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.es_create.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(es_model_desc)]
    lib.es_load_tables.argtypes = [vp, ctypes.POINTER(es_tables_desc)]
    lib.es_set_grid.argtypes = [vp, vp, vp, ip]
    lib.es_set_data.argtypes = [vp, ip, vp, vp, ip]
    lib.es_set_batch.argtypes = [vp, vp, vp, ip, ip, vp]
    lib.es_forward.argtypes = [vp, vp, vp, vp, ip, vp]
    lib.es_loglike.argtypes = [vp, vp, ip, vp]
    lib.es_forward_backward.argtypes = [vp, vp, vp, ip, vp]
    lib.es_loglike_noalloc.argtypes = [vp, vp, vp, ip, vp, vp]
    lib.es_get_flags.argtypes = [vp, vp, ip, vp]
    lib.es_autotune.argtypes = [vp, vp]
    lib.es_probe_rates.argtypes = [ip, ctypes.POINTER(dp), ctypes.POINTER(dp)]
    lib.es_set_graphs.argtypes = [vp, ip]
    lib.es_set_memory_limit.argtypes = [vp, ctypes.c_uint64]
    lib.es_set_test_hooks.argtypes = [vp, ip]
    lib.es_query.argtypes = [vp, ip]
    lib.es_query.restype = ctypes.c_int64
    lib.es_set_profiling.argtypes = [vp, ip]
    lib.es_get_profile.argtypes = [vp, ip, ctypes.c_char_p, ip, ctypes.POINTER(dp), ctypes.POINTER(ctypes.c_int64)]
    lib.es_last_error.argtypes = [vp]
    lib.es_last_error.restype = ctypes.c_char_p
    lib.es_destroy.argtypes = [vp]
    lib.es_destroy.restype = None
    for name in EXPORTS:
        if name not in ("es_query", "es_last_error", "es_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class ExoskryError(RuntimeError):
    pass


def _ptr(a):
    """Pointer of a numpy array (host) or torch tensor (device) or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()       # torch tensor


def _mem(a):
    if a is None or isinstance(a, np.ndarray):
        return ES_MEM_HOST
    return ES_MEM_DEVICE if a.is_cuda else ES_MEM_HOST


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(stream)


def model_desc(model) -> es_model_desc:
    """es_model_desc from a synth.Model-like object."""
    d = es_model_desc()
    d.n_layers = model.n_layers
    d.p_top_bar, d.p_bot_bar, d.p_ref_bar = model.p_top_bar, model.p_bot_bar, model.p_ref_bar
    d.tp_kind, d.cloud_kind, d.n_species = model.tp_kind, model.cloud_kind, model.n_species
    for s, mass in enumerate(model.masses_amu):
        d.species_mass_amu[s] = float(mass)
    d.r_star_cm, d.t_star_k = model.r_star_cm, model.t_star_k
    d.ray_h2_cm2, d.ray_he_cm2, d.ray_nu_ref = model.ray_h2_cm2, model.ray_he_cm2, model.ray_nu_ref
    for k, v in enumerate(model.theta_fixed):
        d.theta_fixed[k] = float(v)
    d.n_free = len(model.free_idx)
    for k, v in enumerate(model.free_idx):
        d.free_idx[k] = int(v)
    d.emission_flux = int(getattr(model, "emission_flux", 0))
    d.distance_cm = float(getattr(model, "distance_cm", 0.0))
    d.cloud_profile = int(getattr(model, "cloud_profile", 0))
    d.cloud_feature = int(getattr(model, "cloud_feature", 0))
    d.emission_quadrature = int(getattr(model, "emission_quadrature", 0))
    d.emission_solver = int(getattr(model, "emission_solver", 0))
    d.cloud_ssa = float(getattr(model, "cloud_ssa", 0.0))
    d.cloud_g = float(getattr(model, "cloud_g", 0.0))
    return d


class Context:
    """One es_ctx. Methods mirror the C entry points of the same name."""

    def __init__(self, model, device: int = 0):
        self.lib = load_library()
        self.handle = ctypes.c_void_p()
        self._desc = model_desc(model)
        st = self.lib.es_create(ctypes.byref(self.handle), device, ctypes.byref(self._desc))
        if st != ES_OK:
            raise ExoskryError("es_create failed: %s" % STATUS_NAMES.get(st, st))
        self.model = model
        self._keep = []

    def _check(self, st, what):
        if st != ES_OK:
            msg = self.lib.es_last_error(self.handle).decode()
            raise ExoskryError("%s: %s (%s)" % (what, STATUS_NAMES.get(st, st), msg))

    def es_load_tables(self, tables, storage="f32"):
        nu = np.ascontiguousarray(tables.nu, np.float64)
        tg = np.ascontiguousarray(tables.t_grid, np.float64)
        pg = np.ascontiguousarray(tables.p_grid_bar, np.float64)
        sig = np.ascontiguousarray(tables.log10_sigma, np.float32)
        ct = np.ascontiguousarray(tables.cia_t_grid, np.float64)
        c1 = np.ascontiguousarray(tables.cia_h2h2, np.float32)
        c2 = np.ascontiguousarray(tables.cia_h2he, np.float32)
        self._keep = [nu, tg, pg, sig, ct, c1, c2]
        d = es_tables_desc()
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        d.n_nu, d.nu = nu.size, nu.ctypes.data_as(dp)
        d.n_t, d.t_grid = tg.size, tg.ctypes.data_as(dp)
        d.n_p, d.p_grid_bar = pg.size, pg.ctypes.data_as(dp)
        d.log10_sigma = sig.ctypes.data_as(fp)
        d.n_t_cia, d.cia_t_grid = ct.size, ct.ctypes.data_as(dp)
        d.cia_h2h2, d.cia_h2he = c1.ctypes.data_as(fp), c2.ctypes.data_as(fp)
        d.storage = ES_TABLE_BF16 if storage == "bf16" else ES_TABLE_F32
        self._check(self.lib.es_load_tables(self.handle, ctypes.byref(d)), "es_load_tables")
        self._keep = []

    def es_set_grid(self, bin_lo_um, bin_hi_um):
        lo = np.ascontiguousarray(bin_lo_um, np.float64)
        hi = np.ascontiguousarray(bin_hi_um, np.float64)
        self._check(self.lib.es_set_grid(self.handle, _ptr(lo), _ptr(hi), lo.size), "es_set_grid")

    def es_set_data(self, kind, y_obs, sigma):
        y = np.ascontiguousarray(y_obs, np.float64)
        s = np.ascontiguousarray(sigma, np.float64)
        self._check(self.lib.es_set_data(self.handle, int(kind), _ptr(y), _ptr(s), y.size), "es_set_data")

    def es_set_batch(self, theta, kind=None, stream=None):
        """theta: numpy float64 [B, n_free] (host) or torch float64 CUDA tensor."""
        mem = _mem(theta)
        if mem == ES_MEM_HOST:
            theta = np.ascontiguousarray(theta, np.float64)
            if kind is not None:
                kind = np.ascontiguousarray(kind, np.int32)
        B = theta.shape[0]
        self._check(self.lib.es_set_batch(self.handle, _ptr(theta), _ptr(kind), B, mem, _stream(stream)),
                    "es_set_batch")

    def es_forward(self, spectrum=None, binned=None, lnl=None, stream=None):
        outs = [a for a in (spectrum, binned, lnl) if a is not None]
        mem = _mem(outs[0]) if outs else ES_MEM_DEVICE
        self._check(self.lib.es_forward(self.handle, _ptr(spectrum), _ptr(binned), _ptr(lnl), mem,
                                        _stream(stream)), "es_forward")

    def es_loglike(self, lnl, stream=None):
        self._check(self.lib.es_loglike(self.handle, _ptr(lnl), _mem(lnl), _stream(stream)), "es_loglike")

    def es_forward_backward(self, lnl, grad, stream=None):
        self._check(self.lib.es_forward_backward(self.handle, _ptr(lnl), _ptr(grad), _mem(lnl),
                                                 _stream(stream)), "es_forward_backward")

    def es_loglike_noalloc(self, theta, kind, lnl, stream=None):
        """ln L without device allocation (theta, kind, lnl: CUDA tensors; kind may be None)."""
        self._check(self.lib.es_loglike_noalloc(self.handle, _ptr(theta), _ptr(kind), int(theta.shape[0]),
                                                _ptr(lnl), _stream(stream)), "es_loglike_noalloc")

    def es_autotune(self, stream=None):
        """Pick the fused kernels' launch shapes (work-item size, item order) by
        timing them on the current batch; returns {kernel: (size, order)} with
        order "chunk-major" or "sample-major" and size 0 for untuned kernels."""
        self._check(self.lib.es_autotune(self.handle, _stream(stream)), "es_autotune")
        return self.launch_shapes()

    def launch_shapes(self):
        bits = self.es_query(16)
        names = ("trans_fwd", "trans_bwd", "emis_fwd", "emis_bwd", "mixed_fwd", "mixed_bwd")
        keys = (8, 9, 12, 13, 14, 15)
        return {n: (self.es_query(k), "sample-major" if (bits >> i) & 1 else "chunk-major")
                for i, (n, k) in enumerate(zip(names, keys))}

    def es_set_graphs(self, on):
        self._check(self.lib.es_set_graphs(self.handle, 1 if on else 0), "es_set_graphs")

    def es_set_memory_limit(self, nbytes):
        self._check(self.lib.es_set_memory_limit(self.handle, int(nbytes)), "es_set_memory_limit")

    def es_set_test_hooks(self, hooks):
        self._check(self.lib.es_set_test_hooks(self.handle, int(hooks)), "es_set_test_hooks")

    def es_get_flags(self, flags, stream=None):
        self._check(self.lib.es_get_flags(self.handle, _ptr(flags), _mem(flags), _stream(stream)),
                    "es_get_flags")

    def es_query(self, key):
        return int(self.lib.es_query(self.handle, int(key)))

    def es_set_profiling(self, on):
        self._check(self.lib.es_set_profiling(self.handle, 1 if on else 0), "es_set_profiling")

    def es_get_profile(self):
        """List of (kernel name, total ms, launches) accumulated since profiling was enabled."""
        out = []
        buf = ctypes.create_string_buffer(128)
        ms, n = ctypes.c_double(), ctypes.c_int64()
        k = 0
        while self.lib.es_get_profile(self.handle, k, buf, 128, ctypes.byref(ms), ctypes.byref(n)) == ES_OK:
            out.append((buf.value.decode(), ms.value, n.value))
            k += 1
        return out

    def es_destroy(self):
        if self.handle:
            self.lib.es_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.es_destroy()
        except Exception:
            pass


def probe_rates(device: int = 0):
    """(ex2 instructions/s, packed FP32x2 FMA instructions/s) measured on `device`."""
    lib = load_library()
    e, f = ctypes.c_double(), ctypes.c_double()
    st = lib.es_probe_rates(int(device), ctypes.byref(e), ctypes.byref(f))
    if st != ES_OK:
        raise RuntimeError("es_probe_rates failed with status %d" % st)
    return e.value, f.value


def context_for(workload, device: int = 0) -> Context:
    """Create a context and load a synth.Workload's tables, grid and data."""
    ctx = Context(workload.model, device)
    ctx.es_load_tables(workload.tables, workload.table_dtype)
    ctx.es_set_grid(workload.bin_lo_um, workload.bin_hi_um)
    for kind in (0, 1):
        ctx.es_set_data(kind, workload.y_obs[kind], workload.sigma[kind])
    return ctx


class LogLikeBatch:
    """ln L of host parameter vectors through one es_set_batch + es_loglike per
    call (host in, host out): the batched likelihood a sampler consumes
    (e.g. nested.run). theta: float64 [B, n_free]; returns float64 [B]."""

    def __init__(self, context, kind=0, stream=None):
        self.context, self.kind, self.stream = context, int(kind), stream
        self.calls = 0

    def __call__(self, theta):
        theta = np.ascontiguousarray(theta, np.float64)
        B = theta.shape[0]
        self.context.es_set_batch(theta, np.full(B, self.kind, np.int32), self.stream)
        lnl = np.empty(B, np.float64)
        self.context.es_loglike(lnl, self.stream)
        self.calls += 1
        return lnl


def _autograd_function():
    import torch

    class LogLikelihood(torch.autograd.Function):
        """ln L(theta) per sample with the hand-written adjoint as backward.
        theta: float64 CUDA tensor [B, n_free]; returns float64 [B]."""

        @staticmethod
        def forward(ctx_, theta, context, kind=None):
            theta = theta.detach().contiguous()
            context.es_set_batch(theta, kind)
            lnl = torch.empty(theta.shape[0], dtype=torch.float64, device=theta.device)
            grad = torch.empty_like(theta)
            context.es_forward_backward(lnl, grad)
            ctx_.save_for_backward(grad)
            return lnl

        @staticmethod
        def backward(ctx_, g):
            (grad,) = ctx_.saved_tensors
            return g[:, None] * grad, None, None

    return LogLikelihood


def loglikelihood(theta, context, kind=None):
    """Differentiable ln L (torch.autograd) through es_forward_backward."""
    return _autograd_function().apply(theta, context, kind)
