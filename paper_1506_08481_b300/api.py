"""Thin ctypes binding over the C ABI declared in include/se_mobility.h.

Argument marshalling only: every step of the product and of the solve runs in
the CUDA library ``libse_b300.so``.  There is no CPU fallback; ``load()`` raises
when the library is missing or fails to load.

Device arrays are passed as torch CUDA tensors (their data pointers) and work is
enqueued on torch's current CUDA stream unless another stream is given.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libse_b300.so")

SE_OK = 0
SE_ERR_ARG, SE_ERR_GRID, SE_ERR_CUTOFF, SE_ERR_CUDA = -1, -2, -3, -4
SE_ERR_STATE, SE_ERR_NONFINITE, SE_ERR_NOT_CONVERGED, SE_ERR_NOMEM = -5, -6, -7, -8
SE_ERR_TOO_LARGE, SE_ERR_OVERLAP = -9, -10
SE_NOALLOC_MAX_N = 8192
SE_F32, SE_F64 = 0, 1
SE_OPT_PRECISION, SE_OPT_SIZE_MODE, SE_OPT_ETA, SE_OPT_SHAPE_M, SE_OPT_RESTART, SE_OPT_PARTS = 1, 2, 3, 4, 5, 6
SE_OPT_TIMING = 7
SE_OPT_OVERLAP = 8
SE_OPT_GATHER = 9
SE_OPT_SPREAD = 12
SE_OPT_OVERLAP_CHECK = 13
SE_OPT_RESIDUAL = 14
SE_OPT_SHEAR = 15
SE_OPT_FF_TABLE = 16
SE_OPT_PC_THETA = 10
SE_OPT_PC_KA = 11
SE_OPT_PC_CMAX = 17
SE_OPT_PAIR_FILL = 18
STAGES = ("permute", "real", "spread", "fft_x_fwd", "fft_y_fwd", "fft_z_scale", "fft_y_inv", "fft_x_inv", "gather")
SE_PRECOND_NONE, SE_PRECOND_BLOCK, SE_PRECOND_LEARNED, SE_PRECOND_SPECTRAL = 0, 1, 2, 3

# every entry point declared in include/se_mobility.h
ABI_SYMBOLS = ("se_create", "se_destroy", "se_set_params", "se_set_option", "se_set_config",
               "se_mobility_apply", "se_mobility_apply_host", "se_solve", "se_brownian_ivp", "se_rigid_solve",
               "se_far_field_diffusivity", "se_high_frequency_viscosity", "se_last_error",
               "se_kernel_launches", "se_stage_times", "se_real_space_apply_noalloc",
               "se_set_learned_weights", "se_learned_features", "se_mlp_forward", "se_mlp_grad",
               "se_mlp_adam_step", "se_batch_create", "se_batch_apply", "se_batch_destroy",
               "se_batch_last_error", "se_batch_status", "se_fp32_fma_probe", "se_batch_set_wait_limit",
               "se_batch_inject_stall")
SE_MLP_NW, SE_MLP_NTRAIN, SE_MLP_SAMPLE = 5544, 5508, 276

_lib = None


class SeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library (raises OSError if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with `python -m paper_1506_08481_b300.build`")
    lib = ctypes.CDLL(path)
    p, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    lib.se_create.argtypes = [ctypes.POINTER(p), i, p]
    lib.se_destroy.argtypes = [p]
    lib.se_set_params.argtypes = [p, d, i, i, d]
    lib.se_set_option.argtypes = [p, i, d]
    lib.se_set_config.argtypes = [p, i64, d, p, p]
    lib.se_mobility_apply.argtypes = [p, i, p, p, i]
    lib.se_mobility_apply_host.argtypes = [p, i, p, p]
    lib.se_solve.argtypes = [p, i, p, p, i, d, i, i, ctypes.POINTER(i), ctypes.POINTER(d)]
    lib.se_brownian_ivp.argtypes = [p, i, d, i, d, i, p, p, ctypes.POINTER(i)]
    lib.se_rigid_solve.argtypes = [p, p, p, p, p, d, i, ctypes.POINTER(i), ctypes.POINTER(d)]
    lib.se_high_frequency_viscosity.argtypes = [p, d, i, ctypes.POINTER(d), ctypes.POINTER(i)]
    lib.se_far_field_diffusivity.argtypes = [p, i, p, p, d, i, ctypes.POINTER(i)]
    lib.se_last_error.argtypes = [p]
    lib.se_last_error.restype = ctypes.c_char_p
    lib.se_kernel_launches.argtypes = [p]
    lib.se_kernel_launches.restype = i64
    lib.se_stage_times.argtypes = [p, ctypes.POINTER(d), i]
    lib.se_stage_times.restype = i
    lib.se_real_space_apply_noalloc.argtypes = [i, p, i64, d, d, d, d, p, p, i, p, p]
    lib.se_real_space_apply_noalloc.restype = i
    lib.se_set_learned_weights.argtypes = [p, p, i]
    lib.se_learned_features.argtypes = [p, p]
    lib.se_mlp_forward.argtypes = [p, p, i, p, p]
    lib.se_mlp_grad.argtypes = [p, p, p, i, p, p, p, ctypes.c_size_t, p]
    lib.se_mlp_adam_step.argtypes = [p, p, p, p, i, ctypes.c_float, p]
    for name in ("se_set_learned_weights", "se_learned_features", "se_mlp_forward", "se_mlp_grad",
                 "se_mlp_adam_step"):
        getattr(lib, name).restype = i
    lib.se_fp32_fma_probe.argtypes = [i, p, i, p, ctypes.POINTER(d), ctypes.POINTER(i)]
    lib.se_fp32_fma_probe.restype = i
    lib.se_batch_create.argtypes = [ctypes.POINTER(p), ctypes.POINTER(p), i, i, p]
    lib.se_batch_apply.argtypes = [p, i, ctypes.POINTER(p), ctypes.POINTER(p), i, i]
    lib.se_batch_destroy.argtypes = [p]
    lib.se_batch_last_error.argtypes = [p]
    lib.se_batch_last_error.restype = ctypes.c_char_p
    lib.se_batch_status.argtypes = [p]
    lib.se_batch_set_wait_limit.argtypes = [p, d]
    lib.se_batch_inject_stall.argtypes = [p, i]
    for name in ("se_batch_create", "se_batch_apply", "se_batch_destroy", "se_batch_status",
                 "se_batch_set_wait_limit", "se_batch_inject_stall"):
        getattr(lib, name).restype = i
    for name in ("se_create", "se_destroy", "se_set_params", "se_set_option", "se_set_config",
                 "se_mobility_apply", "se_mobility_apply_host", "se_solve", "se_brownian_ivp", "se_rigid_solve", "se_far_field_diffusivity",
                 "se_high_frequency_viscosity"):
        getattr(lib, name).restype = i
    _lib = lib
    return lib


def _dtype_code(t):
    import torch
    if t.dtype == torch.float32:
        return SE_F32
    if t.dtype == torch.float64:
        return SE_F64
    raise TypeError("x and y must be float32 or float64 tensors")


class Context:
    """Owns one se_ctx.  Methods mirror the C ABI entry points."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.lib = load()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = ctypes.c_void_p()
        rc = self.lib.se_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream))
        if rc != SE_OK:
            raise SeError(rc, self.lib.se_last_error(None).decode())
        self.h = h
        self.N = 0
        self.L = 0.0
        self._keep = []

    def _check(self, rc):
        if rc != SE_OK:
            raise SeError(rc, self.lib.se_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.se_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return self.lib.se_last_error(self.h).decode()

    def kernel_launches(self) -> int:
        return int(self.lib.se_kernel_launches(self.h))

    def se_stage_times(self) -> tuple[int, dict]:
        """(products, {stage: summed ms}) since the last call (needs SE_OPT_TIMING = 1)."""
        buf = (ctypes.c_double * len(STAGES))()
        n = self.lib.se_stage_times(self.h, buf, len(STAGES))
        if n < 0:
            self._check(n)
        return n, dict(zip(STAGES, list(buf)))

    stage_times = se_stage_times

    # --- se_set_params / se_set_option
    def se_set_params(self, xi: float, M: int, P: int, rc: float):
        self._check(self.lib.se_set_params(self.h, float(xi), int(M), int(P), float(rc)))

    set_params = se_set_params

    def se_set_option(self, key: int, value: float):
        self._check(self.lib.se_set_option(self.h, int(key), float(value)))

    set_option = se_set_option

    # --- se_set_config
    def se_set_config(self, pos, rad, L: float):
        """pos [N,3], rad [N]: numpy arrays or CUDA tensors (copied as FP64)."""
        import torch
        pos_t = torch.as_tensor(np.asarray(pos) if not torch.is_tensor(pos) else pos,
                                dtype=torch.float64, device=f"cuda:{self.device}").contiguous()
        rad_t = torch.as_tensor(np.asarray(rad) if not torch.is_tensor(rad) else rad,
                                dtype=torch.float64, device=f"cuda:{self.device}").contiguous()
        N = rad_t.shape[0]
        if pos_t.numel() != 3 * N:
            raise ValueError("pos must be [N, 3] with N = len(rad)")
        self._check(self.lib.se_set_config(self.h, N, float(L), ctypes.c_void_p(pos_t.data_ptr()),
                                           ctypes.c_void_p(rad_t.data_ptr())))
        self.N, self.L = N, float(L)

    set_config = se_set_config

    # --- se_mobility_apply
    def se_mobility_apply(self, x, y=None, ncomp: int | None = None):
        """y = M_inf . x for CUDA tensors x [N, ncomp] (float32/float64)."""
        import torch
        if ncomp is None:
            ncomp = x.shape[-1]
        if y is None:
            y = torch.empty_like(x)
        if not (x.is_cuda and y.is_cuda and x.is_contiguous() and y.is_contiguous()):
            raise ValueError("x and y must be contiguous CUDA tensors")
        if x.dtype != y.dtype or x.numel() != self.N * ncomp or y.numel() != self.N * ncomp:
            raise ValueError("x and y must be [N, ncomp] tensors of the same dtype")
        self._check(self.lib.se_mobility_apply(self.h, int(ncomp), ctypes.c_void_p(x.data_ptr()),
                                               ctypes.c_void_p(y.data_ptr()), _dtype_code(x)))
        return y

    apply = se_mobility_apply

    def se_mobility_apply_host(self, x: np.ndarray, y: np.ndarray | None = None) -> np.ndarray:
        """Host FP64 arrays [N, ncomp]; copies in, applies, copies out (synchronous)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        ncomp = x.shape[-1]
        if y is None:
            y = np.empty_like(x)
        self._check(self.lib.se_mobility_apply_host(self.h, int(ncomp), x.ctypes.data_as(ctypes.c_void_p),
                                                    y.ctypes.data_as(ctypes.c_void_p)))
        return y

    apply_host = se_mobility_apply_host

    # --- learned preconditioner correction
    def se_set_learned_weights(self, w: np.ndarray):
        w = np.ascontiguousarray(w, dtype=np.float32).reshape(-1)
        self._check(self.lib.se_set_learned_weights(self.h, w.ctypes.data_as(ctypes.c_void_p), w.size))

    set_learned_weights = se_set_learned_weights

    def se_learned_features(self):
        import torch
        f = torch.empty(self.N, 16, device=f"cuda:{self.device}", dtype=torch.float32)
        self._check(self.lib.se_learned_features(self.h, ctypes.c_void_p(f.data_ptr())))
        return f

    learned_features = se_learned_features

    # --- se_solve
    def se_solve(self, b, x=None, rtol: float = 1e-6, maxit: int = 500, precond: int = SE_PRECOND_BLOCK,
                 ncomp: int | None = None, allow_not_converged: bool = False):
        """Solve M_inf x = b (CUDA tensors [N, ncomp]); returns (x, iters, relres)."""
        import torch
        if ncomp is None:
            ncomp = b.shape[-1]
        if x is None:
            x = torch.zeros_like(b)
        iters = ctypes.c_int(0)
        relres = ctypes.c_double(0.0)
        rc = self.lib.se_solve(self.h, int(ncomp), ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                               _dtype_code(b), float(rtol), int(maxit), int(precond), ctypes.byref(iters),
                               ctypes.byref(relres))
        if rc == SE_ERR_NOT_CONVERGED and allow_not_converged:
            return x, iters.value, relres.value
        self._check(rc)
        return x, iters.value, relres.value

    solve = se_solve

    # --- se_brownian_ivp
    def se_brownian_ivp(self, c, nsteps: int = 10, rtol: float = 1e-8, maxit: int = 1000, scale: float = 0.0,
                        ncomp: int | None = None, allow_not_converged: bool = False):
        """x = M^{-1/2} c (FP64 CUDA tensor [N, ncomp], ncomp 3, 6 or 11) by the Swan-Brady
        initial value problem with dtau = 1/nsteps; returns (x, products)."""
        import torch
        if ncomp is None:
            ncomp = c.shape[-1]
        c = c.to(torch.float64).contiguous()
        x = torch.empty_like(c)
        prods = ctypes.c_int(0)
        rc = self.lib.se_brownian_ivp(self.h, int(ncomp), float(scale), int(nsteps), float(rtol), int(maxit),
                                      ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                      ctypes.byref(prods))
        if rc == SE_ERR_NOT_CONVERGED and allow_not_converged:
            return x, prods.value
        self._check(rc)
        return x, prods.value

    brownian_ivp = se_brownian_ivp

    # --- se_rigid_solve / se_far_field_diffusivity
    def se_rigid_solve(self, ft=None, einf=None, rtol: float = 1e-8, maxit: int = 1000,
                       allow_not_converged: bool = False):
        """(U, Omega) [N, 6] and S [N, 5] of rigid spheres under forces and torques ft
        (FP64 CUDA [N, 6] or None) and the imposed strain einf (5 numbers on the
        orthonormal basis or None); returns (uw, s, iters, relres)."""
        import torch
        N = int(self.N)
        dev = torch.device("cuda", self.device)
        if ft is not None:
            ft = ft.to(torch.float64).contiguous()
        uw = torch.empty(N, 6, device=dev, dtype=torch.float64)
        sv = torch.empty(N, 5, device=dev, dtype=torch.float64)
        e = (ctypes.c_double * 5)(*[float(v) for v in einf]) if einf is not None else None
        iters = ctypes.c_int(0)
        relres = ctypes.c_double(0.0)
        rc = self.lib.se_rigid_solve(self.h, ctypes.c_void_p(ft.data_ptr() if ft is not None else 0),
                                     ctypes.cast(e, ctypes.c_void_p) if e is not None else None,
                                     ctypes.c_void_p(uw.data_ptr()), ctypes.c_void_p(sv.data_ptr()), float(rtol),
                                     int(maxit), ctypes.byref(iters), ctypes.byref(relres))
        if not (rc == SE_ERR_NOT_CONVERGED and allow_not_converged):
            self._check(rc)
        return uw, sv, iters.value, relres.value

    rigid_solve = se_rigid_solve

    def se_far_field_diffusivity(self, fr, rtol: float = 1e-6, maxit: int = 1000):
        """Per-particle estimates [N, 2] of tr(mu_ii^tt)/3, tr(mu_ii^rr)/3 from the samples
        fr [nsamples, N, 6] (FP64 CUDA); returns (d, products)."""
        import torch
        fr = fr.to(torch.float64).contiguous()
        d = torch.empty(fr.shape[1], 2, device=fr.device, dtype=torch.float64)
        prods = ctypes.c_int(0)
        rc = self.lib.se_far_field_diffusivity(self.h, int(fr.shape[0]), ctypes.c_void_p(fr.data_ptr()),
                                               ctypes.c_void_p(d.data_ptr()), float(rtol), int(maxit),
                                               ctypes.byref(prods))
        self._check(rc)
        return d, prods.value

    far_field_diffusivity = se_far_field_diffusivity

    def se_high_frequency_viscosity(self, rtol: float = 1e-6, maxit: int = 1000):
        """eta_s / eta of the far-field suspension; returns (ratio, products)."""
        r = ctypes.c_double(0.0)
        prods = ctypes.c_int(0)
        self._check(self.lib.se_high_frequency_viscosity(self.h, float(rtol), int(maxit), ctypes.byref(r),
                                                         ctypes.byref(prods)))
        return r.value, prods.value

    high_frequency_viscosity = se_high_frequency_viscosity


# --- network kernels (stand-alone; device tensors)
def mlp_forward(w, X):
    import torch
    Y = torch.empty(X.shape[0], 4, device=X.device, dtype=torch.float32)
    rc = load().se_mlp_forward(ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(X.data_ptr()), X.shape[0],
                               ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != SE_OK:
        raise SeError(rc, "se_mlp_forward failed")
    return Y


def mlp_grad(w, X, Yt, scratch=None):
    import torch
    n = X.shape[0]
    if scratch is None or scratch.numel() < n * SE_MLP_SAMPLE:
        scratch = torch.empty(n * SE_MLP_SAMPLE, device=X.device, dtype=torch.float32)
    g = torch.empty(SE_MLP_NTRAIN, device=X.device, dtype=torch.float32)
    loss = torch.empty(1, device=X.device, dtype=torch.float32)
    rc = load().se_mlp_grad(ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                            ctypes.c_void_p(Yt.data_ptr()), n, ctypes.c_void_p(g.data_ptr()),
                            ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(scratch.data_ptr()),
                            scratch.numel(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != SE_OK:
        raise SeError(rc, "se_mlp_grad failed")
    return g, loss, scratch


def mlp_adam_step(w, m, v, g, step, lr):
    import torch
    rc = load().se_mlp_adam_step(ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(m.data_ptr()),
                                 ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(g.data_ptr()), int(step),
                                 float(lr), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != SE_OK:
        raise SeError(rc, "se_mlp_adam_step failed")


class Batch:
    """Independent boxes applied together (se_batch_*); contexts must be configured."""

    def __init__(self, contexts, nstreams: int = 8, stream=None):
        import torch
        self.lib = load()
        self.ctxs = list(contexts)
        if stream is None:
            stream = torch.cuda.current_stream(self.ctxs[0].device)
        self.stream = stream
        arr = (ctypes.c_void_p * len(self.ctxs))(*[c.h for c in self.ctxs])
        h = ctypes.c_void_p()
        rc = self.lib.se_batch_create(ctypes.byref(h), arr, len(self.ctxs), int(nstreams),
                                      ctypes.c_void_p(stream.cuda_stream))
        if rc != SE_OK:
            raise SeError(rc, "se_batch_create failed")
        self.h = h

    # se_batch_apply modes
    PER_BOX, GRAPH, PERSISTENT = 0, 1, 2

    def apply(self, xs, ys, use_graph=True):
        """use_graph: False/0 per-box launches, True/1 one CUDA graph of the boxes' kernels,
        2 one persistent launch for every box (Batch.PERSISTENT)."""
        ncomp = xs[0].shape[-1]
        xa = (ctypes.c_void_p * len(xs))(*[x.data_ptr() for x in xs])
        ya = (ctypes.c_void_p * len(ys))(*[y.data_ptr() for y in ys])
        mode = int(use_graph) if not isinstance(use_graph, bool) else int(use_graph)
        rc = self.lib.se_batch_apply(self.h, int(ncomp), xa, ya, _dtype_code(xs[0]), mode)
        if rc != SE_OK:
            raise SeError(rc, self.lib.se_batch_last_error(self.h).decode())

    def status(self):
        """Synchronises; raises if a persistent launch since the last call was aborted."""
        rc = self.lib.se_batch_status(self.h)
        if rc != SE_OK:
            raise SeError(rc, self.lib.se_batch_last_error(self.h).decode())

    def set_wait_limit(self, seconds: float):
        """Time limit of every wait inside a persistent launch (se_batch_set_wait_limit)."""
        rc = self.lib.se_batch_set_wait_limit(self.h, float(seconds))
        if rc != SE_OK:
            raise SeError(rc, "se_batch_set_wait_limit failed")

    def inject_stall(self, box: int):
        """Failure-injection hook for tests (se_batch_inject_stall); -1 turns it off."""
        rc = self.lib.se_batch_inject_stall(self.h, int(box))
        if rc != SE_OK:
            raise SeError(rc, "se_batch_inject_stall failed")

    def close(self):
        if getattr(self, "h", None):
            self.lib.se_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp32_fma_peak(device: int = 0, iters: int = 4096, reps: int = 5) -> tuple[float, int]:
    """Measured FP32 FMA throughput of the device in TFLOP/s (best of `reps` launches of
    se_fp32_fma_probe, timed with CUDA events on torch's current stream) and its SM count."""
    import torch
    lib = load()
    stream = torch.cuda.current_stream(device)
    sink = torch.zeros(1, device=f"cuda:{device}", dtype=torch.float32)
    flop, sms = ctypes.c_double(0.0), ctypes.c_int(0)
    best = None
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = lib.se_fp32_fma_probe(device, ctypes.c_void_p(stream.cuda_stream), iters,
                                   ctypes.c_void_p(sink.data_ptr()), ctypes.byref(flop), ctypes.byref(sms))
        e1.record(stream)
        if rc != SE_OK:
            raise SeError(rc, "se_fp32_fma_probe failed")
        e1.synchronize()
        if r == 0:
            continue                      # the first launch loads the module
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return flop.value / (best * 1e-3) / 1e12, sms.value
