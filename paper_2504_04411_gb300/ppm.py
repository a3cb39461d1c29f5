"""Thin ctypes binding of libppm (include/ppm.h), same names as the C ABI.

Argument marshalling only: every step of the method runs in the CUDA
library.  Tensors are torch CUDA tensors; their device pointers and the
current torch stream are passed straight through.  There is no CPU fallback:
if libppm.so is missing or fails to load, the import of this module's
functions raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libppm.so")

PPM_OK, PPM_EINVAL, PPM_ENOMEM, PPM_ECUDA, PPM_ETIMEOUT, PPM_ESTATE = 0, -1, -2, -3, -4, -5
PPM_EINCOMPLETE = -6
PPM_NGROUPS = 12

c_p = ctypes.c_void_p


class ppm_hitpoints(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("pos", c_p), ("u", c_p), ("v", c_p),
                ("nq", c_p), ("rho", c_p)]


class ppm_photons(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("J", ctypes.c_int64), ("pos", c_p),
                ("flux", c_p), ("channels", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("nq", c_p), ("rho", c_p), ("wq", c_p)]


class ppm_params(ctypes.Structure):
    _fields_ = [("alpha_f", ctypes.c_double), ("k", ctypes.c_float),
                ("rmin_ratio", ctypes.c_float), ("cell_factor", ctypes.c_float),
                ("channels", ctypes.c_int32), ("rgb_test", ctypes.c_int32),
                ("vcm", ctypes.c_int32), ("n_vm", ctypes.c_float),
                ("mapping", ctypes.c_int32), ("tile", ctypes.c_int32), ("test", ctypes.c_int32),
                ("wait_limit", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class ppm_iter_stats(ctypes.Structure):
    _fields_ = [("iter", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("pairs", ctypes.c_int64), ("candidates", ctypes.c_int64),
                ("rejects", ctypes.c_int64), ("pairs_total", ctypes.c_int64),
                ("r_max", ctypes.c_float), ("cell", ctypes.c_float),
                ("launches", ctypes.c_int32), ("gather_ms", ctypes.c_float),
                ("proposals", ctypes.c_int64)]


class ppm_state_view(ctypes.Structure):
    _fields_ = [("r", c_p), ("t", c_p), ("counts", c_p), ("S", c_p), ("Q", c_p),
                ("tau", c_p), ("F", c_p)]


# every symbol include/ppm.h declares
EXPORTS = ("ppm_default_params", "ppm_create", "ppm_set_stream", "ppm_build_grid",
           "ppm_gather_test_update", "ppm_radiance", "ppm_get_state", "ppm_set_state",
           "ppm_set_iteration", "ppm_stats", "ppm_f_critical", "ppm_chi2_critical", "ppm_sort_pairs",
           "ppm_set_hitpoints",
           "ppm_destroy", "ppm_strerror", "ppm_sort_pairs_noalloc",
           "ppm_batch_create", "ppm_batch_iterate", "ppm_batch_radiance",
           "ppm_batch_get_state", "ppm_batch_stats", "ppm_batch_graph_ready",
           "ppm_batch_destroy", "ppm_set_features", "ppm_get_features", "ppm_set_mlp",
           "ppm_mlp_forward", "ppm_mlp_grad", "ppm_mlp_adam", "ppm_mlp_pack",
           "ppm_iterate_host", "ppm_stats_host")

_lib = None


def load(path: str = LIB_PATH):
    """Load libppm.so (built by paper_2504_04411_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libppm.so not built ({path}); run paper_2504_04411_gb300.build.build()")
    L = ctypes.CDLL(path)
    L.ppm_default_params.restype = None
    L.ppm_default_params.argtypes = [ctypes.POINTER(ppm_params)]
    L.ppm_create.restype = ctypes.c_int
    L.ppm_create.argtypes = [ctypes.POINTER(ppm_hitpoints), ctypes.c_float, ctypes.c_float,
                             ctypes.POINTER(ppm_params), c_p, ctypes.POINTER(c_p)]
    L.ppm_set_stream.restype = ctypes.c_int
    L.ppm_set_stream.argtypes = [c_p, c_p]
    L.ppm_set_hitpoints.restype = ctypes.c_int
    L.ppm_set_hitpoints.argtypes = [c_p, ctypes.POINTER(ppm_hitpoints)]
    L.ppm_build_grid.restype = ctypes.c_int
    L.ppm_build_grid.argtypes = [c_p, ctypes.POINTER(ppm_photons)]
    L.ppm_gather_test_update.restype = ctypes.c_int
    L.ppm_gather_test_update.argtypes = [c_p, ctypes.c_int32]
    L.ppm_radiance.restype = ctypes.c_int
    L.ppm_radiance.argtypes = [c_p, c_p]
    L.ppm_get_state.restype = ctypes.c_int
    L.ppm_get_state.argtypes = [c_p, ctypes.POINTER(ppm_state_view)]
    L.ppm_set_state.restype = ctypes.c_int
    L.ppm_set_state.argtypes = [c_p, ctypes.POINTER(ppm_state_view)]
    L.ppm_set_iteration.restype = ctypes.c_int
    L.ppm_set_iteration.argtypes = [c_p, ctypes.c_int32]
    L.ppm_stats.restype = ctypes.c_int
    L.ppm_stats.argtypes = [c_p, ctypes.POINTER(ppm_iter_stats)]
    L.ppm_iterate_host.restype = ctypes.c_int
    L.ppm_iterate_host.argtypes = [c_p, ctypes.POINTER(ppm_photons), ctypes.c_int32]
    L.ppm_stats_host.restype = ctypes.c_int
    L.ppm_stats_host.argtypes = [c_p, ctypes.c_int32, ctypes.POINTER(ppm_iter_stats)]
    L.ppm_f_critical.restype = ctypes.c_int
    L.ppm_f_critical.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_int32, c_p, c_p]
    L.ppm_chi2_critical.restype = ctypes.c_int
    L.ppm_chi2_critical.argtypes = [ctypes.c_int32, ctypes.c_double, c_p, c_p]
    L.ppm_sort_pairs.restype = ctypes.c_int
    L.ppm_sort_pairs.argtypes = [c_p, c_p, c_p, c_p, ctypes.c_int64, ctypes.c_int32, c_p]
    L.ppm_sort_pairs_noalloc.restype = ctypes.c_int
    L.ppm_sort_pairs_noalloc.argtypes = [c_p, c_p, c_p, c_p, ctypes.c_int64, ctypes.c_int32, c_p]
    L.ppm_batch_create.restype = ctypes.c_int
    L.ppm_batch_create.argtypes = [ctypes.c_int32, ctypes.POINTER(ppm_hitpoints), c_p, c_p,
                                   ctypes.c_float, ctypes.POINTER(ppm_params), c_p, c_p,
                                   ctypes.POINTER(c_p)]
    L.ppm_batch_iterate.restype = ctypes.c_int
    L.ppm_batch_iterate.argtypes = [c_p, ctypes.POINTER(ppm_photons), ctypes.c_int32]
    L.ppm_batch_radiance.restype = ctypes.c_int
    L.ppm_batch_radiance.argtypes = [c_p, ctypes.c_int32, c_p]
    L.ppm_batch_get_state.restype = ctypes.c_int
    L.ppm_batch_get_state.argtypes = [c_p, ctypes.c_int32, ctypes.POINTER(ppm_state_view)]
    L.ppm_batch_stats.restype = ctypes.c_int
    L.ppm_batch_stats.argtypes = [c_p, ctypes.POINTER(ppm_iter_stats)]
    L.ppm_batch_graph_ready.restype = ctypes.c_int
    L.ppm_batch_graph_ready.argtypes = [c_p]
    L.ppm_batch_destroy.restype = None
    L.ppm_batch_destroy.argtypes = [c_p]
    L.ppm_set_features.restype = ctypes.c_int
    L.ppm_set_features.argtypes = [c_p, ctypes.c_int32]
    L.ppm_get_features.restype = ctypes.c_int
    L.ppm_get_features.argtypes = [c_p, c_p]
    L.ppm_set_mlp.restype = ctypes.c_int
    L.ppm_set_mlp.argtypes = [c_p, c_p, ctypes.c_float, ctypes.c_float]
    L.ppm_mlp_forward.restype = ctypes.c_int
    L.ppm_mlp_forward.argtypes = [c_p, c_p, ctypes.c_int64, c_p, c_p]
    L.ppm_mlp_grad.restype = ctypes.c_int
    L.ppm_mlp_grad.argtypes = [c_p, c_p, c_p, c_p, ctypes.c_int64, ctypes.c_float, c_p, c_p, c_p]
    L.ppm_mlp_adam.restype = ctypes.c_int
    L.ppm_mlp_adam.argtypes = [c_p, c_p, c_p, c_p, ctypes.c_int32, ctypes.c_float, c_p, c_p]
    L.ppm_mlp_pack.restype = ctypes.c_int
    L.ppm_mlp_pack.argtypes = [c_p, c_p, c_p]
    L.ppm_destroy.restype = None
    L.ppm_destroy.argtypes = [c_p]
    L.ppm_strerror.restype = ctypes.c_char_p
    L.ppm_strerror.argtypes = [ctypes.c_int]
    _lib = L
    return L


class PPMError(RuntimeError):
    def __init__(self, fn: str, code: int):
        msg = load().ppm_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{fn} returned {code} ({msg})")
        self.code = code


def _check(fn: str, rc: int) -> None:
    if rc != PPM_OK:
        raise PPMError(fn, rc)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libppm takes CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("libppm takes contiguous tensors")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(t):
    if t is None:
        return None
    if t.is_cuda:
        raise ValueError("ppm_iterate_host takes host (CPU) tensors")
    if not t.is_contiguous():
        raise ValueError("libppm takes contiguous tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------- C ABI ----
def ppm_default_params() -> ppm_params:
    p = ppm_params()
    load().ppm_default_params(ctypes.byref(p))
    return p


def ppm_create(pos, u, v, r0: float, alpha: float = 0.75, params: ppm_params | None = None,
               nq=None, rho=None, stream=None) -> ctypes.c_void_p:
    """pos, u, v: (n,3) float32 CUDA tensors; nq (n,) int32/uint32 packed
    normals or None; rho (n,2) float32 or None.  Returns the context handle."""
    hp = ppm_hitpoints(pos.shape[0], _ptr(pos), _ptr(u), _ptr(v), _ptr(nq), _ptr(rho))
    ctx = ctypes.c_void_p()
    _check("ppm_create", load().ppm_create(ctypes.byref(hp), r0, alpha,
                                           ctypes.byref(params) if params is not None else None,
                                           _stream(stream), ctypes.byref(ctx)))
    return ctx


def ppm_set_stream(ctx, stream=None) -> None:
    _check("ppm_set_stream", load().ppm_set_stream(ctx, _stream(stream)))


def ppm_set_hitpoints(ctx, pos, u, v, nq=None, rho=None) -> None:
    """Hit points traced anew (same count and order as at ppm_create)."""
    hp = ppm_hitpoints(pos.shape[0], _ptr(pos), _ptr(u), _ptr(v), _ptr(nq), _ptr(rho))
    _check("ppm_set_hitpoints", load().ppm_set_hitpoints(ctx, ctypes.byref(hp)))


def ppm_build_grid(ctx, pos, flux, J: int, nq=None, rho=None, wq=None) -> None:
    channels = 3 if flux.dim() == 2 else 1
    ph = ppm_photons(pos.shape[0], J, _ptr(pos), _ptr(flux), channels, 0,
                     _ptr(nq), _ptr(rho), _ptr(wq))
    _check("ppm_build_grid", load().ppm_build_grid(ctx, ctypes.byref(ph)))


def ppm_gather_test_update(ctx, it: int) -> None:
    _check("ppm_gather_test_update", load().ppm_gather_test_update(ctx, it))


def ppm_radiance(ctx, out) -> None:
    _check("ppm_radiance", load().ppm_radiance(ctx, _ptr(out)))


def ppm_get_state(ctx, r=None, t=None, counts=None, S=None, Q=None, tau=None, F=None) -> None:
    v = ppm_state_view(_ptr(r), _ptr(t), _ptr(counts), _ptr(S), _ptr(Q), _ptr(tau), _ptr(F))
    _check("ppm_get_state", load().ppm_get_state(ctx, ctypes.byref(v)))


def ppm_set_state(ctx, r=None, t=None, counts=None, S=None, Q=None, tau=None, F=None) -> None:
    v = ppm_state_view(_ptr(r), _ptr(t), _ptr(counts), _ptr(S), _ptr(Q), _ptr(tau), _ptr(F))
    _check("ppm_set_state", load().ppm_set_state(ctx, ctypes.byref(v)))


def ppm_set_iteration(ctx, it: int) -> None:
    _check("ppm_set_iteration", load().ppm_set_iteration(ctx, it))


def ppm_stats(ctx) -> ppm_iter_stats:
    s = ppm_iter_stats()
    _check("ppm_stats", load().ppm_stats(ctx, ctypes.byref(s)))
    return s


def ppm_iterate_host(ctx, it: int, pos, flux, J: int, nq=None, rho=None, wq=None) -> None:
    """One iteration from host (CPU) tensors: copy, build, gather/test/update,
    enqueued without waiting (pinned tensors overlap the copy with the
    previous gather).  Keep the tensors alive and unchanged until
    ppm_stats_host(ctx, it) has returned."""
    channels = 3 if flux.dim() == 2 else 1
    ph = ppm_photons(pos.shape[0], J, _host_ptr(pos), _host_ptr(flux), channels, 0,
                     _host_ptr(nq), _host_ptr(rho), _host_ptr(wq))
    _check("ppm_iterate_host", load().ppm_iterate_host(ctx, ctypes.byref(ph), it))


def ppm_stats_host(ctx, it: int) -> ppm_iter_stats:
    s = ppm_iter_stats()
    _check("ppm_stats_host", load().ppm_stats_host(ctx, it, ctypes.byref(s)))
    return s


def ppm_f_critical(J: int, alpha_f: float, t_max: int, out, stream=None) -> None:
    _check("ppm_f_critical", load().ppm_f_critical(J, alpha_f, t_max, _ptr(out), _stream(stream)))


def ppm_chi2_critical(dof: int, alpha: float, out, stream=None) -> None:
    _check("ppm_chi2_critical", load().ppm_chi2_critical(dof, alpha, _ptr(out), _stream(stream)))


def ppm_sort_pairs(keys_in, vals_in, keys_out, vals_out, bits: int, stream=None) -> None:
    """Stable radix sort of uint32 (key, value) pairs (int32 tensors holding
    the bit patterns) on the low ``bits`` bits."""
    _check("ppm_sort_pairs", load().ppm_sort_pairs(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out),
                                                   _ptr(vals_out), keys_in.numel(), bits,
                                                   _stream(stream)))


PPM_NOALLOC_MAX_PAIRS = 1 << 20


def ppm_sort_pairs_noalloc(keys_in, vals_in, keys_out, vals_out, bits: int, stream=None) -> None:
    """ppm_sort_pairs without any device allocation: scratch lives in a
    fixed device array of the library (at most PPM_NOALLOC_MAX_PAIRS pairs;
    calls that overlap on the GPU race on it)."""
    _check("ppm_sort_pairs_noalloc",
           load().ppm_sort_pairs_noalloc(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out),
                                         _ptr(vals_out), keys_in.numel(), bits, _stream(stream)))


PPM_MLP_IN, PPM_MLP_HIDDEN, PPM_MLP_OUT = 12, 64, 2
PPM_MLP_PARAMS = 64 * 12 + 64 * 64 + 2 * 64 + 64 + 64 + 2
PPM_MLP_BLOB_BYTES = 10504


def ppm_set_features(ctx, enable: bool = True) -> None:
    _check("ppm_set_features", load().ppm_set_features(ctx, int(enable)))


def ppm_get_features(ctx, out) -> None:
    _check("ppm_get_features", load().ppm_get_features(ctx, _ptr(out)))


def ppm_set_mlp(ctx, blob, doom_threshold: float = 0.5, min_ratio: float = 0.1) -> None:
    _check("ppm_set_mlp", load().ppm_set_mlp(ctx, _ptr(blob), doom_threshold, min_ratio))


def ppm_mlp_forward(blob, X, Y, stream=None) -> None:
    _check("ppm_mlp_forward", load().ppm_mlp_forward(_ptr(blob), _ptr(X), X.shape[0], _ptr(Y),
                                                     _stream(stream)))


def ppm_mlp_grad(blob, X, Y, M, scale: float, grad, loss, stream=None) -> None:
    _check("ppm_mlp_grad", load().ppm_mlp_grad(_ptr(blob), _ptr(X), _ptr(Y), _ptr(M), X.shape[0],
                                               scale, _ptr(grad), _ptr(loss), _stream(stream)))


def ppm_mlp_adam(master, grad, m, v, step: int, lr: float, blob, stream=None) -> None:
    _check("ppm_mlp_adam", load().ppm_mlp_adam(_ptr(master), _ptr(grad), _ptr(m), _ptr(v), step, lr,
                                               _ptr(blob), _stream(stream)))


def ppm_mlp_pack(master, blob, stream=None) -> None:
    _check("ppm_mlp_pack", load().ppm_mlp_pack(_ptr(master), _ptr(blob), _stream(stream)))


def ppm_destroy(ctx) -> None:
    if ctx:
        load().ppm_destroy(ctx)


def ppm_strerror(code: int) -> str:
    return load().ppm_strerror(code).decode()


# ----------------------------------------------------- convenience class ----
class Estimator:
    """Owns one context; `step(photons, it)` = build_grid + gather_test_update."""

    def __init__(self, hp, r0: float, alpha: float = 0.75, params: ppm_params | None = None,
                 stream=None):
        self.n = int(hp.pos.shape[0])
        self.params = params if params is not None else ppm_default_params()
        self.channels = int(self.params.channels)
        self.ntc = 3 if self.params.rgb_test else 1
        self.ctx = ppm_create(hp.pos, hp.u, hp.v, r0, alpha, self.params,
                              nq=hp.nq, rho=hp.rho if self.params.vcm else None, stream=stream)
        self.it = 0

    def retrace(self, hp) -> None:
        """This iteration's hit points (SPPM-style): same pixels, new
        positions; statistics carry over."""
        ppm_set_hitpoints(self.ctx, hp.pos, hp.u, hp.v, nq=hp.nq,
                          rho=hp.rho if self.params.vcm else None)

    def step(self, ph, J: int | None = None) -> None:
        ppm_build_grid(self.ctx, ph.pos, ph.flux, J if J is not None else ph.pos.shape[0],
                       nq=ph.nq, rho=ph.rho if self.params.vcm else None,
                       wq=ph.wq if self.params.vcm else None)
        self.it += 1
        ppm_gather_test_update(self.ctx, self.it)

    def step_host(self, ph, J: int | None = None) -> int:
        """One iteration from host tensors (ppm_iterate_host); returns its
        iteration number for ppm_stats_host."""
        self.it += 1
        try:
            ppm_iterate_host(self.ctx, self.it, ph.pos, ph.flux, J if J is not None else ph.pos.shape[0],
                             nq=ph.nq, rho=ph.rho if self.params.vcm else None,
                             wq=ph.wq if self.params.vcm else None)
        except Exception:
            self.it -= 1
            raise
        return self.it

    def radiance(self) -> torch.Tensor:
        shape = (self.n,) if self.channels == 1 else (self.n, 3)
        out = torch.empty(shape, device="cuda", dtype=torch.float32)
        ppm_radiance(self.ctx, out)
        return out

    def state(self) -> dict:
        n, d = self.n, "cuda"
        st = {"r": torch.empty(n, device=d), "t": torch.empty(n, device=d, dtype=torch.int32),
              "counts": torch.empty(n, PPM_NGROUPS, device=d, dtype=torch.int32),
              "S": torch.empty(n, self.ntc, PPM_NGROUPS, device=d),
              "Q": torch.empty(n, self.ntc, PPM_NGROUPS, device=d),
              "tau": torch.empty(n, self.channels, device=d, dtype=torch.float64),
              "F": torch.empty(n, device=d)}
        ppm_get_state(self.ctx, **st)
        return st

    def stats(self) -> ppm_iter_stats:
        return ppm_stats(self.ctx)

    def close(self) -> None:
        ppm_destroy(self.ctx)
        self.ctx = None

    def __del__(self):  # pragma: no cover
        try:
            if self.ctx:
                self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- batches ---
def ppm_batch_create(hps, r0s, Js, alpha: float = 0.75, params: ppm_params | None = None,
                     cell_factors=None, stream=None) -> ctypes.c_void_p:
    """hps: list of HitPoints-like objects (pos, u, v, nq, rho CUDA tensors)."""
    import numpy as np
    P = len(hps)
    vcm = bool(params.vcm) if params is not None else False
    arr = (ppm_hitpoints * P)()
    for i, hp in enumerate(hps):
        arr[i] = ppm_hitpoints(hp.pos.shape[0], _ptr(hp.pos), _ptr(hp.u), _ptr(hp.v), _ptr(hp.nq),
                               _ptr(hp.rho) if vcm else None)
    r0 = np.ascontiguousarray(r0s, np.float32)
    J = np.ascontiguousarray(Js, np.int64)
    cf = None if cell_factors is None else np.ascontiguousarray(cell_factors, np.float32)
    b = ctypes.c_void_p()
    _check("ppm_batch_create", load().ppm_batch_create(
        P, arr, r0.ctypes.data_as(c_p), J.ctypes.data_as(c_p), alpha,
        ctypes.byref(params) if params is not None else None,
        None if cf is None else cf.ctypes.data_as(c_p), _stream(stream), ctypes.byref(b)))
    return b


def ppm_batch_iterate(b, photons, it: int, vcm: bool = False) -> None:
    """photons: list (one per problem) of Photons-like objects."""
    P = len(photons)
    arr = (ppm_photons * P)()
    for i, ph in enumerate(photons):
        ch = 3 if ph.flux.dim() == 2 else 1
        n = ph.pos.shape[0]
        arr[i] = ppm_photons(n, n, _ptr(ph.pos), _ptr(ph.flux), ch, 0, _ptr(ph.nq),
                             _ptr(ph.rho) if vcm else None, _ptr(ph.wq) if vcm else None)
    _check("ppm_batch_iterate", load().ppm_batch_iterate(b, arr, it))


def ppm_batch_radiance(b, problem: int, out) -> None:
    _check("ppm_batch_radiance", load().ppm_batch_radiance(b, problem, _ptr(out)))


def ppm_batch_get_state(b, problem: int, r=None, t=None, counts=None, S=None, Q=None, tau=None,
                        F=None) -> None:
    v = ppm_state_view(_ptr(r), _ptr(t), _ptr(counts), _ptr(S), _ptr(Q), _ptr(tau), _ptr(F))
    _check("ppm_batch_get_state", load().ppm_batch_get_state(b, problem, ctypes.byref(v)))


def ppm_batch_stats(b, n_problems: int):
    arr = (ppm_iter_stats * n_problems)()
    _check("ppm_batch_stats", load().ppm_batch_stats(b, arr))
    return list(arr)


def ppm_batch_graph_ready(b) -> bool:
    return bool(load().ppm_batch_graph_ready(b))


def ppm_batch_destroy(b) -> None:
    if b:
        load().ppm_batch_destroy(b)


class Batch:
    """Owns one batch; `step(photon_lists)` runs one iteration of all problems."""

    def __init__(self, hps, r0s, Js, alpha: float = 0.75, params: ppm_params | None = None,
                 cell_factors=None, stream=None):
        self.params = params if params is not None else ppm_default_params()
        self.P = len(hps)
        self.ns = [int(h.pos.shape[0]) for h in hps]
        self.channels = int(self.params.channels)
        self.ntc = 3 if self.params.rgb_test else 1
        self.b = ppm_batch_create(hps, r0s, Js, alpha, self.params, cell_factors, stream)
        self.it = 0

    def step(self, photons) -> None:
        self.it += 1
        ppm_batch_iterate(self.b, photons, self.it, vcm=bool(self.params.vcm))

    def radiance(self, p: int) -> torch.Tensor:
        shape = (self.ns[p],) if self.channels == 1 else (self.ns[p], 3)
        out = torch.empty(shape, device="cuda", dtype=torch.float32)
        ppm_batch_radiance(self.b, p, out)
        return out

    def state(self, p: int) -> dict:
        n, d = self.ns[p], "cuda"
        st = {"r": torch.empty(n, device=d), "t": torch.empty(n, device=d, dtype=torch.int32),
              "counts": torch.empty(n, PPM_NGROUPS, device=d, dtype=torch.int32),
              "S": torch.empty(n, self.ntc, PPM_NGROUPS, device=d),
              "Q": torch.empty(n, self.ntc, PPM_NGROUPS, device=d),
              "tau": torch.empty(n, self.channels, device=d, dtype=torch.float64),
              "F": torch.empty(n, device=d)}
        ppm_batch_get_state(self.b, p, **st)
        return st

    def stats(self):
        return ppm_batch_stats(self.b, self.P)

    def close(self) -> None:
        ppm_batch_destroy(self.b)
        self.b = None
