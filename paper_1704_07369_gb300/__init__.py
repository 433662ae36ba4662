"""Python binding of the GB300 EFM collision library (``include/ef.h``, ``libef.so``).

Argument marshalling only: every step of the collision operator runs in the library's CUDA
kernels.  Torch tensors provide device memory and streams; pointers are passed through the C ABI.
The library must have been built (``build()``); there is no CPU or PyTorch fallback, and a
missing or unloadable ``libef.so`` raises immediately.

Names follow the C API: ``ef_plan_create``, ``ef_plan_create_ex``, ``ef_plan_create_batched``,
``ef_collide``, ``ef_euler_step``, ``ef_moments_entropy``, ``ef_plan_status``, ...
The :class:`Plan` class wraps a handle with the same operations as methods.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libef.so")

EF_OK = 0
EF_ERR_INVALID_ARG = 1
EF_ERR_UNSUPPORTED = 2
EF_ERR_CUDA = 3
EF_ERR_OOM = 4
EF_ERR_TIMEOUT = 5
EF_ERR_POSITIVITY = 6
EF_ERR_NOT_FINITE = 7

EF_PREC_F32 = 0
EF_PREC_F64 = 1
EF_KERNEL_MAXWELL = 0
EF_KERNEL_HARD_SPHERE = 1
EF_DIAG_STRIDE = 10

# every symbol include/ef.h declares
SYMBOLS = ("ef_plan_create", "ef_plan_create_ex", "ef_plan_create_batched", "ef_plan_destroy",
           "ef_collide", "ef_euler_step", "ef_rk3_step", "ef_moments_entropy", "ef_plan_status",
           "ef_plan_set_graph", "ef_plan_info", "ef_plan_class_info", "ef_plan_reserve", "ef_collide_noalloc", "ef_kernel_G",
           "ef_galerkin_create", "ef_galerkin_collide", "ef_galerkin_status", "ef_galerkin_destroy",
           "ef_features", "ef_mlp_create", "ef_mlp_destroy", "ef_mlp_info", "ef_mlp_status", "ef_mlp_params",
           "ef_mlp_forward", "ef_mlp_grad", "ef_mlp_train_step",
           "ef_surrogate_create", "ef_surrogate_destroy", "ef_surrogate_fit_stats", "ef_surrogate_normalize",
           "ef_surrogate_stats", "ef_surrogate_set_policy", "ef_surrogate_set_entropy_gate", "ef_surrogate_infer",
           "ef_surrogate_set_checker",
           "ef_surrogate_infer_ex", "ef_features_inverse",
           "ef_stream_plan_create", "ef_stream_plan_destroy", "ef_stream_plan_info", "ef_stream_euler_step",
           "ef_stream_plan_status", "ef_transport_step", "ef_classical_create", "ef_classical_collide",
           "ef_classical_destroy", "ef_status_string", "ef_last_error")
EF_FEATURE_K = 6
EF_FEATURE_STRIDE = 928


class EfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (status, msg))
        self.status = status


class ef_plan_desc(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("N", ctypes.c_int), ("L", ctypes.c_double),
                ("kernel", ctypes.c_int), ("R", ctypes.c_int), ("prec", ctypes.c_int),
                ("R_tr", ctypes.c_double), ("n_mu", ctypes.c_int), ("n_phi", ctypes.c_int),
                ("n_c", ctypes.c_int), ("J", ctypes.c_int), ("sigma_enabled", ctypes.c_int)]


_lib = None


def build(force: bool = False, verbose: bool = False) -> str:
    from . import buildlib
    return buildlib.build(force=force, verbose=verbose)


def lib():
    """The loaded ``libef.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise RuntimeError("libef.so is not built at %s (call paper_1704_07369_gb300.build())" % LIBPATH)
        L = ctypes.CDLL(LIBPATH)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        pp = ctypes.POINTER(vp)
        L.ef_plan_create.argtypes = [i32, i32, dbl, i32, i32, i32, pp]
        L.ef_plan_create_ex.argtypes = [ctypes.POINTER(ef_plan_desc), pp]
        L.ef_plan_create_batched.argtypes = [i32, i64, ctypes.POINTER(ctypes.c_int), dbl, i32, i32, i32, pp]
        L.ef_plan_destroy.argtypes = [vp]
        L.ef_collide.argtypes = [vp, vp, vp, i64, vp]
        L.ef_collide_noalloc.argtypes = [vp, vp, vp, i64, vp]
        L.ef_features.argtypes = [vp, vp, vp, i64, i32, vp]
        L.ef_mlp_create.argtypes = [i32, i32, i32, i32, i64, ctypes.c_uint64, pp]
        L.ef_mlp_destroy.argtypes = [vp]
        L.ef_mlp_info.argtypes = [vp, ctypes.POINTER(i64)]
        L.ef_mlp_status.argtypes = [vp, i32, i32]
        L.ef_plan_reserve.argtypes = [vp, i64]
        L.ef_kernel_G.argtypes = [vp, i64, vp, vp]
        L.ef_galerkin_create.argtypes = [ctypes.POINTER(ef_plan_desc), i64, pp]
        L.ef_galerkin_collide.argtypes = [vp, vp, vp, i64, vp]
        L.ef_galerkin_status.argtypes = [vp, i32, i32]
        L.ef_galerkin_destroy.argtypes = [vp]
        L.ef_mlp_params.argtypes = [vp, ctypes.POINTER(ctypes.c_float), i32]
        L.ef_mlp_forward.argtypes = [vp, vp, i32, vp, i32, i64, vp]
        L.ef_mlp_grad.argtypes = [vp, vp, i32, vp, i32, vp, vp, i64, vp, vp, vp]
        L.ef_mlp_train_step.argtypes = [vp, vp, i32, vp, i32, vp, vp, i64, ctypes.c_float, vp, vp]
        L.ef_surrogate_create.argtypes = [vp, vp, i64, pp]
        L.ef_surrogate_destroy.argtypes = [vp]
        L.ef_surrogate_fit_stats.argtypes = [vp, vp, vp, vp, vp, vp, vp, i64, vp]
        L.ef_surrogate_normalize.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp]
        L.ef_surrogate_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_float), i32]
        L.ef_surrogate_set_policy.argtypes = [vp, ctypes.c_float, ctypes.c_float]
        L.ef_surrogate_set_entropy_gate.argtypes = [vp, ctypes.c_int]
        L.ef_surrogate_infer.argtypes = [vp, vp, vp, vp, i64, ctypes.c_float, ctypes.c_uint64, ctypes.c_float, vp]
        L.ef_surrogate_set_checker.argtypes = [vp, vp, ctypes.c_float]
        L.ef_surrogate_infer_ex.argtypes = [vp, vp, vp, vp, vp, vp, i64, ctypes.c_float, ctypes.c_uint64, ctypes.c_float, vp]
        L.ef_features_inverse.argtypes = [vp, vp, vp, i64, vp]
        L.ef_euler_step.argtypes = [vp, vp, dbl, i32, vp, i64, vp]
        L.ef_rk3_step.argtypes = [vp, vp, dbl, i32, vp, i64, vp]
        L.ef_stream_plan_create.argtypes = [i32, i64, vp, dbl, i32, i32, i32, i32, ctypes.POINTER(vp)]
        L.ef_stream_plan_destroy.argtypes = [vp]
        L.ef_stream_plan_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
        L.ef_stream_euler_step.argtypes = [vp, vp, dbl, i32, vp, vp]
        L.ef_stream_plan_status.argtypes = [vp, i32, i32]
        L.ef_moments_entropy.argtypes = [vp, vp, vp, vp, i64, vp]
        L.ef_transport_step.argtypes = [vp, vp, vp, i64, dbl, dbl, vp]
        L.ef_classical_create.argtypes = [i32, dbl, dbl, i32, ctypes.POINTER(vp)]
        L.ef_classical_collide.argtypes = [vp, vp, vp, i64, vp]
        L.ef_classical_destroy.argtypes = [vp]
        L.ef_plan_status.argtypes = [vp, i32, i32]
        L.ef_plan_set_graph.argtypes = [vp, i32]
        L.ef_plan_info.argtypes = [vp, ctypes.POINTER(i64)]
        L.ef_plan_class_info.argtypes = [vp, i32, ctypes.POINTER(i64)]
        L.ef_status_string.restype = ctypes.c_char_p
        L.ef_status_string.argtypes = [i32]
        L.ef_last_error.restype = ctypes.c_char_p
        for name in SYMBOLS:
            if name not in ("ef_status_string", "ef_last_error"):
                getattr(L, name).restype = i32
        _lib = L
    return _lib


def _check(st):
    if st != EF_OK:
        L = lib()
        raise EfError(L.ef_status_string(st).decode(), L.ef_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------------ C-API mirrors ----------

def ef_plan_create(d, N, L, kernel, R, prec):
    h = ctypes.c_void_p()
    _check(lib().ef_plan_create(d, N, float(L), kernel, R, prec, ctypes.byref(h)))
    return h


def ef_plan_create_ex(d, N, L, kernel, R, prec, R_tr=0.0, n_mu=0, n_phi=0, n_c=0, J=0, sigma_enabled=-1):
    desc = ef_plan_desc(d, N, float(L), kernel, R, prec, float(R_tr), n_mu, n_phi, n_c, J, sigma_enabled)
    h = ctypes.c_void_p()
    _check(lib().ef_plan_create_ex(ctypes.byref(desc), ctypes.byref(h)))
    return h


def ef_plan_create_batched(d, N_list, L, kernel, R, prec):
    arr = (ctypes.c_int * len(N_list))(*[int(n) for n in N_list])
    h = ctypes.c_void_p()
    _check(lib().ef_plan_create_batched(d, len(N_list), arr, float(L), kernel, R, prec, ctypes.byref(h)))
    return h


def ef_plan_destroy(plan):
    _check(lib().ef_plan_destroy(plan))


def ef_collide(plan, F, Q, ncells, stream=None):
    _check(lib().ef_collide(plan, _ptr(F), _ptr(Q), int(ncells), _stream(stream)))


def ef_collide_noalloc(plan, F, Q, ncells, stream=None):
    """ef_collide without any device allocation (scratch in the library's static device array)."""
    _check(lib().ef_collide_noalloc(plan, _ptr(F), _ptr(Q), int(ncells), _stream(stream)))


def ef_features_inverse(plan, feat, Q, ncells, stream=None):
    """Q on the grid from band modes (the inverse of ef_features on its band)."""
    _check(lib().ef_features_inverse(plan, _ptr(feat), _ptr(Q), int(ncells), _stream(stream)))


def ef_kernel_G(plan, z_index, G, stream=None):
    """G[y] = G^sigma(y, z) of the plan's kernel decomposition at the grid point z (flat index)."""
    _check(lib().ef_kernel_G(plan, int(z_index), _ptr(G), _stream(stream)))


def ef_features(plan, F, feat, ncells, log_input=0, stream=None):
    _check(lib().ef_features(plan, _ptr(F), _ptr(feat), int(ncells), int(log_input), _stream(stream)))


class MLP:
    """Owning wrapper of an ``ef_mlp_t`` (bf16 tensor-core MLP with FP32 master weights)."""

    def __init__(self, nin, nhidden, nlayers, nout, max_batch, seed=0):
        self.handle = ctypes.c_void_p()
        _check(lib().ef_mlp_create(nin, nhidden, nlayers, nout, int(max_batch), int(seed), ctypes.byref(self.handle)))
        info = (ctypes.c_int64 * 8)()
        _check(lib().ef_mlp_info(self.handle, info))
        self.nin, self.nhidden, self.nlayers, self.nout, self.nparams, self.ninp, self.noutp, self.max_batch = list(info)

    def status(self, sync=1, reset=0):
        """The MLP's device status word (EF_ERR_TIMEOUT if a GEMM gave up a bounded wait)."""
        return lib().ef_mlp_status(self.handle, int(sync), int(reset))

    def params(self):
        import numpy as np
        out = np.zeros(self.nparams, dtype=np.float32)
        _check(lib().ef_mlp_params(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 0))
        return out

    def set_params(self, host):
        import numpy as np
        host = np.ascontiguousarray(host, dtype=np.float32)
        _check(lib().ef_mlp_params(self.handle, host.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 1))

    def forward(self, X, Y, batch, stream=None):
        _check(lib().ef_mlp_forward(self.handle, _ptr(X), X.stride(0), _ptr(Y), Y.stride(0), int(batch), _stream(stream)))

    def grad(self, X, T, batch, loss, grad=None, wmask=None, rowweight=None, stream=None):
        _check(lib().ef_mlp_grad(self.handle, _ptr(X), X.stride(0), _ptr(T), T.stride(0), _ptr(wmask),
                                 _ptr(rowweight), int(batch), _ptr(loss), _ptr(grad), _stream(stream)))

    def train_step(self, X, T, batch, lr, loss, wmask=None, rowweight=None, stream=None):
        _check(lib().ef_mlp_train_step(self.handle, _ptr(X), X.stride(0), _ptr(T), T.stride(0), _ptr(wmask),
                                       _ptr(rowweight), int(batch), float(lr), _ptr(loss), _stream(stream)))

    def layout(self):
        """[(W offset, out_p, in_p, b offset)] of the padded FP32 parameter vector."""
        din = [self.ninp] + [(self.nhidden + 63) // 64 * 64] * (self.nlayers - 1)
        dout = [(self.nhidden + 63) // 64 * 64] * (self.nlayers - 1) + [self.noutp]
        out, off = [], 0
        for i, o in zip(din, dout):
            out.append((off, o, i, off + o * i))
            off += o * i + o
        return out

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().ef_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surrogate:
    """Owning wrapper of an ``ef_surrogate_t`` (keeps its plan and MLP alive)."""

    def __init__(self, plan, mlp, max_batch):
        self.plan, self.mlp = plan, mlp
        self.handle = ctypes.c_void_p()
        _check(lib().ef_surrogate_create(plan.handle, mlp.handle, int(max_batch), ctypes.byref(self.handle)))
        self.max_batch = int(max_batch)

    def fit_stats(self, featF, featQ, mom, Xt, Yt, n, rowweight=None, stream=None):
        _check(lib().ef_surrogate_fit_stats(self.handle, _ptr(featF), _ptr(featQ), _ptr(mom), _ptr(Xt), _ptr(Yt),
                                            _ptr(rowweight), int(n), _stream(stream)))

    def normalize(self, featF, featQ, mom, X, Y, n, stream=None):
        _check(lib().ef_surrogate_normalize(self.handle, _ptr(featF), _ptr(featQ), _ptr(mom), _ptr(X), _ptr(Y),
                                            int(n), _stream(stream)))

    def stats(self):
        import numpy as np
        out = np.zeros(4 * EF_FEATURE_STRIDE, dtype=np.float32)
        _check(lib().ef_surrogate_stats(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 0))
        return out

    def set_stats(self, host):
        import numpy as np
        host = np.ascontiguousarray(host, dtype=np.float32)
        _check(lib().ef_surrogate_stats(self.handle, host.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 1))

    def set_policy(self, max_miss_fraction=0.0, xmax=8.0):
        _check(lib().ef_surrogate_set_policy(self.handle, float(max_miss_fraction), float(xmax)))

    def set_entropy_gate(self, on):
        """The band entropy-production gate on or off (off skips the band of ln F)."""
        _check(lib().ef_surrogate_set_entropy_gate(self.handle, int(bool(on))))

    def infer(self, F, qfeat, flags, ncells, audit_fraction=0.05, seed=0, tol=1e-3, stream=None):
        _check(lib().ef_surrogate_infer(self.handle, _ptr(F), _ptr(qfeat), _ptr(flags), int(ncells),
                                        float(audit_fraction), int(seed), float(tol), _stream(stream)))

    def set_checker(self, mlp, tol):
        """Gate every cell on the disagreement of a second network (None switches it off)."""
        self.checker = mlp
        _check(lib().ef_surrogate_set_checker(self.handle, None if mlp is None else mlp.handle, float(tol)))

    def infer_ex(self, F, qfeat, flags, ncells, score=None, Q=None, audit_fraction=0.0, seed=0, tol=1e-3, stream=None):
        _check(lib().ef_surrogate_infer_ex(self.handle, _ptr(F), _ptr(qfeat), _ptr(flags), _ptr(score), _ptr(Q),
                                           int(ncells), float(audit_fraction), int(seed), float(tol), _stream(stream)))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().ef_surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ef_euler_step(plan, F, dt, nsteps, diag, ncells, stream=None):
    _check(lib().ef_euler_step(plan, _ptr(F), float(dt), int(nsteps), _ptr(diag), int(ncells), _stream(stream)))


def ef_plan_reserve(plan, ncells):
    _check(lib().ef_plan_reserve(plan, int(ncells)))


def ef_rk3_step(plan, F, dt, nsteps, diag, ncells, stream=None):
    _check(lib().ef_rk3_step(plan, _ptr(F), float(dt), int(nsteps), _ptr(diag), int(ncells), _stream(stream)))


class StreamPlan:
    """Owning wrapper of an ``ef_stream_plan_t``: a host-resident batch streamed through the GPU in
    ``nchunks`` concurrent chunks (uploads, collision steps and downloads overlap)."""

    def __init__(self, d, N_list, L, kernel, R, prec, nchunks=8):
        arr = (ctypes.c_int * len(N_list))(*[int(n) for n in N_list])
        self.handle = ctypes.c_void_p()
        _check(lib().ef_stream_plan_create(d, len(N_list), arr, float(L), kernel, R, prec, int(nchunks),
                                           ctypes.byref(self.handle)))
        self.ncells = len(N_list)

    def info(self):
        out = (ctypes.c_int64 * 4)()
        _check(lib().ef_stream_plan_info(self.handle, out))
        return {"cells": out[0], "chunks": out[1], "values": out[2], "bytes_per_value": out[3]}

    def euler(self, F_host, dt, nsteps=1, diag_host=None, stream=None):
        """F_host: a (preferably pinned) CPU tensor of the whole batch, updated in place."""
        _check(lib().ef_stream_euler_step(self.handle, _ptr(F_host), float(dt), int(nsteps), _ptr(diag_host),
                                          _stream(stream)))

    def status(self, sync=1, reset=0):
        return lib().ef_stream_plan_status(self.handle, int(sync), int(reset))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().ef_stream_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Galerkin:
    """Owning wrapper of an ``ef_galerkin_t``: the Fourier Galerkin method (unaliased sum over the
    mode set K of the N grid, by zero padding to the 2N grid), the comparison method of Fig. 2."""

    def __init__(self, d, N, L, kernel, R, prec, max_cells, R_tr=0.0, n_mu=0, n_phi=0, n_c=0, J=0, sigma_enabled=0):
        desc = ef_plan_desc(d, N, float(L), kernel, R, prec, float(R_tr), n_mu, n_phi, n_c, J, sigma_enabled)
        self.handle = ctypes.c_void_p()
        _check(lib().ef_galerkin_create(ctypes.byref(desc), int(max_cells), ctypes.byref(self.handle)))
        self.d, self.N = d, N

    def collide(self, F, Q, ncells=None, stream=None):
        n = ncells if ncells is not None else F.numel() // self.N ** self.d
        _check(lib().ef_galerkin_collide(self.handle, _ptr(F), _ptr(Q), int(n), _stream(stream)))

    def status(self, sync=1, reset=0):
        return lib().ef_galerkin_status(self.handle, int(sync), int(reset))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().ef_galerkin_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Classical:
    """Owning wrapper of an ``ef_classical_t``: the entropic Fourier method on the classical form of
    the operator, 3D Maxwell molecules, FP64, summed directly over mode pairs (Table 3 sizes)."""

    def __init__(self, N, L, R_tr=0.0, sigma_enabled=1):
        self.handle = ctypes.c_void_p()
        _check(lib().ef_classical_create(int(N), float(L), float(R_tr), int(sigma_enabled), ctypes.byref(self.handle)))
        self.N = int(N)

    def collide(self, F, Q, ncells=None, stream=None):
        n = ncells if ncells is not None else F.numel() // self.N ** 3
        _check(lib().ef_classical_collide(self.handle, _ptr(F), _ptr(Q), int(n), _stream(stream)))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().ef_classical_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ef_moments_entropy(plan, F, Q, out, ncells, stream=None):
    _check(lib().ef_moments_entropy(plan, _ptr(F), _ptr(Q), _ptr(out), int(ncells), _stream(stream)))


def ef_transport_step(plan, F_in, F_out, ncells, dx, dt, stream=None):
    _check(lib().ef_transport_step(plan, _ptr(F_in), _ptr(F_out), int(ncells), float(dx), float(dt), _stream(stream)))


def ef_plan_status(plan, sync=1, reset=0):
    return lib().ef_plan_status(plan, int(sync), int(reset))


def ef_plan_set_graph(plan, enable):
    _check(lib().ef_plan_set_graph(plan, int(enable)))


def ef_plan_info(plan):
    info = (ctypes.c_int64 * 8)()
    _check(lib().ef_plan_info(plan, info))
    keys = ("d", "classes", "directions", "cluster", "threads", "cells", "prec", "launches")
    return dict(zip(keys, list(info)))


def ef_plan_class_info(plan, i):
    out = (ctypes.c_int64 * 8)()
    _check(lib().ef_plan_class_info(plan, int(i), out))
    keys = ("N", "cells", "cluster", "threads", "planes", "sg_global", "prefetch", "tuned_us")
    return dict(zip(keys, list(out)))


class Plan:
    """Owning wrapper of an ``ef_plan_t``."""

    def __init__(self, d, N, L, kernel, R, prec, batched_N=None, **ex):
        self.d, self.L, self.prec, self.kernel, self.R = d, L, prec, kernel, R
        if batched_N is not None:
            self.N_list = [int(n) for n in batched_N]
            self.handle = ef_plan_create_batched(d, self.N_list, L, kernel, R, prec)
            self.ncells = len(self.N_list)
        else:
            self.N_list = None
            self.N = N
            self.handle = ef_plan_create_ex(d, N, L, kernel, R, prec, **ex) if ex else \
                ef_plan_create(d, N, L, kernel, R, prec)
            self.ncells = None

    def collide(self, F, Q, ncells=None, stream=None):
        ef_collide(self.handle, F, Q, self._n(F, ncells), stream)

    def euler(self, F, dt, nsteps=1, diag=None, ncells=None, stream=None):
        ef_euler_step(self.handle, F, dt, nsteps, diag, self._n(F, ncells), stream)

    def reserve(self, ncells=None):
        """Allocate the SSP-RK3 stage buffers for batches of up to ncells cells (a set-up call:
        it may synchronise the device)."""
        n = int(self.ncells if self.ncells is not None else ncells)
        ef_plan_reserve(self.handle, n)
        self._rk_cells = max(getattr(self, "_rk_cells", 0), n)

    def rk3(self, F, dt, nsteps=1, diag=None, ncells=None, stream=None):
        """SSP-RK3 steps; reserves the stage buffers first if this batch needs more than reserved
        (call reserve() beforehand to keep this call free of allocation, e.g. before graph capture)."""
        n = self._n(F, ncells)
        if getattr(self, "_rk_cells", 0) < n:
            self.reserve(n)
        ef_rk3_step(self.handle, F, dt, nsteps, diag, n, stream)

    def moments(self, F, Q, out, ncells=None, stream=None):
        ef_moments_entropy(self.handle, F, Q, out, self._n(F, ncells), stream)

    def transport(self, F_in, F_out, dx, dt, ncells=None, stream=None):
        """One upwind free-transport step between the batch's cells (a periodic 1D spatial grid)."""
        ef_transport_step(self.handle, F_in, F_out, self._n(F_in, ncells), dx, dt, stream)

    def inhomogeneous(self, F, scratch, dx, dt, nsteps=1, rk3=False, diag=None, stream=None):
        """Lie splitting of dF/dt + v dF/dx = Q(F) on the batch's cells as the points of a periodic 1D
        spatial grid: each step transports the state into the other buffer (F and scratch take
        turns) and applies one collision step (Euler or SSP-RK3) there, in place.  The result ends
        in F (copied back from scratch after an odd number of steps).  diag (optional) receives
        each step's collision diagnostics, [step][cell][k]."""
        import torch
        n = self._n(F, None)
        a, b = F, scratch
        for k in range(int(nsteps)):
            self.transport(a, b, dx, dt, ncells=n, stream=stream)
            d = None if diag is None else diag[k]
            (self.rk3 if rk3 else self.euler)(b, dt, 1, d, ncells=n, stream=stream)
            a, b = b, a
        if a is not F:
            if not F.is_cuda:
                F.copy_(a)
                return
            if stream is None:
                s = torch.cuda.current_stream()
            elif isinstance(stream, int):
                s = torch.cuda.ExternalStream(stream)
            else:
                s = stream
            with torch.cuda.stream(s):
                F.copy_(a)

    def inhomogeneous_sharded(self, F_ext, scratch_ext, dx, dt, nsteps=1, rk3=False, group=None):
        """``inhomogeneous`` for a spatial grid split over ranks (one GPU each): this rank's cells
        are F_ext[1 .. n] of a [n + 2, ...] array whose two ends are halo cells, refreshed before
        every transport step by ``shard.halo_exchange`` (NCCL point-to-point).  Runs on torch's
        current stream; the result ends in F_ext."""
        from . import shard
        n = F_ext.shape[0] - 2

        def transport(a, b):
            self.transport(a, b, dx, dt, ncells=n + 2)

        def collide(view):
            (self.rk3 if rk3 else self.euler)(view, dt, 1, None, ncells=n)

        out = shard.lie_steps_sharded(F_ext, scratch_ext, nsteps, transport, collide, group)
        if out is not F_ext:
            F_ext.copy_(out)

    def status(self, sync=1, reset=0):
        return ef_plan_status(self.handle, sync, reset)

    def set_graph(self, enable=True):
        ef_plan_set_graph(self.handle, enable)

    def info(self):
        return ef_plan_info(self.handle)

    def class_info(self):
        return [ef_plan_class_info(self.handle, i) for i in range(self.info()["classes"])]

    def _n(self, F, ncells):
        if ncells is not None:
            return ncells
        if self.ncells is not None:
            return self.ncells
        return F.numel() // (self.N ** self.d)

    def close(self):
        if getattr(self, "handle", None) is not None:
            ef_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
