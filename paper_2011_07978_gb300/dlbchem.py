"""Thin ctypes binding of libdlbchem (include/dlbchem.h), same entry-point names.

Only argument marshalling lives here: every step of the chemistry runs in the
library's CUDA kernels. PyTorch supplies device memory and streams. If the
library is missing the import fails; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdlbchem.so")

OK, BAD_ARG, BAD_MECH, CUDA, OOM = 0, 1, 2, 3, 4
CELL_SURROGATE = 2
STATIC_MAX_CELLS = 262144
CELL_OK, CELL_MAPPED, CELL_MAX_STEPS, CELL_H_UNDERFLOW, CELL_NONFINITE = 0, 1, -1, -2, -3
SCHED_PLAIN, SCHED_QUEUE = 0, 1


class dlbchem_options(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol", ctypes.c_double), ("max_steps", ctypes.c_int32),
                ("isothermal", ctypes.c_int32), ("hmin_frac", ctypes.c_double), ("schedule", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("mapping", ctypes.c_int32), ("timing", ctypes.c_int32),
                ("map_Ttol", ctypes.c_double), ("map_Ytol", ctypes.c_double), ("map_Tmax", ctypes.c_double),
                ("team_warps", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("predictor", ctypes.c_int32), ("surrogate", ctypes.c_int32), ("gate", ctypes.c_double)]


_vp = ctypes.c_void_p
_lib = None


def load() -> ctypes.CDLL:
    """Load libdlbchem.so (built by paper_2011_07978_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    lib.dlbchem_options_default.argtypes = [ctypes.POINTER(dlbchem_options)]
    lib.dlbchem_create.argtypes = [ctypes.c_char_p, ctypes.POINTER(dlbchem_options), ctypes.POINTER(_vp)]
    lib.dlbchem_set_options.argtypes = [_vp, ctypes.POINTER(dlbchem_options)]
    sig = [_vp, ctypes.c_int64, ctypes.c_double, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    lib.dlbchem_integrate.argtypes = sig
    lib.dlbchem_integrate_host.argtypes = sig
    lib.dlbchem_integrate_static.argtypes = sig[:-2] + [_vp]
    lib.dlbchem_nspecies.argtypes = [_vp]
    lib.dlbchem_table_stats.argtypes = [ctypes.c_char_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]
    lib.dlbchem_lu_stats.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int64)]
    lib.dlbchem_nreactions.argtypes = [_vp]
    lib.dlbchem_last_stats.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
    lib.dlbchem_last_timing.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
    lib.dlbchem_last_worklist.argtypes = [_vp, _vp, ctypes.POINTER(ctypes.c_int64)]
    lib.dlbchem_last_mapping.argtypes = [_vp, _vp, ctypes.POINTER(ctypes.c_int64)]
    lib.dlbchem_check_math.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp]
    lib.dlbchem_rhs.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp, _vp]
    lib.dlbchem_fp64_fma_probe.argtypes = [ctypes.c_int64, _vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), _vp]
    lib.dlbchem_last_error.argtypes = [_vp]
    lib.dlbchem_last_error.restype = ctypes.c_char_p
    lib.dlbchem_destroy.argtypes = [_vp]
    lib.dlbchem_mlp_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)]
    lib.dlbchem_mlp_nparams.argtypes = [_vp]
    lib.dlbchem_mlp_nparams.restype = ctypes.c_int64
    lib.dlbchem_mlp_set_params.argtypes = [_vp, _vp, _vp]
    lib.dlbchem_mlp_get_params.argtypes = [_vp, _vp, _vp]
    _fp = ctypes.POINTER(ctypes.c_float)
    lib.dlbchem_mlp_set_norm.argtypes = [_vp, _fp, _fp, _fp, _fp]
    lib.dlbchem_mlp_forward.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp]
    lib.dlbchem_mlp_grad.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp]
    lib.dlbchem_mlp_adam.argtypes = [_vp, _vp, ctypes.c_float, _vp]
    lib.dlbchem_mlp_train_step.argtypes = [_vp, ctypes.c_int64, _vp, _vp, ctypes.c_float, _vp, _vp]
    lib.dlbchem_mlp_set_fused.argtypes = [_vp, ctypes.c_int]
    lib.dlbchem_mlp_fused.argtypes = [_vp]
    lib.dlbchem_mlp_last_error.argtypes = [_vp]
    lib.dlbchem_mlp_last_error.restype = ctypes.c_char_p
    lib.dlbchem_mlp_destroy.argtypes = [_vp]
    lib.dlbchem_attach_mlp.argtypes = [_vp, _vp]
    lib.dlbchem_batch_create.argtypes = [ctypes.POINTER(dlbchem_options), ctypes.POINTER(_vp)]
    lib.dlbchem_batch_add.argtypes = [_vp, ctypes.c_char_p, ctypes.c_int64, ctypes.c_double] + [_vp] * 7
    lib.dlbchem_batch_tune.argtypes = [_vp, ctypes.c_int64, _vp]
    lib.dlbchem_batch_capture.argtypes = [_vp, _vp]
    lib.dlbchem_batch_launch.argtypes = [_vp, _vp]
    lib.dlbchem_batch_info.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
    lib.dlbchem_batch_last_error.argtypes = [_vp]
    lib.dlbchem_batch_last_error.restype = ctypes.c_char_p
    lib.dlbchem_batch_destroy.argtypes = [_vp]
    _lib = lib
    return lib


def table_stats(mech_path: str, team_warps: int) -> dict:
    """Build and check a mechanism's round tables on the host (no GPU needed):
    dlbchem_table_stats. Raises DlbchemError if a table check fails."""
    lib = load()
    out = (ctypes.c_int64 * 10)()
    rc = lib.dlbchem_table_stats(str(mech_path).encode(), team_warps, out)
    if rc != 0:
        raise DlbchemError(rc, lib.dlbchem_last_error(None).decode())
    keys = ["chunks", "chunk_size", "dslots", "inc_rounds", "tri_rounds", "all_rounds_max_warp", "nsplit",
            "split_off", "nsp", "nrx"]
    return dict(zip(keys, list(out)))


def fp64_fma_probe(iters: int, out, stream=None) -> int:
    """dlbchem_fp64_fma_probe on a CUDA float64 tensor `out` (numel a multiple
    of 256); returns the launch's FP64 flop count."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(out.device)
    flops = ctypes.c_int64(0)
    rc = load().dlbchem_fp64_fma_probe(int(iters), _ptr(out), out.numel(), ctypes.byref(flops),
                                       ctypes.c_void_p(stream.cuda_stream))
    if rc != OK:
        raise DlbchemError(rc, "dlbchem_fp64_fma_probe failed")
    return int(flops.value)


def options_default() -> dlbchem_options:
    o = dlbchem_options()
    load().dlbchem_options_default(ctypes.byref(o))
    return o


class DlbchemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dlbchem error {code}: {msg}")
        self.code = code


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Context:
    """One loaded mechanism on the current CUDA device (dlbchem_create)."""

    def __init__(self, mech_path: str, **opts):
        lib = load()
        o = options_default()
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        h = _vp()
        rc = lib.dlbchem_create(mech_path.encode(), ctypes.byref(o), ctypes.byref(h))
        if rc != OK:
            raise DlbchemError(rc, lib.dlbchem_last_error(None).decode())
        self._h = h
        self.opts = o
        self.nsp = lib.dlbchem_nspecies(h)
        self.nrx = lib.dlbchem_nreactions(h)

    def set_options(self, **opts):
        o = dlbchem_options.from_buffer_copy(self.opts)
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        self._check(load().dlbchem_set_options(self._h, ctypes.byref(o)))
        self.opts = o

    def _check(self, rc):
        if rc != OK:
            raise DlbchemError(rc, load().dlbchem_last_error(self._h).decode())

    def integrate(self, T, p, Y, dt, T_out=None, Y_out=None, steps=None, status=None, Yref=None, stream=None):
        """dlbchem_integrate on CUDA tensors (float64 T[n], p[n], Y[nsp, n] species-major;
        int32 steps/status). Asynchronous on `stream` (default: torch's current stream)."""
        import torch
        n = T.numel()
        for t in (T, p, Y):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError("T, p, Y must be contiguous float64 CUDA tensors")
        if Y.shape != (self.nsp, n) or p.numel() != n:
            raise ValueError("shape mismatch")
        if T_out is None:
            T_out = torch.empty_like(T)
        if Y_out is None:
            Y_out = torch.empty_like(Y)
        if stream is None:
            stream = torch.cuda.current_stream(T.device)
        sh = ctypes.c_void_p(stream.cuda_stream)
        self._check(load().dlbchem_integrate(self._h, n, float(dt), _ptr(T), _ptr(p), _ptr(Y), _ptr(T_out),
                                             _ptr(Y_out), _ptr(steps), _ptr(status), _ptr(Yref), sh))
        return T_out, Y_out

    def integrate_static(self, T, p, Y, dt, T_out, Y_out, steps=None, status=None, stream=None):
        """dlbchem_integrate_static: queued integration with the library's fixed scratch
        array (no device allocation); CUDA tensors as for integrate()."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(T.device)
        self._check(load().dlbchem_integrate_static(self._h, T.numel(), float(dt), _ptr(T), _ptr(p), _ptr(Y),
                                                    _ptr(T_out), _ptr(Y_out), _ptr(steps), _ptr(status),
                                                    ctypes.c_void_p(stream.cuda_stream)))
        return T_out, Y_out

    def integrate_host(self, T, p, Y, dt, T_out, Y_out, steps=None, status=None, Yref=None, stream=None):
        """dlbchem_integrate_host on host numpy arrays or CPU tensors (copies inside)."""
        import numpy as np

        def hp(a):
            if a is None:
                return None
            if isinstance(a, np.ndarray):
                assert a.flags.c_contiguous
                return ctypes.c_void_p(a.ctypes.data)
            return ctypes.c_void_p(a.data_ptr())
        n = int(T.shape[0]) if hasattr(T, "shape") else len(T)
        sh = ctypes.c_void_p(0 if stream is None else stream.cuda_stream)
        self._check(load().dlbchem_integrate_host(self._h, n, float(dt), hp(T), hp(p), hp(Y), hp(T_out), hp(Y_out),
                                                  hp(steps), hp(status), hp(Yref), sh))

    def last_stats(self) -> dict:
        out = (ctypes.c_int64 * 10)()
        self._check(load().dlbchem_last_stats(self._h, out))
        keys = ["integrated", "mapped", "ref", "team_threads", "teams_per_cta", "ctas", "smem_bytes", "launches",
                "fp64_fallbacks", "precision"]
        return dict(zip(keys, list(out)))

    def last_timing(self) -> dict:
        out = (ctypes.c_double * 8)()
        self._check(load().dlbchem_last_timing(self._h, out))
        return dict(zip(["integrator_ms", "classify_ms", "sort_ms", "scatter_ms"], list(out)[:4]))

    def check_math(self, x):
        """Returns a [n, 4] tensor: own exp, CUDA exp, own reciprocal, 1/x."""
        import torch
        out = torch.empty((x.numel(), 4), dtype=torch.float64, device=x.device)
        self._check(load().dlbchem_check_math(self._h, x.numel(), _ptr(x), _ptr(out),
                                              ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)))
        return out

    def last_worklist(self, out):
        """Copy the last work list into the int32 CUDA tensor `out`; returns its length."""
        m = ctypes.c_int64()
        self._check(load().dlbchem_last_worklist(self._h, _ptr(out), ctypes.byref(m)))
        return m.value

    def rhs(self, T, p, Y, fT=None, fY=None, stream=None):
        """dlbchem_rhs: f = (dT/dt, dY/dt) of every cell (CUDA float64 tensors)."""
        import torch
        if fT is None:
            fT = torch.empty_like(T)
        if fY is None:
            fY = torch.empty_like(Y)
        if stream is None:
            stream = torch.cuda.current_stream(T.device)
        self._check(load().dlbchem_rhs(self._h, T.numel(), _ptr(T), _ptr(p), _ptr(Y), _ptr(fT), _ptr(fY),
                                       ctypes.c_void_p(stream.cuda_stream)))
        return fT, fY

    def last_mapping(self, out):
        """dlbchem_last_mapping into the int32 CUDA tensor `out`: the reference of
        each mapped cell, -1 elsewhere. Returns ncells, or -1 without mapping."""
        m = ctypes.c_int64()
        self._check(load().dlbchem_last_mapping(self._h, _ptr(out), ctypes.byref(m)))
        return m.value

    def attach_mlp(self, mlp):
        """dlbchem_attach_mlp: the network used by the predictor / surrogate options."""
        self._mlp = mlp
        self._check(load().dlbchem_attach_mlp(self._h, None if mlp is None else mlp._h))

    def close(self):
        if getattr(self, "_h", None):
            load().dlbchem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several meshes over several mechanisms in one captured CUDA graph
    (dlbchem_batch_*). Arrays are CUDA tensors that must outlive the graph."""

    def __init__(self, **opts):
        lib = load()
        o = options_default()
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        h = _vp()
        if lib.dlbchem_batch_create(ctypes.byref(o), ctypes.byref(h)) != OK:
            raise DlbchemError(BAD_ARG, "batch create failed")
        self._h = h
        self._keep = []

    def _check(self, rc):
        if rc != OK:
            raise DlbchemError(rc, load().dlbchem_batch_last_error(self._h).decode())

    def add(self, mech_path, T, p, Y, dt, T_out, Y_out, steps=None, status=None):
        self._keep.extend([T, p, Y, T_out, Y_out, steps, status])
        self._check(load().dlbchem_batch_add(self._h, mech_path.encode(), T.numel(), float(dt), _ptr(T), _ptr(p),
                                             _ptr(Y), _ptr(T_out), _ptr(Y_out), _ptr(steps), _ptr(status)))

    def tune(self, sample_cells=4096, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        self._check(load().dlbchem_batch_tune(self._h, int(sample_cells), ctypes.c_void_p(s.cuda_stream)))

    def capture(self, stream):
        self._check(load().dlbchem_batch_capture(self._h, ctypes.c_void_p(stream.cuda_stream)))

    def launch(self, stream):
        self._check(load().dlbchem_batch_launch(self._h, ctypes.c_void_p(stream.cuda_stream)))

    def info(self, cls):
        out = (ctypes.c_int64 * 6)()
        self._check(load().dlbchem_batch_info(self._h, cls, out))
        return dict(zip(["meshes", "cells", "team_warps", "chunk", "species", "tune_us"], list(out)))

    def close(self):
        if getattr(self, "_h", None):
            load().dlbchem_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class MLP:
    """dlbchem_mlp_*: the BF16 tensor-core network of the learned predictor."""

    def __init__(self, n_in, n_hidden, n_out):
        h = _vp()
        rc = load().dlbchem_mlp_create(n_in, n_hidden, n_out, ctypes.byref(h))
        if rc != OK:
            raise DlbchemError(rc, "mlp create failed")
        self._h = h
        self.n_in, self.n_hidden, self.n_out = n_in, n_hidden, n_out
        self.nparams = load().dlbchem_mlp_nparams(h)

    def _check(self, rc):
        if rc != OK:
            raise DlbchemError(rc, load().dlbchem_mlp_last_error(self._h).decode())

    def set_params(self, params, stream=None):
        self._check(load().dlbchem_mlp_set_params(self._h, _ptr(params), _stream_ptr(stream)))

    def get_params(self, out, stream=None):
        self._check(load().dlbchem_mlp_get_params(self._h, _ptr(out), _stream_ptr(stream)))
        return out

    def set_norm(self, mu_x, sd_x, mu_y, sd_y):
        import numpy as np
        f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
        arrs = [f(mu_x), f(sd_x), f(mu_y), f(sd_y)]
        self._norm = arrs
        fp = ctypes.POINTER(ctypes.c_float)
        self._check(load().dlbchem_mlp_set_norm(self._h, *[a.ctypes.data_as(fp) for a in arrs]))

    def forward(self, X, out, stream=None):
        self._check(load().dlbchem_mlp_forward(self._h, X.shape[0], _ptr(X), _ptr(out), _stream_ptr(stream)))
        return out

    def set_fused(self, enable: bool):
        """dlbchem_mlp_set_fused: whole-network forward kernel (default) or layer by layer."""
        self._check(load().dlbchem_mlp_set_fused(self._h, 1 if enable else 0))

    @property
    def fused(self) -> bool:
        return load().dlbchem_mlp_fused(self._h) == 1

    def grad(self, X, Y, grad=None, loss=None, stream=None):
        self._check(load().dlbchem_mlp_grad(self._h, X.shape[0], _ptr(X), _ptr(Y), _ptr(grad), _ptr(loss),
                                            _stream_ptr(stream)))

    def adam(self, lr, grad=None, stream=None):
        self._check(load().dlbchem_mlp_adam(self._h, _ptr(grad), float(lr), _stream_ptr(stream)))

    def train_step(self, X, Y, lr, loss=None, stream=None):
        self._check(load().dlbchem_mlp_train_step(self._h, X.shape[0], _ptr(X), _ptr(Y), float(lr), _ptr(loss),
                                                  _stream_ptr(stream)))

    def close(self):
        if getattr(self, "_h", None):
            load().dlbchem_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lu_stats(mech_path: str) -> dict:
    """dlbchem_lu_stats: symbolic sparse-LU analysis of a mechanism (host only)."""
    out = (ctypes.c_int64 * 10)()
    rc = load().dlbchem_lu_stats(mech_path.encode(), out)
    if rc != OK:
        raise DlbchemError(rc, load().dlbchem_last_error(None).decode())
    keys = ("N", "block_nnz", "factor_nnz", "lu_dense", "lu_sparse", "solve_dense", "solve_sparse", "rank1",
            "step_dense", "step_sparse")
    return dict(zip(keys, (int(v) for v in out)))

