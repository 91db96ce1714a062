"""ctypes binding of liblgf.so (include/lgf.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts torch
tensors and numpy block lists into the plain pointers and sizes of the C ABI
and turns status codes into exceptions.  There is no fallback: if liblgf.so
is missing or cannot be loaded, importing the library raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblgf.so")

LGF_OK, LGF_EINVAL, LGF_ENOMEM, LGF_ECUDA, LGF_ETIMEOUT, LGF_EUNSUPPORTED, LGF_ENOTABLE = range(7)
LGF_F32, LGF_F64 = 0, 1
LGF_OP_POISSON, LGF_OP_INTFACTOR, LGF_OP_POISSON_THEN_INTFACTOR, LGF_OP_KINV = 0, 1, 2, 3
LGF_TUNE_OFF, LGF_TUNE_ON, LGF_TUNE_CACHED = 0, 1, 2
LGF_FLAG_BULK_STAGING = 1
LGF_FLAG_BATCH_RAGGED = 2
LGF_FLAG_BATCH_PER_PROBLEM = 4

# Every symbol include/lgf.h declares (checked by the symbol test).
EXPORTS = ("lgf_ctx_create", "lgf_ctx_destroy", "lgf_table_build", "lgf_table_info", "lgf_table_lookup",
           "lgf_kinv_lookup", "lgf_poisson_apply", "lgf_kinv_apply", "lgf_curl", "lgf_curl_adjoint",
           "lgf_velocity_refresh", "lgf_ib_spread", "lgf_ib_interp", "lgf_intfactor_apply", "lgf_intfactor_weights", "lgf_batch_apply",
           "lgf_residual", "lgf_profile_enable", "lgf_profile_read", "lgf_ctx_stats", "lgf_cache_limits",
           "lgf_nested_projection_stage", "lgf_autotune", "lgf_tune_report", "lgf_device_status",
           "lgf_wait_selftest", "lgf_poisson_error_estimate", "lgf_table_save", "lgf_table_load",
           "lgf_intfactor_apply_noalloc",
           "lgf_status_string", "lgf_last_error", "lgf_version")


class lgf_blockset(ctypes.Structure):
    _fields_ = [("b", ctypes.c_int32), ("nblocks", ctypes.c_int32), ("coords", ctypes.POINTER(ctypes.c_int32))]


class lgf_options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("prec", ctypes.c_int32), ("table_radius", ctypes.c_int32),
                ("stencil_radius", ctypes.c_int32), ("device", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class lgf_problem(ctypes.Structure):
    _fields_ = [("src", lgf_blockset), ("tgt", lgf_blockset), ("f_dev", ctypes.c_void_p), ("u_dev", ctypes.c_void_p),
                ("ncomp", ctypes.c_int32), ("nrhs", ctypes.c_int32), ("op", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("alpha", ctypes.c_double), ("dx", ctypes.c_double)]


class lgf_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class lgf_stats(ctypes.Structure):
    _fields_ = [("graphs_cached", ctypes.c_int64), ("poisson_plans", ctypes.c_int64),
                ("intfactor_plans", ctypes.c_int64), ("curl_plans", ctypes.c_int64), ("ib_plans", ctypes.c_int64),
                ("spectra", ctypes.c_int64), ("generation", ctypes.c_int64), ("graphs_dropped", ctypes.c_int64),
                ("evictions", ctypes.c_int64), ("scratch_reallocs", ctypes.c_int64),
                ("scratch_bytes", ctypes.c_int64), ("reserved", ctypes.c_int64 * 5)]


class lgf_stage(ctypes.Structure):
    _fields_ = [("flow", lgf_blockset), ("nmarkers", ctypes.c_int64), ("X_prev_dev", ctypes.c_void_p),
                ("X_dev", ctypes.c_void_p), ("ub_dev", ctypes.c_void_p), ("W1_dev", ctypes.c_void_p),
                ("W2_dev", ctypes.c_void_p), ("r_dev", ctypes.c_void_p), ("u_dev", ctypes.c_void_p),
                ("d_dev", ctypes.c_void_p), ("f_dev", ctypes.c_void_p), ("alpha", ctypes.c_double),
                ("dx", ctypes.c_double), ("reserved", ctypes.c_int32 * 4)]


class lgf_tune_info(ctypes.Structure):
    _fields_ = [("plans_tuned", ctypes.c_int64), ("plans_from_cache", ctypes.c_int64),
                ("candidates_timed", ctypes.c_int64), ("batches_tuned", ctypes.c_int64),
                ("last_branches", ctypes.c_int64), ("shifted_x", ctypes.c_int64), ("shifted_y", ctypes.c_int64),
                ("longer_x", ctypes.c_int64), ("longer_y", ctypes.c_int64), ("longer_z", ctypes.c_int64),
                ("z_variant", ctypes.c_int64), ("tune_ms", ctypes.c_double), ("last_ragged", ctypes.c_int64),
                ("fused_inverse", ctypes.c_int64), ("reserved", ctypes.c_int64 * 2)]


class LgfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lgf status {status}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load liblgf.so (raises if it is missing: build it with build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing; build the CUDA library first "
                          "(python -m paper_1604_01814_gb300.build)")
    L = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    bsp = ctypes.POINTER(lgf_blockset)
    sig = {
        "lgf_ctx_create": [ctypes.POINTER(vp), ctypes.POINTER(lgf_options)],
        "lgf_ctx_destroy": [vp],
        "lgf_table_build": [vp, i32, vp],
        "lgf_table_info": [vp, ctypes.POINTER(i32), ctypes.POINTER(dbl)],
        "lgf_table_lookup": [vp, vp, i64, vp, vp],
        "lgf_poisson_apply": [vp, bsp, bsp, vp, vp, i32, i32, dbl, vp],
        "lgf_kinv_lookup": [vp, dbl, vp, i64, vp, vp],
        "lgf_kinv_apply": [vp, dbl, bsp, bsp, vp, vp, i32, i32, dbl, vp],
        "lgf_curl": [vp, bsp, bsp, vp, vp, i32, dbl, vp],
        "lgf_curl_adjoint": [vp, bsp, bsp, vp, vp, i32, dbl, vp],
        "lgf_velocity_refresh": [vp, bsp, bsp, vp, vp, i32, dbl, vp],
        "lgf_ib_spread": [vp, bsp, i64, vp, vp, vp, i32, dbl, vp],
        "lgf_ib_interp": [vp, bsp, i64, vp, vp, vp, i32, vp],
        "lgf_intfactor_apply": [vp, dbl, bsp, bsp, vp, vp, i32, i32, vp],
        "lgf_intfactor_weights": [vp, dbl, vp, i32, ctypes.POINTER(i32), vp],
        "lgf_batch_apply": [vp, ctypes.POINTER(lgf_problem), i32, vp],
        "lgf_residual": [vp, bsp, vp, vp, dbl, vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), vp],
        "lgf_profile_enable": [vp, i32],
        "lgf_profile_read": [vp, ctypes.POINTER(lgf_kernel_stat), i32, ctypes.POINTER(i32)],
        "lgf_ctx_stats": [vp, ctypes.POINTER(lgf_stats)],
        "lgf_cache_limits": [vp, i32, i32, i32],
        "lgf_nested_projection_stage": [vp, ctypes.POINTER(lgf_stage), vp],
        "lgf_autotune": [vp, i32, ctypes.c_char_p],
        "lgf_device_status": [vp, ctypes.POINTER(i32)],
        "lgf_poisson_error_estimate": [vp, bsp, bsp, vp, vp, i32, i32, dbl, i32, ctypes.POINTER(dbl), vp],
        "lgf_table_save": [vp, ctypes.c_char_p],
        "lgf_table_load": [vp, ctypes.c_char_p],
        "lgf_wait_selftest": [vp, i64, vp],
        "lgf_tune_report": [vp, ctypes.POINTER(lgf_tune_info)],
        "lgf_intfactor_apply_noalloc": [i32, dbl, dbl, bsp, bsp, vp, vp, i32, i32, vp, ctypes.c_char_p, i32],
        "lgf_status_string": [i32],
        "lgf_last_error": [vp],
        "lgf_version": [],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = i32
    L.lgf_status_string.restype = ctypes.c_char_p
    L.lgf_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _blockset(b: int, coords) -> tuple:
    c = np.ascontiguousarray(np.asarray(coords, dtype=np.int32).reshape(-1, 3))
    bs = lgf_blockset(int(b), int(c.shape[0]), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return bs, c   # keep the array alive with the struct


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


class Context:
    """One lgf_ctx: precision, tolerance, G_L table, plans, spectra, scratch."""

    def __init__(self, prec: str = "f32", tol: float = 0.0, table_radius: int = 0, stencil_radius: int = 0,
                 device: int = 0, flags: int = 0):
        self._L = load()
        self.prec = {"f32": LGF_F32, "f64": LGF_F64}[prec]
        opt = lgf_options(float(tol), self.prec, int(table_radius), int(stencil_radius), int(device), int(flags))
        h = ctypes.c_void_p()
        st = self._L.lgf_ctx_create(ctypes.byref(h), ctypes.byref(opt))
        if st != LGF_OK:
            raise LgfError(st, "lgf_ctx_create: " + self._L.lgf_status_string(st).decode())
        self._h = h
        self.device = device

    # -- helpers -------------------------------------------------------------
    def _check(self, st: int, what: str):
        if st != LGF_OK:
            msg = self._L.lgf_last_error(self._h).decode()
            raise LgfError(st, f"{what}: {self._L.lgf_status_string(st).decode()}: {msg}")

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.prec == LGF_F64 else torch.float32

    def _field(self, t, nblk: int, b: int, nf: int, name: str):
        import torch
        if t is None:
            raise ValueError(f"{name} is None")
        if not t.is_cuda or t.dtype != self.dtype or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA tensor of dtype {self.dtype}")
        if t.numel() != nblk * b ** 3 * nf:
            raise ValueError(f"{name} has {t.numel()} elements, expected {nblk * b ** 3 * nf}")
        return t

    def close(self):
        if getattr(self, "_h", None):
            self._L.lgf_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API -----------------------------------------------------------------
    def table_build(self, max_offset: int = 48, stream=None):
        self._check(self._L.lgf_table_build(self._h, int(max_offset), _stream_ptr(stream)), "lgf_table_build")

    def table_info(self):
        r = ctypes.c_int32()
        m = ctypes.c_double()
        self._check(self._L.lgf_table_info(self._h, ctypes.byref(r), ctypes.byref(m)), "lgf_table_info")
        return r.value, m.value

    def table_lookup(self, offsets, stream=None):
        import torch
        off = offsets.to(device=f"cuda:{self.device}", dtype=torch.int32).contiguous()
        out = torch.empty(off.shape[0], dtype=torch.float64, device=off.device)
        self._check(self._L.lgf_table_lookup(self._h, off.data_ptr(), off.shape[0], out.data_ptr(),
                                             _stream_ptr(stream)), "lgf_table_lookup")
        return out

    def kinv_lookup(self, alpha: float, offsets, stream=None):
        import torch
        off = offsets.to(device=f"cuda:{self.device}", dtype=torch.int32).contiguous()
        out = torch.empty(off.shape[0], dtype=torch.float64, device=off.device)
        self._check(self._L.lgf_kinv_lookup(self._h, float(alpha), off.data_ptr(), off.shape[0], out.data_ptr(),
                                            _stream_ptr(stream)), "lgf_kinv_lookup")
        return out

    def kinv_apply(self, alpha: float, b: int, src, tgt, f, u, ncomp: int = 1, nrhs: int = 1, dx: float = 1.0,
                   stream=None):
        s, sa = _blockset(b, src)
        t, ta = _blockset(b, tgt)
        nf = ncomp * nrhs
        if s.nblocks and t.nblocks:
            self._field(f, s.nblocks, b, nf, "f")
        if t.nblocks:
            self._field(u, t.nblocks, b, nf, "u")
        self._check(self._L.lgf_kinv_apply(self._h, float(alpha), ctypes.byref(s), ctypes.byref(t), _ptr(f),
                                           _ptr(u), ncomp, nrhs, float(dx), _stream_ptr(stream)), "lgf_kinv_apply")
        return u

    def _vector_op(self, name: str, b: int, src, tgt, a, out, nrhs: int, dx: float, stream):
        s, sa = _blockset(b, src)
        t, ta = _blockset(b, tgt)
        if s.nblocks and t.nblocks:
            self._field(a, s.nblocks, b, 3 * nrhs, "input")
        if t.nblocks:
            self._field(out, t.nblocks, b, 3 * nrhs, "output")
        self._check(getattr(self._L, name)(self._h, ctypes.byref(s), ctypes.byref(t), _ptr(a), _ptr(out), int(nrhs),
                                           float(dx), _stream_ptr(stream)), name)
        return out

    def curl(self, b: int, src, tgt, u, w, nrhs: int = 1, dx: float = 1.0, stream=None):
        """w = C u (faces -> edges), [nrhs][3][nblocks][b^3] fields."""
        return self._vector_op("lgf_curl", b, src, tgt, u, w, nrhs, dx, stream)

    def curl_adjoint(self, b: int, src, tgt, w, u, nrhs: int = 1, dx: float = 1.0, stream=None):
        """u = C^dagger w (edges -> faces)."""
        return self._vector_op("lgf_curl_adjoint", b, src, tgt, w, u, nrhs, dx, stream)

    def velocity_refresh(self, b: int, src, tgt, u, u_out, nrhs: int = 1, dx: float = 1.0, stream=None):
        """u_out = -C^dagger L^{-1} C u (Eq. vel_refresh)."""
        return self._vector_op("lgf_velocity_refresh", b, src, tgt, u, u_out, nrhs, dx, stream)

    def _markers(self, X):
        import torch
        if not X.is_cuda or X.dtype != torch.float64 or not X.is_contiguous() or X.dim() != 2 or X.shape[1] != 3:
            raise ValueError("X must be a contiguous CUDA float64 tensor of shape [nmarkers, 3]")
        return X

    def _marker_values(self, t, n, name):
        if t.numel() != n or t.dtype != self.dtype or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA tensor of {n} context-precision values")
        return t

    def ib_spread(self, b: int, blocks, X, g, f, nrhs: int = 1, dx: float = 1.0, stream=None):
        """f = R g: marker values g [nrhs][3][nm] onto the face lattices of the blocks."""
        bs, ba = _blockset(b, blocks)
        X = self._markers(X)
        self._marker_values(g, nrhs * 3 * X.shape[0], "g")
        if bs.nblocks:
            self._field(f, bs.nblocks, b, 3 * nrhs, "f")
        self._check(self._L.lgf_ib_spread(self._h, ctypes.byref(bs), X.shape[0], X.data_ptr(), _ptr(g), _ptr(f),
                                          int(nrhs), float(dx), _stream_ptr(stream)), "lgf_ib_spread")
        return f

    def ib_interp(self, b: int, blocks, X, v, U, nrhs: int = 1, stream=None):
        """U = I v at the markers: [nrhs][3][nm]."""
        bs, ba = _blockset(b, blocks)
        X = self._markers(X)
        if bs.nblocks:
            self._field(v, bs.nblocks, b, 3 * nrhs, "v")
        self._marker_values(U, nrhs * 3 * X.shape[0], "U")
        self._check(self._L.lgf_ib_interp(self._h, ctypes.byref(bs), X.shape[0], X.data_ptr(), _ptr(v), _ptr(U),
                                          int(nrhs), _stream_ptr(stream)), "lgf_ib_interp")
        return U

    def poisson_apply(self, b: int, src, tgt, f, u, ncomp: int = 1, nrhs: int = 1, dx: float = 1.0, stream=None):
        s, sa = _blockset(b, src)
        t, ta = _blockset(b, tgt)
        nf = ncomp * nrhs
        if s.nblocks and t.nblocks:
            self._field(f, s.nblocks, b, nf, "f")
        if t.nblocks:
            self._field(u, t.nblocks, b, nf, "u")
        self._check(self._L.lgf_poisson_apply(self._h, ctypes.byref(s), ctypes.byref(t), _ptr(f), _ptr(u),
                                              ncomp, nrhs, float(dx), _stream_ptr(stream)), "lgf_poisson_apply")
        return u

    def intfactor_apply(self, alpha: float, b: int, src, tgt, f, u, ncomp: int = 1, nrhs: int = 1, stream=None):
        s, sa = _blockset(b, src)
        t, ta = _blockset(b, tgt)
        nf = ncomp * nrhs
        if s.nblocks and t.nblocks:
            self._field(f, s.nblocks, b, nf, "f")
        if t.nblocks:
            self._field(u, t.nblocks, b, nf, "u")
        self._check(self._L.lgf_intfactor_apply(self._h, float(alpha), ctypes.byref(s), ctypes.byref(t), _ptr(f),
                                                _ptr(u), ncomp, nrhs, _stream_ptr(stream)), "lgf_intfactor_apply")
        return u

    def intfactor_weights(self, alpha: float, stream=None):
        import torch
        R = ctypes.c_int32()
        self._check(self._L.lgf_intfactor_weights(self._h, float(alpha), None, 0, ctypes.byref(R),
                                                  _stream_ptr(stream)), "lgf_intfactor_weights")
        w = torch.empty(R.value + 1, dtype=torch.float64, device=f"cuda:{self.device}")
        self._check(self._L.lgf_intfactor_weights(self._h, float(alpha), w.data_ptr(), R.value + 1, ctypes.byref(R),
                                                  _stream_ptr(stream)), "lgf_intfactor_weights")
        return R.value, w

    def batch_apply(self, problems: Sequence[dict], stream=None):
        """problems: dicts with b, src, tgt, f, u, ncomp, nrhs, op, alpha, dx."""
        arr = (lgf_problem * max(1, len(problems)))()
        keep = []
        for i, p in enumerate(problems):
            b = int(p["b"])
            s, sa = _blockset(b, p["src"])
            t, ta = _blockset(b, p["tgt"])
            keep += [sa, ta]
            nf = int(p.get("ncomp", 1)) * int(p.get("nrhs", 1))
            if s.nblocks and t.nblocks:
                self._field(p["f"], s.nblocks, b, nf, f"problem {i} f")
            if t.nblocks:
                self._field(p["u"], t.nblocks, b, nf, f"problem {i} u")
            arr[i] = lgf_problem(s, t, _ptr(p.get("f")), _ptr(p.get("u")), int(p.get("ncomp", 1)),
                                 int(p.get("nrhs", 1)), int(p.get("op", LGF_OP_POISSON)), 0,
                                 float(p.get("alpha", 0.0)), float(p.get("dx", 1.0)))
        self._check(self._L.lgf_batch_apply(self._h, arr, len(problems), _stream_ptr(stream)), "lgf_batch_apply")

    def residual(self, b: int, coords, u, f, dx: float = 1.0, stream=None):
        import torch
        c, ca = _blockset(b, coords)
        self._field(u, c.nblocks, b, 1, "u")
        self._field(f, c.nblocks, b, 1, "f")
        r = torch.empty(c.nblocks * b ** 3, dtype=torch.float64, device=u.device)
        ma, mf = ctypes.c_double(), ctypes.c_double()
        self._check(self._L.lgf_residual(self._h, ctypes.byref(c), u.data_ptr(), f.data_ptr(), float(dx),
                                         r.data_ptr(), ctypes.byref(ma), ctypes.byref(mf), _stream_ptr(stream)),
                    "lgf_residual")
        return r, ma.value, mf.value


    def nested_projection_stage(self, b: int, flow, r, u, X_prev=None, X=None, ub=None, W1=None, W2=None,
                                alpha: float = 0.0, dx: float = 1.0, d=None, f=None, stream=None):
        """One stage of Eq. nested_proj on the block set `flow` (see lgf.h):
        r, u [3][nD][b^3]; d [nD][b^3]; markers X_prev, X [nm, 3] float64;
        ub, f [3][nm]; W1, W2 [3nm, 3nm] (W2 None: W1^T)."""
        bs, ba = _blockset(b, flow)
        nm = 0 if X is None else int(X.shape[0])
        if bs.nblocks:
            self._field(r, bs.nblocks, b, 3, "r")
            self._field(u, bs.nblocks, b, 3, "u")
            if d is not None:
                self._field(d, bs.nblocks, b, 1, "d")
        if nm:
            X = self._markers(X)
            X_prev = self._markers(X_prev)
            if X_prev.shape[0] != nm:
                raise ValueError("X_prev and X must hold the same markers")
            self._marker_values(ub, 3 * nm, "ub")
            if f is not None:
                self._marker_values(f, 3 * nm, "f")
            for name, Wm in (("W1", W1), ("W2", W2)):
                if Wm is not None and (Wm.numel() != 9 * nm * nm or Wm.dtype != self.dtype or not Wm.is_cuda
                                       or not Wm.is_contiguous()):
                    raise ValueError(f"{name} must be a contiguous CUDA [3nm, 3nm] tensor of the context dtype")
            if W1 is None:
                raise ValueError("W1 is required when there are markers")
        st = lgf_stage(bs, nm, _ptr(X_prev) if nm else None, _ptr(X) if nm else None, _ptr(ub) if nm else None,
                       _ptr(W1) if nm else None, _ptr(W2) if nm else None, _ptr(r), _ptr(u), _ptr(d),
                       _ptr(f) if nm else None, float(alpha), float(dx))
        self._check(self._L.lgf_nested_projection_stage(self._h, ctypes.byref(st), _stream_ptr(stream)),
                    "lgf_nested_projection_stage")
        return u

    def autotune(self, mode: int = LGF_TUNE_ON, cache_path: Optional[str] = None):
        """Tuning mode (LGF_TUNE_OFF / ON / CACHED) and the file of persisted
        choices (None: $LGF_TUNE_CACHE, if set)."""
        self._check(self._L.lgf_autotune(self._h, int(mode), None if cache_path is None else cache_path.encode()),
                    "lgf_autotune")

    def tune_report(self) -> dict:
        t = lgf_tune_info()
        self._check(self._L.lgf_tune_report(self._h, ctypes.byref(t)), "lgf_tune_report")
        return {name: (float(getattr(t, name)) if name == "tune_ms" else int(getattr(t, name)))
                for name, _ in lgf_tune_info._fields_ if name != "reserved"}

    def poisson_error_estimate(self, b: int, src, tgt, f, u, ncomp: int = 1, nrhs: int = 1, dx: float = 1.0,
                               nsample: int = 64, stream=None) -> float:
        """Largest relative error of u against the FP64 direct sum at nsample targets."""
        s_, sa = _blockset(b, src)
        t_, ta = _blockset(b, tgt)
        nf = ncomp * nrhs
        if s_.nblocks and t_.nblocks:
            self._field(f, s_.nblocks, b, nf, "f")
            self._field(u, t_.nblocks, b, nf, "u")
        e = ctypes.c_double()
        self._check(self._L.lgf_poisson_error_estimate(self._h, ctypes.byref(s_), ctypes.byref(t_), _ptr(f), _ptr(u),
                                                       ncomp, nrhs, float(dx), int(nsample), ctypes.byref(e),
                                                       _stream_ptr(stream)), "lgf_poisson_error_estimate")
        return e.value

    def table_save(self, path: str):
        self._check(self._L.lgf_table_save(self._h, path.encode()), "lgf_table_save")

    def table_load(self, path: str):
        self._check(self._L.lgf_table_load(self._h, path.encode()), "lgf_table_load")

    def device_status(self) -> int:
        """Synchronise and return (and clear) the device error word; raises
        LgfError (LGF_ETIMEOUT) when a bounded device-side wait ran out."""
        w = ctypes.c_int32()
        self._check(self._L.lgf_device_status(self._h, ctypes.byref(w)), "lgf_device_status")
        return w.value

    def wait_selftest(self, cycles: int = 2000000, stream=None):
        self._check(self._L.lgf_wait_selftest(self._h, int(cycles), _stream_ptr(stream)), "lgf_wait_selftest")

    def stats(self) -> dict:
        """Cache state (lgf_ctx_stats): graphs, plans, spectra, invalidations, scratch."""
        st = lgf_stats()
        self._check(self._L.lgf_ctx_stats(self._h, ctypes.byref(st)), "lgf_ctx_stats")
        return {name: int(getattr(st, name)) for name, _ in lgf_stats._fields_ if name != "reserved"}

    def cache_limits(self, max_plans: int = -1, max_spectra: int = -1, max_graphs: int = -1):
        self._check(self._L.lgf_cache_limits(self._h, int(max_plans), int(max_spectra), int(max_graphs)),
                    "lgf_cache_limits")

    def profile_enable(self, enable: bool = True):
        self._check(self._L.lgf_profile_enable(self._h, 1 if enable else 0), "lgf_profile_enable")

    def profile_read(self) -> dict:
        """{kernel name: (launches, total ms)} since the last read (synchronises)."""
        arr = (lgf_kernel_stat * 64)()
        n = ctypes.c_int32()
        self._check(self._L.lgf_profile_read(self._h, arr, 64, ctypes.byref(n)), "lgf_profile_read")
        return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(min(n.value, 64))}


# Module-level names matching the C ABI.
def lgf_ctx_create(prec: str = "f32", **kw) -> Context:
    return Context(prec, **kw)


def lgf_ctx_destroy(ctx: Context):
    ctx.close()


def lgf_table_build(ctx: Context, max_offset: int = 48, stream=None):
    return ctx.table_build(max_offset, stream)


def lgf_table_info(ctx: Context):
    return ctx.table_info()


def lgf_table_lookup(ctx: Context, offsets, stream=None):
    return ctx.table_lookup(offsets, stream)


def lgf_kinv_lookup(ctx: Context, alpha: float, offsets, stream=None):
    return ctx.kinv_lookup(alpha, offsets, stream)


def lgf_poisson_apply(ctx: Context, *a, **kw):
    return ctx.poisson_apply(*a, **kw)


def lgf_kinv_apply(ctx: Context, *a, **kw):
    return ctx.kinv_apply(*a, **kw)


def lgf_curl(ctx: Context, *a, **kw):
    return ctx.curl(*a, **kw)


def lgf_curl_adjoint(ctx: Context, *a, **kw):
    return ctx.curl_adjoint(*a, **kw)


def lgf_velocity_refresh(ctx: Context, *a, **kw):
    return ctx.velocity_refresh(*a, **kw)


def lgf_ib_spread(ctx: Context, *a, **kw):
    return ctx.ib_spread(*a, **kw)


def lgf_ib_interp(ctx: Context, *a, **kw):
    return ctx.ib_interp(*a, **kw)


def lgf_intfactor_apply(ctx: Context, *a, **kw):
    return ctx.intfactor_apply(*a, **kw)


def lgf_intfactor_weights(ctx: Context, alpha: float, stream=None):
    return ctx.intfactor_weights(alpha, stream)


def lgf_batch_apply(ctx: Context, problems, stream=None):
    return ctx.batch_apply(problems, stream)


def lgf_residual(ctx: Context, *a, **kw):
    return ctx.residual(*a, **kw)


def lgf_profile_enable(ctx: Context, enable: bool = True):
    return ctx.profile_enable(enable)


def lgf_profile_read(ctx: Context) -> dict:
    return ctx.profile_read()


def lgf_ctx_stats(ctx: Context) -> dict:
    return ctx.stats()


def lgf_cache_limits(ctx: Context, max_plans: int = -1, max_spectra: int = -1, max_graphs: int = -1):
    return ctx.cache_limits(max_plans, max_spectra, max_graphs)


def lgf_poisson_error_estimate(ctx: Context, *a, **kw) -> float:
    return ctx.poisson_error_estimate(*a, **kw)


def lgf_table_save(ctx: Context, path: str):
    return ctx.table_save(path)


def lgf_table_load(ctx: Context, path: str):
    return ctx.table_load(path)


def lgf_device_status(ctx: Context) -> int:
    return ctx.device_status()


def lgf_wait_selftest(ctx: Context, cycles: int = 2000000, stream=None):
    return ctx.wait_selftest(cycles, stream)


def lgf_autotune(ctx: Context, mode: int = LGF_TUNE_ON, cache_path: Optional[str] = None):
    return ctx.autotune(mode, cache_path)


def lgf_tune_report(ctx: Context) -> dict:
    return ctx.tune_report()


def lgf_nested_projection_stage(ctx: Context, *a, **kw):
    return ctx.nested_projection_stage(*a, **kw)


def lgf_intfactor_apply_noalloc(prec: str, alpha: float, b: int, src, tgt, f, u, ncomp: int = 1, nrhs: int = 1,
                                tol: float = 0.0, stream=None):
    """Allocation-free integrating factor (no context; see include/lgf.h)."""
    L = load()
    s, sa = _blockset(b, src)
    t, ta = _blockset(b, tgt)
    msg = ctypes.create_string_buffer(256)
    st = L.lgf_intfactor_apply_noalloc({"f32": LGF_F32, "f64": LGF_F64}[prec], float(tol), float(alpha),
                                       ctypes.byref(s), ctypes.byref(t), _ptr(f), _ptr(u), int(ncomp), int(nrhs),
                                       _stream_ptr(stream), msg, 256)
    if st != LGF_OK:
        raise LgfError(st, "lgf_intfactor_apply_noalloc: " + msg.value.decode())
    return u


def lgf_status_string(status: int) -> str:
    return load().lgf_status_string(int(status)).decode()


def lgf_version() -> int:
    return int(load().lgf_version())
