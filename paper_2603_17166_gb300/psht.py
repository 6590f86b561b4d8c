"""Thin ctypes binding of the psht C ABI (include/psht.h).

Only argument marshalling happens here: every step of the transform runs in the CUDA library.
PyTorch provides device memory and streams.  Names follow the C entry points.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

PSHT_AUTO, PSHT_FP64, PSHT_FP32, PSHT_FULL_SKY, PSHT_PATCH_FRAME = 0, 1, 2, 4, 8
_PREC = {"auto": PSHT_AUTO, "fp64": PSHT_FP64, "fp32": PSHT_FP32, 64: PSHT_FP64, 32: PSHT_FP32}


class PshtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"psht error {code}: {msg}")
        self.code = code


class PshtInfo(ctypes.Structure):
    _fields_ = [
        ("spin", ctypes.c_int), ("lmax", ctypes.c_int), ("precision", ctypes.c_int),
        ("pole", ctypes.c_int), ("full_sky", ctypes.c_int),
        ("eps", ctypes.c_double), ("theta_star", ctypes.c_double), ("eps_apo", ctypes.c_double),
        ("theta_max", ctypes.c_double), ("alpha", ctypes.c_double), ("dTheta", ctypes.c_double),
        ("Lmax", ctypes.c_int), ("L", ctypes.c_int), ("nring", ctypes.c_int),
        ("M", ctypes.c_int), ("W", ctypes.c_int), ("beta_es", ctypes.c_double),
        ("nTheta", ctypes.c_int), ("nphi", ctypes.c_int), ("r_lo", ctypes.c_int), ("nrows", ctypes.c_int),
        ("npts", ctypes.c_int64), ("ring_mode_pairs", ctypes.c_int64), ("recursion_triples", ctypes.c_int64),
        ("device_bytes", ctypes.c_size_t), ("patch_frame", ctypes.c_int), ("euler", ctypes.c_double * 3),
    ]


class PshtOptions(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int), ("kappa", ctypes.c_double), ("apodisation", ctypes.c_int)]


_WINDOW = {"es": 0, "kb": 1}
_APO = {"paper": 0, "cost": 1}


class PshtRequest(ctypes.Structure):
    _fields_ = [
        ("op", ctypes.c_int), ("spin", ctypes.c_int), ("lmax", ctypes.c_int), ("eps", ctypes.c_double),
        ("flags", ctypes.c_uint32), ("points_key", ctypes.c_uint64), ("theta", ctypes.c_void_p),
        ("phi", ctypes.c_void_p), ("npts", ctypes.c_int64), ("in_a", ctypes.c_void_p), ("in_b", ctypes.c_void_p),
        ("out_a", ctypes.c_void_p), ("out_b", ctypes.c_void_p),
    ]


class PshtResult(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("worker", ctypes.c_int), ("plan_cached", ctypes.c_int),
        ("precision", ctypes.c_int), ("queue_ms", ctypes.c_double), ("plan_ms", ctypes.c_double),
        ("exec_ms", ctypes.c_double), ("total_ms", ctypes.c_double), ("batch", ctypes.c_int),
        ("message", ctypes.c_char * 192),
    ]


class PshtServerStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
        ("plans_created", ctypes.c_int64), ("cache_hits", ctypes.c_int64), ("evictions", ctypes.c_int64),
        ("budget", ctypes.c_size_t), ("bytes_in_use", ctypes.c_size_t), ("bytes_peak", ctypes.c_size_t),
        ("batches", ctypes.c_int64), ("batched_requests", ctypes.c_int64),
    ]


_lib = None


def lib():
    """Load the in-tree libpsht.so; raise if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "(python -m paper_2603_17166_gb300.build)")
        L = ctypes.CDLL(path)
        P, I, D, I64, U32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_uint32
        L.psht_plan_create.argtypes = [I, I, P, P, I64, D, U32, P, ctypes.POINTER(P)]
        L.psht_plan_info.argtypes = [P, ctypes.POINTER(PshtInfo)]
        for name in ("psht_plan_synthesis", "psht_plan_adjoint", "psht_plan_synthesis_packed",
                     "psht_plan_adjoint_packed", "psht_plan_synthesis_host", "psht_plan_adjoint_host",
                     "psht_plan_ring_coeffs", "psht_plan_synthesis_inframe", "psht_plan_adjoint_inframe"):
            getattr(L, name).argtypes = [P, P, P, P, P]
        L.psht_plan_synthesis_batch.argtypes = [P, I, P, P, P, P]
        L.psht_plan_adjoint_batch.argtypes = [P, I, P, P, P, P]
        L.psht_plan_destroy.argtypes = [P]
        L.psht_plan_rings.argtypes = [P, P, P, P]
        L.psht_synthesis.argtypes = [P, P, I, I, P, P, I64, D, P, P]
        L.psht_adjoint_synthesis.argtypes = [P, I, I, P, P, I64, D, P, P, P]
        L.psht_plan_profile.argtypes = [P, I]
        L.psht_plan_status.argtypes = [P, P, P]
        L.psht_plan_stage_times.argtypes = [P, P, P]
        L.psht_ring_synthesis_noalloc.argtypes = [I, I, P, I, P, P, P, P]
        L.psht_noalloc_scratch_bytes.restype = ctypes.c_size_t
        L.psht_plan_create_ex.argtypes = [I, I, P, P, I64, D, U32, ctypes.POINTER(PshtOptions), P, ctypes.POINTER(P)]
        L.psht_predict_error.argtypes = [I, I, D, D, ctypes.POINTER(PshtOptions), P, P, I, P, P]
        L.psht_plan_estimate_points.argtypes = [I, I, P, P, I64, D, U32, P, ctypes.POINTER(ctypes.c_size_t)]
        L.psht_server_create.argtypes = [I, ctypes.c_size_t, ctypes.POINTER(P)]
        L.psht_server_submit.argtypes = [P, ctypes.POINTER(PshtRequest), ctypes.POINTER(I64)]
        L.psht_server_wait.argtypes = [P, I64, ctypes.POINTER(PshtResult)]
        L.psht_server_get_stats.argtypes = [P, ctypes.POINTER(PshtServerStats)]
        L.psht_server_destroy.argtypes = [P]
        L.psht_server_set_batch_limit.argtypes = [P, I]
        L.psht_estimate_bytes.argtypes = [I, I, D, I64, D, U32]
        L.psht_plan_params.argtypes = [I, I, D, D, U32, ctypes.POINTER(PshtOptions), ctypes.POINTER(PshtInfo), P, P,
                                       P]
        L.psht_rotator_create.argtypes = [I, U32, P, ctypes.POINTER(P)]
        L.psht_rotator_apply.argtypes = [P, D, D, D, P, P, P, P, P]
        L.psht_rotator_destroy.argtypes = [P]
        L.psht_rotator_bytes.argtypes = [I, U32]
        L.psht_rotator_bytes.restype = ctypes.c_size_t
        L.psht_rotate_alm.argtypes = [I, D, D, D, P, P, P, P, U32, P]
        L.psht_rotate_points.argtypes = [D, D, D, P, P, I64, P, P, P, P]
        L.psht_patch_rotation.argtypes = [P, P, I64, P, P, P]
        L.psht_estimate_bytes.restype = ctypes.c_size_t
        L.psht_last_error.restype = ctypes.c_char_p
        L.psht_version.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise PshtError(rc, lib().psht_last_error().decode())


def _torch():
    import torch

    return torch


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def nalm(lmax: int) -> int:
    return (lmax + 1) * (lmax + 2) // 2


class Plan:
    """A plan for synthesis general and its adjoint at fixed points (psht_plan_create)."""

    def __init__(self, spin: int, lmax: int, theta, phi, eps: float, precision="auto", stream=None,
                 full_sky: bool = False, window: str = "es", kappa: float = 1.0, patch_frame: bool = False,
                 apodisation: str = "paper"):
        torch = _torch()
        theta = torch.as_tensor(theta, dtype=torch.float64, device="cuda").contiguous()
        phi = torch.as_tensor(phi, dtype=torch.float64, device="cuda").contiguous()
        if theta.shape != phi.shape or theta.dim() != 1:
            raise ValueError("theta and phi must be 1-D tensors of equal length")
        self._h = ctypes.c_void_p()
        flags = _PREC[precision] | (PSHT_FULL_SKY if full_sky else 0) | (PSHT_PATCH_FRAME if patch_frame else 0)
        if window == "es" and kappa == 1.0 and apodisation == "paper":
            _check(lib().psht_plan_create(int(spin), int(lmax), _ptr(theta), _ptr(phi), theta.numel(), float(eps),
                                          flags, _stream(stream), ctypes.byref(self._h)))
        else:
            opt = PshtOptions(_WINDOW[window], float(kappa), _APO[apodisation])
            _check(lib().psht_plan_create_ex(int(spin), int(lmax), _ptr(theta), _ptr(phi), theta.numel(),
                                             float(eps), flags, ctypes.byref(opt), _stream(stream),
                                             ctypes.byref(self._h)))
        self.spin, self.lmax, self.eps, self.npts = int(spin), int(lmax), float(eps), theta.numel()
        i = self.info
        self.precision = i["precision"]
        self.cdtype = torch.complex128 if self.precision == 64 else torch.complex64
        self.np_cdtype = np.complex128 if self.precision == 64 else np.complex64

    @property
    def info(self) -> dict:
        inf = PshtInfo()
        _check(lib().psht_plan_info(self._h, ctypes.byref(inf)))
        d = {name: getattr(inf, name) for name, _ in PshtInfo._fields_}
        d["euler"] = tuple(d["euler"])
        return d

    def _alm_in(self, a):
        torch = _torch()
        if a is None:
            return None
        a = torch.as_tensor(a, device="cuda").to(self.cdtype).contiguous()
        if a.numel() != nalm(self.lmax):
            raise ValueError(f"a_lm must hold {nalm(self.lmax)} packed coefficients")
        return a

    def synthesis(self, g, c=None, out=None, stream=None, packed_grad: bool = False, in_frame: bool = False):
        """f_p = -sum (g_lm + i c_lm) sY_lm(theta_p, phi_p) (psht_plan_synthesis); with packed_grad
        the m > 0 inputs count half (psht_plan_synthesis_packed); with in_frame the a_lm are in a
        patch-frame plan's own frame (psht_plan_synthesis_inframe)."""
        torch = _torch()
        g, c = self._alm_in(g), self._alm_in(c)
        f = out if out is not None else torch.empty(self.npts, dtype=self.cdtype, device="cuda")
        if in_frame and packed_grad:
            raise ValueError("in_frame and packed_grad do not combine")
        fn = lib().psht_plan_synthesis_packed if packed_grad else lib().psht_plan_synthesis
        if in_frame:
            fn = lib().psht_plan_synthesis_inframe
        _check(fn(self._h, _ptr(g), _ptr(c), _ptr(f), _stream(stream)))
        return f

    def adjoint(self, f, g_out=None, c_out=None, want_c: bool = True, stream=None, packed_grad: bool = False,
                in_frame: bool = False):
        """(g~, c~) of adjoint synthesis general (psht_plan_adjoint); with packed_grad the m > 0
        outputs are doubled (psht_plan_adjoint_packed); with in_frame they stay in a patch-frame
        plan's own frame (psht_plan_adjoint_inframe)."""
        torch = _torch()
        f = torch.as_tensor(f, device="cuda").to(self.cdtype).contiguous()
        if f.numel() != self.npts:
            raise ValueError("f must hold one value per point")
        n = nalm(self.lmax)
        g = g_out if g_out is not None else torch.empty(n, dtype=self.cdtype, device="cuda")
        c = (c_out if c_out is not None else torch.empty(n, dtype=self.cdtype, device="cuda")) if want_c else None
        if in_frame and packed_grad:
            raise ValueError("in_frame and packed_grad do not combine")
        fn = lib().psht_plan_adjoint_packed if packed_grad else lib().psht_plan_adjoint
        if in_frame:
            fn = lib().psht_plan_adjoint_inframe
        _check(fn(self._h, _ptr(f), _ptr(g), _ptr(c), _stream(stream)))
        return g, c

    def synthesis_batch(self, gs, cs=None, outs=None, stream=None):
        """Synthesis of several a_lm sets on this plan (psht_plan_synthesis_batch): the sets share the
        Wigner-d recursion's column evaluations.  gs: list of packed a_lm; cs: None or a list of
        the same length (entries may be None); returns the list of maps."""
        torch = _torch()
        n = len(gs)
        gs = [self._alm_in(g) for g in gs]
        cs = [None] * n if cs is None else [self._alm_in(c) for c in cs]
        if len(cs) != n:
            raise ValueError("gs and cs must have the same length")
        fs = list(outs) if outs is not None else [torch.empty(self.npts, dtype=self.cdtype, device="cuda")
                                                    for _ in range(n)]
        for f in fs:
            if f.numel() != self.npts or f.dtype != self.cdtype or not f.is_contiguous():
                raise ValueError("outs must be contiguous tensors of one value per point in the plan's precision")
        arr = ctypes.c_void_p * n
        ga = arr(*[g.data_ptr() for g in gs])
        ca = arr(*[0 if c is None else c.data_ptr() for c in cs])
        fa = arr(*[f.data_ptr() for f in fs])
        _check(lib().psht_plan_synthesis_batch(self._h, n, ga, None if all(c is None for c in cs) else ca, fa,
                                               _stream(stream)))
        return fs

    def adjoint_batch(self, fs, want_c: bool = True, stream=None):
        """Adjoint of several maps on this plan (psht_plan_adjoint_batch) -> list of (g~, c~)."""
        torch = _torch()
        n = len(fs)
        fs = [torch.as_tensor(f, device="cuda").to(self.cdtype).contiguous() for f in fs]
        for f in fs:
            if f.numel() != self.npts:
                raise ValueError("f must hold one value per point")
        na = nalm(self.lmax)
        gs = [torch.empty(na, dtype=self.cdtype, device="cuda") for _ in range(n)]
        cs = [torch.empty(na, dtype=self.cdtype, device="cuda") for _ in range(n)] if want_c else None
        arr = ctypes.c_void_p * n
        _check(lib().psht_plan_adjoint_batch(self._h, n, arr(*[f.data_ptr() for f in fs]),
                                             arr(*[g.data_ptr() for g in gs]),
                                             None if cs is None else arr(*[c.data_ptr() for c in cs]),
                                             _stream(stream)))
        return [(g, None if cs is None else cs[k]) for k, g in enumerate(gs)]

    def synthesis_host(self, g: np.ndarray, c, f: np.ndarray, stream=None):
        """Host-buffer synthesis (psht_plan_synthesis_host); g, c, f numpy arrays (pinned memory ok)."""
        _check(lib().psht_plan_synthesis_host(self._h, ctypes.c_void_p(g.ctypes.data),
                                              None if c is None else ctypes.c_void_p(c.ctypes.data),
                                              ctypes.c_void_p(f.ctypes.data), _stream(stream)))
        return f

    def adjoint_host(self, f: np.ndarray, g: np.ndarray, c, stream=None):
        _check(lib().psht_plan_adjoint_host(self._h, ctypes.c_void_p(f.ctypes.data), ctypes.c_void_p(g.ctypes.data),
                                            None if c is None else ctypes.c_void_p(c.ctypes.data), _stream(stream)))
        return g, c

    def rings(self):
        """(theta_j, w_j, M_j) of the planner (psht_plan_rings)."""
        n = self.info["nring"]
        th, w, mj = np.zeros(n), np.zeros(n), np.zeros(n, dtype=np.int32)
        _check(lib().psht_plan_rings(self._h, ctypes.c_void_p(th.ctypes.data), ctypes.c_void_p(w.ctypes.data),
                                     ctypes.c_void_p(mj.ctypes.data)))
        return th, w, mj

    def ring_coeffs(self, g, c=None, stream=None):
        """Ring Fourier coefficients F[j, m + M] (psht_plan_ring_coeffs)."""
        torch = _torch()
        i = self.info
        g, c = self._alm_in(g), self._alm_in(c)
        F = torch.empty((i["nring"], 2 * i["M"] + 1), dtype=self.cdtype, device="cuda")
        _check(lib().psht_plan_ring_coeffs(self._h, _ptr(g), _ptr(c), _ptr(F), _stream(stream)))
        return F

    STAGES = ("rec_synthesis", "theta_synthesis", "phi_synthesis", "gather", "scatter", "phi_adjoint",
              "theta_adjoint", "rec_adjoint")

    def profile(self, enable: bool = True):
        """Record CUDA events around each stage of later calls (psht_plan_profile)."""
        _check(lib().psht_plan_profile(self._h, 1 if enable else 0))

    def stage_times(self) -> dict:
        """{stage: (summed ms, launches)} since the last call (psht_plan_stage_times)."""
        ms = np.zeros(8)
        calls = np.zeros(8, dtype=np.int64)
        _check(lib().psht_plan_stage_times(self._h, ctypes.c_void_p(ms.ctypes.data), ctypes.c_void_p(calls.ctypes.data)))
        return {name: (float(ms[i]), int(calls[i])) for i, name in enumerate(self.STAGES)}

    def status(self, stream=None) -> int:
        """0 if every bounded wait in earlier calls completed (psht_plan_status); clears it."""
        st = ctypes.c_int(0)
        _check(lib().psht_plan_status(self._h, ctypes.byref(st), _stream(stream)))
        return st.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().psht_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def synthesis(g, c, spin: int, lmax: int, theta, phi, eps: float, stream=None):
    """One-shot synthesis general (psht_synthesis); precision chosen from eps."""
    torch = _torch()
    theta = torch.as_tensor(theta, dtype=torch.float64, device="cuda").contiguous()
    phi = torch.as_tensor(phi, dtype=torch.float64, device="cuda").contiguous()
    cd = torch.complex64 if eps >= 1e-5 else torch.complex128
    g = torch.as_tensor(g, device="cuda").to(cd).contiguous()
    c = None if c is None else torch.as_tensor(c, device="cuda").to(cd).contiguous()
    f = torch.empty(theta.numel(), dtype=cd, device="cuda")
    _check(lib().psht_synthesis(_ptr(g), _ptr(c), int(spin), int(lmax), _ptr(theta), _ptr(phi), theta.numel(),
                                float(eps), _ptr(f), _stream(stream)))
    return f


def adjoint_synthesis(f, spin: int, lmax: int, theta, phi, eps: float, stream=None):
    """One-shot adjoint synthesis general (psht_adjoint_synthesis) -> (g~, c~)."""
    torch = _torch()
    theta = torch.as_tensor(theta, dtype=torch.float64, device="cuda").contiguous()
    phi = torch.as_tensor(phi, dtype=torch.float64, device="cuda").contiguous()
    cd = torch.complex64 if eps >= 1e-5 else torch.complex128
    f = torch.as_tensor(f, device="cuda").to(cd).contiguous()
    g = torch.empty(nalm(lmax), dtype=cd, device="cuda")
    c = torch.empty(nalm(lmax), dtype=cd, device="cuda")
    _check(lib().psht_adjoint_synthesis(_ptr(f), int(spin), int(lmax), _ptr(theta), _ptr(phi), theta.numel(),
                                        float(eps), _ptr(g), _ptr(c), _stream(stream)))
    return g, c


def estimate_bytes(spin: int, lmax: int, theta_star: float, npts: int, eps: float, precision="auto") -> int:
    return int(lib().psht_estimate_bytes(int(spin), int(lmax), float(theta_star), int(npts), float(eps),
                                         _PREC[precision]))


def ring_synthesis_noalloc(spin: int, lmax: int, theta_rings, g, c=None, out=None, stream=None):
    """Ring Fourier coefficients F[j, m + lmax] at the given ring colatitudes without allocating
    inside the library (psht_ring_synthesis_noalloc): FP64, lmax <= 511, at most 4096 rings.
    The library's fixed scratch array is shared by all calls; order overlapping calls yourself."""
    torch = _torch()
    th = torch.as_tensor(theta_rings, dtype=torch.float64, device="cuda").contiguous()
    if th.dim() != 1:
        raise ValueError("theta_rings must be a 1-D array of ring colatitudes")
    g = torch.as_tensor(g, device="cuda").to(torch.complex128).contiguous()
    c = None if c is None else torch.as_tensor(c, device="cuda").to(torch.complex128).contiguous()
    # the C entry point takes no buffer sizes: check them here, before anything reaches the device
    n = nalm(int(lmax))
    if g.numel() != n or (c is not None and c.numel() != n):
        raise ValueError(f"g and c must hold nalm(lmax) = {n} packed coefficients")
    shape = (th.numel(), 2 * int(lmax) + 1)
    if out is not None:
        if (not out.is_cuda or out.dtype != torch.complex128 or tuple(out.shape) != shape
                or not out.is_contiguous()):
            raise ValueError(f"out must be a contiguous complex128 CUDA tensor of shape {shape}")
        F = out
    else:
        F = torch.empty(shape, dtype=torch.complex128, device="cuda")
    _check(lib().psht_ring_synthesis_noalloc(int(spin), int(lmax), _ptr(th), th.numel(), _ptr(g), _ptr(c), _ptr(F),
                                             _stream(stream)))
    return F


class Server:
    """Request server of the library (psht_server_*): nstreams workers, a plan cache and admission
    against a device-memory budget (bytes; 0 = 80 % of the free memory).  submit() takes device
    tensors, which the caller keeps alive until wait() has returned for the ticket."""

    SYNTHESIS, ADJOINT = 0, 1

    def __init__(self, nstreams: int = 4, budget_bytes: int = 0, max_batch: int = 8):
        _torch().cuda.current_device()
        self._h = ctypes.c_void_p()
        _check(lib().psht_server_create(int(nstreams), int(budget_bytes), ctypes.byref(self._h)))
        self._keep = {}
        if max_batch != 8:
            self.set_batch_limit(max_batch)

    def set_batch_limit(self, max_batch: int):
        """Largest batch the workers form (psht_server_set_batch_limit; 1 = no batching)."""
        _check(lib().psht_server_set_batch_limit(self._h, int(max_batch)))

    def submit(self, op: int, points_key: int, spin: int, lmax: int, eps: float, theta, phi, in_a, in_b=None,
               out_a=None, out_b=None, precision="auto") -> int:
        r = PshtRequest(int(op), int(spin), int(lmax), float(eps), _PREC[precision], int(points_key),
                        theta.data_ptr(), phi.data_ptr(), theta.numel(), in_a.data_ptr(),
                        None if in_b is None else in_b.data_ptr(), out_a.data_ptr(),
                        None if out_b is None else out_b.data_ptr())
        t = ctypes.c_int64()
        _check(lib().psht_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        self._keep[t.value] = (theta, phi, in_a, in_b, out_a, out_b)
        return t.value

    def wait(self, ticket: int) -> dict:
        res = PshtResult()
        _check(lib().psht_server_wait(self._h, int(ticket), ctypes.byref(res)))
        self._keep.pop(ticket, None)
        out = {name: getattr(res, name) for name, _ in PshtResult._fields_}
        out["message"] = res.message.decode(errors="replace")
        return out

    def stats(self) -> dict:
        st = PshtServerStats()
        _check(lib().psht_server_get_stats(self._h, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in PshtServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().psht_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def estimate_points(spin: int, lmax: int, theta, phi, eps: float, precision="auto", stream=None) -> int:
    """Device bytes of a plan for these points (psht_plan_estimate_points)."""
    b = ctypes.c_size_t()
    _check(lib().psht_plan_estimate_points(int(spin), int(lmax), _ptr(theta), _ptr(phi), theta.numel(), float(eps),
                                           _PREC[precision], _stream(stream), ctypes.byref(b)))
    return b.value


def predict_error(spin: int, lmax: int, theta_star: float, eps: float, cl, beta, window: str = "es",
                  kappa: float = 1.0, stream=None) -> np.ndarray:
    """Predicted relative rms error of the partial-sky route at angles beta from the pole for an
    isotropic field with spectrum cl (psht_predict_error)."""
    cl = np.ascontiguousarray(cl, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    if cl.size != lmax + 1:
        raise ValueError("cl must hold lmax + 1 values")
    out = np.zeros(beta.size)
    opt = PshtOptions(_WINDOW[window], float(kappa), 0)
    _check(lib().psht_predict_error(int(spin), int(lmax), float(theta_star), float(eps), ctypes.byref(opt),
                                    ctypes.c_void_p(cl.ctypes.data), ctypes.c_void_p(beta.ctypes.data), beta.size,
                                    ctypes.c_void_p(out.ctypes.data), _stream(stream)))
    return out


class Rotator:
    """Wigner-D rotation of a_lm sets at one band limit (psht_rotator_create / _apply)."""

    def __init__(self, lmax: int, precision="fp64", stream=None):
        self.lmax = int(lmax)
        self.precision = 32 if _PREC[precision] == PSHT_FP32 else 64
        self._h = ctypes.c_void_p()
        _check(lib().psht_rotator_create(self.lmax, _PREC[precision], _stream(stream), ctypes.byref(self._h)))
        torch = _torch()
        self.cdtype = torch.complex128 if self.precision == 64 else torch.complex64

    def _in(self, a):
        torch = _torch()
        if a is None:
            return None
        a = torch.as_tensor(a, device="cuda").to(self.cdtype).contiguous()
        if a.numel() != nalm(self.lmax):
            raise ValueError(f"a_lm must hold {nalm(self.lmax)} packed coefficients")
        return a

    def apply(self, g, c=None, alpha: float = 0.0, beta: float = 0.0, gamma: float = 0.0, g_out=None, c_out=None,
              stream=None):
        """Rotated (g', c') = D(alpha, beta, gamma) (g, c); c may be None."""
        torch = _torch()
        g, c = self._in(g), self._in(c)
        go = g_out if g_out is not None else torch.empty_like(g)
        co = None if c is None else (c_out if c_out is not None else torch.empty_like(c))
        _check(lib().psht_rotator_apply(self._h, float(alpha), float(beta), float(gamma), _ptr(g), _ptr(c), _ptr(go),
                                        _ptr(co), _stream(stream)))
        return go, co

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().psht_rotator_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rotate_alm(g, c=None, alpha: float = 0.0, beta: float = 0.0, gamma: float = 0.0, lmax: int = None,
               precision=None, stream=None):
    """One-shot rotation of packed a_lm (psht_rotate_alm); precision follows g's dtype by default."""
    torch = _torch()
    g = torch.as_tensor(g, device="cuda")
    if precision is None:
        precision = "fp32" if g.dtype == torch.complex64 else "fp64"
    cd = torch.complex64 if _PREC[precision] == PSHT_FP32 else torch.complex128
    g = g.to(cd).contiguous()
    c = None if c is None else torch.as_tensor(c, device="cuda").to(cd).contiguous()
    if lmax is None:
        lmax = int(round((np.sqrt(8 * g.numel() + 1) - 3) / 2))
    if g.numel() != nalm(lmax) or (c is not None and c.numel() != nalm(lmax)):
        raise ValueError(f"a_lm must hold {nalm(lmax)} packed coefficients")
    go = torch.empty_like(g)
    co = None if c is None else torch.empty_like(c)
    _check(lib().psht_rotate_alm(int(lmax), float(alpha), float(beta), float(gamma), _ptr(g), _ptr(c), _ptr(go),
                                 _ptr(co), _PREC[precision], _stream(stream)))
    return go, co


def rotate_points(theta, phi, alpha: float, beta: float, gamma: float, want_psi: bool = True, stream=None):
    """Rotated points (theta', phi') and the spin-basis angle psi (psht_rotate_points)."""
    torch = _torch()
    theta = torch.as_tensor(theta, dtype=torch.float64, device="cuda").contiguous()
    phi = torch.as_tensor(phi, dtype=torch.float64, device="cuda").contiguous()
    t2, p2 = torch.empty_like(theta), torch.empty_like(phi)
    psi = torch.empty_like(theta) if want_psi else None
    _check(lib().psht_rotate_points(float(alpha), float(beta), float(gamma), _ptr(theta), _ptr(phi), theta.numel(),
                                    _ptr(t2), _ptr(p2), _ptr(psi), _stream(stream)))
    return t2, p2, psi


def patch_rotation(theta, phi, stream=None):
    """Euler angles of the rotation taking the centre of the points' smallest cap to the north pole,
    and the cap radius (psht_patch_rotation)."""
    torch = _torch()
    theta = torch.as_tensor(theta, dtype=torch.float64, device="cuda").contiguous()
    phi = torch.as_tensor(phi, dtype=torch.float64, device="cuda").contiguous()
    eul = (ctypes.c_double * 3)()
    ts = ctypes.c_double()
    _check(lib().psht_patch_rotation(_ptr(theta), _ptr(phi), theta.numel(), eul, ctypes.byref(ts), _stream(stream)))
    return (eul[0], eul[1], eul[2]), ts.value


def plan_params(spin: int, lmax: int, theta_star: float, eps: float, precision="auto", full_sky: bool = False,
                window: str = "es", kappa: float = 1.0, apodisation: str = "paper", patch_frame: bool = False):
    """The planner's parameters and ring set for theta_star about the north pole, on the host
    (psht_plan_params): (info dict, theta_j, w_j, Mj)."""
    flags = _PREC[precision] | (PSHT_FULL_SKY if full_sky else 0) | (PSHT_PATCH_FRAME if patch_frame else 0)
    opt = PshtOptions(_WINDOW[window], float(kappa), _APO[apodisation])
    inf = PshtInfo()
    _check(lib().psht_plan_params(int(spin), int(lmax), float(theta_star), float(eps), flags, ctypes.byref(opt),
                                  ctypes.byref(inf), None, None, None))
    n = inf.nring
    th, w, mj = np.zeros(n), np.zeros(n), np.zeros(n, dtype=np.int32)
    _check(lib().psht_plan_params(int(spin), int(lmax), float(theta_star), float(eps), flags, ctypes.byref(opt),
                                  ctypes.byref(inf), ctypes.c_void_p(th.ctypes.data), ctypes.c_void_p(w.ctypes.data),
                                  ctypes.c_void_p(mj.ctypes.data)))
    d = {name: getattr(inf, name) for name, _ in PshtInfo._fields_}
    d["euler"] = tuple(d["euler"])
    return d, th, w, mj
