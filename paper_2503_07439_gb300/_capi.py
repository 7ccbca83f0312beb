"""ctypes marshalling for the C ABI in include/me.h (no computation here)."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

ME_OK = 0
ME_ERR_ARG = -1
ME_ERR_OOM = -2
ME_ERR_PROCESS = -3
ME_ERR_TIMEOUT = -4
ME_ERR_CUDA = -5
ME_ERR_BUSY = -6
ME_PREC_FP64 = 0
ME_PREC_MIXED = 1
ME_PARAMS_VERSION = 4
ME_RESCUE_POINTS = 0
ME_RESCUE_ITEMS = 1
ME_TERMS_MASKED, ME_TERMS_QUEUED, ME_TERMS_AUTO = 0, 1, 2
ME_KIND_BORN = 0
ME_KIND_REAL_SUBTRACTED = 1
ME_KIND_NBODY_NLO = 2
KINDS = {"born": ME_KIND_BORN, "real_subtracted": ME_KIND_REAL_SUBTRACTED, "nbody_nlo": ME_KIND_NBODY_NLO}

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libme_gb300.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "me.h")


class MEError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class MEParams(ctypes.Structure):
    _fields_ = [("version", ctypes.c_uint32), ("precision", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("alpha_s", ctypes.c_double), ("mt", ctypes.c_double), ("xi_cut", ctypes.c_double),
                ("delta", ctypes.c_double), ("xi_thr", ctypes.c_double), ("y_thr", ctypes.c_double),
                ("tol", ctypes.c_double), ("me_eps", ctypes.c_double), ("device", ctypes.c_int32),
                ("lanes_per_event", ctypes.c_int32), ("queued_rescue", ctypes.c_int32),
                ("rescue", ctypes.c_int32), ("term_queues", ctypes.c_int32), ("cut_pt_min", ctypes.c_double),
                ("cut_abs_y_max", ctypes.c_double), ("cut_abs_cos_axis_max", ctypes.c_double),
                ("cut_thrust_max", ctypes.c_double)]


class MEServerParams(ctypes.Structure):
    _fields_ = [("version", ctypes.c_uint32), ("device", ctypes.c_int32), ("n_slots", ctypes.c_int32),
                ("max_queue", ctypes.c_int32), ("mem_budget_bytes", ctypes.c_int64), ("params", MEParams),
                ("use_graphs", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("persistent_idle_us", ctypes.c_int32)]


class MERequest(ctypes.Structure):
    _fields_ = [("process", ctypes.c_char_p), ("kind", ctypes.c_int32), ("momenta", ctypes.c_void_p),
                ("ps_weights", ctypes.c_void_p), ("n", ctypes.c_int64), ("out", ctypes.c_void_p)]


class MEResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n", ctypes.c_int64), ("n_rescued", ctypes.c_int64),
                ("sum_w", ctypes.c_double), ("sum_w2", ctypes.c_double), ("t_queue_us", ctypes.c_double),
                ("t_device_us", ctypes.c_double), ("t_total_us", ctypes.c_double)]


_lib = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load the CUDA library (fails loudly if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} not found: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    sig = {
        "me_default_params": (None, [ctypes.POINTER(MEParams)]),
        "me_init": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(MEParams), ctypes.POINTER(vp)]),
        "me_n_external": (ctypes.c_int, [vp]),
        "me_eval_born": (ctypes.c_int, [vp, vp, vp, i64, vp]),
        "me_eval_nbody_nlo": (ctypes.c_int, [vp, vp, vp, i64, vp]),
        "me_eval_real_subtracted": (ctypes.c_int, [vp, vp, vp, i64, vp]),
        "me_last_rescued": (ctypes.c_int, [vp, ctypes.POINTER(i64)]),
        "me_last_rescue_work": (ctypes.c_int, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "me_last_rescue_configs": (ctypes.c_int, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "me_get_accumulators": (ctypes.c_int, [vp, dp]),
        "me_set_accumulators": (ctypes.c_int, [vp, dp]),
        "me_set_stream": (ctypes.c_int, [vp, vp]),
        "me_enable_stage_timers": (ctypes.c_int, [vp, ctypes.c_int]),
        "me_stage_times": (ctypes.c_int, [vp, dp, ctypes.POINTER(i64)]),
        "me_synchronize": (ctypes.c_int, [vp]),
        "me_destroy": (None, [vp]),
        "me_last_error": (ctypes.c_char_p, []),
        "me_default_server_params": (None, [ctypes.POINTER(MEServerParams)]),
        "me_server_create": (ctypes.c_int, [ctypes.POINTER(MEServerParams), ctypes.POINTER(vp)]),
        "me_submit": (ctypes.c_int, [vp, ctypes.POINTER(MERequest), ctypes.POINTER(ctypes.c_uint64)]),
        "me_poll": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.POINTER(MEResult), i64]),
        "me_server_destroy": (None, [vp]),
        "me_server_stats": (ctypes.c_int, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "me_server_persistent_stats": (ctypes.c_int, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                                      ctypes.POINTER(i64)]),
        "me_generate_flat": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_uint32, i64, ctypes.c_double, i64, vp, vp]),
        "me_generate_fks": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_uint32, i64, ctypes.c_double, i64, vp, vp]),
        "me_unweight": (ctypes.c_int, [vp, vp, i64, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32, i64, vp, vp,
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int64)]),
        "me_eval_real_subtracted_noalloc": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(MEParams), vp, vp, i64,
                                                           vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def library() -> ctypes.CDLL:
    return load_library()


def declared_symbols(header: str = HEADER) -> list[str]:
    """Function names declared in the C header."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(me_[a-z0-9_]+)\s*\(", text)))


def _check(rc: int):
    if rc != ME_OK:
        raise MEError(rc, library().me_last_error().decode())


def default_params(**kw) -> MEParams:
    p = MEParams()
    library().me_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(x):
    """(address, keepalive) of a numpy array or torch tensor (host or CUDA)."""
    if x is None:
        return None, None
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            x = np.ascontiguousarray(x, dtype=np.float64)
        return x.ctypes.data, x
    if hasattr(x, "data_ptr"):  # torch.Tensor
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError("tensors must be contiguous float64")
        return x.data_ptr(), x
    raise TypeError(type(x))


class Handle:
    """One process on one device (me_init ... me_destroy)."""

    def __init__(self, process: str, precision: int = ME_PREC_FP64, **params):
        self.lib = library()
        self.params = default_params(precision=precision, **params)
        h = ctypes.c_void_p()
        _check(self.lib.me_init(process.encode(), ctypes.byref(self.params), ctypes.byref(h)))
        self.h = h
        self.process = process
        self.n_ext = self.lib.me_n_external(self.h)
        # with device buffers the library returns once the work is enqueued on its
        # stream; unless the caller hands in its own stream, wait for it here
        self.sync = True

    def _call(self, fn, p, w, out):
        n = p.shape[-1]
        if p.shape[:2] != (4, self.n_ext):
            raise ValueError(f"momenta must be [4][{self.n_ext}][n], got {tuple(p.shape)}")
        if out is None:
            if isinstance(p, np.ndarray):
                out = np.empty(n)
            else:
                import torch
                out = torch.empty(n, dtype=torch.float64, device=p.device)
        pp, kp = _ptr(p)
        wp, kw = _ptr(w)
        op, ko = _ptr(out)
        _check(fn(self.h, pp, wp, n, op))
        if self.sync:
            _check(self.lib.me_synchronize(self.h))
        if isinstance(out, np.ndarray) and ko is not out:
            out[...] = ko
        return out

    def born(self, p, w=None, out=None):
        return self._call(self.lib.me_eval_born, p, w, out)

    def nbody_nlo(self, p, w=None, out=None):
        return self._call(self.lib.me_eval_nbody_nlo, p, w, out)

    def real_subtracted(self, p, w=None, out=None):
        return self._call(self.lib.me_eval_real_subtracted, p, w, out)

    def _generate(self, fn, n, seed, sqrt_s, first_point, stream, out):
        import torch
        if out is None:
            p = torch.empty((4, self.n_ext, n), dtype=torch.float64, device=f"cuda:{self.params.device}")
            w = torch.empty(n, dtype=torch.float64, device=p.device)
        else:
            p, w = out
        _check(fn(self.h, seed, stream, first_point, float(sqrt_s), n, ctypes.c_void_p(p.data_ptr()),
                  ctypes.c_void_p(w.data_ptr())))
        if self.sync:
            _check(self.lib.me_synchronize(self.h))
        return p, w

    def generate_flat(self, n: int, seed: int, sqrt_s: float, first_point: int = 0, stream: int = 0, out=None):
        """Flat phase-space points of this process generated on the device (torch tensors
        momenta [4][n_ext][n] and weights [n] on the handle's device, or `out` = (p, w))."""
        return self._generate(self.lib.me_generate_flat, n, seed, sqrt_s, first_point, stream, out)

    def generate_fks(self, n: int, seed: int, sqrt_s: float, first_point: int = 0, stream: int = 0, out=None):
        """Real-emission points generated on the device in FKS-sector variables (soft and
        collinear regions sampled more densely; multichannel weights), as generate_flat."""
        return self._generate(self.lib.me_generate_fks, n, seed, sqrt_s, first_point, stream, out)

    def unweight(self, w, w_max: float = 0.0, seed: int = 0, stream: int = 1, first_point: int = 0):
        """Unweighted events from the device weights `w` (torch float64 CUDA tensor):
        (indices of the kept points, their event weights, w_max applied, overweight count).
        w_max <= 0 takes the batch maximum of |w|."""
        import torch
        n = int(w.shape[0])
        kept = torch.empty(max(n, 1), dtype=torch.int32, device=w.device)
        kw = torch.empty(max(n, 1), dtype=torch.float64, device=w.device)
        nk, wm, no = ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64()
        wp, _keep = _ptr(w)
        _check(self.lib.me_unweight(self.h, wp, n, float(w_max), seed, stream, first_point,
                                    ctypes.c_void_p(kept.data_ptr()), ctypes.c_void_p(kw.data_ptr()),
                                    ctypes.byref(nk), ctypes.byref(wm), ctypes.byref(no)))
        return kept[:nk.value], kw[:nk.value], wm.value, no.value

    def last_rescued(self) -> int:
        v = ctypes.c_int64()
        _check(self.lib.me_last_rescued(self.h, ctypes.byref(v)))
        return v.value

    def last_rescue_work(self) -> tuple[int, int, int]:
        """(flagged points, real blocks, Born-value sets) re-evaluated in float64 by the
        last subtracted-real call (item rescue)."""
        v = [ctypes.c_int64() for _ in range(3)]
        _check(self.lib.me_last_rescue_work(self.h, *(ctypes.byref(x) for x in v)))
        return tuple(x.value for x in v)

    def last_rescue_configs(self) -> tuple[int, int]:
        """Float64 Born configurations of the last subtracted-real call that ran the
        per-term queues: (soft or sector-1, collinear or sector-2)."""
        v = [ctypes.c_int64() for _ in range(2)]
        _check(self.lib.me_last_rescue_configs(self.h, *(ctypes.byref(x) for x in v)))
        return tuple(x.value for x in v)

    def accumulators(self):
        a = (ctypes.c_double * 3)()
        _check(self.lib.me_get_accumulators(self.h, a))
        return tuple(a)

    def set_accumulators(self, vals):
        a = (ctypes.c_double * 3)(*vals)
        _check(self.lib.me_set_accumulators(self.h, a))

    def enable_stage_timers(self, on: bool = True):
        _check(self.lib.me_enable_stage_timers(self.h, 1 if on else 0))

    def stage_times(self):
        """(main kernel ms, rescue ms, reduction ms, calls) summed since the last read."""
        t = (ctypes.c_double * 3)()
        c = ctypes.c_int64()
        _check(self.lib.me_stage_times(self.h, t, ctypes.byref(c)))
        return t[0], t[1], t[2], c.value

    def set_stream(self, stream_ptr: int | None):
        """Run on the caller's CUDA stream (e.g. torch.cuda.Stream().cuda_stream); calls
        then return without waiting and the caller orders work on that stream."""
        _check(self.lib.me_set_stream(self.h, stream_ptr))
        self.sync = stream_ptr is None

    def synchronize(self):
        _check(self.lib.me_synchronize(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.me_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request loop (me_server_create / me_submit / me_poll / me_server_destroy)."""

    def __init__(self, device: int = 0, n_slots: int = 4, max_queue: int = 4096, mem_budget_bytes: int = 0,
                 precision: int = ME_PREC_MIXED, use_graphs: bool = True, persistent: bool = False,
                 persistent_idle_us: int = 0, **params):
        self.lib = library()
        sp = MEServerParams()
        self.lib.me_default_server_params(ctypes.byref(sp))
        sp.device = device
        sp.n_slots = n_slots
        sp.max_queue = max_queue
        sp.use_graphs = 1 if use_graphs else 0
        sp.persistent = 1 if persistent else 0
        if persistent_idle_us:
            sp.persistent_idle_us = persistent_idle_us
        if mem_budget_bytes:
            sp.mem_budget_bytes = mem_budget_bytes
        sp.params = default_params(precision=precision, device=device, **params)
        s = ctypes.c_void_p()
        _check(self.lib.me_server_create(ctypes.byref(sp), ctypes.byref(s)))
        self.s = s
        self._keep = {}

    def submit(self, process: str, kind: str, p: np.ndarray, w=None, out=None) -> int:
        n = p.shape[-1]
        out = np.empty(n) if out is None else out
        pp, kp = _ptr(p)
        wp, kw = _ptr(w)
        op, ko = _ptr(out)
        req = MERequest(process.encode(), KINDS[kind], pp, wp, n, op)
        t = ctypes.c_uint64()
        _check(self.lib.me_submit(self.s, ctypes.byref(req), ctypes.byref(t)))
        self._keep[t.value] = (kp, kw, ko, req)
        return t.value

    def poll(self, ticket: int, timeout_us: int = -1) -> dict:
        r = MEResult()
        rc = self.lib.me_poll(self.s, ctypes.c_uint64(ticket), ctypes.byref(r), timeout_us)
        if rc == ME_ERR_TIMEOUT:
            return {"status": ME_ERR_TIMEOUT}
        _check(rc)
        kp, kw, ko, _ = self._keep.pop(ticket)
        return {"status": r.status, "n": r.n, "n_rescued": r.n_rescued, "sum_w": r.sum_w, "sum_w2": r.sum_w2,
                "t_queue_us": r.t_queue_us, "t_device_us": r.t_device_us, "t_total_us": r.t_total_us,
                "out": ko}

    def stats(self) -> dict:
        """Requests run by replaying a captured CUDA graph and by ordinary launches; with
        persistent kernels also their launches, idle exits (ME_ERR_TIMEOUT) and requests."""
        g, p = ctypes.c_int64(), ctypes.c_int64()
        _check(self.lib.me_server_stats(self.s, ctypes.byref(g), ctypes.byref(p)))
        la, to, rq = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(self.lib.me_server_persistent_stats(self.s, ctypes.byref(la), ctypes.byref(to), ctypes.byref(rq)))
        return {"graph_runs": g.value, "plain_runs": p.value, "persistent_launches": la.value,
                "persistent_idle_timeouts": to.value, "persistent_requests": rq.value}

    def close(self):
        if getattr(self, "s", None):
            self.lib.me_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
