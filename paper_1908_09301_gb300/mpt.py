"""ctypes binding of libmpt (the C ABI in ``include/mpt.h``).

Argument marshalling only: every step of the Taylor method runs in the CUDA
kernels of ``libmpt.so``.  There is no CPU fallback -- if the library cannot
be loaded the import of :func:`lib` raises.

Numbers cross the boundary in the interchange layout of ``include/mpt.h``:
``signs[n]`` (int32, 0/1), ``exps[n]`` (int32, limb exponent) and
``limbs[n, L]`` (uint32, least significant first).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpt.so")

MPT_OK, MPT_EINVAL, MPT_ENOMEM, MPT_ERANGE, MPT_ETIMEDOUT, MPT_ECUDA = 0, -1, -2, -3, -4, -5

_lock = threading.Lock()
_lib = None

i32p = ctypes.POINTER(ctypes.c_int32)
u32p = ctypes.POINTER(ctypes.c_uint32)
vp = ctypes.c_void_p

# name -> (restype, argtypes); every symbol include/mpt.h declares
SIGNATURES = {
    "mpt_limbs_for_digits": (ctypes.c_int, [ctypes.c_int]),
    "mpt_init": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p,
                                ctypes.c_uint64]),
    "mpt_destroy": (None, [vp]),
    "mpt_parse_number": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int, vp, vp, vp]),
    "mpt_get_dims": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "mpt_set_state": (ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p]),
    "mpt_set_state_raw": (ctypes.c_int, [vp, vp, vp, vp]),
    "mpt_get_state": (ctypes.c_int, [vp, vp, vp, vp]),
    "mpt_get_params": (ctypes.c_int, [vp, vp, vp, vp]),
    "mpt_step": (ctypes.c_int, [vp]),
    "mpt_integrate": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.c_int64, vp, vp, vp]),
    "mpt_get_coefficients": (ctypes.c_int, [vp, vp, vp, vp]),
    "mpt_launch": (ctypes.c_int, [vp, ctypes.c_int64]),
    "mpt_set_profiling": (ctypes.c_int, [vp, ctypes.c_int]),
    "mpt_set_wait_limit": (ctypes.c_int, [vp, ctypes.c_int64]),
    "mpt_get_profile": (ctypes.c_int, [vp, vp, ctypes.c_int]),
    "mpt_wait": (ctypes.c_int, [vp]),
    "mpt_set_exact": (ctypes.c_int, [vp, ctypes.c_int]),
    "mpt_set_pipe_batch": (ctypes.c_int, [vp, ctypes.c_int]),
    "mpt_integrate_batch_shape": (ctypes.c_int, [ctypes.c_int, vp, vp, ctypes.c_int64, ctypes.c_char_p,
                                                 ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p, vp, vp,
                                                 vp, vp, ctypes.c_uint64]),
    "mpt_get_counters": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "mpt_set_launch": (ctypes.c_int, [vp, ctypes.c_int]),
    "mpt_get_launch": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int)]),
    "mpt_set_kernel": (ctypes.c_int, [vp, ctypes.c_int]),
    "mpt_get_kernel": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int)]),
    "mpt_set_system": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int, vp]),
    "mpt_int_peak_run": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int)]),
    "mpt_integrate_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int64, vp, vp,
                                             vp, vp, vp, vp, ctypes.c_uint64]),
    "mpt_integrate_batch": (ctypes.c_int, [ctypes.c_int, vp, vp, ctypes.c_int64, ctypes.c_char_p,
                                           ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p, vp, vp,
                                           vp, ctypes.c_uint64]),
    "mpt_integrate_batch_params": (ctypes.c_int, [ctypes.c_int, vp, vp, ctypes.c_int64, ctypes.c_char_p,
                                                  vp, vp, vp, vp, vp, vp, ctypes.c_uint64]),
    "mpt_backward": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_char_p,
                                    ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p, vp, vp, ctypes.c_int,
                                    vp, vp, vp, ctypes.c_uint64]),
    "mpt_backward_raw": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int64, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                        vp, vp, vp, ctypes.c_uint64]),
    "mpt_jacobian_fd": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                       ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p,
                                       vp, ctypes.c_int, vp, ctypes.c_uint64]),
    "mpt_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "mpt_last_error": (ctypes.c_char_p, []),
}


class MPTError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mpt error {code}: {msg}")
        self.code = code


def lib(build_if_missing: bool = True) -> ctypes.CDLL:
    """The loaded libmpt.so (built in-tree by ``build.py`` when absent)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                from . import build as _build
                _build.build()
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libmpt.so not found at {LIB_PATH}: run the build first")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc: int):
    if rc != MPT_OK:
        msg = lib().mpt_last_error().decode(errors="replace")
        raise MPTError(rc, msg)


def limbs_for_digits(K: int) -> int:
    rc = lib().mpt_limbs_for_digits(int(K))
    if rc < 0:
        _check(rc)
    return rc


def parse_number(text: str, L: int):
    """trunc_L of a decimal or rational string: (sign, exp, limbs[L]) (host only)."""
    s = np.zeros(1, np.int32)
    e = np.zeros(1, np.int32)
    l = np.zeros(L, np.uint32)
    _check(lib().mpt_parse_number(str(text).encode(), int(L), _ptr(s), _ptr(e), _ptr(l)))
    return int(s[0]), int(e[0]), [int(x) for x in l]


def _ptr(a):
    """Pointer of a numpy array or a torch tensor (host or device)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("buffers passed to libmpt must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors passed to libmpt must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError(f"unsupported buffer type {type(a)}")


_I32, _U32 = "torch.int32", "torch.uint32"


def _check_noalloc_buffer(t, name: str, numel: int, dtypes):
    """A contiguous CUDA tensor of exactly ``numel`` elements of a 32-bit
    dtype from ``dtypes``; ValueError otherwise."""
    if not hasattr(t, "data_ptr") or not hasattr(t, "is_cuda"):
        raise ValueError(f"{name} must be a torch tensor, got {type(t).__name__}")
    if not t.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device, got {t.device}")
    if str(t.dtype) not in dtypes:
        raise ValueError(f"{name} must have dtype {' or '.join(dtypes)}, got {t.dtype}")
    if t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _current_stream() -> int:
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:  # pragma: no cover
        pass
    return 0


class Context:
    """One integrator context (``mpt_init`` .. ``mpt_destroy``)."""

    def __init__(self, N: int, L: int = 0, K: int = 0, tau: str = "0.01", sigma: str = "10",
                 R: str = "28", b: str = "8/3", stream: int | None = None):
        self._h = vp()
        if stream is None:
            stream = _current_stream()
        _check(lib().mpt_init(ctypes.byref(self._h), int(K), int(N), int(L), str(tau).encode(),
                              str(sigma).encode(), str(R).encode(), str(b).encode(),
                              ctypes.c_uint64(int(stream))))
        l, n = ctypes.c_int(), ctypes.c_int()
        _check(lib().mpt_get_dims(self._h, ctypes.byref(l), ctypes.byref(n)))
        self.L, self.N = l.value, n.value

    def close(self):
        if self._h:
            lib().mpt_destroy(self._h)
            self._h = vp()

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- numbers
    def _empty(self, n: int):
        return (np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros((n, self.L), np.uint32))

    def set_state(self, x0: str, y0: str, z0: str):
        _check(lib().mpt_set_state(self._h, str(x0).encode(), str(y0).encode(), str(z0).encode()))

    def set_state_raw(self, signs, exps, limbs):
        s = np.ascontiguousarray(signs, np.int32)
        e = np.ascontiguousarray(exps, np.int32)
        l = np.ascontiguousarray(limbs, np.uint32).reshape(3, self.L)
        _check(lib().mpt_set_state_raw(self._h, _ptr(s), _ptr(e), _ptr(l)))

    def get_state(self):
        s, e, l = self._empty(3)
        _check(lib().mpt_get_state(self._h, _ptr(s), _ptr(e), _ptr(l)))
        return s, e, l

    def params(self):
        s, e, l = self._empty(4)
        _check(lib().mpt_get_params(self._h, _ptr(s), _ptr(e), _ptr(l)))
        return s, e, l

    def coefficients(self):
        s, e, l = self._empty(3 * (self.N + 1))
        _check(lib().mpt_get_coefficients(self._h, _ptr(s), _ptr(e), _ptr(l)))
        return s, e, l

    # -- stepping
    def step(self):
        _check(lib().mpt_step(self._h))

    def integrate(self, nsteps: int, record_every: int = 0, out=None):
        """nsteps steps in one launch.  With record_every > 0 the records go to
        ``out`` = (signs, exps, limbs) (numpy arrays or torch tensors, host or
        device) or to new numpy arrays, which are returned."""
        nrec = nsteps // record_every if record_every > 0 else 0
        if nrec == 0:
            _check(lib().mpt_integrate(self._h, int(nsteps), 0, None, None, None))
            return None
        if out is None:
            out = (np.zeros((nrec, 3), np.int32), np.zeros((nrec, 3), np.int32),
                   np.zeros((nrec, 3, self.L), np.uint32))
        _check(lib().mpt_integrate(self._h, int(nsteps), int(record_every), _ptr(out[0]),
                                   _ptr(out[1]), _ptr(out[2])))
        return out

    def launch_async(self, nsteps: int = 1):
        """Queue nsteps steps on the context's stream (``mpt_launch``)."""
        _check(lib().mpt_launch(self._h, int(nsteps)))

    def wait(self):
        """Finish queued steps and report device-side errors (``mpt_wait``)."""
        _check(lib().mpt_wait(self._h))

    def set_exact(self, on: bool = True):
        """Every launch with all products in full (``mpt_set_exact``)."""
        _check(lib().mpt_set_exact(self._h, int(bool(on))))

    def set_pipe_batch(self, tb: int):
        """Worker terms per staged batch of the pipelined kernel (0 = the
        largest that fits) (``mpt_set_pipe_batch``)."""
        _check(lib().mpt_set_pipe_batch(self._h, int(tb)))

    def counters(self):
        """(full reruns so far, limb-product chunks of the last launch)
        (``mpt_get_counters``)."""
        r, c = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().mpt_get_counters(self._h, ctypes.byref(r), ctypes.byref(c)))
        return r.value, c.value

    PROFILE_SLOTS = ["place", "stage", "mac", "flush", "barrier", "close", "horner", "horner_mac",
                     "horner_close", "total", "x1", "x2", "x3", "x4", "x5", "x6"]

    def set_wait_limit(self, polls: int = 0):
        """Bound of device-side waits in polls (0 = default) (``mpt_set_wait_limit``)."""
        _check(lib().mpt_set_wait_limit(self._h, int(polls)))

    def set_profiling(self, on: bool = True):
        _check(lib().mpt_set_profiling(self._h, int(bool(on))))

    def profile(self):
        """Per-phase SM cycles of the last launch: {cta: {phase: cycles}} for
        the first and the last CTA, and under "ctas" one row of raw counters
        per CTA (pipelined kernel; zeros otherwise)."""
        rows = 2 + self.launch()
        buf = np.zeros(16 * rows, np.int64)
        _check(lib().mpt_get_profile(self._h, _ptr(buf), int(buf.size)))
        out = {}
        for k, cta in enumerate(("first", "last")):
            out[cta] = {n: int(buf[16 * k + j]) for j, n in enumerate(self.PROFILE_SLOTS)}
        out["ctas"] = buf[32:].reshape(-1, 16)
        return out

    TIMELINE_ROWS = ("beta_start", "beta_waited", "beta_published", "last_edge_done", "last_worker_done",
                     "gamma_published", "last_edge_seen", "last_edge_mac_start", "last_edge_mac_end")
    MAX_N = 4096

    def timeline(self, sms: int):
        """Per-index global-timer stamps (ns) of the last step of the last
        launch (pipelined kernel, profiling on): {row: int64 array [N]},
        rows as TIMELINE_ROWS; ``sms`` is the device's SM count."""
        n = (2 + int(sms)) * 16 + len(self.TIMELINE_ROWS) * (self.MAX_N + 1)
        buf = np.zeros(n, np.int64)
        _check(lib().mpt_get_profile(self._h, _ptr(buf), int(buf.size)))
        tl = buf[(2 + int(sms)) * 16:].reshape(len(self.TIMELINE_ROWS), self.MAX_N + 1)
        return {name: tl[k, :self.N].copy() for k, name in enumerate(self.TIMELINE_ROWS)}

    def set_launch(self, ctas: int):
        _check(lib().mpt_set_launch(self._h, int(ctas)))

    def set_kernel(self, kind: int):
        """0 = library choice, 1 = lock-step, 2 = pipelined (``mpt_set_kernel``)."""
        _check(lib().mpt_set_kernel(self._h, int(kind)))

    def set_system(self, system):
        """A general three-component quadratic system (``mpt_set_system``):
        a dict with ``params`` (strings), ``fixed`` ((target, neg, p, j)
        tuples) and ``quad`` ((target, neg, i, j) tuples)."""
        params = [str(p).encode() for p in system.get("params", [])]
        fixed = np.ascontiguousarray(np.asarray(system.get("fixed", []), np.int32).reshape(-1, 4))
        quad = np.ascontiguousarray(np.asarray(system.get("quad", []), np.int32).reshape(-1, 4))
        arr = (ctypes.c_char_p * max(1, len(params)))(*params)
        _check(lib().mpt_set_system(self._h, len(params), ctypes.cast(arr, ctypes.c_void_p),
                                    len(fixed), _ptr(fixed), len(quad), _ptr(quad)))

    def kernel(self) -> int:
        k = ctypes.c_int()
        _check(lib().mpt_get_kernel(self._h, ctypes.byref(k)))
        return k.value

    def launch(self) -> int:
        c = ctypes.c_int()
        _check(lib().mpt_get_launch(self._h, ctypes.byref(c)))
        return c.value


def integrate_noalloc(L: int, N: int, nsteps: int, params, state, stream: int | None = None):
    """nsteps Taylor steps through ``mpt_integrate_noalloc``, which keeps its
    working memory in a static device array instead of allocating, for callers
    that may not allocate device memory while they step.

    ``params`` = (signs[4], exps[4], limbs[4, L]) for sigma, R, b, tau and
    ``state`` = (signs[3], exps[3], limbs[3, L]), which is overwritten with the
    new state: contiguous torch tensors (int32 / int32 / int32 or uint32
    viewed as 32-bit) on the current CUDA device.  Calls that overlap on the
    GPU race on the shared array."""
    ps, pe, pl = params
    ss, se, sl = state
    # the C ABI cannot see buffer sizes: check them here, before any pointer
    # crosses it
    _check_noalloc_buffer(ps, "par_signs", 4, (_I32,))
    _check_noalloc_buffer(pe, "par_exps", 4, (_I32,))
    _check_noalloc_buffer(pl, "par_limbs", 4 * int(L), (_I32, _U32))
    _check_noalloc_buffer(ss, "signs", 3, (_I32,))
    _check_noalloc_buffer(se, "exps", 3, (_I32,))
    _check_noalloc_buffer(sl, "limbs", 3 * int(L), (_I32, _U32))
    devs = {t.device for t in (ps, pe, pl, ss, se, sl)}
    if len(devs) != 1:
        raise ValueError(f"all six tensors must be on one CUDA device, got {sorted(map(str, devs))}")
    if stream is None:
        stream = _current_stream()
    _check(lib().mpt_integrate_noalloc(int(L), int(N), int(nsteps), _ptr(ps), _ptr(pe), _ptr(pl),
                                       _ptr(ss), _ptr(se), _ptr(sl), ctypes.c_uint64(int(stream))))


def integrate_batch(Ls, Ns, nsteps: int, states, tau: str = "0.01", sigma="10",
                    R="28", b="8/3", stream: int = 0, shape=None):
    """nsteps Taylor steps of B independent trajectories through
    ``mpt_integrate_batch``.  ``Ls``, ``Ns``: per-trajectory limbs and order;
    ``states``: per trajectory (signs[3], exps[3], limbs[3, L_j]) in the
    interchange layout (host).  ``sigma``, ``R``, ``b``: one string each, or a
    list of B strings each (``mpt_integrate_batch_params``).  ``shape``:
    (kernel variant, terms per staging batch, window copies), see
    ``mpt_integrate_batch_shape`` (one set of parameters only).  Returns the
    new states in the same form."""
    B = len(Ls)
    if B != len(Ns) or B != len(states):
        raise ValueError("Ls, Ns and states must have the same length")
    Lv = np.ascontiguousarray(np.asarray(Ls, np.int32))
    Nv = np.ascontiguousarray(np.asarray(Ns, np.int32))
    signs = np.ascontiguousarray(np.concatenate([np.asarray(st[0], np.int32).reshape(3) for st in states]))
    exps = np.ascontiguousarray(np.concatenate([np.asarray(st[1], np.int32).reshape(3) for st in states]))
    limbs = np.ascontiguousarray(np.concatenate(
        [np.asarray(st[2], np.uint32).reshape(3 * int(L)) for st, L in zip(states, Ls)]))
    if isinstance(sigma, (list, tuple)):
        if not (len(sigma) == len(R) == len(b) == B):
            raise ValueError("per-trajectory sigma, R, b need B strings each")
        arrs = [(ctypes.c_char_p * B)(*[str(v).encode() for v in vs]) for vs in (sigma, R, b)]
        _check(lib().mpt_integrate_batch_params(
            int(B), _ptr(Lv), _ptr(Nv), int(nsteps), str(tau).encode(),
            *[ctypes.cast(a, ctypes.c_void_p) for a in arrs],
            _ptr(signs), _ptr(exps), _ptr(limbs), ctypes.c_uint64(int(stream))))
    elif shape is not None:
        sh = np.ascontiguousarray(np.asarray(shape, np.int32).reshape(3))
        _check(lib().mpt_integrate_batch_shape(int(B), _ptr(Lv), _ptr(Nv), int(nsteps), str(tau).encode(),
                                               str(sigma).encode(), str(R).encode(), str(b).encode(),
                                               _ptr(signs), _ptr(exps), _ptr(limbs), _ptr(sh),
                                               ctypes.c_uint64(int(stream))))
    else:
        _check(lib().mpt_integrate_batch(int(B), _ptr(Lv), _ptr(Nv), int(nsteps), str(tau).encode(),
                                         str(sigma).encode(), str(R).encode(), str(b).encode(),
                                         _ptr(signs), _ptr(exps), _ptr(limbs),
                                         ctypes.c_uint64(int(stream))))
    out, off = [], 0
    for j, L in enumerate(Ls):
        L = int(L)
        out.append((signs[3 * j:3 * j + 3].copy(), exps[3 * j:3 * j + 3].copy(),
                    limbs[off:off + 3 * L].reshape(3, L).copy()))
        off += 3 * L
    return out


def _strings(x0s):
    strs = [str(v).encode() for p in x0s for v in p]
    if len(strs) != 3 * len(x0s):
        raise ValueError("each initial point needs three values")
    return (ctypes.c_char_p * len(strs))(*strs)


def backward(x0s, g, L: int, N: int, nsteps: int, tau: str = "0.01", sigma: str = "10", R: str = "28",
             b: str = "8/3", checkpoint_every: int = 50, with_jacobian: bool = False, stream: int = 0):
    """``mpt_backward`` (the reverse sweep): for initial points x0s (B triples
    of strings) and the upstream gradients g [B, 3], returns g^T J with
    respect to the points [B, 3] and to (sigma, R, b) [3], and the Jacobians
    [B, 3, 6] if asked (three sweeps per point)."""
    B = len(x0s)
    arr = _strings(x0s)
    gv = np.ascontiguousarray(np.asarray(g, np.float64).reshape(B, 3))
    gx = np.zeros((B, 3), np.float64)
    gp = np.zeros(3, np.float64)
    J = np.zeros((B, 3, 6), np.float64) if with_jacobian else None
    _check(lib().mpt_backward(int(B), int(L), int(N), int(nsteps), str(tau).encode(), str(sigma).encode(),
                              str(R).encode(), str(b).encode(), ctypes.cast(arr, ctypes.c_void_p), _ptr(gv),
                              int(checkpoint_every), _ptr(gx), _ptr(gp), _ptr(J) if J is not None else None,
                              ctypes.c_uint64(int(stream))))
    return gx, gp, J


def backward_raw(par, states, gbar, G: int, L: int, N: int, nsteps: int, checkpoint_every: int = 50,
                 stream: int = 0):
    """``mpt_backward_raw``: par = (signs[4], exps[4], limbs[4, L]) for sigma,
    R, b, tau; states = (signs[3B], exps[3B], limbs[3B, L]); gbar = the
    adjoints of the final states, 3 B G numbers (item j G + g belongs to
    trajectory j).  Returns (the adjoints of the initial states, the adjoints
    of (sigma, R, b)), 3 B G numbers each, in the interchange layout."""
    ps, pe, pl = (np.ascontiguousarray(x) for x in (par[0], par[1], par[2]))
    ss, se, sl = (np.ascontiguousarray(x) for x in (states[0], states[1], states[2]))
    B = len(ss) // 3
    gs = np.ascontiguousarray(np.asarray(gbar[0], np.int32).copy())
    ge = np.ascontiguousarray(np.asarray(gbar[1], np.int32).copy())
    gl = np.ascontiguousarray(np.asarray(gbar[2], np.uint32).reshape(-1, L).copy())
    if len(gs) != 3 * B * G or len(ps) != 4:
        raise ValueError("gbar needs 3 B G numbers and par 4")
    ts = np.zeros(3 * B * G, np.int32)
    te = np.zeros(3 * B * G, np.int32)
    tl = np.zeros((3 * B * G, L), np.uint32)
    _check(lib().mpt_backward_raw(int(B), int(G), int(L), int(N), int(nsteps), int(checkpoint_every),
                                  _ptr(np.asarray(ps, np.int32)), _ptr(np.asarray(pe, np.int32)),
                                  _ptr(np.asarray(pl, np.uint32)), _ptr(np.asarray(ss, np.int32)),
                                  _ptr(np.asarray(se, np.int32)), _ptr(np.asarray(sl, np.uint32)),
                                  _ptr(gs), _ptr(ge), _ptr(gl), _ptr(ts), _ptr(te), _ptr(tl),
                                  ctypes.c_uint64(int(stream))))
    return (gs, ge, gl), (ts, te, tl)


def jacobian_fd(x0s, L: int, N: int, nsteps: int, tau: str = "0.01", sigma: str = "10", R: str = "28",
                b: str = "8/3", h_digits: int = 100, stream: int = 0):
    """``mpt_jacobian_fd``: the 3 x 6 Jacobians [B, 3, 6] by central
    differences (h = 10^-h_digits) of bit-exact runs."""
    B = len(x0s)
    arr = _strings(x0s)
    J = np.zeros((B, 3, 6), np.float64)
    _check(lib().mpt_jacobian_fd(int(B), int(L), int(N), int(nsteps), str(tau).encode(), str(sigma).encode(),
                                 str(R).encode(), str(b).encode(), ctypes.cast(arr, ctypes.c_void_p),
                                 int(h_digits), _ptr(J), ctypes.c_uint64(int(stream))))
    return J


def int_peak(variant: int, iters: int = 20000, threads: int = 1024):
    """INT32 multiply-add probe: (results per SM per clock, ms, sms, grid)."""
    cyc, ms = ctypes.c_double(), ctypes.c_double()
    ds, g = ctypes.c_int(), ctypes.c_int()
    rc = lib().mpt_int_peak_run(int(variant), int(threads), int(iters), ctypes.byref(cyc),
                                ctypes.byref(ms), ctypes.byref(ds), ctypes.byref(g))
    if rc != 0:
        raise MPTError(MPT_ECUDA, f"int peak probe failed with CUDA error {rc}")
    per_clk = iters * 8 * threads / cyc.value
    return per_clk, ms.value, ds.value, g.value
