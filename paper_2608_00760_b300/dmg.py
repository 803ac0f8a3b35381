"""Thin ctypes binding of libdmg.so (include/dmg.h), with the same names.

Argument marshalling only: every array argument may be a torch tensor (CUDA or
CPU), a numpy array, or None where the C API allows NULL; each must be a
C-contiguous float64 array of nx*ny*nz elements in [nz][ny][nx] order (nz = 1:
a 2D grid [ny][nx]). The
stream defaults to torch's current CUDA stream. Every computation runs in the
library's CUDA kernels; when the library is missing the first call raises.
A context set up with ``batch = B`` takes B such fields back to back,
[B][nz][ny][nx].

``Solver`` is a small convenience owner of one context (setup/destroy) whose
methods allocate torch outputs and raise ``DMGError`` on a failing status.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libdmg.so")
_CHECK_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libdmg_check.so")


def use_check_library():
    """Load the bounds-checked build (libdmg_check.so) instead of libdmg.so; call
    before the first use of the library in the process."""
    global _LIB_PATH
    if _lib is not None and _LIB_PATH != _CHECK_PATH:
        raise RuntimeError("the library is already loaded")
    _LIB_PATH = _CHECK_PATH

DMG_OK, DMG_EINVAL, DMG_ENOMEM, DMG_ECUDA, DMG_ENOCONV, DMG_ENAN, DMG_ETIMEOUT = range(7)
DMG_FP64, DMG_MIXED = 0, 1
DMG_FACE_ARITHMETIC, DMG_FACE_HARMONIC = 0, 1
DMG_COARSEN_FULL_WEIGHTING, DMG_COARSEN_INJECTION = 0, 1
(DMG_KERNEL_SMOOTH, DMG_KERNEL_RESTRICT, DMG_KERNEL_PROLONG, DMG_KERNEL_RESIDUAL, DMG_KERNEL_GRAD,
 DMG_KERNEL_TAIL) = range(6)
DMG_HIST_LEN = 64
DMG_PHASE_FORWARD, DMG_PHASE_TANGENT, DMG_PHASE_ADJOINT = range(3)


class dmg_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("symmetric", ctypes.c_int), ("max_cycles", ctypes.c_int), ("rtol", ctypes.c_double),
                ("fixed_cycles", ctypes.c_int), ("precision", ctypes.c_int), ("face_mean", ctypes.c_int),
                ("coarsen", ctypes.c_int), ("inner_cycles", ctypes.c_int), ("batch", ctypes.c_int),
                ("autotune", ctypes.c_int), ("split_prolong", ctypes.c_int),
                ("twin_adjoint", ctypes.c_int)]


class dmg_info(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("outer", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("hist", ctypes.c_double * DMG_HIST_LEN)]

    def history(self):
        n = min(self.outer, DMG_HIST_LEN)
        return [self.hist[i] for i in range(n)]


EXPORTS = ("dmg_default_params", "dmg_setup", "dmg_solve", "dmg_jvp", "dmg_vjp", "dmg_residual",
           "dmg_destroy", "dmg_strerror", "dmg_last_error", "dmg_levels", "dmg_level_shape",
           "dmg_launch_count", "dmg_profile_begin", "dmg_profile_end", "dmg_residual_static",
           "dmg_batch_info", "dmg_slot_load", "dmg_slot_begin", "dmg_step_launch", "dmg_step_finish",
           "dmg_slot_result", "dmg_slot_read", "dmg_device_bytes", "dmg_response", "dmg_response_jvp",
           "dmg_response_vjp", "dmg_vjp_unrolled", "dmg_tile", "dmg_debug_fail_alloc", "dmg_solve_vjp",
           "dmg_debug_grad_per_vertex",
           "dmg_debug_oob_count", "dmg_set_coefficients", "dmg_probe_fma", "dmg_solve_vjp_many",
           "dmg_setup_pyramid")

_lib = None


class DMGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (_strerror(status), status, msg))
        self.status = status


def lib():
    """Load libdmg.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError("libdmg.so not found at %s: build it with "
                               "`python -m paper_2608_00760_b300.build`" % _LIB_PATH)
        L = ctypes.CDLL(_LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        P = ctypes.POINTER
        sig = {
            "dmg_default_params": (None, [P(dmg_params)]),
            "dmg_setup": (i, [P(dmg_params), vp, vp, vp, P(vp)]),
            "dmg_solve": (i, [vp, vp, vp, P(dmg_info), vp]),
            "dmg_jvp": (i, [vp, vp, vp, vp, vp, vp, P(dmg_info), vp]),
            "dmg_vjp": (i, [vp, vp, vp, i, vp, vp, vp, P(dmg_info), vp]),
            "dmg_residual": (i, [vp, vp, vp, P(d), vp]),
            "dmg_destroy": (i, [vp]),
            "dmg_strerror": (ctypes.c_char_p, [i]),
            "dmg_last_error": (ctypes.c_char_p, [vp]),
            "dmg_levels": (i, [vp]),
            "dmg_level_shape": (i, [vp, i, P(i), P(i), P(i)]),
            "dmg_launch_count": (ctypes.c_ulonglong, [vp]),
            "dmg_profile_begin": (i, [vp, i, i, i, i]),
            "dmg_profile_end": (i, [vp, P(ctypes.c_longlong), P(d)]),
            "dmg_residual_static": (i, [P(dmg_params), vp, vp, vp, vp, P(d), vp]),
            "dmg_batch_info": (i, [vp, P(i), P(d)]),
            "dmg_slot_load": (i, [vp, i, vp, vp, vp]),
            "dmg_slot_begin": (i, [vp, i, i, vp, vp, vp, vp]),
            "dmg_step_launch": (i, [vp, vp]),
            "dmg_step_finish": (i, [vp, vp, P(i), P(i)]),
            "dmg_slot_result": (i, [vp, i, P(i), P(i), P(d)]),
            "dmg_slot_read": (i, [vp, i, vp, vp, vp, vp, vp]),
            "dmg_device_bytes": (ctypes.c_size_t, [vp]),
            "dmg_response": (i, [vp, vp, d, vp, vp, P(dmg_info), vp]),
            "dmg_vjp_unrolled": (i, [vp, vp, vp, i, i, vp, vp, vp, vp, vp]),
            "dmg_tile": (i, [vp, i, i, P(i), P(i)]),
            "dmg_solve_vjp": (i, [vp, vp, vp, vp, vp, vp, vp, P(dmg_info), P(dmg_info), vp]),
            "dmg_debug_fail_alloc": (None, [ctypes.c_longlong]),
            "dmg_debug_grad_per_vertex": (None, [ctypes.c_int]),
            "dmg_debug_oob_count": (ctypes.c_longlong, []),
            "dmg_response_jvp": (i, [vp, vp, vp, vp, vp, d, vp, P(dmg_info), vp]),
            "dmg_response_vjp": (i, [vp, vp, vp, d, vp, vp, vp, P(dmg_info), vp]),
            "dmg_set_coefficients": (i, [vp, vp, vp, vp]),
            "dmg_probe_fma": (i, [i, P(d), vp]),
            "dmg_solve_vjp_many": (i, [vp, i, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
            "dmg_setup_pyramid": (i, [P(dmg_params), P(i), i, vp, P(vp)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _strerror(status):
    try:
        return lib().dmg_strerror(int(status)).decode()
    except Exception:
        return "status"


def _ptr(x, n=None):
    """Raw address of an array argument (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    mod = type(x).__module__
    if mod.startswith("torch"):
        if x.dtype.itemsize != 8 or not x.is_floating_point() or not x.is_contiguous():
            raise ValueError("expected a contiguous float64 tensor")
        if n is not None and x.numel() != n:
            raise ValueError("expected %d elements, got %d" % (n, x.numel()))
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            raise ValueError("expected a C-contiguous float64 numpy array")
        if n is not None and x.size != n:
            raise ValueError("expected %d elements, got %d" % (n, x.size))
        return x.ctypes.data
    raise TypeError("unsupported array type %r" % type(x))


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else getattr(stream, "cuda_stream", stream)
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def dmg_default_params(**kw) -> dmg_params:
    p = dmg_params()
    lib().dmg_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError("dmg_params has no field %r" % k)
        setattr(p, k, v)
    return p


def dmg_setup(params: dmg_params, D, mu, stream=None):
    """Returns (status, ctx). ctx is an opaque c_void_p (None on failure)."""
    n = params.nx * params.ny * params.nz * max(params.batch, 1)
    out = ctypes.c_void_p()
    st = lib().dmg_setup(ctypes.byref(params), _ptr(D, n), _ptr(mu, n), _stream(stream), ctypes.byref(out))
    return st, (out if st == DMG_OK else None)


def dmg_setup_pyramid(params: dmg_params, slots_per_level, stream=None):
    """Returns (status, ctx): a pool whose slots_per_level[k] slots serve grids of level k of params' grid."""
    k = len(slots_per_level)
    arr = (ctypes.c_int * max(k, 1))(*[int(x) for x in slots_per_level])
    out = ctypes.c_void_p()
    st = lib().dmg_setup_pyramid(ctypes.byref(params), arr, k, _stream(stream), ctypes.byref(out))
    return st, (out if st == DMG_OK else None)


def dmg_solve(ctx, q, u, info=None, stream=None, n=None):
    return lib().dmg_solve(ctx, _ptr(q, n), _ptr(u, n), ctypes.byref(info) if info is not None else None,
                           _stream(stream))


def dmg_jvp(ctx, u, dq, dD, dmu, du, info=None, stream=None, n=None):
    return lib().dmg_jvp(ctx, _ptr(u, n), _ptr(dq, n), _ptr(dD, n), _ptr(dmu, n), _ptr(du, n),
                         ctypes.byref(info) if info is not None else None, _stream(stream))


def dmg_solve_vjp(ctx, q, w, u, qbar, Dbar, mubar, info_fwd=None, info_adj=None, stream=None, n=None):
    return lib().dmg_solve_vjp(ctx, _ptr(q, n), _ptr(w, n), _ptr(u, n), _ptr(qbar, n), _ptr(Dbar, n),
                               _ptr(mubar, n), ctypes.byref(info_fwd) if info_fwd is not None else None,
                               ctypes.byref(info_adj) if info_adj is not None else None, _stream(stream))


def dmg_solve_vjp_many(ctx, q, w, u=None, qbar=None, Dbar=None, mubar=None, info_fwd=None, info_adj=None,
                       stream=None, n=None):
    """npairs fwd+VJP pairs with overlapped host transfers. q, w: sequences of
    arrays (one per pair); u, qbar, Dbar, mubar: sequences of output arrays or
    None; info_fwd / info_adj: ctypes arrays of dmg_info (e.g. (dmg_info * n)())
    or None."""
    m = len(q)
    if len(w) != m:
        raise ValueError("q and w need one array per pair")

    def ptrs(seq):
        if seq is None:
            return None
        if len(seq) != m:
            raise ValueError("expected %d arrays" % m)
        arr = (ctypes.c_void_p * m)(*[_ptr(x, n) for x in seq])
        return arr

    keep = [ptrs(x) for x in (q, w, u, qbar, Dbar, mubar)]
    return lib().dmg_solve_vjp_many(ctx, m, *keep, info_fwd, info_adj, _stream(stream))


def dmg_vjp(ctx, u, w, cycles, qbar, Dbar, mubar, info=None, stream=None, n=None):
    return lib().dmg_vjp(ctx, _ptr(u, n), _ptr(w, n), int(cycles), _ptr(qbar, n), _ptr(Dbar, n),
                         _ptr(mubar, n), ctypes.byref(info) if info is not None else None, _stream(stream))


def dmg_residual(ctx, q, u, stream=None, n=None, batch=1):
    """(status, (||q_0 - A u_0||, ||q_0||, ||q_1 - A u_1||, ...)): 2 * batch norms."""
    out = (ctypes.c_double * (2 * batch))()
    st = lib().dmg_residual(ctx, _ptr(q, n), _ptr(u, n), out, _stream(stream))
    return st, tuple(out)


def dmg_batch_info(ctx, batch):
    """(status, cycles, rel): per-sample report of the last solve/jvp/vjp."""
    cyc = (ctypes.c_int * batch)()
    rel = (ctypes.c_double * batch)()
    st = lib().dmg_batch_info(ctx, cyc, rel)
    return st, list(cyc), list(rel)


def dmg_residual_static(params: dmg_params, D, mu, q, u, stream=None):
    """Context-free, allocation-free residual norm: (status, (||q - A u||, ||q||)).
    D, mu, q, u must be device arrays of the current device."""
    n = params.nx * params.ny * params.nz
    out = (ctypes.c_double * 2)()
    st = lib().dmg_residual_static(ctypes.byref(params), _ptr(D, n), _ptr(mu, n), _ptr(q, n), _ptr(u, n), out,
                                   _stream(stream))
    return st, (out[0], out[1])


def dmg_vjp_unrolled(ctx, q, w, m, stride, u, qbar, Dbar, mubar, stream=None, n=None):
    return lib().dmg_vjp_unrolled(ctx, _ptr(q, n), _ptr(w, n), int(m), int(stride), _ptr(u, n), _ptr(qbar, n),
                                  _ptr(Dbar, n), _ptr(mubar, n), _stream(stream))


def dmg_response(ctx, q, edge, Le, u=None, info=None, stream=None, n=None):
    return lib().dmg_response(ctx, _ptr(q, n), float(edge), _ptr(Le, n), _ptr(u, n),
                              ctypes.byref(info) if info is not None else None, _stream(stream))


def dmg_response_jvp(ctx, u, dq, dD, dmu, edge, dLe, info=None, stream=None, n=None):
    return lib().dmg_response_jvp(ctx, _ptr(u, n), _ptr(dq, n), _ptr(dD, n), _ptr(dmu, n), float(edge),
                                  _ptr(dLe, n), ctypes.byref(info) if info is not None else None, _stream(stream))


def dmg_response_vjp(ctx, u, rbar, edge, qbar, Dbar, mubar, info=None, stream=None, n=None):
    return lib().dmg_response_vjp(ctx, _ptr(u, n), _ptr(rbar, n), float(edge), _ptr(qbar, n), _ptr(Dbar, n),
                                  _ptr(mubar, n), ctypes.byref(info) if info is not None else None,
                                  _stream(stream))


def dmg_set_coefficients(ctx, D, mu, stream=None, n=None):
    return lib().dmg_set_coefficients(ctx, _ptr(D, n), _ptr(mu, n), _stream(stream))


def dmg_probe_fma(fp64=True, stream=None):
    """(status, FMA instructions per second) of the current device."""
    out = ctypes.c_double()
    st = lib().dmg_probe_fma(int(bool(fp64)), ctypes.byref(out), _stream(stream))
    return st, out.value


def dmg_slot_load(ctx, slot, D, mu, stream=None, n=None):
    return lib().dmg_slot_load(ctx, int(slot), _ptr(D, n), _ptr(mu, n), _stream(stream))


def dmg_slot_begin(ctx, slot, phase, a=None, b=None, c=None, stream=None, n=None):
    return lib().dmg_slot_begin(ctx, int(slot), int(phase), _ptr(a, n), _ptr(b, n), _ptr(c, n), _stream(stream))


def dmg_step_launch(ctx, stream=None):
    return lib().dmg_step_launch(ctx, _stream(stream))


def dmg_step_finish(ctx, batch, stream=None):
    """(status, [slots whose phase ended])."""
    ended = (ctypes.c_int * max(batch, 1))()
    n = ctypes.c_int(0)
    st = lib().dmg_step_finish(ctx, _stream(stream), ended, ctypes.byref(n))
    return st, [ended[k] for k in range(n.value)]


def dmg_slot_result(ctx, slot):
    """(status, phase status (-1 while running), cycles, rel)."""
    a, b, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    st = lib().dmg_slot_result(ctx, int(slot), ctypes.byref(a), ctypes.byref(b), ctypes.byref(r))
    return st, a.value, b.value, r.value


def dmg_slot_read(ctx, slot, u=None, x=None, Dbar=None, mubar=None, stream=None, n=None):
    return lib().dmg_slot_read(ctx, int(slot), _ptr(u, n), _ptr(x, n), _ptr(Dbar, n), _ptr(mubar, n),
                               _stream(stream))


def dmg_device_bytes(ctx):
    return lib().dmg_device_bytes(ctx)


def dmg_destroy(ctx):
    return lib().dmg_destroy(ctx)


def dmg_strerror(status):
    return lib().dmg_strerror(int(status)).decode()


def dmg_last_error(ctx=None):
    return lib().dmg_last_error(ctx).decode()


def dmg_levels(ctx):
    return lib().dmg_levels(ctx)


def dmg_level_shape(ctx, level):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    st = lib().dmg_level_shape(ctx, level, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return st, (c.value, b.value, a.value)


def dmg_debug_fail_alloc(n):
    """Testing hook: the n-th device allocation from now on fails with DMG_ENOMEM (n <= 0: off)."""
    lib().dmg_debug_fail_alloc(int(n))


def dmg_debug_grad_per_vertex(on):
    """Testing hook: 1 forms D-bar and mu-bar with the per-vertex gradient kernels (0: the tiled ones)."""
    lib().dmg_debug_grad_per_vertex(1 if on else 0)


def dmg_debug_oob_count():
    """Accesses counted outside their arrays (bounds-checked build), -1 in normal builds."""
    return lib().dmg_debug_oob_count()


def dmg_tile(ctx, level, fp32=False):
    a, b = ctypes.c_int(), ctypes.c_int()
    st = lib().dmg_tile(ctx, int(level), int(bool(fp32)), ctypes.byref(a), ctypes.byref(b))
    return st, (a.value, b.value)


def dmg_launch_count(ctx):
    return lib().dmg_launch_count(ctx)


def dmg_profile_begin(ctx, kernel, level=0, fp32=False, max_launches=4096):
    return lib().dmg_profile_begin(ctx, int(kernel), int(level), int(bool(fp32)), int(max_launches))


def dmg_profile_end(ctx):
    n, ms = ctypes.c_longlong(), ctypes.c_double()
    st = lib().dmg_profile_end(ctx, ctypes.byref(n), ctypes.byref(ms))
    return st, n.value, ms.value


class Solver:
    """Owns one dmg context for fixed (D, mu) on a grid of shape (nz, ny, nx),
    or a batch of B problems of shape (B, nz, ny, nx).

    Array arguments are float64 torch tensors (device or host) or numpy arrays;
    results are new torch tensors on ``device`` (default cuda). ``strict``:
    raise on DMG_ENOCONV too (default True).
    """

    def __init__(self, D, mu, h, shape=None, stream=None, strict=True, dim=3, **params):
        import torch
        self.torch = torch
        shape = tuple(shape if shape is not None else D.shape)
        if dim == 2:   # a 2D grid (ny, nx), or a batch (B, ny, nx): nz = 1
            if len(shape) == 3:
                self.batch, (ny, nx), nz = shape[0], shape[1:], 1
            elif len(shape) == 2:
                self.batch, (ny, nx), nz = 1, shape, 1
            else:
                raise ValueError("expected a shape (ny, nx) or (B, ny, nx), got %r" % (shape,))
        elif len(shape) == 4:
            self.batch, (nz, ny, nx) = shape[0], shape[1:]
        elif len(shape) == 3:
            self.batch, (nz, ny, nx) = 1, shape
        else:
            raise ValueError("expected a shape (nz, ny, nx) or (B, nz, ny, nx), got %r" % (shape,))
        self.dim = dim
        self.shape, self.n = shape, nx * ny * nz * self.batch
        self.params = dmg_default_params(nx=nx, ny=ny, nz=nz, h=float(h), batch=self.batch, **params)
        self.strict = strict
        self.last_info = dmg_info()
        st, self.ctx = dmg_setup(self.params, D, mu, stream)
        if st != DMG_OK:
            raise DMGError(st, dmg_last_error(None))

    def close(self):
        if getattr(self, "ctx", None) is not None:
            dmg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st == DMG_OK or (st == DMG_ENOCONV and not self.strict):
            return
        raise DMGError(st, dmg_last_error(self.ctx))

    def _empty(self, like=None, device=None):
        t = self.torch
        dev = device if device is not None else (like.device if like is not None and hasattr(like, "device")
                                                 else t.device("cuda"))
        return t.empty(self.shape, dtype=t.float64, device=dev)

    def levels(self):
        return [dmg_level_shape(self.ctx, l)[1] for l in range(dmg_levels(self.ctx))]

    def set_coefficients(self, D, mu, stream=None):
        """Rebuild the coefficient hierarchy in place from new D, mu (same shape)."""
        self._check(dmg_set_coefficients(self.ctx, D, mu, stream, n=self.n))

    def tiles(self, fp32=False):
        """Block shape (threads along the half-row, rows) of the colour kernels per level."""
        return [dmg_tile(self.ctx, l, fp32)[1] for l in range(dmg_levels(self.ctx))]

    def solve(self, q, out=None, stream=None):
        u = out if out is not None else self._empty(q)
        info = dmg_info()
        self._check(dmg_solve(self.ctx, q, u, info, stream, n=self.n))
        self.last_info = info
        return u

    def jvp(self, u, dq=None, dD=None, dmu=None, out=None, stream=None):
        like = next((x for x in (dq, dD, dmu, u) if x is not None), None)
        du = out if out is not None else self._empty(like)
        info = dmg_info()
        self._check(dmg_jvp(self.ctx, u, dq, dD, dmu, du, info, stream, n=self.n))
        self.last_info = info
        return du

    def vjp(self, u, w, cycles=0, need=(True, True, True), stream=None):
        qb = self._empty(w) if need[0] else None
        Db = self._empty(w) if need[1] else None
        mb = self._empty(w) if need[2] else None
        info = dmg_info()
        self._check(dmg_vjp(self.ctx, u if (need[1] or need[2]) else None, w, cycles, qb, Db, mb, info,
                            stream, n=self.n))
        self.last_info = info
        return qb, Db, mb

    def vjp_unrolled(self, q, w, m, stride=0, stream=None):
        """(u, qbar, Dbar, mubar): u = S_m(q) and the exact gradient of <w, S_m(q; D, mu)>."""
        u, qb, Db, mb = (self._empty(q) for _ in range(4))
        self._check(dmg_vjp_unrolled(self.ctx, q, w, m, stride, u, qb, Db, mb, stream, n=self.n))
        return u, qb, Db, mb

    def response(self, q, edge, stream=None):
        """(Le, u): Le = M(mu S(q)) with the edge mask of depth `edge` (see dmg_response)."""
        Le, u = self._empty(q), self._empty(q)
        info = dmg_info()
        self._check(dmg_response(self.ctx, q, edge, Le, u, info, stream, n=self.n))
        self.last_info = info
        return Le, u

    def response_jvp(self, u, edge, dq=None, dD=None, dmu=None, stream=None):
        dLe = self._empty(u)
        info = dmg_info()
        self._check(dmg_response_jvp(self.ctx, u, dq, dD, dmu, edge, dLe, info, stream, n=self.n))
        self.last_info = info
        return dLe

    def response_vjp(self, u, rbar, edge, stream=None):
        qb, Db, mb = self._empty(rbar), self._empty(rbar), self._empty(rbar)
        info = dmg_info()
        self._check(dmg_response_vjp(self.ctx, u, rbar, edge, qb, Db, mb, info, stream, n=self.n))
        self.last_info = info
        return qb, Db, mb

    def residual(self, q, u, stream=None):
        """(||q - A u||, ||q||), or a list of such pairs for a batch."""
        st, r = dmg_residual(self.ctx, q, u, stream, n=self.n, batch=self.batch)
        self._check(st)
        if self.batch == 1 and len(self.shape) == self.dim:
            return r
        return [(r[2 * b], r[2 * b + 1]) for b in range(self.batch)]

    def batch_info(self):
        """Per-sample (cycles, rel_residual) lists of the last solve/jvp/vjp."""
        st, cyc, rel = dmg_batch_info(self.ctx, self.batch)
        self._check(st)
        return cyc, rel
