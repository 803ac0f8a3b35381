"""FP64 CPU oracle for the DMGS hot path (arXiv 2608.00760).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference leg of ``bench.py`` may import this package. The product
package never imports it, and the two share no code: the oracle is the plain
C file ``dmg_oracle.c`` (compiled with ``-O2 -ffp-contract=off``) plus this
ctypes wrapper, which only marshals numpy arrays.

Every array is a C-contiguous float64 numpy array of shape (nz, ny, nx) over
all vertices, boundary planes included.

Parity status: pinned. Each function is checked by CPU tests against something
other than itself (closed-form eigenmodes, the PDE to O(h^2), a library sparse
direct solve, trilinear interpolation by a library routine, brute-force
transposes, finite differences); see ``tests/test_oracle_*.py``. The strength of
those pins is itself tested: ``tests/test_oracle_mutants.py`` plants single
mistakes in copies of this package and requires each to fail a pin.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dmg_oracle.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")

_dp = ctypes.POINTER(ctypes.c_double)
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, FP64, no FMA contraction)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    """The compiled oracle. The environment variable DMG_ORACLE_LIB names another
    build of dmg_oracle.c to load instead; the mutation test uses it to run the
    pins against copies with planted mistakes."""
    global _lib
    if _lib is None:
        L = ctypes.CDLL(os.environ.get("DMG_ORACLE_LIB") or build())
        i, d, p = ctypes.c_int, ctypes.c_double, _dp
        sig = {
            "orc_face": (d, [d, d, i]),
            "orc_apply": (None, [i, i, i, d, i, p, p, p, p]),
            "orc_residual": (None, [i, i, i, d, i, p, p, p, p, p]),
            "orc_gs_half": (None, [i, i, i, d, i, p, p, p, p, i]),
            "orc_restrict": (None, [i, i, i, p, p]),
            "orc_prolong_add": (None, [i, i, i, p, p]),
            "orc_coarsen": (None, [i, i, i, i, p, p]),
            "orc_count_levels": (i, [i, i, i]),
            "orc_create": (ctypes.c_void_p, [i, i, i, d, i, i, i, i, i, p, p]),
            "orc_free": (None, [ctypes.c_void_p]),
            "orc_levels": (i, [ctypes.c_void_p]),
            "orc_level_dims": (None, [ctypes.c_void_p, i, ctypes.POINTER(ctypes.c_int)]),
            "orc_level_coeffs": (None, [ctypes.c_void_p, i, p, p]),
            "orc_rel_residual": (d, [ctypes.c_void_p, p, p]),
            "orc_solve": (i, [ctypes.c_void_p, p, p, d, i, i, p, i]),
            "orc_adjoint": (i, [ctypes.c_void_p, p, p, d, i, i, p, i]),
            "orc_vcycle": (None, [ctypes.c_void_p, p, p, i]),
            "orc_adjoint_literal": (None, [ctypes.c_void_p, p, p, i]),
            "orc_grad": (None, [i, i, i, d, i, p, p, p, p, p]),
            "orc_dA_apply": (None, [i, i, i, d, i, p, p, p, p, p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _arr(x):
    a = np.ascontiguousarray(x, dtype=np.float64)
    return a


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _dims(a):
    nz, ny, nx = a.shape
    return nx, ny, nz


def apply(D, mu, h, u, harmonic=False):
    """A u (Eq. 1, 7-point, interior only; zero on the boundary)."""
    D, mu, u = _arr(D), _arr(mu), _arr(u)
    out = np.zeros_like(u)
    lib().orc_apply(*_dims(u), h, int(harmonic), _ptr(D), _ptr(mu), _ptr(u), _ptr(out))
    return out


def residual(D, mu, h, f, u, harmonic=False):
    """f - A u on interior vertices (the defect, Sec. 2.3.2)."""
    D, mu, f, u = _arr(D), _arr(mu), _arr(f), _arr(u)
    r = np.zeros_like(u)
    lib().orc_residual(*_dims(u), h, int(harmonic), _ptr(D), _ptr(mu), _ptr(f), _ptr(u), _ptr(r))
    return r


def gs_half(D, mu, h, f, u, color, harmonic=False):
    """One Gauss-Seidel half-sweep over colour (i+j+k)%2 == color (Eq. 9); returns the new u."""
    D, mu, f = _arr(D), _arr(mu), _arr(f)
    u = _arr(u).copy()
    lib().orc_gs_half(*_dims(u), h, int(harmonic), _ptr(D), _ptr(mu), _ptr(f), _ptr(u), int(color))
    return u


def coarse_shape(shape):
    return tuple((n - 1) // 2 + 1 for n in shape)


def restrict(r):
    """Full-weighting restriction 1/4[1 2 1]^3 (Eq. 7) onto coarse interior vertices."""
    r = _arr(r)
    fc = np.zeros(coarse_shape(r.shape))
    lib().orc_restrict(*_dims(r), _ptr(r), _ptr(fc))
    return fc


def prolong_add(e, uf):
    """uf + I e with I = 2^3 R^T (Eq. 17) on fine interior vertices."""
    e = _arr(e)
    uf = _arr(uf).copy()
    lib().orc_prolong_add(*_dims(e), _ptr(e), _ptr(uf))
    return uf


def coarsen(X, inject=False):
    """Coarse vertex coefficient field (full weighting interior, injection boundary)."""
    X = _arr(X)
    Xc = np.zeros(coarse_shape(X.shape))
    lib().orc_coarsen(*_dims(X), int(inject), _ptr(X), _ptr(Xc))
    return Xc


def count_levels(shape):
    nz, ny, nx = shape
    return lib().orc_count_levels(nx, ny, nz)


def grad(D, h, u, lam, harmonic=False):
    """(Dbar, mubar) = gradients of <w, u> given u and lam = A^{-1} w."""
    D, u, lam = _arr(D), _arr(u), _arr(lam)
    Db, mb = np.zeros_like(u), np.zeros_like(u)
    lib().orc_grad(*_dims(u), h, int(harmonic), _ptr(D), _ptr(u), _ptr(lam), _ptr(Db), _ptr(mb))
    return Db, mb


def dA_apply(D, h, dD, dmu, u, harmonic=False):
    """(dA) u for the coefficient tangents (dD, dmu); either may be None."""
    D, u = _arr(D), _arr(u)
    dD = None if dD is None else _arr(dD)
    dmu = None if dmu is None else _arr(dmu)
    out = np.zeros_like(u)
    lib().orc_dA_apply(*_dims(u), h, int(harmonic), _ptr(D), _ptr(dD), _ptr(dmu), _ptr(u),
                       _ptr(out))
    return out


class Hierarchy:
    """The multigrid hierarchy and solver (Sec. 2.2) with its adjoints (Sec. 2.4).

    nu1/nu2: pre/post RB-GS sweeps; symmetric: post-smoothing black->red
    (then S_m is symmetric when nu1 == nu2); harmonic: harmonic face mean;
    inject: coefficient coarsening by injection instead of full weighting.
    """

    def __init__(self, D, mu, h, nu1=2, nu2=2, harmonic=False, inject=False, symmetric=False):
        self.D, self.mu = _arr(D), _arr(mu)
        self.h = float(h)
        self.shape = self.D.shape
        self.harmonic = bool(harmonic)
        nx, ny, nz = _dims(self.D)
        self._h = lib().orc_create(nx, ny, nz, self.h, int(harmonic), int(inject), int(nu1),
                                   int(nu2), int(symmetric), _ptr(self.D), _ptr(self.mu))
        if not self._h:
            raise ValueError("oracle: invalid grid %r or non-SPD coarsest matrix" % (self.shape,))

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_free(self._h)
            self._h = None

    @property
    def nlev(self):
        return lib().orc_levels(self._h)

    def level_shape(self, l):
        d = (ctypes.c_int * 3)()
        lib().orc_level_dims(self._h, l, d)
        return (d[2], d[1], d[0])

    def level_coeffs(self, l):
        s = self.level_shape(l)
        D, mu = np.zeros(s), np.zeros(s)
        lib().orc_level_coeffs(self._h, l, _ptr(D), _ptr(mu))
        return D, mu

    def rel_residual(self, f, u):
        f, u = _arr(f), _arr(u)
        return lib().orc_rel_residual(self._h, _ptr(f), _ptr(u))

    def solve(self, q, rtol=1e-10, max_cycles=100, fixed=0):
        """V-cycles from u = 0: to rtol, or exactly `fixed` cycles. Returns (u, cycles, hist)."""
        q = _arr(q)
        u = np.zeros_like(q)
        hist = np.zeros(max(max_cycles, fixed, 1))
        c = lib().orc_solve(self._h, _ptr(q), _ptr(u), rtol, max_cycles, fixed, _ptr(hist), len(hist))
        return u, c, hist[:c].copy()

    def adjoint(self, w, rtol=1e-10, max_cycles=100, fixed=0):
        """Transposed V-cycle iteration: S_m^T w (fixed=m) or A^{-1} w to rtol."""
        w = _arr(w)
        lam = np.zeros_like(w)
        hist = np.zeros(max(max_cycles, fixed, 1))
        c = lib().orc_adjoint(self._h, _ptr(w), _ptr(lam), rtol, max_cycles, fixed, _ptr(hist),
                              len(hist))
        return lam, c, hist[:c].copy()

    def adjoint_literal(self, w, m):
        """S_m^dagger w as the reversed composition of per-operation adjoints (Eq. 18)."""
        w = _arr(w)
        qb = np.zeros_like(w)
        lib().orc_adjoint_literal(self._h, _ptr(w), _ptr(qb), int(m))
        return qb

    def vcycle(self, f, u, transposed=False):
        f = _arr(f)
        u = _arr(u).copy()
        lib().orc_vcycle(self._h, _ptr(f), _ptr(u), int(transposed))
        return u

    def vjp(self, u, w, rtol=1e-10, max_cycles=100, fixed=0):
        """(qbar, Dbar, mubar) of <w, u(q, D, mu)>; fixed=m uses the count-matched adjoint."""
        lam, c, _ = self.adjoint(w, rtol=rtol, max_cycles=max_cycles, fixed=fixed)
        Db, mb = grad(self.D, self.h, u, lam, self.harmonic)
        return lam, Db, mb, c

    def jvp(self, u, dq, dD=None, dmu=None, rtol=1e-10, max_cycles=100, fixed=0):
        """du = S(dq - dA u) (Sec. 2.3: the push-forward applies S to the perturbation)."""
        rhs = _arr(dq).copy()
        if dD is not None or dmu is not None:
            rhs = rhs - dA_apply(self.D, self.h, dD, dmu, u, self.harmonic)
        du, c, _ = self.solve(rhs, rtol=rtol, max_cycles=max_cycles, fixed=fixed)
        return du, c


def interior_index(shape):
    nz, ny, nx = shape
    kk, jj, ii = np.meshgrid(np.arange(1, nz - 1), np.arange(1, ny - 1), np.arange(1, nx - 1),
                             indexing="ij")
    return np.ravel_multi_index((kk.ravel(), jj.ravel(), ii.ravel()), shape)


def assemble(D, mu, h, harmonic=False):
    """Sparse matrix of the oracle's A on interior unknowns, built column by column
    by applying `apply` to unit vectors (for library direct solves on small grids)."""
    import scipy.sparse as sp
    shape = D.shape
    idx = interior_index(shape)
    n = idx.size
    pos = -np.ones(int(np.prod(shape)), dtype=np.int64)
    pos[idx] = np.arange(n)
    rows, cols, vals = [], [], []
    e = np.zeros(shape)
    ef = e.reshape(-1)
    for c in range(n):
        ef[idx[c]] = 1.0
        col = apply(D, mu, h, e, harmonic).reshape(-1)
        ef[idx[c]] = 0.0
        nz_ = np.nonzero(col)[0]
        rows.append(pos[nz_])
        cols.append(np.full(nz_.size, c))
        vals.append(col[nz_])
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    return A, idx


def direct_solve(D, mu, h, q, harmonic=False):
    """u = A^{-1} q by scipy's sparse direct solver on the assembled oracle matrix."""
    import scipy.sparse.linalg as spla
    A, idx = assemble(D, mu, h, harmonic)
    u = np.zeros(D.shape)
    u.reshape(-1)[idx] = spla.spsolve(A.tocsc(), _arr(q).reshape(-1)[idx])
    return u


# ---------------------------------------------------------------------------
# The application's forward model (Sec. 2.5.3, Eq. response): R(q) = M(mu S(q)),
# the absorbed energy density L_e = mu rho on the voxels outside the masked edge
# region (Sec. 2.5.1: data masked to a depth of 0.2 cm on all edges). Reading:
# a vertex at coordinate x = i h on an axis of length (n-1) h is kept when its
# distance to both faces, min(x, (n-1) h - x), is at least the edge depth (with a
# relative slack of 1e-12 for the rounding of i h); fields are returned on the
# full grid with the other voxels set to 0.

def edge_mask(shape, h, edge):
    """Boolean mask of the kept voxels (Eq. response's M), from the distances."""
    keep = np.ones(shape, dtype=bool)
    for axis, n in enumerate(shape):
        x = np.arange(n) * h
        dist = np.minimum(x, (n - 1) * h - x)
        ok = dist >= edge * (1.0 - 1e-12)
        sl = [None] * len(shape)
        sl[axis] = slice(None)
        keep &= ok[tuple(sl)]
    return keep


def response(H, q, edge, rtol=1e-10):
    """(L_e, u): u = S(q) by the oracle's V-cycles, L_e = M(mu u)."""
    u, _, _ = H.solve(q, rtol=rtol)
    return np.where(edge_mask(H.shape, H.h, edge), H.mu * u, 0.0), u


def response_jvp(H, u, dq, dD, dmu, edge, rtol=1e-10):
    """Tangent of L_e: M(dmu u + mu du), du = S(dq - dA u)."""
    dq = np.zeros(H.shape) if dq is None else dq
    du, _ = H.jvp(u, dq, dD, dmu, rtol=rtol)
    t = H.mu * du
    if dmu is not None:
        t = t + _arr(dmu) * u
    return np.where(edge_mask(H.shape, H.h, edge), t, 0.0)


def response_vjp(H, u, rbar, edge, rtol=1e-10):
    """Pull-back of a cotangent rbar on L_e. The chain rule through L_e = M(mu u):
    the cotangent of u is w = mu M^T rbar (interior), the solve's VJP gives
    (qbar, Dbar, mubar_S), and the explicit factor mu adds u M^T rbar to mubar."""
    m = edge_mask(H.shape, H.h, edge)
    w = np.where(m, H.mu * _arr(rbar), 0.0)
    w[0, :, :] = w[-1, :, :] = 0.0
    w[:, 0, :] = w[:, -1, :] = 0.0
    w[:, :, 0] = w[:, :, -1] = 0.0
    qb, Db, mb, _ = H.vjp(u, w, rtol=rtol)
    mb = mb + np.where(m, u * _arr(rbar), 0.0)
    return qb, Db, mb
