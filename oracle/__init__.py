"""FP64 CPU oracle for the Stokeslet + stresslet treecode (arXiv:1811.12498).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports, links or calls anything here.

This module is a ctypes wrapper around ``oracle.c`` (plain C11 + OpenMP),
which follows the paper step by step:

* ``direct``            -- eq. (1.3), the velocity sum, from its definition;
* ``direct_grad``       -- gradients of sum g.u of that sum (f, h, nu, x),
                           from the derivatives of S and T;
* ``coulomb_coeffs``    -- recurrence (3.2) for the Coulomb coefficients b^k;
* ``taylor_stokeslet``  -- eq. (3.4), explicit a^k_ij;
* ``taylor_stresslet``  -- eq. (3.7), explicit a~^k_ijl;
* ``far_contracted``    -- eqs. (4.4) and (4.9), the contracted far field;
* ``far_explicit``      -- eq. (2.9), sum of a^k M^k + a~^k M~^k;
* ``moments``           -- the cluster moments of Section 2;
* ``Tree``              -- the octree of Section 5; per target, the
                           interaction list of the MAC (eq. 5.1) and its sum
                           (``treecode``, Algorithm 1's result); the same
                           lists decided at other positions with moved
                           particles (``treecode_frozen``), and the
                           far-field particle count per target
                           (``far_mass``).

Every function is pinned in ``tests/test_oracle_pins.py`` to something other
than itself: hand-computed values and the Stokes equations (``direct``),
finite differences (``direct_grad``), closed forms and the Legendre
generating function (``coulomb_coeffs``), an independent power-series
expansion (``taylor_*``), the explicit sum and the truncation rate against
the direct sum (``far_*``), the binomial translation identity (``moments``),
structural invariants, a plain walk of Algorithm 1, limits that reduce to the
direct sum, exact scaling laws and the paper's Tables 1 and 2 (``Tree``).
Parity unpinned: only the internal flattening order of the moments.

Arrays are float64, row-major ``(count, 3)``.  Multi-index quantities use
cubes of shape ``(P+1, P+1, P+1)`` (zero where ||k|| > P).
"""
import ctypes
import os

import numpy as np

from ._build import build as _build_lib, LIB_PATH

_lib = None
_P = ctypes.POINTER
_d = _P(ctypes.c_double)
_i64 = _P(ctypes.c_int64)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(
            os.path.join(os.path.dirname(__file__), "oracle.c")):
        _build_lib()
    lib = ctypes.CDLL(LIB_PATH)
    c_int, c_i64, c_dbl, vp = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    sig = {
        "orc_stokeslet": (None, [_d, _d, _d]),
        "orc_stresslet": (None, [_d, _d, _d]),
        "orc_direct": (None, [_d, _d, _d, _d, c_i64, _d, c_i64, _d, c_int]),
        "orc_direct_grad": (None, [_d, _d, _d, _d, c_i64, _d, _d, _d, _d, _d, c_int]),
        "orc_coulomb_coeffs": (None, [_d, c_int, _d]),
        "orc_taylor_stokeslet": (None, [_d, c_int, _d]),
        "orc_taylor_stresslet": (None, [_d, c_int, _d]),
        "orc_far_contracted": (None, [_d, c_int, _d, _d, _d]),
        "orc_far_explicit": (None, [_d, c_int, _d, _d, _d]),
        "orc_moments": (None, [_d, _d, _d, _d, vp, c_i64, _d, c_int, _d, _d]),
        "orc_tree_build": (vp, [_d, c_i64, c_int, c_int]),
        "orc_tree_free": (None, [vp]),
        "orc_tree_num_nodes": (c_i64, [vp]),
        "orc_tree_root": (None, [vp, _d, _d]),
        "orc_tree_export": (None, [vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "orc_tree_order": (None, [vp, _i64]),
        "orc_tree_quantized": (None, [vp, vp]),
        "orc_tree_moments": (c_int, [vp, _d, _d, _d, c_int]),
        "orc_tree_export_moments": (None, [vp, c_i64, _d, _d]),
        "orc_treecode": (c_int, [vp, _d, c_i64, c_dbl, c_int, _d, vp, vp, vp, c_int]),
        "orc_far_mass": (None, [vp, _d, c_i64, c_dbl, _i64]),
        "orc_treecode_frozen": (c_int, [vp, _d, _d, _d, _d, c_int, _d, _d, c_i64, c_dbl, _d, c_int]),
        "orc_max_threads": (c_int, []),
        "orc_stokeslet_reg": (None, [_d, _d, c_dbl, _d]),
        "orc_stresslet_reg": (None, [_d, _d, c_dbl, _d]),
        "orc_direct_reg": (None, [_d, _d, _d, _d, c_i64, _d, c_i64, c_dbl, _d, c_int]),
        "orc_coeffs_nu": (None, [_d, c_dbl, c_int, c_int, _d]),
        "orc_taylor_stokeslet_reg": (None, [_d, c_dbl, c_int, _d]),
        "orc_taylor_stresslet_reg": (None, [_d, c_dbl, c_int, _d]),
        "orc_far_reg": (None, [_d, c_dbl, c_int, _d, _d, _d]),
        "orc_treecode_eps": (c_int, [vp, _d, c_i64, c_dbl, c_int, c_dbl, _d, vp, vp, vp, c_int]),
        "orc_set_threads": (None, [c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    return a.ctypes.data_as(_d)


def _c3(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def max_threads():
    return _load().orc_max_threads()


_all_threads = None


def set_threads(n):
    """Threads of every later oracle call (n <= 0: all of the host's)."""
    global _all_threads
    lib = _load()
    if _all_threads is None:
        _all_threads = lib.orc_max_threads()
    lib.orc_set_threads(int(n) if n > 0 else _all_threads)


def stokeslet(x, y):
    """S_ij(x, y) of eq. (1.2a) as a 3x3 array."""
    out = np.empty(9)
    _load().orc_stokeslet(_ptr(_c3(x)), _ptr(_c3(y)), _ptr(out))
    return out.reshape(3, 3)


def stresslet(x, y):
    """T_ijl(x, y) of eq. (1.2b) as a 3x3x3 array."""
    out = np.empty(27)
    _load().orc_stresslet(_ptr(_c3(x)), _ptr(_c3(y)), _ptr(out))
    return out.reshape(3, 3, 3)


def direct(x, f, h, nu, targets=None, nthreads=0):
    """Velocity of eq. (1.3) at the targets (default: the sources), FP64."""
    x, f, h, nu = (_c3(a) for a in (x, f, h, nu))
    t = x if targets is None else _c3(targets)
    u = np.empty((t.shape[0], 3))
    _load().orc_direct(_ptr(x), _ptr(f), _ptr(h), _ptr(nu), x.shape[0], _ptr(t), t.shape[0], _ptr(u), nthreads)
    return u


def direct_grad(x, f, h, nu, g, nthreads=0):
    """Gradients of L = sum_m g_m . u_m (u the direct sum at the particles)
    with respect to f, h, nu and x, each (N, 3), from the derivatives of S and
    T as defined (FP64)."""
    x, f, h, nu, g = (_c3(a) for a in (x, f, h, nu, g))
    N = x.shape[0]
    out = {k: np.empty((N, 3)) for k in ("f", "h", "nu", "x")}
    _load().orc_direct_grad(_ptr(x), _ptr(f), _ptr(h), _ptr(nu), N, _ptr(g), _ptr(out["f"]), _ptr(out["h"]),
                            _ptr(out["nu"]), _ptr(out["x"]), nthreads)
    return out


def stokeslet_reg(x, y, eps):
    """Regularized Stokeslet S^eps_ij(x, y) (oracle.c), 3x3."""
    out = np.empty(9)
    _load().orc_stokeslet_reg(_ptr(_c3(x)), _ptr(_c3(y)), float(eps), _ptr(out))
    return out.reshape(3, 3)


def stresslet_reg(x, y, eps):
    """Regularized stresslet T^eps_ijl(x, y) (oracle.c), 3x3x3."""
    out = np.empty(27)
    _load().orc_stresslet_reg(_ptr(_c3(x)), _ptr(_c3(y)), float(eps), _ptr(out))
    return out.reshape(3, 3, 3)


def direct_reg(x, f, h, nu, eps, targets=None, nthreads=0):
    """Velocity of eq. (1.3) with the regularized kernels, FP64."""
    x, f, h, nu = (_c3(a) for a in (x, f, h, nu))
    t = x if targets is None else _c3(targets)
    u = np.empty((t.shape[0], 3))
    _load().orc_direct_reg(_ptr(x), _ptr(f), _ptr(h), _ptr(nu), x.shape[0], _ptr(t), t.shape[0], float(eps), _ptr(u),
                           nthreads)
    return u


def coeffs_nu(d, eps, two_nu, P):
    """Taylor coefficients of (|x - y|^2 + eps^2)^(-two_nu/2) in y about y_c
    for ||k|| <= P (the generalized recurrence); d = x - y_c."""
    c = np.empty((P + 1,) * 3)
    _load().orc_coeffs_nu(_ptr(_c3(d)), float(eps), int(two_nu), P, _ptr(c))
    return c


def taylor_stokeslet_reg(d, eps, p):
    a = np.empty((9,) + (p + 1,) * 3)
    _load().orc_taylor_stokeslet_reg(_ptr(_c3(d)), float(eps), p, _ptr(a))
    return a.reshape((3, 3) + (p + 1,) * 3)


def taylor_stresslet_reg(d, eps, p):
    t = np.empty((27,) + (p + 1,) * 3)
    _load().orc_taylor_stresslet_reg(_ptr(_c3(d)), float(eps), p, _ptr(t))
    return t.reshape((3, 3, 3) + (p + 1,) * 3)


def far_reg(d, eps, p, Mf, Mt):
    """Regularized far field of one cluster (explicit Taylor coefficients)."""
    u = np.empty(3)
    _load().orc_far_reg(_ptr(_c3(d)), float(eps), p, _ptr(_c3(Mf)), _ptr(_c3(Mt)), _ptr(u))
    return u


def coulomb_coeffs(d, P):
    """b^k(x, y_c) for ||k|| <= P by recurrence (3.2); d = x - y_c."""
    b = np.empty((P + 1,) * 3)
    _load().orc_coulomb_coeffs(_ptr(_c3(d)), P, _ptr(b))
    return b


def taylor_stokeslet(d, p):
    """a^k_ij of eq. (3.4), shape (3, 3, p+1, p+1, p+1)."""
    a = np.empty((9,) + (p + 1,) * 3)
    _load().orc_taylor_stokeslet(_ptr(_c3(d)), p, _ptr(a))
    return a.reshape((3, 3) + (p + 1,) * 3)


def taylor_stresslet(d, p):
    """a~^k_ijl of eq. (3.7), shape (3, 3, 3, p+1, p+1, p+1)."""
    t = np.empty((27,) + (p + 1,) * 3)
    _load().orc_taylor_stresslet(_ptr(_c3(d)), p, _ptr(t))
    return t.reshape((3, 3, 3) + (p + 1,) * 3)


def moments(y, f, h, nu, yc, p):
    """Cluster moments (Section 2): Mf (3, cube), Mt (3, 3, cube)."""
    y, f, h, nu = (_c3(a) for a in (y, f, h, nu))
    n3 = (p + 1) ** 3
    Mf = np.empty(3 * n3)
    Mt = np.empty(9 * n3)
    _load().orc_moments(_ptr(y), _ptr(f), _ptr(h), _ptr(nu), None, y.shape[0], _ptr(_c3(yc)), p, _ptr(Mf),
                        _ptr(Mt))
    return Mf.reshape((3,) + (p + 1,) * 3), Mt.reshape((3, 3) + (p + 1,) * 3)


def far_contracted(d, p, Mf, Mt):
    """Far-field velocity of one cluster by eqs. (4.4) + (4.9)."""
    u = np.empty(3)
    _load().orc_far_contracted(_ptr(_c3(d)), p, _ptr(_c3(Mf)), _ptr(_c3(Mt)), _ptr(u))
    return u


def far_explicit(d, p, Mf, Mt):
    """Far-field velocity of one cluster by eq. (2.9) with explicit a^k, a~^k."""
    u = np.empty(3)
    _load().orc_far_explicit(_ptr(_c3(d)), p, _ptr(_c3(Mf)), _ptr(_c3(Mt)), _ptr(u))
    return u


class Tree:
    """Octree of Section 5 over positions x (N,3); see ``oracle.c``."""

    def __init__(self, x, N0, shrink=True):
        self.x = _c3(x)
        self.N = self.x.shape[0]
        self.N0 = int(N0)
        self.shrink = bool(shrink)
        self._h = _load().orc_tree_build(_ptr(self.x), self.N, self.N0, int(self.shrink))
        if not self._h:
            raise ValueError("oracle tree build rejected its arguments")
        self._keep = []
        self.p = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_tree_free(h)
            self._h = None

    @property
    def num_nodes(self):
        return int(_load().orc_tree_num_nodes(self._h))

    def root(self):
        lo = np.empty(3)
        side = np.empty(1)
        _load().orc_tree_root(self._h, _ptr(lo), _ptr(side))
        return lo, float(side[0])

    def nodes(self):
        n = self.num_nodes
        out = dict(begin=np.empty(n, np.int64), count=np.empty(n, np.int64), level=np.empty(n, np.int32),
                   cell=np.empty((n, 3), np.int64), nchild=np.empty(n, np.int32), child=np.empty((n, 8), np.int64),
                   yc=np.empty((n, 3)), rc2=np.empty(n))
        _load().orc_tree_export(self._h, *(out[k].ctypes.data for k in
                                           ("begin", "count", "level", "cell", "nchild", "child", "yc", "rc2")))
        return out

    def order(self):
        o = np.empty(self.N, np.int64)
        _load().orc_tree_order(self._h, o.ctypes.data_as(_i64))
        return o

    def quantized(self):
        q = np.empty((self.N, 3), np.uint32)
        _load().orc_tree_quantized(self._h, q.ctypes.data)
        return q

    def set_moments(self, f, h, nu, p):
        f, h, nu = _c3(f), _c3(h), _c3(nu)
        self._keep = [f, h, nu]
        rc = _load().orc_tree_moments(self._h, _ptr(f), _ptr(h), _ptr(nu), int(p))
        if rc != 0:
            raise ValueError("oracle moments rejected p=%d" % p)
        self.p = int(p)

    def node_moments(self, node):
        p = self.p
        n3 = (p + 1) ** 3
        Mf = np.empty(3 * n3)
        Mt = np.empty(9 * n3)
        _load().orc_tree_export_moments(self._h, node, _ptr(Mf), _ptr(Mt))
        return Mf.reshape((3,) + (p + 1,) * 3), Mt.reshape((3, 3) + (p + 1,) * 3)

    def treecode(self, targets, theta, p=None, counts=False, nthreads=0):
        """Treecode velocity (Algorithm 1's result) at each target: its
        interaction list by the MAC of eq. (5.1), then the sum of that list;
        returns u (M,3) [and per-target counts]."""
        p = self.p if p is None else int(p)
        t = _c3(targets)
        M = t.shape[0]
        u = np.empty((M, 3))
        nf = np.empty(M, np.int64)
        nl = np.empty(M, np.int64)
        npairs = np.empty(M, np.int64)
        rc = _load().orc_treecode(self._h, _ptr(t), M, float(theta), p, _ptr(u), nf.ctypes.data, nl.ctypes.data,
                                  npairs.ctypes.data, nthreads)
        if rc != 0:
            raise ValueError("oracle treecode needs moments of order >= p")
        if counts:
            return u, dict(far=nf, near_leaves=nl, near_pairs=npairs)
        return u

    def treecode_reg(self, targets, theta, eps, p=None, nthreads=0):
        """The same lists summed with the regularized kernels (eps > 0)."""
        p = self.p if p is None else int(p)
        t = _c3(targets)
        u = np.empty((t.shape[0], 3))
        rc = _load().orc_treecode_eps(self._h, _ptr(t), t.shape[0], float(theta), p, float(eps), _ptr(u), None, None,
                                      None, nthreads)
        if rc != 0:
            raise ValueError("oracle treecode needs moments of order >= p and eps >= 0")
        return u

    def treecode_frozen(self, xe, f, h, nu, p, td, te, theta, nthreads=0):
        """Frozen-structure velocity: MAC decisions at td, moments and direct
        sums at the moved sources xe, evaluation at the moved targets te."""
        xe, f, h, nu, td, te = (_c3(a) for a in (xe, f, h, nu, td, te))
        u = np.empty((te.shape[0], 3))
        rc = _load().orc_treecode_frozen(self._h, _ptr(xe), _ptr(f), _ptr(h), _ptr(nu), int(p), _ptr(td), _ptr(te),
                                         te.shape[0], float(theta), _ptr(u), nthreads)
        if rc != 0:
            raise ValueError("oracle frozen treecode rejected p")
        return u

    def far_mass(self, targets, theta):
        t = _c3(targets)
        m = np.empty(t.shape[0], np.int64)
        _load().orc_far_mass(self._h, _ptr(t), t.shape[0], float(theta), m.ctypes.data_as(_i64))
        return m


def rel_l2(a, b):
    """Relative L2 error of eq. (6.1): ||a - b|| / ||b||."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.sqrt(np.sum(b * b))
    return float(np.sqrt(np.sum((a - b) ** 2)) / den) if den > 0 else float(np.sqrt(np.sum(a * a)))
