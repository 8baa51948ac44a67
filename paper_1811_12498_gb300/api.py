"""Thin Python binding of the C ABI (include/tc.h) over torch CUDA tensors.

Only argument marshalling happens here: every step of the treecode runs in
the CUDA kernels of libtc.so.  Arrays of 3-vectors are float64 CUDA tensors
of shape (3, count) (structure of arrays), the layout of the C ABI.
``soa`` converts an (count, 3) tensor.

    tc = Treecode(precision="mixed", shrink=True)
    tc.build(x, N0=2000)          # eq. (1.3) sources, Section 5 octree
    tc.moments(f, h, nu, p=8)     # Section 2 moments
    u = tc.eval(theta=0.5, p=8)   # Algorithm 1 at the sources
"""
import ctypes

import torch

from ._lib import PHASES, TCConfig, lib

TC_FP64, TC_MIXED = 0, 1
_STATUS = {0: "TC_OK", 1: "TC_EINVAL", 2: "TC_ENOMEM", 3: "TC_ECUDA", 4: "TC_ESTATE", 5: "TC_ETIMEOUT",
           6: "TC_EDEVICE"}


class TCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


def _prec(precision):
    if precision in (TC_FP64, "fp64", "FP64"):
        return TC_FP64
    if precision in (TC_MIXED, "mixed", "MIXED"):
        return TC_MIXED
    raise ValueError("precision must be 'fp64' or 'mixed'")


def _check(status, handle=None):
    if status != 0:
        msg = lib().tc_last_error(handle)
        raise TCError(status, msg.decode() if msg else "")


def soa(a):
    """(count, 3) -> contiguous (3, count) float64 on the same device."""
    return a.t().contiguous().to(torch.float64)


def _vec3(a, name, count=None):
    if a is None:
        return None
    if not isinstance(a, torch.Tensor) or not a.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if a.dtype != torch.float64 or a.dim() != 2 or a.shape[0] != 3 or not a.is_contiguous():
        raise ValueError("%s must be a contiguous float64 tensor of shape (3, n)" % name)
    if count is not None and a.shape[1] != count:
        raise ValueError("%s has %d entries, expected %d" % (name, a.shape[1], count))
    return a


def _host3(a, name, count=None):
    if not isinstance(a, torch.Tensor) or a.is_cuda:
        raise TypeError("%s must be a host (CPU) tensor" % name)
    if a.dtype != torch.float64 or a.dim() != 2 or a.shape[0] != 3 or not a.is_contiguous():
        raise ValueError("%s must be a contiguous float64 tensor of shape (3, n)" % name)
    if count is not None and a.shape[1] != count:
        raise ValueError("%s has %d entries, expected %d" % (name, a.shape[1], count))
    return a


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.data_ptr())


def _stream_ptr(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Treecode:
    """One treecode context (tc_ctx): tree, moments and interaction lists."""

    def __init__(self, precision="mixed", shrink=True, stream=None, rec64=False, reg_eps=0.0):
        """rec64: in mixed precision, run the far-field recurrence in FP64 for
        p >= 8 (tc_config.rec64).  reg_eps > 0: the regularized Stokeslet and
        stresslet with that eps (tc_config.reg_eps)."""
        self.precision = _prec(precision)
        self.stream = torch.cuda.current_stream() if stream is None else stream
        cfg = TCConfig(self.precision, int(bool(shrink)), _stream_ptr(self.stream), int(bool(rec64)), 0,
                       float(reg_eps))
        h = ctypes.c_void_p()
        _check(lib().tc_create(ctypes.byref(h), ctypes.byref(cfg)))
        self._h = h
        self.N = 0
        self.p = None
        self._keep = ()

    def close(self):
        if getattr(self, "_h", None):
            lib().tc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        _check(st, self._h)

    def build(self, x, N0):
        x = _vec3(x, "x")
        self.N = x.shape[1]
        self._chk(lib().tc_build(self._h, _ptr(x), self.N, int(N0)))
        return self

    def moments(self, f, h, nu, p):
        f, h, nu = (_vec3(a, n, self.N) for a, n in ((f, "f"), (h, "h"), (nu, "nu")))
        self._chk(lib().tc_moments(self._h, _ptr(f), _ptr(h), _ptr(nu), int(p)))
        self._keep = (f, h, nu)  # inputs must outlive the enqueued kernels
        self.p = int(p)
        return self

    def eval(self, theta, p=None, targets=None, out=None):
        p = self.p if p is None else int(p)
        t = _vec3(targets, "targets")
        M = self.N if t is None else t.shape[1]
        if out is None:
            with torch.cuda.stream(self.stream):
                out = torch.empty((3, M), dtype=torch.float64, device="cuda")
        _vec3(out, "out", M)
        self._chk(lib().tc_eval(self._h, _ptr(t), M, float(theta), p, _ptr(out)))
        self._M = M
        self._keep_t = t
        return out

    def velocity_host(self, x, f, h, nu, N0, theta, p, out=None):
        """build + moments + eval from HOST tensors (tc_velocity_host): x, f,
        h, nu are (3, N) float64 CPU tensors (pinned memory copies
        asynchronously); returns u as a (3, N) CPU tensor, complete on return
        (pinned when x is)."""
        x = _host3(x, "x")
        N = x.shape[1]
        f, h, nu = (_host3(a, n, N) for a, n in ((f, "f"), (h, "h"), (nu, "nu")))
        if out is None:
            out = torch.empty((3, N), dtype=torch.float64, pin_memory=x.is_pinned())
        _host3(out, "out", N)
        self._chk(lib().tc_velocity_host(self._h, _ptr(x), _ptr(f), _ptr(h), _ptr(nu), N, int(N0), float(theta),
                                         int(p), _ptr(out)))
        self.N, self.p, self._M = N, int(p), N
        self._keep, self._keep_t = (), None
        return out

    def update_positions(self, x):
        """Move the particles (tc_update_positions): tree, centres, radii and
        the last eval's lists stay; moments and tables are recomputed."""
        x = _vec3(x, "x", self.N)
        self._chk(lib().tc_update_positions(self._h, _ptr(x)))
        self._keep_x = x
        return self

    def eval_frozen(self, out=None):
        """Velocity at the moved particles with the last eval's lists
        (tc_eval_frozen); (3, N)."""
        if out is None:
            with torch.cuda.stream(self.stream):
                out = torch.empty((3, self.N), dtype=torch.float64, device="cuda")
        _vec3(out, "out", self.N)
        self._chk(lib().tc_eval_frozen(self._h, _ptr(out)))
        return out

    def sync(self):
        self._chk(lib().tc_sync(self._h))

    def adjoint(self, g, f=True, h=True, nu=True, x=True, t=False):
        """Gradients of L = sum_m g^m . u^m with the structure of the last eval
        frozen (tc_adjoint).  g: (3, M).  Returns a dict with the requested
        entries among f, h, nu, x (each (3, N)) and t (targets, (3, M))."""
        M = self._M
        g = _vec3(g, "g", M)
        out = {}
        with torch.cuda.stream(self.stream):
            for k, want, n in (("f", f, self.N), ("h", h, self.N), ("nu", nu, self.N), ("x", x, self.N),
                               ("t", t, M)):
                if want:
                    out[k] = torch.empty((3, n), dtype=torch.float64, device="cuda")
        self._chk(lib().tc_adjoint(self._h, _ptr(g), _ptr(out.get("f")), _ptr(out.get("h")), _ptr(out.get("nu")),
                                   _ptr(out.get("x")), _ptr(out.get("t"))))
        self._keep_g = g
        return out

    def profile(self, enable=True):
        """Enable per-phase CUDA-event timing (see phase_times).  enable=2
        runs every phase on one stream, one after the other, so that each
        phase time is that work's own duration (by default the moment passes,
        the far field and the adjoint's far-gradient passes run beside the
        near field)."""
        self._chk(lib().tc_profile(self._h, int(enable) if enable in (0, 1, 2) else int(bool(enable))))

    def phase_times(self):
        """ms of the most recent run of each phase (None if not run)."""
        ms = (ctypes.c_double * len(PHASES))()
        self._chk(lib().tc_phase_times(self._h, ms))
        return {k: (v if v >= 0 else None) for k, v in zip(PHASES, ms)}

    def stats(self):
        near, far, nodes = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._chk(lib().tc_stats(self._h, ctypes.byref(near), ctypes.byref(far), ctypes.byref(nodes)))
        return dict(near_pairs=near.value, far_interactions=far.value, clusters=nodes.value)

    def list_stats(self):
        """Interaction-list sizes of the last eval and the fraction of kernel
        lanes doing useful work in the far and near kernels."""
        fe, ne, ns = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._chk(lib().tc_list_stats(self._h, ctypes.byref(fe), ctypes.byref(ne), ctypes.byref(ns)))
        st = self.stats()
        return dict(far_entries=fe.value, near_entries=ne.value, near_entry_sources=ns.value,
                    far_lane_use=st["far_interactions"] / max(1, 32 * fe.value),
                    near_lane_use=st["near_pairs"] / max(1, 32 * ns.value))

    def tune(self, x, f, h, nu, thetas, orders, leaf_sizes, sample, target_E):
        """Fastest (theta, p, N0) of the grid whose error E at the sampled
        particles reaches target_E (tc_tune).  x, f, h, nu: (3, N) CUDA
        tensors; thetas, orders, leaf_sizes: sequences; sample: indices in
        [0, N).  Returns dict(best=(theta, p, N0) or None, table=[(theta, p,
        N0, seconds, E), ...] in the candidate order of tc_tune)."""
        import numpy as np
        x = _vec3(x, "x")
        N = x.shape[1]
        f, h, nu = (_vec3(a, n, N) for a, n in ((f, "f"), (h, "h"), (nu, "nu")))
        th = np.ascontiguousarray(thetas, dtype=np.float64)
        ps = np.ascontiguousarray(orders, dtype=np.int32)
        n0 = np.ascontiguousarray(leaf_sizes, dtype=np.int32)
        smp = np.ascontiguousarray(sample, dtype=np.int64)
        ncand = th.size * ps.size * n0.size
        sec = np.zeros(max(ncand, 1), np.float64)
        err = np.zeros(max(ncand, 1), np.float64)
        best = ctypes.c_int32(-1)
        vp = ctypes.c_void_p
        self._chk(lib().tc_tune(self._h, _ptr(x), _ptr(f), _ptr(h), _ptr(nu), N, vp(th.ctypes.data), th.size,
                                vp(ps.ctypes.data), ps.size, vp(n0.ctypes.data), n0.size, vp(smp.ctypes.data),
                                smp.size, float(target_E), vp(sec.ctypes.data), vp(err.ctypes.data),
                                ctypes.byref(best)))
        table = []
        k = 0
        for nl in n0:
            for p in ps:
                for t in th:
                    table.append((float(t), int(p), int(nl), float(sec[k]), float(err[k])))
                    k += 1
        self.N = N
        self.p = int(ps[-1])
        self._keep = (f, h, nu)
        b = best.value
        return dict(best=None if b < 0 else table[b][:3], table=table)

    def eval_counts(self):
        M = self.N if getattr(self, "_M", None) is None else self._M
        nf = torch.empty(M, dtype=torch.int64, device="cuda")
        nn = torch.empty(M, dtype=torch.int64, device="cuda")
        self._chk(lib().tc_eval_counts(self._h, _ptr(nf), _ptr(nn)))
        return nf, nn

    def tree_info(self):
        n, d = ctypes.c_int64(), ctypes.c_int32()
        lo = (ctypes.c_double * 3)()
        side = ctypes.c_double()
        self._chk(lib().tc_tree_info(self._h, ctypes.byref(n), ctypes.byref(d), lo, ctypes.byref(side)))
        return dict(nnodes=n.value, depth=d.value, lo=list(lo), side=side.value)

    def tree_export(self):
        import numpy as np
        n = self.tree_info()["nnodes"]
        out = dict(begin=np.empty(n, np.int32), count=np.empty(n, np.int32), level=np.empty(n, np.int32),
                   cell=np.empty((n, 3), np.int32), parent=np.empty(n, np.int32), first_child=np.empty(n, np.int32),
                   nchild=np.empty(n, np.int32), yc=np.empty((n, 3)), rc2=np.empty(n))
        keys = ("begin", "count", "level", "cell", "parent", "first_child", "nchild", "yc", "rc2")
        self._chk(lib().tc_tree_export(self._h, *(ctypes.c_void_p(out[k].ctypes.data) for k in keys)))
        return out

    def tree_order(self):
        import numpy as np
        o = np.empty(self.N, np.int32)
        self._chk(lib().tc_tree_order(self._h, ctypes.c_void_p(o.ctypes.data)))
        return o

    def moments_export(self, node):
        import numpy as np
        q = self.p + 1
        Mf = np.empty((3, q, q, q))
        Mt = np.empty((3, 3, q, q, q))
        self._chk(lib().tc_moments_export(self._h, int(node), ctypes.c_void_p(Mf.ctypes.data),
                                          ctypes.c_void_p(Mt.ctypes.data)))
        return Mf, Mt


def direct(x, f, h, nu, targets=None, precision="fp64", out=None, stream=None):
    """Direct sum of eq. (1.3) (tc_direct); returns u of shape (3, M)."""
    x = _vec3(x, "x")
    N = x.shape[1]
    f, h, nu = (_vec3(a, n, N) for a, n in ((f, "f"), (h, "h"), (nu, "nu")))
    t = _vec3(targets, "targets")
    M = N if t is None else t.shape[1]
    if out is None:
        out = torch.empty((3, M), dtype=torch.float64, device=x.device)
    _vec3(out, "out", M)
    _check(lib().tc_direct(_ptr(x), _ptr(f), _ptr(h), _ptr(nu), N, _ptr(t), M, _prec(precision),
                           _stream_ptr(stream), _ptr(out)))
    return out


def direct_reg(x, f, h, nu, eps, targets=None, precision="fp64", out=None, stream=None):
    """O(N M) sum of eq. (1.3) with the regularized kernels (tc_direct_reg)."""
    x = _vec3(x, "x")
    N = x.shape[1]
    f, h, nu = (_vec3(a, n, N) for a, n in ((f, "f"), (h, "h"), (nu, "nu")))
    t = _vec3(targets, "targets")
    M = N if t is None else t.shape[1]
    if out is None:
        out = torch.empty((3, M), dtype=torch.float64, device="cuda")
    _vec3(out, "out", M)
    _check(lib().tc_direct_reg(_ptr(x), _ptr(f), _ptr(h), _ptr(nu), N, _ptr(t), M, float(eps), _prec(precision),
                               _stream_ptr(stream), _ptr(out)))
    return out


class Batch:
    """Many independent systems evaluated together (tc_batch_*).

    Arrays are segmented (3, ntot) float64 CUDA tensors; `offsets` is a list
    of nsys + 1 particle offsets.  eval() runs all systems' far and near
    fields as persistent kernels replayed from a CUDA graph."""

    def __init__(self, precision="mixed", shrink=True, stream=None, autotune=True, graph=True, rec64=False):
        self.stream = torch.cuda.current_stream() if stream is None else stream
        cfg = TCConfig(_prec(precision), int(bool(shrink)), _stream_ptr(self.stream), int(bool(rec64)), 0)
        h = ctypes.c_void_p()
        _check(lib().tc_batch_create(ctypes.byref(h), ctypes.byref(cfg)))
        self._h = h
        self._chk(lib().tc_batch_set(h, int(bool(autotune)), int(bool(graph))))
        self.offsets = None
        self._keep = ()

    def _chk(self, st):
        if st != 0:
            msg = lib().tc_batch_last_error(self._h)
            raise TCError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None):
            lib().tc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build(self, x, offsets, N0):
        x = _vec3(x, "x", int(offsets[-1]))
        self.offsets = [int(v) for v in offsets]
        off = (ctypes.c_int64 * len(self.offsets))(*self.offsets)
        self._chk(lib().tc_batch_build(self._h, _ptr(x), len(self.offsets) - 1, off, int(N0)))
        self._keep_x = x
        return self

    def moments(self, f, h, nu, p):
        n = self.offsets[-1]
        f, h, nu = (_vec3(a, k, n) for a, k in ((f, "f"), (h, "h"), (nu, "nu")))
        self._chk(lib().tc_batch_moments(self._h, _ptr(f), _ptr(h), _ptr(nu), int(p)))
        self._keep = (f, h, nu)
        return self

    def eval(self, theta, p, out=None):
        n = self.offsets[-1]
        if out is None:
            with torch.cuda.stream(self.stream):
                out = torch.empty((3, n), dtype=torch.float64, device="cuda")
        _vec3(out, "out", n)
        self._chk(lib().tc_batch_eval(self._h, float(theta), int(p), _ptr(out)))
        return out

    def eval_separate(self, theta, p, outs=None):
        """One ordinary tc_eval per system; returns the list of (3, n_s) outputs."""
        sizes = [b - a for a, b in zip(self.offsets[:-1], self.offsets[1:])]
        if outs is None:
            with torch.cuda.stream(self.stream):
                outs = [torch.empty((3, n), dtype=torch.float64, device="cuda") for n in sizes]
        arr = (ctypes.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
        self._chk(lib().tc_batch_eval_separate(self._h, float(theta), int(p), arr))
        return outs

    def info(self):
        sh = (ctypes.c_int32 * 4)()
        ms = (ctypes.c_float * 2)()
        self._chk(lib().tc_batch_info(self._h, sh, ms))
        return dict(far_warps=sh[0], far_blocks=sh[1], near_warps=sh[2], near_blocks=sh[3],
                    far_ms=ms[0], near_ms=ms[1])

    def system_stats(self, s):
        h = lib().tc_batch_system(self._h, int(s))
        near, far, nodes = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().tc_stats(h, ctypes.byref(near), ctypes.byref(far), ctypes.byref(nodes)), h)
        return dict(near_pairs=near.value, far_interactions=far.value, clusters=nodes.value)


class StokesTreecode(torch.autograd.Function):
    """u = treecode velocity (eq. 1.3 by Algorithm 1) as a differentiable op.

    forward(x, f, h, nu, theta, p, N0, precision, shrink): x, f, h, nu are
    (3, N) float64 CUDA tensors; returns u (3, N) at the particles.
    backward: the adjoint with the tree and interaction lists of the forward
    pass frozen (tc_adjoint); gradients for x, f, h and nu.
    """

    @staticmethod
    def forward(ctx, x, f, h, nu, theta, p, N0, precision="mixed", shrink=True):
        tc = Treecode(precision, shrink)
        tc.build(x.detach(), N0).moments(f.detach(), h.detach(), nu.detach(), p)
        u = tc.eval(theta, p)
        ctx.tc = tc
        return u

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, gu):
        tc = ctx.tc
        if tc is None:
            raise RuntimeError("StokesTreecode: backward ran twice on one forward pass; the adjoint releases the "
                               "frozen tree and lists after its first run (use a fresh forward pass)")
        need = ctx.needs_input_grad
        gr = tc.adjoint(gu.contiguous(), f=need[1], h=need[2], nu=need[3], x=need[0])
        tc.sync()
        tc.close()
        ctx.tc = None
        return gr.get("x"), gr.get("f"), gr.get("h"), gr.get("nu"), None, None, None, None, None


def stokes_velocity(x, f, h, nu, theta, p, N0, precision="mixed", shrink=True):
    """Differentiable treecode velocity at the particles (see StokesTreecode)."""
    return StokesTreecode.apply(x, f, h, nu, theta, p, N0, precision, shrink)


def kernel_launches():
    """Kernels launched by libtc.so in this process so far."""
    return int(lib().tc_kernel_launches())


def fma_peak(precision="mixed", stream=None):
    """Measured FP32 (precision "mixed") or FP64 FMA peak of the current
    device in TFLOP/s (tc_fma_peak)."""
    out = ctypes.c_double()
    _check(lib().tc_fma_peak(_prec(precision), _stream_ptr(stream), ctypes.byref(out)))
    return out.value


def fail_allocations(after):
    """Host-side injection: after `after` further device allocations by the
    library every allocation fails as out of memory (TC_ENOMEM); after < 0
    switches it off (tc_fail_allocations)."""
    lib().tc_fail_allocations(int(after))


def velocity(x, f, h, nu, theta, p, N0, precision="mixed", shrink=True, targets=None):
    """One-shot treecode velocity (build + moments + eval); u of shape (3, M)."""
    tc = Treecode(precision, shrink)
    try:
        tc.build(x, N0).moments(f, h, nu, p)
        u = tc.eval(theta, p, targets)
        tc.sync()
        return u
    finally:
        tc.close()
