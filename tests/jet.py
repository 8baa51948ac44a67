"""Truncated multivariate power series ("jets") in t = (t1, t2, t3).

Used by the tests to expand the kernels S(x, y_c + t) and T(x, y_c + t) in t
directly from their definitions (eqs. 1.2a,b), independently of the
recurrences (3.2), (3.4) and (3.7).  A jet of order P is a cube c[k1,k2,k3]
holding the coefficient of t^k for ||k|| <= P (zero elsewhere).
"""
import numpy as np


class Jet:
    def __init__(self, P, c=None):
        self.P = P
        self.c = np.zeros((P + 1,) * 3) if c is None else c

    @classmethod
    def const(cls, P, v):
        j = cls(P)
        j.c[0, 0, 0] = v
        return j

    @classmethod
    def var(cls, P, axis, v0=0.0):
        """The series v0 + t_axis."""
        j = cls.const(P, v0)
        idx = [0, 0, 0]
        idx[axis] = 1
        if P >= 1:
            j.c[tuple(idx)] = 1.0
        return j

    def _mask(self):
        k = np.arange(self.P + 1)
        return (k[:, None, None] + k[None, :, None] + k[None, None, :]) <= self.P

    def __add__(self, o):
        if not isinstance(o, Jet):
            o = Jet.const(self.P, o)
        return Jet(self.P, self.c + o.c)

    __radd__ = __add__

    def __neg__(self):
        return Jet(self.P, -self.c)

    def __sub__(self, o):
        return self + (-o if isinstance(o, Jet) else -o)

    def __rsub__(self, o):
        return (-self) + o

    def __mul__(self, o):
        if not isinstance(o, Jet):
            return Jet(self.P, self.c * o)
        P = self.P
        out = np.zeros_like(self.c)
        nz = np.argwhere(self.c != 0)
        for a1, a2, a3 in nz:
            if a1 + a2 + a3 > P:
                continue
            v = self.c[a1, a2, a3]
            out[a1:, a2:, a3:] += v * o.c[:P + 1 - a1, :P + 1 - a2, :P + 1 - a3]
        out[~self._mask()] = 0.0
        return Jet(P, out)

    __rmul__ = __mul__

    def rpow(self, alpha):
        """self^(-alpha) for a jet with a positive constant term (binomial series)."""
        P = self.P
        s0 = self.c[0, 0, 0]
        eps = Jet(P, self.c.copy())
        eps.c[0, 0, 0] = 0.0
        eps = eps * (1.0 / s0)
        out = Jet.const(P, 1.0)
        term = Jet.const(P, 1.0)
        coef = 1.0
        for n in range(1, P + 1):
            coef *= (-alpha - (n - 1)) / n  # binomial(-alpha, n)
            term = term * eps
            out = out + term * coef
        return out * (s0 ** -alpha)

    def rpow_half(self):
        """self^(-1/2) for a jet with a positive constant term."""
        return self.rpow(0.5)


def kernel_jets(d, P):
    """Jets of G, S_ij and T_ijl at y = y_c + t, with d = x - y_c."""
    t = [Jet.var(P, a) for a in range(3)]
    dm = [t[a] * -1.0 + d[a] for a in range(3)]  # components of x - y = d - t
    r2 = dm[0] * dm[0] + dm[1] * dm[1] + dm[2] * dm[2]
    G = r2.rpow_half()
    G3 = G * G * G
    G5 = G3 * G * G
    S = [[(Jet.const(P, 1.0) * G if i == j else Jet(P)) + dm[i] * dm[j] * G3 for j in range(3)] for i in range(3)]
    T = [[[dm[i] * dm[j] * dm[l] * G5 for l in range(3)] for j in range(3)] for i in range(3)]
    return G, S, T


def reg_kernel_jets(d, eps, P):
    """Jets of the regularized kernels at y = y_c + t, d = x - y_c, straight
    from their definitions: with s = |x - y|^2 + eps^2,
    S^eps_ij = (delta_ij (|x - y|^2 + 2 eps^2) + (x - y)_i (x - y)_j) s^(-3/2),
    T^eps_ijl = ((x - y)_i (x - y)_j (x - y)_l + (eps^2 / 2)(delta_ij (x - y)_l
    + delta_jl (x - y)_i + delta_il (x - y)_j)) s^(-5/2)."""
    t = [Jet.var(P, a) for a in range(3)]
    dm = [t[a] * -1.0 + d[a] for a in range(3)]
    r2 = dm[0] * dm[0] + dm[1] * dm[1] + dm[2] * dm[2]
    s = r2 + eps * eps
    s32 = s.rpow(1.5)
    s52 = s.rpow(2.5)
    e2 = eps * eps
    S = [[((r2 + 2.0 * e2) if i == j else Jet(P)) * s32 + dm[i] * dm[j] * s32 for j in range(3)] for i in range(3)]
    T = [[[(dm[i] * dm[j] * dm[l]
            + ((dm[l] if i == j else Jet(P)) + (dm[i] if j == l else Jet(P)) + (dm[j] if i == l else Jet(P)))
            * (0.5 * e2)) * s52
           for l in range(3)] for j in range(3)] for i in range(3)]
    return S, T
