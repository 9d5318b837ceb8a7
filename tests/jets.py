"""Truncated multivariate Taylor arithmetic ("jets") over numpy arrays.

A Jet holds the Taylor coefficients c_a = (d^a f)/a! of a function of the four
variables (t, x, y, z) about a set of evaluation points, for every multi-index
a of total degree <= order.  Arithmetic and elementary functions propagate the
coefficients exactly (up to rounding), so derivatives of composite
expressions come out without finite differencing.  Used only by the tests to
evaluate exact solutions; it knows nothing of the method under test.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

NVAR = 4
MAXORD = 3
# multi-indices of total degree <= MAXORD, sorted by degree
MIDX = sorted((a for a in itertools.product(range(MAXORD + 1), repeat=NVAR) if sum(a) <= MAXORD),
              key=lambda a: (sum(a), tuple(-v for v in a)))
POS = {a: i for i, a in enumerate(MIDX)}
DEG = np.array([sum(a) for a in MIDX])
NC = len(MIDX)


def _pairs(order):
    """For each output coefficient c (degree <= order), index pairs (a, b) with a + b = c."""
    out = []
    for c in MIDX:
        if sum(c) > order:
            out.append((np.zeros(0, int), np.zeros(0, int)))
            continue
        ia, ib = [], []
        for a in MIDX:
            b = tuple(ci - ai for ci, ai in zip(c, a))
            if min(b) >= 0:
                ia.append(POS[a])
                ib.append(POS[b])
        out.append((np.array(ia), np.array(ib)))
    return out


_PAIRS = {o: _pairs(o) for o in range(MAXORD + 1)}


class Jet:
    __slots__ = ("c", "order")

    def __init__(self, c, order):
        self.c = c  # shape (NC, ...)
        self.order = order

    # ---- construction
    @staticmethod
    def const(v, shape, order=MAXORD):
        c = np.zeros((NC,) + shape)
        c[0] = v
        return Jet(c, order)

    @staticmethod
    def var(k, v, order=MAXORD):
        v = np.asarray(v, dtype=np.float64)
        c = np.zeros((NC,) + v.shape)
        c[0] = v
        e = [0] * NVAR
        e[k] = 1
        c[POS[tuple(e)]] = 1.0
        return Jet(c, order)

    @property
    def shape(self):
        return self.c.shape[1:]

    @property
    def val(self):
        return self.c[0]

    def _mask(self, order):
        c = self.c.copy()
        c[DEG > order] = 0.0
        return c

    # ---- arithmetic
    def _lift(self, o):
        if isinstance(o, Jet):
            return o
        return Jet.const(o, self.shape, MAXORD)

    def __add__(self, o):
        o = self._lift(o)
        order = min(self.order, o.order)
        return Jet(self._mask(order) + o._mask(order), order)

    __radd__ = __add__

    def __neg__(self):
        return Jet(-self.c, self.order)

    def __sub__(self, o):
        return self + (-self._lift(o))

    def __rsub__(self, o):
        return self._lift(o) - self

    def __mul__(self, o):
        if not isinstance(o, Jet):
            return Jet(self.c * o, self.order)
        order = min(self.order, o.order)
        out = np.zeros((NC,) + np.broadcast_shapes(self.shape, o.shape))
        for ci, (ia, ib) in enumerate(_PAIRS[order]):
            if len(ia):
                out[ci] = np.sum(self.c[ia] * o.c[ib], axis=0)
        return Jet(out, order)

    __rmul__ = __mul__

    def __truediv__(self, o):
        if not isinstance(o, Jet):
            return Jet(self.c / o, self.order)
        return self * o.recip()

    def __rtruediv__(self, o):
        return self._lift(o) * self.recip()

    def __pow__(self, p):
        return self.apply(lambda v, n: _powder(v, n, p))

    # ---- elementary functions by Taylor composition
    def apply(self, derivs):
        """f(self) where derivs(v, n) returns d^n f / dv^n at v."""
        v0 = self.c[0]
        d = Jet(self.c.copy(), self.order)
        d.c[0] = 0.0
        out = Jet.const(derivs(v0, 0), self.shape, self.order)
        power = Jet.const(1.0, self.shape, self.order)
        for n in range(1, self.order + 1):
            power = power * d
            out = out + power * (derivs(v0, n) / math.factorial(n))
        out.order = self.order
        return out

    def recip(self):
        return self ** -1.0

    def sqrt(self):
        return self ** 0.5

    def log(self):
        def f(v, n):
            if n == 0:
                return np.log(v)
            return (-1.0) ** (n - 1) * math.factorial(n - 1) / v ** n
        return self.apply(f)

    def exp(self):
        return self.apply(lambda v, n: np.exp(v))

    def sin(self):
        return self.apply(lambda v, n: [np.sin, np.cos, lambda u: -np.sin(u), lambda u: -np.cos(u)][n % 4](v))

    def cos(self):
        return self.apply(lambda v, n: [np.cos, lambda u: -np.sin(u), lambda u: -np.cos(u), np.sin][n % 4](v))

    # ---- derivative
    def d(self, k):
        """Partial derivative with respect to variable k (order drops by one)."""
        out = np.zeros_like(self.c)
        for ci, a in enumerate(MIDX):
            if sum(a) >= self.order:
                continue
            b = list(a)
            b[k] += 1
            out[ci] = self.c[POS[tuple(b)]] * b[k]
        return Jet(out, self.order - 1)


def _powder(v, n, p):
    coef = 1.0
    for m in range(n):
        coef *= (p - m)
    return coef * v ** (p - n)


def sin(j):
    return j.sin()


def cos(j):
    return j.cos()


def sqrt(j):
    return j.sqrt()


def log(j):
    return j.log()
