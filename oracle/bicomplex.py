"""Bicomplex numbers for second-order complex steps (X-SLAM Sec. 3: the second derivatives come from
two imaginary units).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A bicomplex number is z = z1 + z2 i2 with z1, z2 complex (imaginary unit i1) and i1^2 = i2^2 = -1,
i1 i2 = i2 i1. With x = x0 + h i1 e_j + h i2 e_k, f(x) = f(x0) + h i1 df_j + h i2 df_k + h^2 i1 i2 d2f_jk
+ O(h^2) real and O(h^3) imaginary parts, so d2f_jk = Im(z2) / h^2 (the i1 i2 part) with no
subtraction of nearly equal numbers. Arrays: z1, z2 are numpy complex arrays of one shape.

Products and quotients are exact bicomplex operations. A function g(z) that is analytic at z1 is
evaluated as g(z1) + g'(z1) z2 i2: the dropped term is -g''(z1) z2^2 / 2, a real part of order h^2
relative (below double precision for h = 1e-20) with imaginary parts of order h^3.
"""
from __future__ import annotations

import numpy as np


class Bicomplex:
    __array_priority__ = 1000  # numpy defers to our operators

    def __init__(self, z1, z2=None):
        self.z1 = np.asarray(z1, np.complex128)
        self.z2 = np.zeros_like(self.z1) if z2 is None else np.asarray(z2, np.complex128)

    # -- parts ----------------------------------------------------------------------------------
    @property
    def real(self):
        return self.z1.real

    def i1(self):
        return self.z1.imag

    def i2(self):
        return self.z2.real

    def i1i2(self):
        return self.z2.imag

    # -- arithmetic -----------------------------------------------------------------------------
    @staticmethod
    def _lift(o):
        return o if isinstance(o, Bicomplex) else Bicomplex(o)

    def __add__(self, o):
        o = self._lift(o)
        return Bicomplex(self.z1 + o.z1, self.z2 + o.z2)

    __radd__ = __add__

    def __neg__(self):
        return Bicomplex(-self.z1, -self.z2)

    def __sub__(self, o):
        return self + (-self._lift(o))

    def __rsub__(self, o):
        return self._lift(o) - self

    def __mul__(self, o):
        o = self._lift(o)
        return Bicomplex(self.z1 * o.z1 - self.z2 * o.z2, self.z1 * o.z2 + self.z2 * o.z1)

    __rmul__ = __mul__

    def __truediv__(self, o):
        o = self._lift(o)
        d = o.z1 * o.z1 + o.z2 * o.z2  # (w1 + w2 i2)(w1 - w2 i2)
        return self * Bicomplex(o.z1 / d, -o.z2 / d)

    def __rtruediv__(self, o):
        return self._lift(o) / self

    def __getitem__(self, idx):
        return Bicomplex(self.z1[idx], self.z2[idx])

    @property
    def shape(self):
        return self.z1.shape


def sqrt(z: Bicomplex) -> Bicomplex:
    """Principal square root near z1 (see the module docstring)."""
    s = np.sqrt(z.z1)
    return Bicomplex(s, z.z2 / (2.0 * s))


def stack(xs, axis=-1) -> Bicomplex:
    return Bicomplex(np.stack([x.z1 for x in xs], axis), np.stack([x.z2 for x in xs], axis))


def where(mask, a: Bicomplex, b) -> Bicomplex:
    b = Bicomplex._lift(b)
    return Bicomplex(np.where(mask, a.z1, b.z1), np.where(mask, a.z2, b.z2))
