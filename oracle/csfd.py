"""Complex-step finite difference (X-SLAM Sec. 3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The oracle uses full complex arithmetic (numpy complex128), not the simplified products of
Eq. csfd_simplify_multiplication / csfd_simplify_division, so that it is independent of the GPU's
lane arithmetic; with h = 1e-20 the dropped b1*b2 terms are below double precision anyway.
"""
from __future__ import annotations

import numpy as np

H_ORACLE = 1e-20  # imaginary step of the oracle; O(h^2) truncation vanishes in double


def promote(x, h: float = H_ORACLE):
    """x* = x + h i (Eq. complex_taylor)."""
    return np.asarray(x, np.complex128) + 1j * h


def derivative(fz, h: float = H_ORACLE):
    """f'(x) ~ Im(f*(x + h i)) / h (Eq. csfd)."""
    return np.imag(fz) / h


def table1_f(x):
    """The worked example of Sec. 3 / Table 1: f(x) = (e^x + x^3 + x) / (x + 1)."""
    return (np.exp(x) + x ** 3 + x) / (x + 1)


def table1_fprime(x):
    """Closed-form derivative of table1_f (quotient rule)."""
    x = np.asarray(x, np.float64)
    num = np.exp(x) + x ** 3 + x
    dnum = np.exp(x) + 3 * x ** 2 + 1
    return (dnum * (x + 1) - num) / (x + 1) ** 2


def relative_error(v0, v):
    """e_relative = |(v0 - v) / v| (Sec. 3, relative-error definition used by Table 1)."""
    return np.abs((np.asarray(v0) - np.asarray(v)) / np.asarray(v))
