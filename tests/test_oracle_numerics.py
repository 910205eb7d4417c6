"""Pins of the oracle's CSFD extraction and SE(3) algebra against closed forms and scipy.

X-SLAM Sec. 3 (Eq. csfd, Table 1) and Sec. 4.1 (Eq. lie, rotvector, rotation_jacobi)."""
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import csfd, se3

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_table1():
    out = {}
    for line in open(os.path.join(GOLDEN, "table1_csfd.txt")):
        if line.startswith("#") or line.startswith("method"):
            continue
        k, v = line.split()
        out[k] = float(v)
    return out


def test_table1_example_csfd_exact():
    """Eq. csfd on the Sec. 3 worked example: complex128 CSFD at h = 1e-20 reproduces the analytic
    derivative to rounding, and beats the paper's printed CSFD error (Table 1)."""
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, 10000)
    d = csfd.derivative(csfd.table1_f(csfd.promote(x)))
    err = csfd.relative_error(d, csfd.table1_fprime(x))
    assert err.max() < 2e-15
    g = _golden_table1()
    assert err.max() < g["CSFD"]
    # no subtractive cancellation: the same accuracy at h = 1e-8 (the paper's depth step) and 1e-100
    for h in (1e-8, 1e-100):
        e = csfd.relative_error(csfd.derivative(csfd.table1_f(csfd.promote(x, h)), h), csfd.table1_fprime(x))
        assert e.max() < 1e-14


def test_forward_difference_cancellation():
    """Eq. forward_difference loses digits as h shrinks (the motivation of Sec. 3)."""
    x = np.linspace(0.05, 0.95, 50)
    ref = csfd.table1_fprime(x)
    e_fd = csfd.relative_error((csfd.table1_f(x + 1e-13) - csfd.table1_f(x)) / 1e-13, ref)
    assert e_fd.max() > 1e-4


def _twist_matrix(xi):
    M = np.zeros((4, 4), np.result_type(xi, np.float64))
    M[:3, :3] = se3.hat(xi[:3])
    M[:3, 3] = xi[3:]
    return M


@pytest.mark.parametrize("scale", [1e-7, 1e-3, 0.3, 2.5])
def test_se3_exp_matches_matrix_exponential(scale):
    """Eq. lie / rotvector / rotation_jacobi against scipy's matrix exponential of the 4x4 twist."""
    rng = np.random.default_rng(int(scale * 1e7) % 1000)
    for _ in range(5):
        xi = rng.standard_normal(6) * scale
        E = scipy.linalg.expm(_twist_matrix(xi))[:3]
        assert np.abs(se3.se3_exp(xi) - E).max() < 1e-13
        # complex argument (a CSFD lane on top of a real twist)
        xc = xi + 1j * 1e-20 * rng.standard_normal(6)
        Ec = scipy.linalg.expm(_twist_matrix(xc))[:3]
        T = se3.se3_exp(xc)
        assert np.abs(T.real - Ec.real).max() < 1e-13
        assert np.abs(T.imag - Ec.imag).max() < 1e-13 * 1e-20 * 10


def test_series_branch_continuity():
    """The power-series branch (|theta^2| < 1e-4) and the closed form agree across the threshold."""
    rng = np.random.default_rng(5)
    axis = rng.standard_normal(3)
    axis /= np.linalg.norm(axis)
    for th in (0.00999, 0.01001):
        xi = np.concatenate([axis * th, rng.standard_normal(3)])
        E = scipy.linalg.expm(_twist_matrix(xi))[:3]
        assert np.abs(se3.se3_exp(xi) - E).max() < 1e-15 * 10


def test_generators_at_identity():
    """Im exp(h i e_j) / h is exactly the j-th generator; Re is exactly the identity."""
    for j in range(6):
        T = se3.promote_pose(np.eye(3, 4), j, 1e-20)
        G = np.zeros((3, 4))
        e = np.zeros(6)
        e[j] = 1.0
        G[:, :3] = se3.hat(e[:3])
        G[:, 3] = e[3:]
        assert np.array_equal(T.real, np.eye(3, 4))
        assert np.abs(T.imag / 1e-20 - G).max() < 1e-15


def test_rotation_orthonormal_and_inverse():
    rng = np.random.default_rng(7)
    for _ in range(10):
        xi = rng.standard_normal(6)
        T = se3.se3_exp(xi)
        R = T[:, :3]
        assert np.abs(R.T @ R - np.eye(3)).max() < 1e-14
        assert abs(np.linalg.det(R) - 1) < 1e-14
        assert np.abs(se3.compose(T, se3.inverse(T)) - np.eye(3, 4)).max() < 1e-14


def test_readout_recovers_left_twist():
    """For T* = exp(h i xi) T the read-out gives dT = xi^ T and the left twist xi exactly."""
    rng = np.random.default_rng(11)
    T = se3.se3_exp(rng.standard_normal(6))
    xi = rng.standard_normal(6)
    Tc = se3.compose(se3.se3_exp(1j * 1e-20 * xi), T.astype(complex))
    Re, dT, tw = se3.readout(Tc, 1e-20)
    assert np.abs(Re - T).max() < 1e-15
    assert np.abs(dT - _twist_matrix(xi)[:3] @ np.vstack([T, [0, 0, 0, 1]])).max() < 1e-14
    assert np.abs(tw - xi).max() < 1e-14
