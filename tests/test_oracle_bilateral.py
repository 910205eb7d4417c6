"""Pins of the oracle's bilateral filter of the raw depth (X-SLAM Sec. 4.1, surface measurement).

The paper names the filter but not its parameters; the readings are a 7x7 window, a spatial Gaussian of
sigma 4.5 pixels, a range Gaussian of sigma 0.03 m, valid taps only, and an invalid output where the
centre is invalid. Each test compares against a value fixed by that definition and worked out by hand
(a constant map, an affine ramp, a step far above the range sigma, two-tap and one-tap windows in
closed form) or against central differences of the real filter, so that a swapped sigma, a dropped
centre tap, a wrong normalisation, a wrong window radius or a lost range-weight derivative fails."""
import math

import numpy as np
import pytest

from oracle import measure

SS, SR = 4.5, 0.03  # the readings' spatial (pixels) and range (metres) sigmas


def test_constant_map_is_unchanged():
    D = np.full((20, 30), 1.7)
    D[4, 5] = 0.0  # invalid taps do not pull the average down
    out = measure.bilateral(D)
    valid = D > 0
    assert np.abs(out[valid] - 1.7).max() < 1e-15
    assert out[4, 5] == 0.0


def test_affine_ramp_reproduced_with_wide_range_sigma():
    """With a range sigma far above the ramp's spread the filter is a normalised symmetric Gaussian,
    which reproduces an affine function exactly at every pixel whose window lies inside the image."""
    H, W = 24, 32
    v, u = np.mgrid[0:H, 0:W].astype(float)
    D = 1.0 + 0.003 * u - 0.002 * v
    out = measure.bilateral(D, sigma_r=1e6)
    inner = (slice(3, H - 3), slice(3, W - 3))
    assert np.abs(out[inner] - D[inner]).max() < 1e-13
    # at the border the window is one-sided and the ramp is not reproduced
    assert abs(out[0, 16] - D[0, 16]) > 1e-4


def test_step_far_above_range_sigma_keeps_both_sides():
    """A 0.25 m step (8.3 range sigmas: a cross weight below e^-34) is left sharp."""
    H, W = 16, 20
    u = np.arange(W)[None, :].repeat(H, 0)
    D = np.where(u < 10, 1.0, 1.25)
    out = measure.bilateral(D)
    assert np.abs(out - D).max() < 1e-12


def test_two_tap_window_closed_form():
    """Centre c with two valid neighbours: (u+1, v) at c + SR and (u, v+2) at c. Weights, by hand:
    centre 1; first exp(-1/(2 SS^2)) exp(-1/2); second exp(-4/(2 SS^2)). The output is
    c + w1 SR / (1 + w1 + w2)."""
    c = 2.0
    D = np.zeros((9, 9))
    D[4, 4] = c
    D[4, 5] = c + SR
    D[6, 4] = c
    w1 = math.exp(-1.0 / (2 * SS * SS)) * math.exp(-0.5)
    w2 = math.exp(-4.0 / (2 * SS * SS))
    out = measure.bilateral(D)
    assert abs(out[4, 4] - (c + w1 * SR / (1 + w1 + w2))) < 1e-15
    # seen from (u+1, v): its own weight 1, the centre at (-1, 0) with range difference -SR, the third
    # tap at (-1, +2) with range difference -SR
    wa = math.exp(-1.0 / (2 * SS * SS) - 0.5)
    wb = math.exp(-5.0 / (2 * SS * SS) - 0.5)
    assert abs(out[4, 5] - ((c + SR) - SR * (wa + wb) / (1 + wa + wb))) < 1e-15


def test_window_radius_is_three():
    """A tap 3 pixels away contributes, one 4 pixels away does not."""
    D = np.zeros((11, 11))
    D[5, 5] = 1.0
    D[5, 8] = 1.01
    near = measure.bilateral(D)[5, 5]
    w = math.exp(-9.0 / (2 * SS * SS) - (0.01 ** 2) / (2 * SR * SR))
    assert abs(near - (1.0 + 0.01 * w / (1 + w))) < 1e-15
    D2 = np.zeros((11, 11))
    D2[5, 5] = 1.0
    D2[5, 9] = 1.01
    assert measure.bilateral(D2)[5, 5] == 1.0


def test_shift_invariance():
    """The range weights depend on depth differences only: filtering D + s gives the filtered D + s."""
    rng = np.random.default_rng(3)
    D = rng.uniform(1.0, 1.1, (15, 17))
    D[rng.random(D.shape) < 0.1] = 0.0
    a = measure.bilateral(D)
    b = measure.bilateral(np.where(D > 0, D + 0.37, 0.0))
    valid = D > 0
    assert np.abs((b - a)[valid] - 0.37).max() < 1e-13
    assert np.all(a[~valid] == 0) and np.all(b[~valid] == 0)


def test_all_pixel_depth_perturbation_stays_h():
    """D + h i on every valid pixel: the range weights see no imaginary difference, so the filtered
    perturbation is h at every valid pixel (the GPU's all-pixel DEPTH lane relies on this)."""
    rng = np.random.default_rng(4)
    D = rng.uniform(1.0, 1.2, (12, 14))
    D[rng.random(D.shape) < 0.15] = 0.0
    h = 1e-20
    out = measure.bilateral(np.where(D > 0, D + 1j * h, 0))
    valid = D > 0
    assert np.abs(out.imag[valid] / h - 1.0).max() < 1e-13
    assert np.all(out.imag[~valid] == 0)


@pytest.mark.parametrize("pix", [(6, 7), (0, 0), (6, 12)])
def test_single_pixel_perturbation_matches_central_differences(pix):
    """D + h i at one pixel: the complex step through the range weights equals central differences
    of the real filter at every output pixel of the window."""
    rng = np.random.default_rng(5)
    D = rng.uniform(1.0, 1.06, (13, 15))
    D[2, 3] = 0.0
    e = np.zeros_like(D)
    e[pix] = 1.0
    h, hfd = 1e-20, 1e-7
    cs = measure.bilateral(D + 1j * h * e).imag / h
    fd = (measure.bilateral(D + hfd * e) - measure.bilateral(D - hfd * e)) / (2 * hfd)
    assert np.abs(cs - fd).max() < 1e-6 * np.abs(cs).max()
    # the derivative is confined to the 7x7 window around the perturbed pixel
    mask = np.zeros(D.shape, bool)
    mask[max(0, pix[0] - 3):pix[0] + 4, max(0, pix[1] - 3):pix[1] + 4] = True
    assert np.all(cs[~mask] == 0) and np.all(cs[mask & (D > 0)] != 0)
