"""Pins of the oracle's supersampling anti-aliasing (Sec. 3.1.2
"Anti-aliasing"): the area filter against hand-worked weights and the
textbook box average, its normalisation and its adjoint, and the
supersampled camera against the original camera's rays.  No GPU."""
import numpy as np
import pytest

import oracle
import synth
from oracle import antialias


def test_area_weights_hand_worked():
    """Three pixels onto two (s = 1.5): target 0 covers [0, 1.5): all of
    pixel 0 and half of pixel 1; target 1 covers [1.5, 3)."""
    M = antialias.area_weights(3, 2)
    assert np.allclose(M, [[2 / 3, 1 / 3, 0], [0, 1 / 3, 2 / 3]], rtol=0, atol=1e-15)


def test_integer_factor_is_the_box_average():
    rng = np.random.default_rng(0)
    img = rng.normal(size=(3, 8, 12))
    want = img.reshape(3, 4, 2, 6, 2).mean(axis=(2, 4))
    assert np.allclose(antialias.downsample(img, 4, 6), want, rtol=0, atol=1e-14)


@pytest.mark.parametrize("n_in,n_out", [(11, 10), (1408, 1280), (924, 840), (15, 10), (7, 7), (33, 16)])
def test_rows_and_columns(n_in, n_out):
    """Every target pixel averages (weights sum to 1, so constants pass
    through); every source pixel spreads a total of n_out / n_in."""
    M = antialias.area_weights(n_in, n_out)
    assert np.allclose(M.sum(1), 1.0, rtol=0, atol=1e-12)
    assert np.allclose(M.sum(0), n_out / n_in, rtol=0, atol=1e-12)
    assert (M >= 0).all()
    # a source pixel touches at most two target pixels when n_in >= n_out
    assert ((M > 0).sum(0) <= 2).all()


def test_adjoint():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 17, 23))
    y = rng.normal(size=(2, 12, 20))
    lhs = (antialias.downsample(x, 12, 20) * y).sum()
    rhs = (x * antialias.downsample_adjoint(y, 17, 23)).sum()
    assert abs(lhs - rhs) < 1e-11 * (abs(lhs) + 1)


@pytest.mark.parametrize("h_ss", [1.1, 1.5, 2.0])
def test_supersampled_camera_rays(h_ss):
    """The supersampled pixel (X, Y) looks along the original camera's ray
    through the same point of the image plane, (X + 1/2) / s - 1/2 in the
    original pixel coordinates."""
    cam = synth.orbit_camera(5, 64, 40)
    ss = antialias.supersampled_camera(cam, h_ss)
    assert (ss.width, ss.height) == antialias.supersampled_size(64, 40, h_ss)
    sx, sy = ss.width / cam.width, ss.height / cam.height
    for X, Y in ((0, 0), (ss.width - 1, ss.height - 1), (17, 9), (ss.width // 2, ss.height // 3)):
        ro1, rd1 = oracle.pixel_ray(ss, X, Y)
        ro0, rd0 = oracle.pixel_ray(cam, (X + 0.5) / sx - 0.5, (Y + 0.5) / sy - 0.5)
        assert np.allclose(ro1, ro0, rtol=0, atol=1e-12)
        # float32 intrinsics of the scaled camera: equal up to their rounding
        assert np.allclose(rd1, rd0, rtol=1e-6, atol=1e-7)
