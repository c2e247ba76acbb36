"""Pins of the oracle's regularisers (Eq. 4, 5, 14) to closed forms and to
central finite differences."""
import numpy as np
import pytest

from oracle import regularizers as R

pytest.importorskip("torch")


def test_opacity_loss_is_the_mean_transmittance():
    rng = np.random.default_rng(0)
    T = rng.uniform(0, 1, (7, 9))
    L, g = R.opacity_loss(1.0 - T)
    assert abs(L - T.mean()) < 1e-15
    np.testing.assert_allclose(g[T > 0], -1.0 / T.size)
    assert R.opacity_loss(np.ones((3, 4)))[0] == 0.0


def test_scale_loss_closed_forms():
    smax = 0.05
    L, g = R.scale_loss(np.full((10, 2), 0.04), smax)
    assert L == 0.0 and np.all(g == 0)
    L, g = R.scale_loss(np.array([[2 * smax, 0.5 * smax]]), smax)
    assert abs(L - 1.0) < 1e-14 and abs(g[0, 0] - 2.0 / smax) < 1e-9 and g[0, 1] == 0.0
    L, g = R.scale_loss(np.array([[1.5 * smax, 1.5 * smax], [0.1 * smax, 0.2 * smax]]), smax)
    assert abs(L - 0.25 / 2) < 1e-14
    np.testing.assert_allclose(g[0], [0.5 / smax / 2, 0.5 / smax / 2], rtol=1e-12)  # tie: split evenly
    assert np.all(g[1] == 0)


def test_env_tv_ramps_pin_the_wrap_reading():
    H, W = 5, 8
    cols = np.broadcast_to(np.arange(W, dtype=float)[None, :, None], (H, W, 3))
    rows = np.broadcast_to(np.arange(H, dtype=float)[:, None, None], (H, W, 3))
    assert R.env_tv(np.full((H, W, 3), 0.3))[0] == 0.0
    assert abs(R.env_tv(cols)[0] - 2.0 * (W - 1) / W) < 1e-14  # wraps in azimuth
    assert abs(R.env_tv(rows)[0] - (H - 1) / H) < 1e-14        # no wrap across the poles


@pytest.mark.parametrize("which", ["opacity", "scale", "tv"])
def test_regulariser_gradients_match_central_differences(which):
    rng = np.random.default_rng(4)
    if which == "opacity":
        x = rng.uniform(0.2, 0.9, (4, 5))
        f = lambda v: R.opacity_loss(v)[0]
        g = R.opacity_loss(x)[1]
    elif which == "scale":
        x = rng.uniform(0.02, 0.09, (6, 2))
        f = lambda v: R.scale_loss(v, 0.05)[0]
        g = R.scale_loss(x, 0.05)[1]
    else:
        x = rng.uniform(0, 1, (4, 6, 3))
        f = lambda v: R.env_tv(v)[0]
        g = R.env_tv(x)[1]
    h = 1e-7
    for idx in [tuple(rng.integers(0, s) for s in x.shape) for _ in range(6)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        assert abs((f(xp) - f(xm)) / (2 * h) - g[idx]) < 1e-6
