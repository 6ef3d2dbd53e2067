"""Pins of the oracle's spectrum, anisotropy and anisotropy-suppressing loss (Eqs. psd-as)."""
import numpy as np
import pytest

import oracle as O


def test_dft_matches_numpy_fft():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(16, 16)) + 1j * rng.normal(size=(16, 16))
    np.testing.assert_allclose(O.dft2(x), np.fft.fft2(x), atol=1e-10)
    np.testing.assert_allclose(O.dft2(x, inverse=True), np.fft.ifft2(x) * 256, atol=1e-10)


def test_parseval():
    rng = np.random.default_rng(1)
    q = rng.random((32, 32))
    r = O.anisotropy_loss(q)
    assert abs(r["psd"].sum() - (q * q).sum()) < 1e-9


def test_checkerboard_peaks_at_half_cycle():
    n = 32
    q = np.indices((n, n)).sum(0) % 2 * 1.0
    psd = O.anisotropy_loss(q)["psd"]
    psd[0, 0] = 0.0                                    # DC
    k = np.unravel_index(np.argmax(psd), psd.shape)
    assert k == (n // 2, n // 2)                       # (1/2, 1/2) cycles per pixel
    assert abs(psd[n // 2, n // 2] - n * n / 4) < 1e-9


def test_radially_symmetric_pattern_has_small_anisotropy():
    n = 64
    y, x = np.indices((n, n)) - n // 2
    q = np.exp(-(x * x + y * y) / (2 * 1.5 ** 2))
    an = O.anisotropy_loss(q)["aniso"]
    # The only spread inside a ring of width 1 is the radial slope of the spectrum:
    # P ~ exp(-rho^2 (2 pi s / n)^2)  =>  A(rho) ~ (2 rho (2 pi s / n)^2)^2 / 12.
    rho = np.arange(1, n // 4)
    bound = (2 * rho * (2 * np.pi * 1.5 / n) ** 2) ** 2 / 12
    assert np.all(an[1:n // 4] < 2 * bound + 1e-3)
    assert np.nanmax(an[1:n // 4]) < 0.05              # vs ~1 for white noise
    rb = O.anisotropy_loss(q, mode=1)
    assert rb["loss"] < 0.05


def test_white_noise_anisotropy_is_one():
    """Periodogram of i.i.d. noise: exponential spread, A(f_rho) ~ 1 (0 dB) on average."""
    rng = np.random.default_rng(2)
    vals = []
    for _ in range(4):
        q = (rng.random((64, 64)) < 0.5).astype(np.float64)
        an = O.anisotropy_loss(q)["aniso"]
        vals.append(np.nanmean(an[4:32]))
    assert abs(np.mean(vals) - 1.0) < 0.15


def test_directional_pattern_is_anisotropic():
    n = 32
    q = (np.indices((n, n))[1] % 4 < 2) * 1.0           # vertical stripes
    q += 0.01 * np.random.default_rng(3).random((n, n))
    assert O.anisotropy_loss(q, mode=1)["loss"] > 0.5     # vs < 0.05 for a symmetric one
    assert np.nanmax(O.anisotropy_loss(q)["aniso"]) > 5.0


@pytest.mark.parametrize("mode", [0, 1])
def test_dc_and_scale_invariances(mode):
    rng = np.random.default_rng(4)
    q = rng.random((32, 32))
    a = O.anisotropy_loss(q, mode=mode)["loss"]
    b = O.anisotropy_loss(q + 0.37, mode=mode)["loss"]   # changes the DC sample only
    assert abs(a - b) < 1e-9 * abs(a)
    if mode == 1:                                        # variance / mean^2 is scale free
        assert abs(O.anisotropy_loss(3 * q, mode=1)["loss"] - a) < 1e-9 * a
    else:                                                # numerator scales with the 4th power
        assert abs(O.anisotropy_loss(2 * q, mode=0)["loss"] - 16 * a) < 1e-8 * a


@pytest.mark.parametrize("mode", [0, 1])
def test_gradient_matches_finite_differences(mode):
    rng = np.random.default_rng(5)
    n = 16
    q = rng.random((n, n))
    r = O.anisotropy_loss(q, mode=mode, n_rad=4, n_ang=4, grad=True)
    g = r["grad"]
    eps = 1e-6
    for (i, j) in [(0, 0), (3, 7), (8, 8), (15, 1), (5, 12)]:
        qp, qm = q.copy(), q.copy()
        qp[i, j] += eps; qm[i, j] -= eps
        fd = (O.anisotropy_loss(qp, mode, 4, 4)["loss"] - O.anisotropy_loss(qm, mode, 4, 4)["loss"]) / (2 * eps)
        assert abs(fd - g[i, j]) < 1e-6 * max(1.0, abs(fd)), (i, j, fd, g[i, j])
