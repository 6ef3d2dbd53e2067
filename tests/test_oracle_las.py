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


# ---------------------------------------------------------------------------
# Closed forms for a spectrum that is flat except at one conjugate pair.
# q = delta at the origin + eps cos(2 pi (u0 a + v0 b) / n) has F = 1 everywhere except
# F(+-f0) = 1 + eps N / 2, so P = 1/N except P(+-f0) = (1 + eps N / 2)^2 / N.  Every ring or
# bin without f0 is then flat and contributes nothing, and the loss is a closed form in the
# number of samples of f0's ring (paper form) or of f0's radial and angular bins (binned
# form).  Those counts are taken here from exact integer tests on s = u^2 + v^2 and on the
# direction, not from the oracle's square roots, rounding and atan2, so a misplaced ring
# or bin edge, a wrong radial scale or swapped angle axes in the oracle change the loss.
# ---------------------------------------------------------------------------
import math

_N_SP = 32
_EPS_SP = 0.25


def _spike(n, u0, v0, eps=_EPS_SP):
    a, b = np.indices((n, n))
    q = eps * np.cos(2 * np.pi * (u0 * a + v0 * b) / n)
    q[0, 0] += 1.0
    N = n * n
    return q, 1.0 / N, (1.0 + eps * N / 2) ** 2 / N


def _lattice(n):
    r = np.arange(-(n // 2), n // 2)
    return [(int(u), int(v)) for u in r for v in r]


def _ring_of(s):
    """Paper-form ring of a frequency with u^2 + v^2 = s: rho = round(sqrt(s)), i.e. the rho
    with rho^2 - rho + 1 <= s <= rho^2 + rho ((rho +- 1/2)^2 is never an integer)."""
    rho = math.isqrt(s)
    while not (rho * rho - rho + 1 <= s <= rho * rho + rho):
        rho += 1
    return rho


def _radial_bin(s, n, n_rad):
    """floor(n_rad r / (n/2)) for r = sqrt(s) < n/2: floor(sqrt(x)) = isqrt(floor(x))."""
    half = n // 2
    return math.isqrt((n_rad * n_rad * s) // (half * half))


def _angular_bin(u, v, n_ang):
    """Number of bin edges j pi / n_ang (j = 1 .. n_ang - 1) at or before the direction's
    angle theta = atan2(u, v) mod pi, by the sign of a cross product; the edges at 45, 90 and
    135 degrees, where lattice directions can lie exactly, by integer comparisons."""
    if u < 0 or (u == 0 and v < 0):
        u, v = -u, -v
    bt = 0
    for j in range(1, n_ang):
        if 4 * j == n_ang:
            past = u >= v
        elif 2 * j == n_ang:
            past = v <= 0
        elif 4 * j == 3 * n_ang:
            past = v <= -u
        else:
            a = j * np.pi / n_ang
            past = np.cos(a) * u - np.sin(a) * v >= 0
        bt += bool(past)
    return bt


F0S = [(3, 5), (0, 7), (4, 4), (5, -5), (-6, 2), (9, 11), (1, 7), (7, 1), (2, -13), (12, 3), (15, 5), (-11, 11)]


@pytest.mark.parametrize("f0", F0S)
def test_paper_form_single_pair_closed_form(f0):
    n = _N_SP
    u0, v0 = f0
    q, p0, ps = _spike(n, u0, v0)
    r = O.anisotropy_loss(q, mode=0)
    psd = r["psd"]
    assert psd[u0 % n, v0 % n] == pytest.approx(ps, rel=1e-9) and psd[1, 0] == pytest.approx(p0, rel=1e-9)
    rho = _ring_of(u0 * u0 + v0 * v0)
    c = sum(1 for (u, v) in _lattice(n) if (u, v) != (0, 0) and _ring_of(u * u + v * v) == rho)
    mean = (2 * ps + (c - 2) * p0) / c
    dev2 = 2 * (ps - mean) ** 2 + (c - 2) * (p0 - mean) ** 2
    assert r["loss"] == pytest.approx(dev2, rel=1e-9)
    assert r["aniso"][rho] == pytest.approx(dev2 / (c - 1) / mean ** 2, rel=1e-9)
    others = [k for k in range(1, len(r["aniso"])) if k != rho and np.isfinite(r["aniso"][k])]
    assert others and max(abs(r["aniso"][k]) for k in others) < 1e-12


@pytest.mark.parametrize("f0", [f for f in F0S if f[0] ** 2 + f[1] ** 2 < (_N_SP // 2) ** 2])
def test_binned_form_single_pair_closed_form(f0):
    n, n_rad, n_ang = _N_SP, 32, 16
    u0, v0 = f0
    q, p0, ps = _spike(n, u0, v0)
    got = O.anisotropy_loss(q, mode=1, n_rad=n_rad, n_ang=n_ang)["loss"]
    counts = {}
    for (u, v) in _lattice(n):
        s = u * u + v * v
        if s == 0 or s >= (n // 2) ** 2:
            continue
        key = (_radial_bin(s, n, n_rad), _angular_bin(u, v, n_ang))
        counts[key] = counts.get(key, 0) + 1
    K = {}
    for (br, bt) in counts:
        K[br] = K.get(br, 0) + 1
    n_used = sum(1 for br in K if K[br] >= 2)
    B = _radial_bin(u0 * u0 + v0 * v0, n, n_rad)
    jstar = _angular_bin(u0, v0, n_ang)
    assert _angular_bin(-u0, -v0, n_ang) == jstar
    R = sum(c for (br, _), c in counts.items() if br == B)
    nstar = counts[(B, jstar)]
    m = (2 * ps + (R - 2) * p0) / R
    astar = (2 * ps + (nstar - 2) * p0) / nstar
    A = ((astar - m) ** 2 + (K[B] - 1) * (p0 - m) ** 2) / ((K[B] - 1) * m * m)
    assert K[B] >= 2
    assert got == pytest.approx(A / n_used, rel=1e-9), (f0, B, jstar, R, nstar, K[B], n_used)
