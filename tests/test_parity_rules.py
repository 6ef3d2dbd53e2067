"""The comparison rules the GPU parity tests apply (tests/_cases.py), checked on hand-made
cases at the margin: which pixels count as decided by the oracle, and that mismatches are
counted only there.  A rule that silently decided nothing would make the parity tests
vacuous; the last test bounds the decided fraction on realistic inputs."""
import numpy as np

from _cases import MARGIN, compare_levels, decided_mask


def test_sigmoid_rule():
    p = np.array([[[0.5, 0.5 + 0.5 * MARGIN, 0.5 + 2 * MARGIN, 0.7, 0.2]]])
    u = np.full((1, 5), 0.5)
    assert decided_mask(p, u, 0).tolist() == [[False, False, True, True, True]]
    u2 = np.array([[0.1, 0.9, 0.5 + 2 * MARGIN, 0.7 + 0.5 * MARGIN, 0.2 - 3 * MARGIN]])
    assert decided_mask(p, u2, 1).tolist() == [[True, True, False, False, True]]


def test_softmax_rules():
    q = np.array([0.25, 0.25, 0.25, 0.25])[:, None, None] * np.ones((4, 1, 3))
    u = np.array([[0.25 + 0.5 * MARGIN, 0.6, 1.0 - 0.5 * MARGIN]])
    # Bernoulli: decided unless u lies within the margin of a partial sum 0.25, 0.5, 0.75, 1
    assert decided_mask(q, u, 1).tolist() == [[False, True, False]]
    # threshold: decided when the two largest probabilities differ by more than the margin
    qt = np.stack([np.array([[0.4, 0.3, 0.3 + 0.5 * MARGIN]]), np.array([[0.3, 0.3, 0.3]]),
                   np.array([[0.2, 0.2, 0.2]]), np.array([[0.1, 0.2, 0.2 - 0.5 * MARGIN]])])
    assert decided_mask(qt, np.full((1, 3), 0.5), 0).tolist() == [[True, False, False]]


def test_mismatches_count_only_where_decided():
    gpu = np.array([[0, 1, 1, 0]])
    ref = np.array([[0, 0, 1, 1]])
    decided = np.array([[True, True, False, False]])
    assert compare_levels(gpu, ref, decided) == (2, 1)


def test_decided_fraction_on_realistic_inputs():
    rng = np.random.default_rng(0)
    p = rng.random((1, 256, 256))
    u = rng.random((256, 256))
    frac = decided_mask(p, u, 1).mean()
    assert 0.999 < frac < 1.0                      # |p - u| <= 1e-4 has probability ~2e-4
    q = rng.dirichlet(np.ones(4), size=(256, 256)).transpose(2, 0, 1)
    assert 0.998 < decided_mask(q, u, 1).mean() < 1.0


def test_unexplained_mismatches():
    """A mismatch counts as explained only where u lies within |p_gpu - p_or| of p_or."""
    from _cases import unexplained
    p_or = np.array([[0.30, 0.50, 0.70, 0.90]])
    p_gpu = np.array([[0.31, 0.50, 0.70, 0.90]])
    u = np.array([[0.305, 0.2, 0.6, 0.95]])
    lev_or = (u < p_or).astype(np.uint8)
    lev_gpu = lev_or.copy()
    lev_gpu[0, 0] ^= 1                      # u between the two p: explained
    dec = np.ones_like(u, bool)
    assert unexplained(lev_gpu, lev_or, p_gpu, p_or, u, dec) == 0
    lev_gpu[0, 2] ^= 1                      # p equal on both sides: a fault
    assert unexplained(lev_gpu, lev_or, p_gpu, p_or, u, dec) == 1
    dec[0, 2] = False
    assert unexplained(lev_gpu, lev_or, p_gpu, p_or, u, dec) == 0
