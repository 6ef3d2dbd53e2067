"""Shared helpers for the GPU parity tests (comparison rules, not method arithmetic)."""
import numpy as np

MARGIN = 1e-4


def decided_mask(p_or: np.ndarray, u: np.ndarray, mode: int, margin: float = MARGIN) -> np.ndarray:
    """Pixels whose action the FP64 oracle decides by more than `margin`:
    sigmoid: |p - u| > margin (u = 0.5 in threshold mode); softmax (p_or [K][h][w]):
    Bernoulli -> u is farther than margin from every partial sum of q, threshold -> the
    top-two probabilities differ by more than margin."""
    if p_or.shape[0] == 1:
        return np.abs(p_or[0] - u) > margin
    if mode == 1:
        cdf = np.cumsum(p_or, axis=0)
        return np.all(np.abs(cdf - u[None]) > margin, axis=0)
    s = np.sort(p_or, axis=0)
    return (s[-1] - s[-2]) > margin


def compare_levels(gpu: np.ndarray, ref: np.ndarray, decided: np.ndarray):
    mism = (gpu != ref) & decided
    return int(decided.sum()), int(mism.sum())
