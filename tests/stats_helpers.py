"""Two-sample tests of per-primary layer profiles (rows: primaries, columns:
layers), used to compare the CUDA path and the oracle run with independent
random seeds, where histories differ one by one but their distributions must
not."""
import numpy as np
from scipy import stats


def layer_profile_tests(a, b):
    """Per-layer Welch tests (Bonferroni over the layers) and Hotelling's T^2
    on the whole layer vector with the pooled covariance (layers are strongly
    correlated, so the per-layer tests alone would miss a shift spread over
    many layers). Layers with no deposit in either sample are dropped.
    Returns (min per-layer p-value x layers, Hotelling p-value, layers used)."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    na, nb = len(a), len(b)
    keep = (a.var(0) > 0) | (b.var(0) > 0)
    a, b = a[:, keep], b[:, keep]
    k = a.shape[1]
    va, vb = a.var(0, ddof=1), b.var(0, ddof=1)
    z = (a.mean(0) - b.mean(0)) / np.sqrt(va / na + vb / nb)
    p_layer = 2.0 * stats.norm.sf(np.abs(z))
    p_bonf = min(1.0, float(p_layer.min()) * k)
    d = a.mean(0) - b.mean(0)
    S = ((na - 1) * np.cov(a.T) + (nb - 1) * np.cov(b.T)) / (na + nb - 2)
    t2 = na * nb / (na + nb) * float(d @ np.linalg.solve(S, d))
    f = (na + nb - k - 1) / (k * (na + nb - 2)) * t2
    p_t2 = float(stats.f.sf(f, k, na + nb - k - 1))
    return p_bonf, p_t2, k
