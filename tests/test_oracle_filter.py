"""Pins of the oracle's Gaussian filtering (Sec. 3.2, "Gaussian filtering": keep
the Gaussians with the largest beta_i, the sum of their weights): a brute-force
rank count on small inputs with many ties, the edge cases of the keep count,
and beta from the oracle's own uplift."""
import numpy as np
import pytest

import oracle
from paper_2410_14462_gb300 import inputs


def _brute(beta, keep):
    """i is kept iff fewer than `keep` Gaussians rank above it: a larger beta,
    or the same beta and a lower index."""
    b = [max(float(x), 0.0) if x == x else 0.0 for x in beta]
    out = []
    for i in range(len(b)):
        above = sum(1 for j in range(len(b)) if b[j] > b[i] or (b[j] == b[i] and j < i))
        if above < keep:
            out.append(i)
    return np.array(out, np.int32)


@pytest.mark.parametrize("seed", range(6))
def test_matches_rank_count_with_ties(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 90))
    beta = rng.choice(np.array([0.0, 0.25, 0.5, 0.5, 1.0, 3.0, -1.0], np.float32), size=n)
    for keep in {0, 1, n // 2, n - n // 2, n - 1, n}:
        if keep < 0:
            continue
        got = oracle.beta_select(beta, keep)
        assert np.array_equal(got, _brute(beta, keep)), (n, keep)
        assert got.size == keep and np.all(np.diff(got) > 0)


def test_all_equal_keeps_lowest_indices_and_nan_ranks_as_zero():
    assert np.array_equal(oracle.beta_select(np.full(10, 2.0), 4), np.arange(4))
    beta = np.array([np.nan, 0.0, 1.0, -3.0, np.nan, 0.5], np.float32)
    assert np.array_equal(oracle.beta_select(beta, 2), [2, 5])
    assert np.array_equal(oracle.beta_select(beta, 4), [0, 1, 2, 5])   # zeros by index: 0, 1


def test_beta_from_the_uplift_keeps_the_contributing_half():
    """On the tiny scene, beta = sum of weights (Eq. 3's normaliser); keeping
    the top half keeps only contributing Gaussians when more than half
    contribute, and every kept beta is >= every dropped one."""
    wl = inputs.tiny_mask_workload()
    _, beta = oracle.uplift(wl.scene, wl.cams, lambda v: wl.features(v), views=range(4))
    keep = wl.scene.n - wl.scene.n // 2
    idx = oracle.beta_select(beta, keep)
    mask = np.zeros(wl.scene.n, bool)
    mask[idx] = True
    assert beta[mask].min() >= beta[~mask].max()
    assert ((beta > 0).sum() >= keep) == (beta[mask] > 0).all()
