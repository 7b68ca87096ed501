"""Pins of the oracle's graph diffusion (Sec. 3.3): exact kNN on Gaussian
centres, the union edge set, the edge weights of Eq. 7 / the diffusion
workload, and the power iteration of Eq. 8 (closed forms, the dominant
eigenvector from numpy, binarised-graph reachability, scipy/ dense matvec)."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.spatial import cKDTree

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_knn_golden_line():
    g = json.load(open(os.path.join(GOLDEN, "knn_line.json")))
    x = np.array(g["points_x"], np.float32)
    means = np.stack([x, np.zeros_like(x), np.zeros_like(x)], 1)
    idx, _ = oracle.knn(means, g["k"])
    assert idx.tolist() == g["neighbours"]
    r, c = oracle.union_edges(idx)
    und = sorted({(min(a, b), max(a, b)) for a, b in zip(r.tolist(), c.tolist())})
    assert [list(e) for e in und] == g["union_edges"]


def test_knn_matches_kdtree():
    rng = np.random.default_rng(4)
    pts = rng.uniform(-1, 1, size=(3000, 3)).astype(np.float32)
    idx, d2 = oracle.knn(pts, 16)
    tree = cKDTree(pts.astype(np.float64))
    dd, ii = tree.query(pts.astype(np.float64), k=17)
    assert (ii[:, 0] == np.arange(len(pts))).all()
    assert np.array_equal(idx, ii[:, 1:])
    np.testing.assert_allclose(d2, dd[:, 1:] ** 2, rtol=1e-5)
    # subset queries give the same rows
    q = np.array([5, 17, 2999])
    idx2, _ = oracle.knn(pts, 16, queries=q)
    assert np.array_equal(idx2, idx[q])


def test_knn_duplicates_and_small_n():
    means = np.zeros((4, 3), np.float32)   # all coincident: order by index
    idx, d2 = oracle.knn(means, 5)
    assert idx.tolist() == [[1, 2, 3, -1, -1], [0, 2, 3, -1, -1], [0, 1, 3, -1, -1], [0, 1, 2, -1, -1]]
    assert np.isinf(d2[:, 3:]).all()


def test_edge_weight_values():
    means = np.array([[0, 0, 0], [0.1, 0, 0], [0, 0.2, 0]], np.float32)
    feats = np.array([[1, 0], [1, 1], [-1, 0.5]], np.float32)
    rows = np.array([0, 1, 0, 2, 1, 2])
    cols = np.array([1, 0, 2, 0, 2, 1])
    w = oracle.edge_weights_spatial_cos(means, feats, rows, cols, h=0.01)
    d01 = float(np.float32(0.1)) ** 2
    d02 = float(np.float32(0.2)) ** 2
    d12 = d01 + d02
    e01 = np.exp(-d01 / 0.01) * (1 / np.sqrt(2))
    e02 = 0.0                                   # cosine -0.894 clipped to 0
    e12 = np.exp(-d12 / 0.01) * max(0.0, (-1 + 0.5) / (np.sqrt(2) * np.sqrt(1.25)))
    np.testing.assert_allclose(w, [e01, e01, e02, e02, e12, e12], rtol=1e-12, atol=1e-300)


def _ring_graph(n, k=2, seed=0):
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        for d in range(1, k + 1):
            j = (i + d) % n
            w = rng.uniform(0.2, 1.0)
            rows += [i, j]
            cols += [j, i]
            vals += [w, w]
    return np.array(rows), np.array(cols), np.array(vals)


def test_row_normalised_diffusion_of_ones_is_uniform():
    """With rows summing to 1, A 1 = 1, so g_t = 1/sqrt(n) for every t >= 1."""
    n = 50
    r, c, v = _ring_graph(n)
    A = oracle.csr(n, r, c, v, row_normalize=True)
    for t in (1, 2, 7):
        g = oracle.diffuse(A, np.ones(n), t)
        np.testing.assert_allclose(g, 1 / np.sqrt(n), rtol=1e-14)


def test_power_iteration_reaches_dominant_eigenvector():
    """Eq. 8 on the raw symmetric A is the power method (Sec. 3.3)."""
    n = 40
    r, c, v = _ring_graph(n, k=3, seed=1)
    A = oracle.csr(n, r, c, v, row_normalize=False)
    assert abs(A - A.T).max() == 0
    lam, vec = np.linalg.eigh(A.toarray())
    top = vec[:, np.argmax(np.abs(lam))]
    x0 = np.random.default_rng(3).uniform(0.1, 1.0, n)
    g = oracle.diffuse(A, x0, 3000)
    cos = abs(g @ top) / np.linalg.norm(g)
    assert cos > 1 - 1e-8


def test_binarised_support_is_walk_reachability():
    """With A thresholded to 0/1 (Sec. 4.1 uses 1e-5), supp(g_T) is the set of
    nodes reached by a walk of exactly T edges from supp(g_0)."""
    rng = np.random.default_rng(8)
    n = 60
    rows = rng.integers(0, n, 150)
    cols = rng.integers(0, n, 150)
    keep = rows != cols
    rows, cols = rows[keep], cols[keep]
    vals = rng.choice([1e-7, 1e-3, 0.5], size=rows.size)
    R = np.concatenate([rows, cols])
    C = np.concatenate([cols, rows])
    V = np.concatenate([vals, vals])
    A = oracle.csr(n, R, C, V, row_normalize=True, binarize=1e-5)
    adj = {i: set() for i in range(n)}
    for a, b, w in zip(R, C, V):
        if w > 1e-5:
            adj[a].add(b)
    x0 = np.zeros(n)
    x0[[0, 1]] = 1.0
    S = {0, 1}
    for T in range(1, 6):
        S = {j for i in S for j in adj[i]}
        g = oracle.diffuse(A, x0, T)
        assert set(np.flatnonzero(g > 0).tolist()) == S


def test_diffusion_matches_dense_matvec_multi_query():
    n = 30
    r, c, v = _ring_graph(n, seed=5)
    A = oracle.csr(n, r, c, v, row_normalize=True)
    Ad = A.toarray()
    np.testing.assert_allclose(Ad.sum(1), 1.0, rtol=1e-14)
    x0 = np.random.default_rng(6).normal(size=(n, 3))
    x0[:, 2] = 0.0                       # a zero column stays zero
    g = oracle.diffuse(A, x0, 4)
    ref = x0.copy()
    for _ in range(4):
        nrm = np.linalg.norm(ref, axis=0)
        ref = Ad @ (ref / np.where(nrm > 0, nrm, 1.0))
    np.testing.assert_allclose(g, ref, rtol=1e-13, atol=1e-15)
    assert (g[:, 2] == 0).all()


# ---- paper-form diffusion (Eq. 7 with the appendix's S_f and P, Sec. 4.1) ----

def _tri():
    f = np.array([[1, 0], [0, 1], [1, 1]], np.float32)
    rows = np.array([0, 1, 0, 2, 1, 2])
    cols = np.array([1, 0, 2, 0, 2, 1])
    return f, rows, cols


def test_feature_scale_closed_form_and_scale_invariance():
    """f^ = (1,0), (0,1), (1,1)/sqrt2: the six directed edge distances are
    sqrt2 twice and sqrt(2 - sqrt2) four times, so the median is sqrt(2 - sqrt2);
    scaling feature rows by positive factors changes nothing."""
    f, r, c = _tri()
    assert abs(oracle.feature_scale(f, r, c) - np.sqrt(2 - np.sqrt(2))) < 1e-15
    f2 = f * np.array([[3.0], [0.25], [7.0]], np.float32)
    assert abs(oracle.feature_scale(f2, r, c) - oracle.feature_scale(f, r, c)) < 1e-15
    # an even count takes the mean of the two middle values
    assert abs(oracle.feature_scale(f, r[:4], c[:4]) - (np.sqrt(2) + np.sqrt(2 - np.sqrt(2))) / 2) < 1e-15


def test_rbf_unary_edge_weights_closed_form():
    """A_ij = exp(-||f^_i - f^_j||^2 / (b s^2)) sqrt(P_i P_j) by hand."""
    f, r, c = _tri()
    b, s = 0.5, 0.8
    P = np.array([0.25, 1.0, 0.64])
    w = oracle.edge_weights_rbf_unary(f, r, c, b, s, unary=P)
    d01, d02 = 2.0, 2 - np.sqrt(2)
    e = lambda d2, pi, pj: np.exp(-d2 / (b * s * s)) * np.sqrt(pi * pj)
    ref = [e(d01, .25, 1), e(d01, 1, .25), e(d02, .25, .64), e(d02, .64, .25), e(d02, 1, .64), e(d02, .64, 1)]
    np.testing.assert_allclose(w, ref, rtol=1e-12)
    np.testing.assert_allclose(oracle.edge_weights_rbf_unary(f, r, c, b, s), [e(x, 1, 1) for x in
                               (d01, d01, d02, d02, d02, d02)], rtol=1e-12)


def test_unary_anchor_closed_form():
    """Anchors along e1: f_bar = e1, so P = 1 on rows along e1, exp(-2/(b s^2))
    on rows along e2, exp(-(2 - sqrt2)/(b s^2)) on the diagonal; no anchors:
    f_bar = 0 and P = exp(-1/(b s^2)) on every non-zero row."""
    f = np.array([[2, 0], [0, 1], [1, 1], [0.5, 0], [0, 0]], np.float32)
    g0 = np.array([1.0, 0, 0, 0.3, 0])
    b, s = 0.5, 0.7
    P = oracle.unary_anchor(f, g0, b, s)
    k = b * s * s
    np.testing.assert_allclose(P, [1, np.exp(-2 / k), np.exp(-(2 - np.sqrt(2)) / k), 1, np.exp(-1 / k)],
                               rtol=1e-12)
    # anchors e1 and e2: the mean (1/2, 1/2) normalises to the diagonal
    P2 = oracle.unary_anchor(f, np.array([0, 1.0, 0, 1.0, 0]), b, s)
    np.testing.assert_allclose(P2[2], 1.0, rtol=1e-12)
    np.testing.assert_allclose(P2[:2], [np.exp(-(2 - np.sqrt(2)) / k)] * 2, rtol=1e-12)
    P0 = oracle.unary_anchor(f, np.zeros(5), b, s)
    np.testing.assert_allclose(P0, [np.exp(-1 / k)] * 4 + [1.0], rtol=1e-12)


def _brute_top(u, percent):
    u = [float(x) for x in u]
    pos = [i for i in range(len(u)) if u[i] > 0]
    keep = (len(pos) * percent + 99) // 100
    out = np.zeros(len(u))
    for i in pos:
        above = sum(1 for j in pos if u[j] > u[i] or (u[j] == u[i] and j < i))
        if above < keep:
            out[i] = u[i]
    return out


@pytest.mark.parametrize("seed", range(5))
def test_topfrac_positive_rank_count(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 120))
    u = rng.choice(np.array([0.0, -0.5, 0.2, 0.2, 0.7, 1.0], np.float32), size=n)
    for pct in (10, 50, 100, 1):
        assert np.array_equal(oracle.topfrac_positive(u, pct), _brute_top(u, pct)), (n, pct)
    assert (oracle.topfrac_positive(np.zeros(7), 10) == 0).all()


def test_reach_weight_is_support_of_diffusion():
    """h = P on supp(g_T) (Eq. 8 on the binarised A, compared with the float64
    power iteration where it cannot underflow) and on the BFS walk set."""
    rng = np.random.default_rng(11)
    n = 50
    rows = rng.integers(0, n, 120)
    cols = rng.integers(0, n, 120)
    ok = rows != cols
    R = np.concatenate([rows[ok], cols[ok]])
    C = np.concatenate([cols[ok], rows[ok]])
    V = rng.choice([1e-7, 0.3], size=R.size)
    A = oracle.csr(n, R, C, V, row_normalize=False, binarize=1e-5)
    g0 = np.zeros((n, 2))
    g0[[3, 4], 0] = [0.5, 1.0]
    g0[7, 1] = 2.0
    P = rng.uniform(0.1, 1.0, n)
    for T in (1, 2, 5):
        h = oracle.reach_weight(A, g0, T, P)
        g = oracle.diffuse(A, g0, T)
        assert np.array_equal(h > 0, g > 0)
        np.testing.assert_array_equal(h, np.where(g > 0, P[:, None], 0.0))
