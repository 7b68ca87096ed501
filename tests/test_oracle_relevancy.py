"""Pins of the oracle's relevancy score (appendix, "Relevancy scores"):
r_iq = min_k exp(T f.phi_q) / (exp(T f.phi_q) + exp(T f.phi_cano^k)) on
l2-normalised vectors, checked against closed forms, a scalar brute force and
the sigmoid identity r = min_k 1 / (1 + exp(T (s_k - s_q)))."""
import math

import numpy as np

import oracle


def test_closed_forms():
    e = np.eye(4)
    # f orthogonal to every embedding: every ratio is 1/2
    r = oracle.relevancy(e[[0]], e[[1]], e[[2, 3]], 10.0)
    assert abs(r[0, 0] - 0.5) < 1e-15
    # f along the query, orthogonal to the canonical phrases: e^T / (e^T + 1)
    r = oracle.relevancy(e[[1]] * 3.0, e[[1]], e[[2, 3]], 10.0)
    assert abs(r[0, 0] - math.exp(10) / (math.exp(10) + 1)) < 1e-15
    # f along a canonical phrase: 1 / (1 + e^T), the minimum over k
    r = oracle.relevancy(e[[2]], e[[1]], e[[2, 3]], 10.0)
    assert abs(r[0, 0] - 1 / (1 + math.exp(10))) < 1e-15
    # a query equal to a canonical phrase scores exactly 1/2 wherever f points
    rng = np.random.default_rng(0)
    r = oracle.relevancy(rng.normal(size=(5, 4)), e[[3]], e[[2, 3]], 10.0)
    assert np.all(r <= 0.5 + 1e-15) and np.any(np.abs(r - 0.5) < 1e-15)


def test_brute_force_and_sigmoid_identity():
    rng = np.random.default_rng(1)
    f = rng.normal(size=(7, 6))
    f[3] = 0.0                                     # a zero feature: all dots 0, r = 1/2
    pq = rng.normal(size=(3, 6))
    pc = rng.normal(size=(4, 6))
    r = oracle.relevancy(f, pq, pc, 10.0)
    for i in range(7):
        nf = np.linalg.norm(f[i])
        fi = f[i] / nf if nf > 0 else f[i]
        for q in range(3):
            sq = fi @ (pq[q] / np.linalg.norm(pq[q]))
            vals = []
            for k in range(4):
                sk = fi @ (pc[k] / np.linalg.norm(pc[k]))
                vals.append(math.exp(10 * sq) / (math.exp(10 * sq) + math.exp(10 * sk)))
                assert abs(vals[-1] - 1 / (1 + math.exp(10 * (sk - sq)))) < 1e-15
            assert abs(r[i, q] - min(vals)) < 1e-15
    assert np.allclose(r[3], 0.5)
    # scale invariance of every input row
    r2 = oracle.relevancy(f * 4.0, pq * 0.1, pc * 7.0, 10.0)
    assert np.allclose(r, r2, rtol=0, atol=1e-14)
