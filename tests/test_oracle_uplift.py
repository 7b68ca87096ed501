"""Pins of the oracle's compositing weights (Sec. 3.1, Eq. 1) and uplift
(Sec. 3.2, Eq. 3 and its matrix form Eq. 5, and the one-gradient-step reading
of Eq. 6): closed forms, hand-derived golden cases, exact invariants, and dense
linear algebra on tiny scenes."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2410_14462_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _axis_scene(depths, opacity, scale=0.01):
    n = len(depths)
    means = np.zeros((n, 3), np.float32)
    means[:, 2] = depths
    return inputs.Scene(means, np.full((n, 3), scale, np.float32),
                        np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
                        np.asarray(opacity, np.float32))


def _cam_from(c):
    p = np.zeros(16, np.float32)
    p[:9] = c["R"]
    p[9:12] = c["t"]
    p[12:16] = (c["fx"], c["fy"], c["cx"], c["cy"])
    return p, c["width"], c["height"]


def _weights_at(res, pixel_index, n):
    w = np.zeros(n)
    sel = res["pix"] == pixel_index
    w[res["gid"][sel]] = res["w64"][sel]
    return w


@pytest.mark.parametrize("mode", [oracle.MODE_HYBRID, oracle.MODE_FP64])
def test_golden_composite_cases(mode):
    g = json.load(open(os.path.join(GOLDEN, "composite_cases.json")))
    cam, w, h = _cam_from(g["camera"])
    u, v = g["pixel"]
    for case in g["cases"]:
        sc = _axis_scene(case["depths"], case["opacity"])
        res = oracle.view_uplift(sc, cam, w, h, mode=mode, triplets=True, t_final=True)
        got = _weights_at(res, v * w + u, sc.n)
        np.testing.assert_allclose(got, case["weights"], rtol=1e-6, atol=1e-9, err_msg=case["name"])
        assert abs(res["t_final"][v, u] - case["t_final"]) < 1e-6, case["name"]


def test_single_gaussian_closed_form():
    """One axis-aligned Gaussian on the optical axis: the Jacobian's depth column
    vanishes, so Sigma_2D = diag(fx^2 sx^2, fy^2 sy^2)/z^2 + 0.3 I exactly and
    w(p) = o * exp(-dx^2/(2a) - dy^2/(2c)); w = o at the pixel under the mean."""
    fx, fy, z = 120.0, 90.0, 4.0
    sx, sy = 0.05, 0.09
    o = 0.7
    cam = np.zeros(16, np.float32)
    cam[[0, 4, 8]] = 1
    cam[12:16] = (fx, fy, 40.5, 30.5)
    sc = inputs.Scene(np.array([[0, 0, z]], np.float32), np.array([[sx, sy, 0.02]], np.float32),
                      np.array([[1, 0, 0, 0]], np.float32), np.array([o], np.float32))
    W, H = 81, 61
    res = oracle.view_uplift(sc, cam, W, H, mode=oracle.MODE_FP64, triplets=True)
    a = (fx * float(np.float32(sx))) ** 2 / z ** 2 + 0.3
    c = (fy * float(np.float32(sy))) ** 2 / z ** 2 + 0.3
    op = float(np.float32(o))
    expect = {}
    for v in range(H):
        for u in range(W):
            dx, dy = u + 0.5 - 40.5, v + 0.5 - 30.5
            r = math.ceil(3 * math.sqrt(max(a, c)))
            if abs(dx) > 16 * 5 or abs(dy) > 16 * 5:
                continue
            wv = min(0.99, op * math.exp(-0.5 * (dx * dx / a + dy * dy / c)))
            if wv >= 1 / 255:
                expect[v * W + u] = wv
    got = dict(zip(res["pix"].tolist(), res["w64"].tolist()))
    assert set(got) == set(expect)
    for k in expect:
        assert abs(got[k] - expect[k]) < 1e-12
    assert abs(got[30 * W + 40] - op) < 1e-15
    # uplift of a ramp: f = sum_p w F / sum_p w by hand
    F = (np.arange(H * W, dtype=np.float32) / (H * W)).reshape(H, W, 1)
    num = np.zeros((1, 1))
    den = np.zeros(1)
    oracle.view_uplift(sc, cam, W, H, F, num, den, mode=oracle.MODE_FP64)
    hand = sum(wv * float(F.reshape(-1)[k]) for k, wv in expect.items()) / sum(expect.values())
    assert abs(num[0, 0] / den[0] - hand) < 1e-12


@pytest.mark.parametrize("mode", [oracle.MODE_HYBRID, oracle.MODE_FP64])
def test_weights_plus_transmittance_is_one(mode):
    """sum_i w_i(p) + T_final(p) = 1 exactly in exact arithmetic (telescoping
    product of Eq. 1); float64 rounding only."""
    wl = inputs.tiny_mask_workload()
    for v in (0, 3):
        res = oracle.view_uplift(wl.scene, wl.cams.params[v], 128, 128, mode=mode,
                                 triplets=True, t_final=True)
        s = np.bincount(res["pix"], weights=res["w64"], minlength=128 * 128)
        np.testing.assert_allclose(s + res["t_final"].ravel(), 1.0, rtol=0, atol=1e-12)
        assert res["count"] > 10_000


def test_constant_map_uplifts_to_constant():
    """Eq. 3 is a convex combination, so F = c gives f_i = c wherever beta_i > 0."""
    wl = inputs.small_field_workload(n=5000, views=2, d=3)
    c = np.array([0.25, -1.5, 3.0], np.float32)
    f, beta = oracle.uplift(wl.scene, wl.cams,
                            lambda v: np.broadcast_to(c, (wl.cams.height, wl.cams.width, 3)))
    pos = beta > 0
    assert pos.sum() > 1000
    np.testing.assert_allclose(f[pos], np.broadcast_to(c, f[pos].shape), rtol=0, atol=1e-12)
    assert (f[~pos] == 0).all()


def _dense_w(wl, views, mode=oracle.MODE_HYBRID):
    """W as a dense (views*pixels) x n matrix from the oracle's triplets."""
    P = wl.cams.height * wl.cams.width
    Wm = np.zeros((len(views) * P, wl.scene.n))
    for k, v in enumerate(views):
        res = oracle.view_uplift(wl.scene, wl.cams.params[v], wl.cams.width, wl.cams.height,
                                 mode=mode, triplets=True)
        Wm[k * P + res["pix"], res["gid"]] = res["w64"]
    return Wm


def test_matrix_form_and_gradient_step():
    """f = D^-1 W^T F (Eq. 5) with D = diag(W^T 1), and f = -D^-1 grad L(0) for
    L(f) = 0.5 ||F - W f||^2 (Eq. 6)."""
    wl = inputs.small_field_workload(n=600, views=2, d=5, width=40, height=31)
    views = [0, 1]
    Wm = _dense_w(wl, views)
    F = np.concatenate([wl.features(v).numpy().reshape(-1, 5) for v in views]).astype(np.float64)
    f, beta = oracle.uplift(wl.scene, wl.cams, lambda v: wl.features(v), views=views)
    Dg = Wm.sum(axis=0)
    np.testing.assert_allclose(beta, Dg, rtol=1e-13, atol=1e-15)
    pos = Dg > 0
    ref = np.zeros_like(f)
    ref[pos] = (Wm.T @ F)[pos] / Dg[pos, None]
    np.testing.assert_allclose(f, ref, rtol=1e-12, atol=1e-14)
    grad0 = Wm.T @ (Wm @ np.zeros_like(f) - F)
    step = np.zeros_like(f)
    step[pos] = -grad0[pos] / Dg[pos, None]
    np.testing.assert_allclose(f, step, rtol=1e-12, atol=1e-14)


def test_linearity_view_split_and_channel_independence():
    wl = inputs.small_field_workload(n=3000, views=3, d=6)
    H, W = wl.cams.height, wl.cams.width
    feats = {v: wl.features(v).numpy() for v in range(3)}
    n = wl.scene.n

    def sums(views, fmap):
        num = np.zeros((n, fmap(0).shape[-1]))
        den = np.zeros(n)
        for v in views:
            oracle.view_uplift(wl.scene, wl.cams.params[v], W, H, fmap(v), num, den)
        return num, den

    numA, denA = sums([0, 1, 2], lambda v: feats[v])
    num01, den01 = sums([0, 1], lambda v: feats[v])
    num2, den2 = sums([2], lambda v: feats[v])
    np.testing.assert_allclose(numA, num01 + num2, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(denA, den01 + den2, rtol=1e-12, atol=1e-13)
    # linearity in F: a power-of-two scale is exact in float32, so the sums scale
    # bit for bit; adding a constant map adds c * beta
    numB, _ = sums([0, 1, 2], lambda v: 4.0 * feats[v])
    assert np.array_equal(numB, 4.0 * numA)
    numK, _ = sums([0, 1, 2], lambda v: np.full((H, W, 2), 0.5, np.float32))
    np.testing.assert_allclose(numK, 0.5 * np.stack([denA, denA], 1), rtol=1e-13, atol=1e-15)
    # channel 4 alone equals channel 4 of the joint run, bit for bit
    numC, denC = sums([0, 1, 2], lambda v: np.ascontiguousarray(feats[v][..., 4:5]))
    assert np.array_equal(numC[:, 0], numA[:, 4])
    assert np.array_equal(denC, denA)


def test_index_permutation_permutes_output():
    wl = inputs.small_field_workload(n=2000, views=2, d=4)
    perm = np.random.default_rng(2).permutation(wl.scene.n)
    f, beta = oracle.uplift(wl.scene, wl.cams, lambda v: wl.features(v))
    f2, beta2 = oracle.uplift(wl.scene.subset(perm), wl.cams, lambda v: wl.features(v))
    # the scene's depths are distinct, so only the order changes
    np.testing.assert_allclose(f2, f[perm], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(beta2, beta[perm], rtol=1e-13, atol=1e-15)


def test_hybrid_decisions_track_fp64_definition():
    """The float32 decision track only flips near-threshold decisions: uplift
    from both modes agrees to float32-level error on the tiny workload."""
    wl = inputs.tiny_mask_workload()
    fh, bh = oracle.uplift(wl.scene, wl.cams, lambda v: wl.features(v), mode=oracle.MODE_HYBRID)
    f6, b6 = oracle.uplift(wl.scene, wl.cams, lambda v: wl.features(v), mode=oracle.MODE_FP64)
    pos = (bh > 0) & (b6 > 0)
    assert (bh > 0).sum() == (b6 > 0).sum()
    rel = np.linalg.norm(fh[pos] - f6[pos]) / np.linalg.norm(f6[pos])
    assert rel < 1e-4
    assert np.linalg.norm(bh - b6) / np.linalg.norm(b6) < 1e-4


def test_exp32_accuracy():
    x = np.concatenate([np.linspace(-87.0, 0.0, 20001), -np.logspace(-8, 1.9, 2000), [0.0, -0.5, -1e-30]])
    x = x.astype(np.float32)
    e = oracle.exp32(x)
    ref = np.exp(x.astype(np.float64))
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    assert (np.abs(e - ref) / ulp).max() <= 1.0
    assert oracle.exp32(np.array([0.0], np.float32))[0] == 1.0
    assert oracle.exp32(np.array([-100.0], np.float32))[0] == 0.0


def test_count_normalised_uplift():
    """GaussianEditor's normaliser (appendix): f_i = sum w F / |S_i|.  One
    Gaussian: |S| is the number of pixels with w >= 1/255 (the closed form of
    the single-Gaussian pin); in general f_count * count = f * beta = num."""
    fx, fy, z = 120.0, 90.0, 4.0
    cam = np.zeros(16, np.float32)
    cam[[0, 4, 8]] = 1
    cam[12:16] = (fx, fy, 40.5, 30.5)
    sc = inputs.Scene(np.array([[0, 0, z]], np.float32), np.array([[0.05, 0.09, 0.02]], np.float32),
                      np.array([[1, 0, 0, 0]], np.float32), np.array([0.7], np.float32))
    W, H = 81, 61
    a = (fx * float(np.float32(0.05))) ** 2 / z ** 2 + 0.3
    c = (fy * float(np.float32(0.09))) ** 2 / z ** 2 + 0.3
    op = float(np.float32(0.7))
    F = (np.arange(H * W, dtype=np.float32) / (H * W)).reshape(H, W, 1)
    cams = inputs.Cameras(cam[None, :], W, H)
    fc, cnt = oracle.uplift(sc, cams, lambda v: F, mode=oracle.MODE_FP64, count_normalise=True)
    ws = {}
    for v in range(H):
        for u in range(W):
            dx, dy = u + 0.5 - 40.5, v + 0.5 - 30.5
            wv = min(0.99, op * math.exp(-0.5 * (dx * dx / a + dy * dy / c)))
            if wv >= 1 / 255:
                ws[v * W + u] = wv
    assert cnt[0] == len(ws)
    assert abs(fc[0, 0] - sum(w * float(F.reshape(-1)[k]) for k, w in ws.items()) / len(ws)) < 1e-12
    wl = inputs.small_field_workload(n=3000, views=2, d=4)
    f, beta = oracle.uplift(wl.scene, wl.cams, lambda v: wl.features(v))
    fc, cnt = oracle.uplift(wl.scene, wl.cams, lambda v: wl.features(v), count_normalise=True)
    assert np.array_equal(cnt > 0, beta > 0) and (cnt == np.round(cnt)).all()
    np.testing.assert_allclose(fc * cnt[:, None], f * beta[:, None], rtol=1e-12, atol=1e-12)
