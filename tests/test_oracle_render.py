"""Pins of the oracle's rendering operator F_hat = W f (Sec. 3.2, Eq. 4): the
hand-derived compositing weights of the golden cases, the adjoint identity with
the uplift's numerator (W^T F, Eq. 5), the telescoping sum of the weights
(Eq. 1), the dense matrix built from the weight triplets, and a single Gaussian
in closed form."""
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


@pytest.mark.parametrize("mode", [oracle.MODE_HYBRID, oracle.MODE_FP64])
def test_golden_cases_one_hot_features(mode):
    """With f_i = e_i (one-hot rows) the rendered pixel is the weight vector of
    the hand-derived cases."""
    g = json.load(open(os.path.join(GOLDEN, "composite_cases.json")))
    c = g["camera"]
    cam = np.zeros(16, np.float32)
    cam[:9] = c["R"]
    cam[9:12] = c["t"]
    cam[12:16] = (c["fx"], c["fy"], c["cx"], c["cy"])
    u, v = g["pixel"]
    for case in g["cases"]:
        sc = _axis_scene(case["depths"], case["opacity"])
        out, _ = oracle.view_render(sc, cam, c["width"], c["height"], np.eye(sc.n), mode=mode)
        np.testing.assert_allclose(out[v, u], case["weights"], rtol=1e-6, atol=1e-9, err_msg=case["name"])


def test_adjoint_of_the_uplift_numerator():
    """<W f, F> = <f, W^T F>: the render and the uplift's accumulation (two
    separately written sums) are transposes of each other, per view."""
    wl = inputs.small_field_workload(n=4000, views=3, d=7, width=70, height=45)
    n, d = wl.scene.n, 7
    f = inputs.gaussian_features(n, d, seed=3).astype(np.float64)
    for v in range(3):
        F = wl.features(v).numpy()
        Fh, count = oracle.view_render(wl.scene, wl.cams.params[v], wl.cams.width, wl.cams.height, f)
        num = np.zeros((n, d))
        den = np.zeros(n)
        oracle.view_uplift(wl.scene, wl.cams.params[v], wl.cams.width, wl.cams.height, F, num, den)
        lhs = float(np.sum(Fh * F.astype(np.float64)))
        rhs = float(np.sum(f * num))
        assert count > 5000
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs)) * count ** 0.5
        # and with constant F = 1: <W f, 1> = <f, beta>
        assert abs(Fh.sum() - float((f.T @ den).sum())) <= 1e-10


@pytest.mark.parametrize("mode", [oracle.MODE_HYBRID, oracle.MODE_FP64])
def test_rendering_ones_gives_opacity(mode):
    """f = 1 renders sum_i w_i(p) = 1 - T_final(p) (telescoping product of Eq. 1)."""
    wl = inputs.tiny_mask_workload()
    for v in (1, 5):
        Fh, _ = oracle.view_render(wl.scene, wl.cams.params[v], 128, 128, np.ones((wl.scene.n, 2)), mode=mode)
        res = oracle.view_uplift(wl.scene, wl.cams.params[v], 128, 128, mode=mode, t_final=True)
        np.testing.assert_allclose(Fh[..., 0], 1.0 - res["t_final"], rtol=0, atol=1e-12)
        assert np.array_equal(Fh[..., 0], Fh[..., 1])
        assert (Fh[..., 0] > 0.5).sum() > 1000


def test_dense_matrix_and_layout():
    """F_hat[v, y, x, :] = row (y*W + x) of the dense W (from the weight
    triplets) times f; pixels without a contributor render to 0."""
    wl = inputs.small_field_workload(n=500, views=2, d=3, width=37, height=29)
    n = wl.scene.n
    f = inputs.gaussian_features(n, 5, seed=11, normalise=False).astype(np.float64)
    Fh = oracle.render(wl.scene, wl.cams, f)
    assert Fh.shape == (2, 29, 37, 5)
    for v in range(2):
        res = oracle.view_uplift(wl.scene, wl.cams.params[v], 37, 29, triplets=True)
        Wm = np.zeros((29 * 37, n))
        Wm[res["pix"], res["gid"]] = res["w64"]
        np.testing.assert_allclose(Fh[v].reshape(-1, 5), Wm @ f, rtol=1e-13, atol=1e-15)
        empty = Wm.sum(axis=1) == 0
        assert empty.any() and (Fh[v].reshape(-1, 5)[empty] == 0).all()


def test_single_gaussian_closed_form():
    """One axis-aligned Gaussian on the optical axis (Sigma_2D diagonal, see the
    uplift pins): F_hat(p) = w(p) f with w = o exp(-dx^2/(2a) - dy^2/(2c))."""
    fx, fy, z = 120.0, 90.0, 4.0
    sx, sy = 0.05, 0.09
    o = 0.7
    cam = np.zeros(16, np.float32)
    cam[[0, 4, 8]] = 1
    cam[12:16] = (fx, fy, 40.5, 30.5)
    sc = inputs.Scene(np.array([[0, 0, z]], np.float32), np.array([[sx, sy, 0.02]], np.float32),
                      np.array([[1, 0, 0, 0]], np.float32), np.array([o], np.float32))
    W, H = 81, 61
    f = np.array([[0.5, -2.0, 3.25]])
    Fh, count = oracle.view_render(sc, cam, W, H, f, mode=oracle.MODE_FP64)
    a = (fx * float(np.float32(sx))) ** 2 / z ** 2 + 0.3
    c = (fy * float(np.float32(sy))) ** 2 / z ** 2 + 0.3
    op = float(np.float32(o))
    expect = np.zeros((H, W))
    for v in range(H):
        for u in range(W):
            dx, dy = u + 0.5 - 40.5, v + 0.5 - 30.5
            if abs(dx) > 16 * 5 or abs(dy) > 16 * 5:
                continue
            wv = min(0.99, op * math.exp(-0.5 * (dx * dx / a + dy * dy / c)))
            if wv >= 1 / 255:
                expect[v, u] = wv
    assert count == int((expect > 0).sum())
    np.testing.assert_allclose(Fh, expect[..., None] * f[0], rtol=0, atol=1e-12)


def test_empty_inputs():
    sc = _axis_scene([], [])
    cam = np.zeros(16, np.float32)
    cam[[0, 4, 8]] = 1
    cam[12:16] = (50, 50, 8, 8)
    Fh, count = oracle.view_render(sc, cam, 17, 9, np.zeros((0, 4)))
    assert count == 0 and Fh.shape == (9, 17, 4) and (Fh == 0).all()
    wl = inputs.tiny_mask_workload()
    Fh, count = oracle.view_render(wl.scene, wl.cams.params[0], 128, 128, np.zeros((wl.scene.n, 0)))
    assert Fh.shape == (128, 128, 0) and count > 10_000


def test_tile_selection_matches_full_render():
    """Rendering a subset of tiles gives those tiles' pixels of the full render
    exactly and leaves the rest zero."""
    wl = inputs.small_field_workload(n=3000, views=1, d=4, width=70, height=45)
    f = inputs.gaussian_features(wl.scene.n, 4, seed=2).astype(np.float64)
    full, cf = oracle.view_render(wl.scene, wl.cams.params[0], 70, 45, f)
    tiles = np.zeros((3, 5), bool)
    tiles[0, 1] = tiles[2, 4] = tiles[1, 2] = True
    part, cp = oracle.view_render(wl.scene, wl.cams.params[0], 70, 45, f, tiles=tiles)
    pix = np.kron(tiles, np.ones((16, 16), bool))[:45, :70]
    assert np.array_equal(part[pix], full[pix]) and (part[~pix] == 0).all()
    assert 0 < cp < cf
