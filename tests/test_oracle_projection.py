"""Pins of the oracle's projection (Sec. 3.1: Gaussians projected onto the image
plane; EWA covariance and tile rules of the 3DGS rasteriser the paper uses,
Sec. 5) against computations that do not share its code: scipy's quaternion
rotation, a finite-difference Jacobian of the pinhole map, numpy eigenvalues,
Monte-Carlo projection of samples, and the brute-force tile-rectangle rule."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2410_14462_gb300 import inputs


def _cam(R=np.eye(3), t=(0, 0, 0), f=(300.0, 280.0), c=(200.0, 150.0), w=400, h=300):
    p = np.zeros(16, np.float32)
    p[:9] = np.asarray(R, np.float64).reshape(-1)
    p[9:12] = t
    p[12:14] = f
    p[14:16] = c
    return p, w, h


def _pinhole(cam, X):
    R = cam[:9].astype(np.float64).reshape(3, 3)
    t = cam[9:12].astype(np.float64)
    x = X @ R.T + t
    return np.stack([cam[12] * x[..., 0] / x[..., 2] + cam[14],
                     cam[13] * x[..., 1] / x[..., 2] + cam[15]], axis=-1)


def _reference_cov2d(scene, i, cam):
    """Sigma_2D = J R_c Sigma R_c^T J^T + 0.3 I with Sigma from scipy's rotation
    and J the central-difference Jacobian of the pinhole map."""
    q = scene.quats[i].astype(np.float64)
    Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()   # scipy is scalar-last
    S = np.diag(scene.scales[i].astype(np.float64) ** 2)
    Sigma = Rq @ S @ Rq.T
    mu = scene.means[i].astype(np.float64)
    h = 1e-5
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (_pinhole(cam, mu + e) - _pinhole(cam, mu - e)) / (2 * h)
    return J @ Sigma @ J.T + 0.3 * np.eye(2)


def _random_onscreen_scene(n=200, seed=3):
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-1, 1, n), rng.uniform(-0.8, 0.8, n), rng.uniform(3, 6, n)], 1)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    scales = np.exp(rng.normal(-3.0, 0.7, size=(n, 3)))
    op = rng.uniform(0.05, 0.95, n)
    return inputs.Scene(means.astype(np.float32), scales.astype(np.float32),
                        q.astype(np.float32), op.astype(np.float32))


def test_mean2d_matches_pinhole():
    sc = _random_onscreen_scene()
    R = Rotation.from_euler("xyz", [0.1, -0.2, 0.05]).as_matrix()
    cam, w, h = _cam(R=R, t=(0.1, -0.05, 0.3))
    pr = oracle.project(sc, cam, w, h)
    ref = _pinhole(cam, sc.means.astype(np.float64))
    vis = pr["visible"]
    assert vis.sum() > 150
    np.testing.assert_allclose(pr["p64"][vis, :2], ref[vis], rtol=0, atol=1e-9)
    np.testing.assert_allclose(pr["p32"][vis, :2], ref[vis], rtol=0, atol=2e-3)


def test_conic_is_inverse_of_ewa_covariance():
    sc = _random_onscreen_scene()
    R = Rotation.from_euler("xyz", [0.1, -0.2, 0.05]).as_matrix()
    cam, w, h = _cam(R=R, t=(0.1, -0.05, 0.3))
    pr = oracle.project(sc, cam, w, h)
    checked = 0
    for i in np.flatnonzero(pr["visible"]):
        # the Jacobian clamp (1.3 x half-FOV) is inactive for on-screen means
        cov = _reference_cov2d(sc, i, cam)
        conic = np.linalg.inv(cov)
        got64 = np.array([[pr["p64"][i, 3], pr["p64"][i, 4]], [pr["p64"][i, 4], pr["p64"][i, 5]]])
        got32 = np.array([[pr["p32"][i, 3], pr["p32"][i, 4]], [pr["p32"][i, 4], pr["p32"][i, 5]]])
        np.testing.assert_allclose(got64, conic, rtol=1e-6, atol=1e-9 * np.abs(conic).max())
        np.testing.assert_allclose(got32, conic, rtol=2e-3, atol=2e-4 * np.abs(conic).max())
        checked += 1
    assert checked > 150


def test_radius_from_largest_eigenvalue():
    sc = _random_onscreen_scene()
    cam, w, h = _cam()
    pr = oracle.project(sc, cam, w, h)
    for i in np.flatnonzero(pr["visible"]):
        cov = _reference_cov2d(sc, i, cam)
        lam = np.linalg.eigvalsh(cov)
        if (lam[1] - lam[0]) ** 2 / 4 <= 0.2:      # the 0.1 discriminant floor is active
            continue
        r = math.ceil(3 * math.sqrt(lam[1]))
        assert pr["p64"][i, 6] == r
        assert abs(pr["p32"][i, 7] - r) <= 1


def test_monte_carlo_projection_matches_ewa():
    """Sampled 3D points pushed through the exact perspective map have the EWA
    covariance (minus the 0.3 px^2 dilation) to first order for small splats."""
    rng = np.random.default_rng(11)
    sc = _random_onscreen_scene(n=6, seed=5)
    sc.scales[:] = np.float32(0.01)
    sc.scales[:, 0] = np.float32(0.03)
    cam, w, h = _cam()
    pr = oracle.project(sc, cam, w, h)
    for i in range(sc.n):
        q = sc.quats[i].astype(np.float64)
        Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        X = rng.normal(size=(400_000, 3)) * sc.scales[i].astype(np.float64)
        X = X @ Rq.T + sc.means[i]
        emp = np.cov(_pinhole(cam, X).T)
        a, b, c = pr["p64"][i, 3:6]
        cov = np.linalg.inv(np.array([[a, b], [b, c]])) - 0.3 * np.eye(2)
        np.testing.assert_allclose(cov, emp, rtol=0.03, atol=0.03 * np.abs(emp).max())


def test_culling_rules():
    cam, w, h = _cam()
    means = np.array([[0, 0, 0.1],      # in front of the near plane (z <= 0.2)
                      [0, 0, -3.0],     # behind the camera
                      [50, 0, 3.0],     # far off screen to the right
                      [0, 0, 3.0]],     # visible
                     np.float32)
    sc = inputs.Scene(means, np.full((4, 3), 0.02, np.float32),
                      np.tile(np.array([1, 0, 0, 0], np.float32), (4, 1)), np.full(4, 0.5, np.float32))
    pr = oracle.project(sc, cam, w, h)
    assert pr["visible"].tolist() == [False, False, False, True]
    assert (pr["rect"][:3] == 0).all()


def test_tile_rect_rule_bruteforce():
    sc = _random_onscreen_scene(n=400, seed=9)
    cam, w, h = _cam(w=397, h=301)     # ragged last tile column / row
    pr = oracle.project(sc, cam, w, h)
    TX, TY = (w + 15) // 16, (h + 15) // 16
    for i in np.flatnonzero(pr["visible"]):
        mx, my = float(pr["p32"][i, 0]), float(pr["p32"][i, 1])
        r = float(pr["p32"][i, 7])
        tiles_x = [tx for tx in range(TX) if math.floor((mx - r) / 16) <= tx <= math.floor((mx + r) / 16)]
        tiles_y = [ty for ty in range(TY) if math.floor((my - r) / 16) <= ty <= math.floor((my + r) / 16)]
        x0, y0, x1, y1 = pr["rect"][i]
        assert list(range(x0, x1)) == tiles_x
        assert list(range(y0, y1)) == tiles_y


def test_tile_lists_are_rect_members_in_depth_order():
    wl = inputs.tiny_mask_workload()
    sc = wl.scene.subset(np.arange(3000))
    cams = wl.cams
    for v in (0, 5):
        pr = oracle.project(sc, cams.params[v], cams.width, cams.height)
        ranges, lst = oracle.tile_lists(sc, cams.params[v], cams.width, cams.height)
        TX = (cams.width + 15) // 16
        rect = pr["rect"]
        vis = pr["visible"]
        for t in range(ranges.shape[0]):
            tx, ty = t % TX, t // TX
            got = lst[ranges[t, 0]:ranges[t, 1]]
            member = np.flatnonzero(vis & (rect[:, 0] <= tx) & (tx < rect[:, 2]) &
                                    (rect[:, 1] <= ty) & (ty < rect[:, 3]))
            assert sorted(got.tolist()) == member.tolist()
            z = pr["p32"][got, 2]
            key = list(zip(z.tolist(), got.tolist()))
            assert key == sorted(key)


def test_near_singular_conic_uses_float64_inverse():
    """An edge-on needle without dilation would be singular; with the 0.3 px^2
    dilation its float32 conic must still match the float64 inverse."""
    cam, w, h = _cam()
    q = Rotation.from_euler("z", 0.7).as_quat()   # scalar-last
    sc = inputs.Scene(np.array([[0.05, 0.02, 2.0]], np.float32),
                      np.array([[0.6, 1e-6, 1e-6]], np.float32),
                      np.array([[q[3], q[0], q[1], q[2]]], np.float32), np.array([0.5], np.float32))
    pr = oracle.project(sc, cam, w, h)
    assert pr["visible"][0]
    np.testing.assert_allclose(pr["p32"][0, 3:6], pr["p64"][0, 3:6], rtol=1e-4)
