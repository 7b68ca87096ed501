"""Seeded synthetic workloads shaped like the paper's uplifting experiments.

This module only *produces data*: Gaussian scenes, pinhole cameras and 2D
feature maps.  It holds none of the uplifting arithmetic (no projection, no
compositing, no aggregation) so that both the CUDA path and the CPU oracle can
consume exactly the same bytes.

Workloads (paper Sec. 5 and App. B.1 describe the real ones: trained 3DGS
scenes of ~600k Gaussians, 131-299 views of about 724x986 pixels, DINOv2
ViT-g/14 patch features, SAM masks):

* tiny scene: 20,000 Gaussians, means U[-1,1]^3, log-scales N(-4,0.5), random
  unit quaternions, opacity sigmoid(N(0,1.5)); 8 cameras on a radius-3 sphere,
  128x128 px, fx=fy=120; one binary mask per view (rays passing within 0.4 of
  the origin), seed 0.
* paper-scale scene: 1,000,000 Gaussians drawn around 40 cluster centres
  (U[-2,2]^3, per-axis sigma 0.15, clipped to [-2,2]^3); 150 cameras on the
  upper hemisphere of radius 4, 980x546 px, fx=fy=900; per-view smooth random
  feature field (bilinear upsample of an N(0,1) grid at 1/14 resolution, the
  DINOv2 patch size, L2-normalised per pixel), seed 1.

Scales are produced as *linear* standard deviations: the log-scale draw is
exponentiated once here in float64 and rounded to float32, so neither side of a
parity test depends on a float32 ``exp`` of the scales.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

TILE = 16


@dataclasses.dataclass
class Scene:
    """A Gaussian Splatting scene in structure-of-arrays float32 layout."""

    means: np.ndarray     # [N,3]
    scales: np.ndarray    # [N,3] linear per-axis standard deviations
    quats: np.ndarray     # [N,4] (w,x,y,z), unit norm up to float32 rounding
    opacity: np.ndarray   # [N]   in (0,1), post-sigmoid

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx].copy(), self.scales[idx].copy(),
                     self.quats[idx].copy(), self.opacity[idx].copy())


@dataclasses.dataclass
class Cameras:
    """Pinhole cameras sharing one image size.

    ``params`` is float32 [V,16]: a row-major world->camera rotation R (9),
    translation t (3), fx, fy, cx, cy.  Camera axes follow OpenCV: x right,
    y down, z forward; a world point X maps to camera point R X + t and to the
    pixel (fx x/z + cx, fy y/z + cy); pixel (u,v) has its centre at
    (u+0.5, v+0.5).
    """

    params: np.ndarray    # [V,16] float32
    width: int
    height: int

    @property
    def v(self) -> int:
        return int(self.params.shape[0])

    def centers(self) -> np.ndarray:
        """Camera centres in world space (float64), C = -R^T t."""
        p = self.params.astype(np.float64)
        R = p[:, :9].reshape(-1, 3, 3)
        t = p[:, 9:12]
        return -np.einsum("vji,vj->vi", R, t)

    def subset(self, idx) -> "Cameras":
        return Cameras(self.params[idx].copy(), self.width, self.height)


def _rng(seed: int, *stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, *stream])))


def _finish_scene(rng: np.random.Generator, means: np.ndarray) -> Scene:
    n = means.shape[0]
    log_scales = rng.normal(-4.0, 0.5, size=(n, 3))
    q = rng.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    logit = rng.normal(0.0, 1.5, size=n)
    opacity = 1.0 / (1.0 + np.exp(-logit))
    return Scene(means.astype(np.float32),
                 np.exp(log_scales).astype(np.float32),
                 q.astype(np.float32),
                 opacity.astype(np.float32))


def scene_uniform(n: int, seed: int, extent: float = 1.0) -> Scene:
    """Means uniform in [-extent, extent]^3 (the tiny workload)."""
    rng = _rng(seed, 0)
    means = rng.uniform(-extent, extent, size=(n, 3))
    return _finish_scene(rng, means)


def scene_clusters(n: int, seed: int, n_clusters: int = 40, sigma: float = 0.15,
                   extent: float = 2.0) -> Scene:
    """Means around ``n_clusters`` centres (the paper-scale workload)."""
    rng = _rng(seed, 0)
    centres = rng.uniform(-extent, extent, size=(n_clusters, 3))
    which = rng.integers(0, n_clusters, size=n)
    means = centres[which] + rng.normal(0.0, sigma, size=(n, 3))
    np.clip(means, -extent, extent, out=means)
    return _finish_scene(rng, means)


def cluster_centres(seed: int, n_clusters: int = 40, extent: float = 2.0) -> np.ndarray:
    """The centres :func:`scene_clusters` used for the same seed."""
    rng = _rng(seed, 0)
    return rng.uniform(-extent, extent, size=(n_clusters, 3))


def look_at(center: np.ndarray, target=(0.0, 0.0, 0.0)) -> tuple[np.ndarray, np.ndarray]:
    """World->camera (R, t) in float64 for a camera at ``center`` looking at ``target``.

    World up is +z; when the viewing direction is (anti)parallel to it, +y is
    used instead.
    """
    c = np.asarray(center, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - c
    f /= np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0])
    x = np.cross(f, up)
    if np.linalg.norm(x) < 1e-6:
        x = np.cross(f, np.array([0.0, 1.0, 0.0]))
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])
    t = -R @ c
    return R, t


def fibonacci_points(n: int, hemisphere: bool) -> np.ndarray:
    """n unit vectors spread by the golden-angle spiral (upper half if asked)."""
    i = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - i / n if hemisphere else 1.0 - 2.0 * i / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def cameras_orbit(n: int, radius: float, width: int, height: int, focal: float,
                  hemisphere: bool) -> Cameras:
    """Cameras on a sphere (or upper hemisphere) looking at the origin."""
    pts = fibonacci_points(n, hemisphere) * radius
    params = np.zeros((n, 16), dtype=np.float64)
    for v, c in enumerate(pts):
        R, t = look_at(c)
        params[v, :9] = R.reshape(-1)
        params[v, 9:12] = t
        params[v, 12:16] = (focal, focal, width / 2.0, height / 2.0)
    return Cameras(params.astype(np.float32), width, height)


def pixel_rays(cams: Cameras, v: int) -> tuple[np.ndarray, np.ndarray]:
    """World-space origin and unit directions [H,W,3] through pixel centres (float64)."""
    p = cams.params[v].astype(np.float64)
    R = p[:9].reshape(3, 3)
    fx, fy, cx, cy = p[12:16]
    u = np.arange(cams.width, dtype=np.float64) + 0.5
    w = np.arange(cams.height, dtype=np.float64) + 0.5
    uu, vv = np.meshgrid(u, w)
    d_cam = np.stack([(uu - cx) / fx, (vv - cy) / fy, np.ones_like(uu)], axis=-1)
    d = d_cam @ R          # R^T d_cam, row-vector form
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    return cams.centers()[v], d


def sphere_masks(cams: Cameras, radius: float = 0.4, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Binary masks [V,H,W,1] float32: 1 where the pixel ray passes within
    ``radius`` of ``center`` (a projected sphere, thresholded): the synthetic
    stand-in for a reference frame's foreground mask."""
    out = np.zeros((cams.v, cams.height, cams.width, 1), dtype=np.float32)
    c = np.asarray(center, dtype=np.float64)
    for v in range(cams.v):
        o, d = pixel_rays(cams, v)
        # distance from the centre to the line o + s d (the sphere is in front)
        cr = np.cross(np.broadcast_to(o - c, d.shape), d)
        out[v, :, :, 0] = (np.linalg.norm(cr, axis=-1) < radius).astype(np.float32)
    return out


def field_grid_shape(height: int, width: int, patch: int = 14) -> tuple[int, int]:
    return max(1, round(height / patch)), max(1, round(width / patch))


def field_grid(seed: int, view: int, d: int, height: int, width: int) -> np.ndarray:
    """The N(0,1) coarse grid [D,gh,gw] float32 behind view ``view``'s feature map."""
    gh, gw = field_grid_shape(height, width)
    return _rng(seed, 1, view).standard_normal((d, gh, gw), dtype=np.float32)


def feature_field(seed: int, view: int, d: int, height: int, width: int, device="cpu",
                  dtype=None):
    """Smooth random feature map [H,W,D] (torch tensor, channels-last).

    The coarse grid is upsampled bilinearly with half-pixel centres and edge
    clamping, then every pixel's D-vector is L2-normalised (a zero vector stays
    zero).  Built with torch so that paper-scale maps can be produced directly
    in device memory.
    """
    import torch
    import torch.nn.functional as tF

    g = torch.from_numpy(field_grid(seed, view, d, height, width)).to(device)
    up = tF.interpolate(g[None], size=(height, width), mode="bilinear", align_corners=False)[0]
    f = up.permute(1, 2, 0).contiguous()
    nrm = torch.linalg.vector_norm(f, dim=-1, keepdim=True)
    f = torch.where(nrm > 0, f / torch.where(nrm > 0, nrm, torch.ones_like(nrm)), f)
    if dtype is not None:
        f = f.to(dtype)
    return f


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

def gaussian_features(n: int, d: int, seed: int, normalise: bool = True) -> np.ndarray:
    """Per-Gaussian features [n,d] float32 to render back (Eq. 4): N(0,1) rows,
    L2-normalised like the uplifted DINOv2 features (zero rows stay zero)."""
    f = _rng(seed, 7).standard_normal((n, d))
    if normalise and d > 0:
        nrm = np.linalg.norm(f, axis=1, keepdims=True)
        f = np.divide(f, nrm, out=np.zeros_like(f), where=nrm > 0)
    return f.astype(np.float32)


@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    cams: Cameras
    d: int
    seed: int
    kind: str          # "mask" or "field"

    def features_d(self, view: int, d: int, device="cpu", dtype=None):
        """The same smooth field with another channel count (precision form)."""
        return feature_field(self.seed, view, d, self.cams.height, self.cams.width, device=device, dtype=dtype)

    def features(self, view: int, device="cpu", dtype=None):
        """Feature map [H,W,D] of one view as a torch tensor."""
        import torch
        if self.kind == "mask":
            m = sphere_masks(self.cams.subset([view]))[0]
            t = torch.from_numpy(m).to(device)
            return t.to(dtype) if dtype is not None else t
        return feature_field(self.seed, view, self.d, self.cams.height, self.cams.width,
                             device=device, dtype=dtype)


def tiny_mask_workload() -> Workload:
    """20k Gaussians, 8 views of 128x128, D=1 sphere masks, seed 0."""
    scene = scene_uniform(20_000, seed=0)
    cams = cameras_orbit(8, 3.0, 128, 128, 120.0, hemisphere=False)
    return Workload("tiny-mask-20k-8v-128px-d1", scene, cams, 1, 0, "mask")


def paper_scale_workload(n: int = 1_000_000, views: int = 150, d: int = 384,
                         width: int = 980, height: int = 546, seed: int = 1) -> Workload:
    """1M clustered Gaussians, 150 hemisphere views of 980x546, D=384 field."""
    scene = scene_clusters(n, seed=seed)
    cams = cameras_orbit(views, 4.0, width, height, 900.0 * width / 980.0, hemisphere=True)
    return Workload(f"clusters-{n}-{views}v-{width}x{height}-d{d}", scene, cams, d, seed, "field")


def small_field_workload(n: int = 20_000, views: int = 4, d: int = 48, width: int = 100,
                         height: int = 75, seed: int = 5) -> Workload:
    """Parity-test sized field workload with ragged tile edges."""
    scene = scene_clusters(n, seed=seed, n_clusters=8, sigma=0.25, extent=1.0)
    cams = cameras_orbit(views, 3.0, width, height, 0.9 * width, hemisphere=True)
    return Workload(f"clusters-{n}-{views}v-{width}x{height}-d{d}", scene, cams, d, seed, "field")


# --------------------------------------------------------------------------
# batched and serving forms: many uplifts of uneven size on shared pools
# --------------------------------------------------------------------------

FORM_WIDTH, FORM_HEIGHT, FORM_FOCAL = 640, 480, 600.0


def form_cameras(views: int = 200) -> Cameras:
    """Camera set shared by the jobs and requests: a hemisphere of radius 4
    looking at the origin, 640x480, fx = fy = 600 (about the field of view of
    the paper-scale cameras)."""
    return cameras_orbit(views, 4.0, FORM_WIDTH, FORM_HEIGHT, FORM_FOCAL, hemisphere=True)


def form_pool(d: int, cams: Cameras, seed: int = 5, device="cuda", dtype=None):
    """Feature pool [V,H,W,d] (bfloat16 by default) built view by view on the
    device: d = 1 holds each view's sphere mask (radius 0.4 at the origin),
    any other d the smooth unit-norm field of ``feature_field``."""
    import torch
    dtype = dtype or torch.bfloat16
    out = torch.empty((cams.v, cams.height, cams.width, d), dtype=dtype, device=device)
    for v in range(cams.v):
        if d == 1:
            out[v] = torch.from_numpy(sphere_masks(cams.subset([v]))[0]).to(device=device, dtype=dtype)
        else:
            out[v] = feature_field(seed, v, d, cams.height, cams.width, device=device, dtype=dtype)
    return out


@dataclasses.dataclass
class JobSpec:
    n: int          # Gaussians (scene_clusters with the paper-scale layout)
    seed: int       # scene seed
    views: int
    v0: int         # first view of the pool
    d: int


def batch_jobs(count: int = 32, seed: int = 3, pool_views: int = 200, dims=(1, 3, 64, 384, 512),
               n_range=(50_000, 1_000_000), views_range=(20, 200)) -> list[JobSpec]:
    """Seeded uneven jobs: N log-uniform in ``n_range``, V uniform in
    ``views_range`` (a contiguous range of the pool's views), D uniform over
    ``dims``; job j's scene has seed 100 + j."""
    rng = _rng(seed, 9)
    jobs = []
    for j in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        v = int(rng.integers(views_range[0], views_range[1] + 1))
        v0 = int(rng.integers(0, pool_views - v + 1))
        d = int(dims[int(rng.integers(0, len(dims)))])
        jobs.append(JobSpec(n, 100 + j, v, v0, d))
    return jobs


SERVING_SCENES = ((250_000, 40), (500_000, 41), (750_000, 42), (1_000_000, 43))   # (N, seed)
