"""CPU oracle for LUDVIG uplifting and graph diffusion (arXiv 2410.14462).

TEST INFRASTRUCTURE ONLY.  Nothing in the library's compute path imports,
links or runs this package; only ``tests/``, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline / reference leg use it.  It shares no code with
the CUDA library: the two meet only through the seeded input generators.

* ``ludvig_oracle.c`` (plain C, float64 values, float32 decision track):
  projection, tile lists, per-pixel compositing (Eq. 1), uplift sums
  (Eq. 3 / Eq. 5), rendering of per-Gaussian features (Eq. 4), exact kNN on
  Gaussian centres (Sec. 3.3).
* this module (numpy / scipy): the similarity graph (Eq. 7 and the edge
  weight of the diffusion workload), row normalisation, and the power
  iteration g_{t+1} = A g_t / ||g_t||_2 (Eq. 8), the selection of the
  most important Gaussians by beta (Sec. 3.2, Gaussian filtering), the
  paper-form diffusion pieces (appendix), relevancy scores, and the FP8-E4M3
  storage of features (OCP 8-bit format: encode, decode, per-view absmax
  quantiser).

Parity pins live in ``tests/test_oracle_*.py``.  "Parity unpinned": absolute
agreement with the paper's own rasteriser (no code or printed values exist)
and every task metric (no datasets).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ludvig_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_HYBRID = 32   # float32 decisions (the kernel's precision), float64 values
MODE_FP64 = 64     # every decision in float64


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (no contraction of a*b+c into fma)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            i64, i32, f32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_float
            p = ctypes.c_void_p
            L.orc_exp32.argtypes = [f32]
            L.orc_exp32.restype = f32
            L.orc_project.argtypes = [i64, p, p, p, p, p, i32, i32, p, p, p, p, i32]
            L.orc_project.restype = i32
            L.orc_tile_lists.argtypes = [i64, p, p, p, p, p, i32, i32, i32, p, i64, p, i32]
            L.orc_tile_lists.restype = i64
            L.orc_view_uplift.argtypes = [i64, p, p, p, p, p, i32, i32, p, i32, i32, p, p, p, p,
                                          i64, p, p, p, p, i32]
            L.orc_view_uplift.restype = i64
            L.orc_view_render.argtypes = [i64, p, p, p, p, p, i32, i32, p, i32, i32, p, p, i32]
            L.orc_view_render.restype = i64
            L.orc_normalise.argtypes = [i64, i32, p, p, p]
            L.orc_normalise.restype = None
            L.orc_knn.argtypes = [i64, p, i32, i64, p, p, p, i32]
            L.orc_knn.restype = i32
            _lib = L
    return _lib


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _scene_arrays(scene):
    return (_c(scene.means, np.float32), _c(scene.scales, np.float32),
            _c(scene.quats, np.float32), _c(scene.opacity, np.float32))


# ---------------------------------------------------------------------------
# rasteriser pieces
# ---------------------------------------------------------------------------

def exp32(x) -> np.ndarray:
    """The float32 exponential of the decision track, elementwise."""
    L = lib()
    x = np.asarray(x, dtype=np.float32)
    return np.array([L.orc_exp32(float(v)) for v in x.ravel()], dtype=np.float32).reshape(x.shape)


def project(scene, cam_params, width, height, nthreads=None):
    """Per-Gaussian projection of one view.

    Returns dict: ``p32`` [N,8] (mx,my,z,ca,cb,cc,opacity,radius),
    ``rect`` [N,4] (x0,y0,x1,y1 tiles, half-open), ``p64`` [N,8]
    (mx,my,z,ca,cb,cc,radius,visible), ``visible`` [N] (float32 track).
    """
    m, s, q, o = _scene_arrays(scene)
    n = m.shape[0]
    cam = _c(cam_params, np.float32)
    out32 = np.zeros((n, 8), np.float32)
    rect = np.zeros((n, 4), np.int32)
    out64 = np.zeros((n, 8), np.float64)
    vis = np.zeros(n, np.uint8)
    rc = lib().orc_project(n, _ptr(m), _ptr(s), _ptr(q), _ptr(o), _ptr(cam), width, height,
                           _ptr(out32), _ptr(rect), _ptr(out64), _ptr(vis),
                           nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"orc_project failed: {rc}")
    return {"p32": out32, "rect": rect, "p64": out64, "visible": vis.astype(bool)}


def tile_lists(scene, cam_params, width, height, mode=MODE_HYBRID, nthreads=None):
    """Depth-ordered candidate list of every 16x16 tile: (ranges [T,2], list)."""
    m, s, q, o = _scene_arrays(scene)
    n = m.shape[0]
    cam = _c(cam_params, np.float32)
    ntiles = ((width + 15) // 16) * ((height + 15) // 16)
    ranges = np.zeros((ntiles, 2), np.int64)
    L = lib()
    args = (n, _ptr(m), _ptr(s), _ptr(q), _ptr(o), _ptr(cam), width, height, mode, _ptr(ranges))
    total = L.orc_tile_lists(*args, 0, None, nthreads or default_threads())
    if total < 0:
        raise RuntimeError(f"orc_tile_lists failed: {total}")
    lst = np.zeros(max(total, 1), np.int32)
    L.orc_tile_lists(*args, total, _ptr(lst), nthreads or default_threads())
    return ranges, lst[:total]


def view_uplift(scene, cam_params, width, height, feats=None, num=None, den=None,
                mode=MODE_HYBRID, want=None, t_final=False, triplets=False, nthreads=None):
    """Adds one view's contribution to ``num`` [N,D] / ``den`` [N] (float64).

    ``feats``: [H,W,D] float32 (or None).  Returns a dict with the number of
    contributions and, on request, ``t_final`` [H,W] and the sparse weight
    triplets (pixel, gaussian, w64, w32).
    """
    m, s, q, o = _scene_arrays(scene)
    n = m.shape[0]
    cam = _c(cam_params, np.float32)
    d = 0
    fptr = None
    if feats is not None:
        feats = _c(feats, np.float32)
        d = feats.shape[-1]
        fptr = _ptr(feats)
    if num is not None:
        assert num.dtype == np.float64 and num.flags.c_contiguous and num.shape == (n, d)
    if den is not None:
        assert den.dtype == np.float64 and den.flags.c_contiguous and den.shape == (n,)
    wmask = None if want is None else _c(want, np.uint8)
    tf = np.zeros((height, width), np.float64) if t_final else None
    L = lib()
    nt = nthreads or default_threads()
    res = {}

    def call(cap, tp, tg, tw, tw32):
        return L.orc_view_uplift(n, _ptr(m), _ptr(s), _ptr(q), _ptr(o), _ptr(cam), width, height,
                                 fptr, d, mode, _ptr(wmask), _ptr(num), _ptr(den), _ptr(tf),
                                 cap, _ptr(tp), _ptr(tg), _ptr(tw), _ptr(tw32), nt)

    if triplets:
        # count the contributions first (no accumulation), then run for real
        total = L.orc_view_uplift(n, _ptr(m), _ptr(s), _ptr(q), _ptr(o), _ptr(cam), width,
                                  height, None, 0, mode, _ptr(wmask), None, None, None,
                                  0, None, None, None, None, nt)
        if total < 0:
            raise RuntimeError(f"orc_view_uplift failed: {total}")
        tp = np.zeros(max(total, 1), np.int32)
        tg = np.zeros(max(total, 1), np.int32)
        tw = np.zeros(max(total, 1), np.float64)
        tw32 = np.zeros(max(total, 1), np.float32)
        total2 = call(total, tp, tg, tw, tw32)
        assert total2 == total
        res.update(pix=tp[:total], gid=tg[:total], w64=tw[:total], w32=tw32[:total])
    else:
        total = call(0, None, None, None, None)
        if total < 0:
            raise RuntimeError(f"orc_view_uplift failed: {total}")
    res["count"] = int(total)
    if t_final:
        res["t_final"] = tf
    return res


def view_render(scene, cam_params, width, height, f, mode=MODE_HYBRID, tiles=None, nthreads=None):
    """Renders per-Gaussian features into one view (Eq. 4, F_hat = W f).

    ``f``: [N,D] features (any float type, taken as float64); ``tiles``:
    optional [ntiles] bool mask of the 16x16 tiles to render (the others stay
    zero).  Returns (F_hat [H,W,D] float64, number of contributions)."""
    m, s, q, o = _scene_arrays(scene)
    n = m.shape[0]
    f = np.asarray(f)
    f = _c(f.reshape(n, 1) if f.ndim == 1 else f, np.float64)
    if f.ndim != 2 or f.shape[0] != n:
        raise ValueError(f"features must be [{n}, d], got {f.shape}")
    d = f.shape[1]
    out = np.zeros((height, width, d), np.float64)
    ntiles = ((width + 15) // 16) * ((height + 15) // 16)
    tm = None if tiles is None else _c(np.asarray(tiles).reshape(ntiles).astype(np.uint8), np.uint8)
    rc = lib().orc_view_render(n, _ptr(m), _ptr(s), _ptr(q), _ptr(o), _ptr(_c(cam_params, np.float32)),
                               width, height, _ptr(f), d, mode, _ptr(tm), _ptr(out),
                               nthreads or default_threads())
    if rc < 0:
        raise RuntimeError(f"orc_view_render failed: {rc}")
    return out, int(rc)


def render(scene, cams, f, views=None, mode=MODE_HYBRID, nthreads=None):
    """F_hat = W f over ``views`` (default all): [V,H,W,D] float64 (Eq. 4)."""
    views = list(range(cams.v)) if views is None else list(views)
    return np.stack([view_render(scene, cams.params[v], cams.width, cams.height, f, mode=mode,
                                 nthreads=nthreads)[0] for v in views])


def beta_select(beta, keep: int) -> np.ndarray:
    """Gaussian filtering by importance (Sec. 3.2, "Gaussian filtering"): the
    indices of the ``keep`` Gaussians with the largest beta_i, ties to the lower
    index, returned in ascending index order.  beta values <= 0 (and NaN) rank
    as 0."""
    b = np.asarray(beta, dtype=np.float64).ravel()
    b = np.where(b > 0, b, 0.0)
    order = np.lexsort((np.arange(b.size), -b))   # by -beta, then index
    return np.sort(order[:keep]).astype(np.int32)


def normalise(num: np.ndarray, den: np.ndarray) -> np.ndarray:
    """f_i = num_i / beta_i, and 0 where beta_i = 0 (Eq. 3)."""
    out = np.zeros_like(num)
    pos = den > 0
    out[pos] = num[pos] / den[pos, None]
    return out


def uplift(scene, cams, features, views=None, mode=MODE_HYBRID, want=None, nthreads=None,
           count_normalise=False):
    """Uplift over ``views`` (default all): returns (f [N,D], beta [N]) in float64.

    ``features(v)`` returns the [H,W,D] float32 map of view v (numpy or torch).
    With ``count_normalise`` the normaliser is GaussianEditor's (appendix,
    comparison with GaussianEditor): the number of (view, pixel) pairs with
    w_i > 0, returned in place of beta.
    """
    views = range(cams.v) if views is None else views
    num = den = None
    cnt = np.zeros(scene.n, np.float64)
    for v in views:
        F = features(v)
        F = F.cpu().numpy() if hasattr(F, "cpu") else np.asarray(F)
        F = _c(F, np.float32)
        if num is None:
            num = np.zeros((scene.n, F.shape[-1]), np.float64)
            den = np.zeros(scene.n, np.float64)
        res = view_uplift(scene, cams.params[v], cams.width, cams.height, F, num, den, mode=mode,
                          want=want, nthreads=nthreads, triplets=count_normalise)
        if count_normalise:
            cnt += np.bincount(res["gid"], minlength=scene.n)
    if count_normalise:
        return normalise(num, cnt), cnt
    return normalise(num, den), den


# ---------------------------------------------------------------------------
# graph diffusion (Sec. 3.3)
# ---------------------------------------------------------------------------

def knn(means, k, queries=None, nthreads=None):
    """Exact k nearest neighbours (float32 squared distances, ties to the lower
    index, self excluded).  Returns (idx [m,k] int32, d2 [m,k] float32)."""
    m = _c(means, np.float32)
    n = m.shape[0]
    q = None if queries is None else _c(queries, np.int64)
    mq = n if q is None else q.shape[0]
    idx = np.zeros((mq, k), np.int32)
    d2 = np.zeros((mq, k), np.float32)
    rc = lib().orc_knn(n, _ptr(m), k, mq, _ptr(q), _ptr(idx), _ptr(d2), nthreads or default_threads())
    if rc != 0:
        raise RuntimeError("orc_knn failed")
    return idx, d2


def union_edges(nbr: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Undirected edge set {i,j}: j in N(i) or i in N(j), no self loops.
    Returns (rows, cols) of the symmetric pattern sorted by (row, col)."""
    n, k = nbr.shape
    r = np.repeat(np.arange(n, dtype=np.int64), k)
    c = nbr.reshape(-1).astype(np.int64)
    ok = (c >= 0) & (c != r)
    r, c = r[ok], c[ok]
    rows = np.concatenate([r, c])
    cols = np.concatenate([c, r])
    key = np.unique(rows * n + cols)
    return key // n, key % n


def edge_weights_spatial_cos(means, feats, rows, cols, h=0.01):
    """Diffusion-workload edge weight exp(-||x_i-x_j||^2/h) * max(0, cos(f_i,f_j))
    in float64 (a zero feature vector has cosine 0)."""
    x = np.asarray(means, np.float64)
    f = np.asarray(feats, np.float64)
    d2 = np.sum((x[rows] - x[cols]) ** 2, axis=1)
    nf = np.linalg.norm(f, axis=1)
    dot = np.sum(f[rows] * f[cols], axis=1)
    den = nf[rows] * nf[cols]
    cos = np.where(den > 0, dot / np.where(den > 0, den, 1.0), 0.0)
    return np.exp(-d2 / h) * np.maximum(0.0, cos)


def edge_weights_rbf_unary(feats, rows, cols, bandwidth, s_f, unary=None):
    """Eq. 7 with the RBF similarity of the appendix:
    A_ij = exp(-||f^_i - f^_j||^2 / (b s_f^2)) * sqrt(P_i) sqrt(P_j), with f^ the
    l2-normalised features and P the unary term (1 when omitted)."""
    f = np.asarray(feats, np.float64)
    nf = np.linalg.norm(f, axis=1, keepdims=True)
    fh = np.where(nf > 0, f / np.where(nf > 0, nf, 1.0), 0.0)
    d2 = np.sum((fh[rows] - fh[cols]) ** 2, axis=1)
    w = np.exp(-d2 / (bandwidth * s_f * s_f))
    if unary is not None:
        p = np.sqrt(np.asarray(unary, np.float64))
        w = w * p[rows] * p[cols]
    return w


def _unit_rows(f):
    f = np.asarray(f, np.float64)
    nf = np.linalg.norm(f, axis=1, keepdims=True)
    return np.where(nf > 0, f / np.where(nf > 0, nf, 1.0), 0.0)


def feature_scale(feats, rows, cols):
    """s_f of the RBF similarity (appendix, diffusion): the median of the l2
    distances between l2-normalised features, taken over the graph's edges
    (all n^2 pairs are out of reach at scale); numpy's median (the mean of
    the two middle values for an even count)."""
    fh = _unit_rows(feats)
    d = np.sqrt(np.sum((fh[rows] - fh[cols]) ** 2, axis=1))
    return float(np.median(d)) if d.size else 0.0


def unary_anchor(feats, g0, bandwidth, s_f):
    """Unary term of Eq. 7 when scribbles are given (appendix, diffusion):
    P_i = S_f(f_i, f_bar) = exp(-||f^_i - f_bar||^2 / (b s_f^2)), with f_bar the
    l2-normalised mean of the normalised features of the anchor nodes
    {i : g0_i > 0} (zero when there are none)."""
    fh = _unit_rows(feats)
    anchors = np.asarray(g0, np.float64).reshape(len(fh), -1)[:, 0] > 0
    fbar = fh[anchors].sum(axis=0) if anchors.any() else np.zeros(fh.shape[1])
    fbar = _unit_rows(fbar[None, :])[0]
    d2 = np.sum((fh - fbar[None, :]) ** 2, axis=1)
    return np.exp(-d2 / (bandwidth * s_f * s_f))


def topfrac_positive(u, percent: int):
    """g_0 of the segmentation task (appendix, diffusion): the uplifted mask u
    keeps its values on the top `percent` % of the Gaussians with u_i > 0
    (ceil(npos * percent / 100) of them, larger u first, ties to the lower
    index) and is zero elsewhere."""
    u = np.asarray(u, np.float64).ravel()
    pos = u > 0
    keep = (int(pos.sum()) * int(percent) + 99) // 100
    key = np.where(pos, u, 0.0)
    order = np.lexsort((np.arange(u.size), -key))[:keep]
    g0 = np.zeros_like(u)
    g0[order] = u[order]
    return g0


def reach_weight(A, g0, T, unary=None):
    """Segmentation weight after T diffusion steps (Sec. 4.1 and appendix):
    S = {i : g_T,i > 0} for the non-negative A and g_0 >= 0, which in exact
    arithmetic is the set reached from supp(g_0) by walks of exactly T edges
    of A (taken here as that boolean walk, immune to underflow); h_i = P_i on
    S (1 without a unary term) and 0 elsewhere.  Columns of g0 are separate
    queries."""
    g = np.asarray(g0, np.float64)
    squeeze = g.ndim == 1
    s = (g[:, None] if squeeze else g) > 0
    pat = A.copy().tocsr()
    pat.data = (pat.data > 0).astype(np.float64)
    for _ in range(T):
        s = (pat @ s.astype(np.float64)) > 0
    p = np.ones(s.shape[0]) if unary is None else np.asarray(unary, np.float64)
    h = np.where(s, p[:, None], 0.0)
    return h[:, 0] if squeeze else h


def relevancy(feats, phi_queries, phi_canon, temperature=10.0):
    """Relevancy of uplifted CLIP features to text queries (appendix, relevancy
    scores): r_iq = min_k exp(T s_iq) / (exp(T s_iq) + exp(T s_ik)), with s the
    dot products of the l2-normalised feature f^_i with the l2-normalised query
    and canonical-phrase embeddings.  Returns [n, q] float64."""
    fh = _unit_rows(feats)
    pq = _unit_rows(phi_queries)
    pc = _unit_rows(phi_canon)
    sq = fh @ pq.T                                  # [n, q]
    sc = fh @ pc.T                                  # [n, k]
    eq = np.exp(temperature * sq)[:, :, None]
    ec = np.exp(temperature * sc)[:, None, :]
    return np.min(eq / (eq + ec), axis=2)


def csr(n, rows, cols, vals, row_normalize=True, binarize=0.0):
    """scipy CSR matrix of the graph.  With ``binarize`` > 0 every weight above
    the threshold becomes 1 and the rest 0 (the segmentation variant of Sec. 4.1
    thresholds A at 1e-5); with ``row_normalize`` each row is then divided by
    its sum (rows summing to 0 stay 0)."""
    import scipy.sparse as sp
    vals = np.asarray(vals, np.float64)
    if binarize > 0:
        vals = (vals > binarize).astype(np.float64)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A.sum_duplicates()
    if row_normalize:
        s = np.asarray(A.sum(axis=1)).ravel()
        inv = np.where(s > 0, 1.0 / np.where(s > 0, s, 1.0), 0.0)
        A = sp.diags(inv) @ A
        A = A.tocsr()
    return A


def diffuse(A, x0, iters):
    """Power iteration of Eq. 8 on each column: g_{t+1} = A (g_t / ||g_t||_2).
    A column whose norm reaches 0 stays 0.  Returns g_iters (float64)."""
    g = np.array(x0, dtype=np.float64, copy=True)
    squeeze = g.ndim == 1
    if squeeze:
        g = g[:, None]
    for _ in range(iters):
        nrm = np.linalg.norm(g, axis=0)
        scale = np.where(nrm > 0, 1.0 / np.where(nrm > 0, nrm, 1.0), 0.0)
        g = A @ (g * scale[None, :])
    return g[:, 0] if squeeze else g


# --------------------------------------------------------------------------
# FP8-E4M3 storage of features (the precision form's 8-bit variant; the
# format is the OCP 8-bit floating point one, not the paper's): 1 sign bit,
# 4 exponent bits with bias 7, 3 mantissa bits, no infinities, code 0x7F
# (and 0xFF) NaN.  Normal codes hold 2^(E-7) (1 + M/8), E = 1..15; E = 0
# holds the subnormals M 2^-9.  The largest finite value is 448 (0x7E).
# --------------------------------------------------------------------------

E4M3_MAX = 448.0


def e4m3_encode(x) -> np.ndarray:
    """Codes (uint8) of the values x rounded to E4M3: round to nearest, ties
    to the even code, magnitudes above 448 saturated to 448, NaN to 0x7F.
    Every step is exact in float64 (scaling by powers of two)."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    code = np.zeros(x.shape, dtype=np.int64)
    fin = np.isfinite(a) & (a > 0)
    # exponent of the leading bit: a = m 2^k with m in [0.5, 1) -> e = k - 1
    _, k = np.frexp(np.where(fin, a, 1.0))
    e = np.maximum(k - 1, -6)                  # below 2^-6 the quantum stays 2^-9
    q = np.rint(np.where(fin, a, 0.0) / np.ldexp(1.0, e - 3))   # units of the quantum; rint ties to even
    # normal range: code = (e + 7) * 8 + (q - 8); subnormal (e = -6, q < 8):
    # code = q; both forms agree at q = 8 and carry q = 16 into the next exponent
    c = np.where(q < 8, q, (e + 7) * 8 + (q - 8)).astype(np.int64)
    code = np.where(fin, np.minimum(c, 0x7E), code)
    code = np.where(np.isinf(a) | (fin & (a > E4M3_MAX)), 0x7E, code)
    code = np.where(np.isnan(x), 0x7F, code)
    code = code | np.where(np.signbit(x) & ~np.isnan(x), 0x80, 0)
    return code.astype(np.uint8)


def e4m3_decode(code) -> np.ndarray:
    """float64 values of E4M3 codes (NaN for 0x7F / 0xFF)."""
    c = np.asarray(code, dtype=np.int64)
    E, M = (c >> 3) & 15, c & 7
    mag = np.where(E == 0, M * 2.0 ** -9, np.ldexp(1.0 + M / 8.0, E - 7))
    mag = np.where((c & 0x7F) == 0x7F, np.nan, mag)
    return np.where(c & 0x80, -mag, mag)


def fp8_quantize(views) -> tuple[np.ndarray, np.ndarray]:
    """Per-view absmax scaling then E4M3 rounding, for float32 views [V, ...]:
    s_v = max|x| / 448 in float32 (1 when the view is all zero), codes of
    float32(x / s_v).  Returns (codes uint8 [V, ...], s float32 [V])."""
    xs = np.asarray(views, dtype=np.float32)
    V = xs.shape[0]
    s = np.ones(V, dtype=np.float32)
    q = np.zeros(xs.shape, dtype=np.uint8)
    for v in range(V):
        amax = np.float32(np.max(np.abs(xs[v]))) if xs[v].size else np.float32(0)
        if amax > 0:
            s[v] = amax / np.float32(E4M3_MAX)
        q[v] = e4m3_encode(xs[v] / s[v])
    return q, s


def fp8_dequantize(q, s) -> np.ndarray:
    """x = decode(q) s_v in float64 (the values an FP8 uplift averages)."""
    q = np.asarray(q)
    s = np.asarray(s, dtype=np.float64).reshape((-1,) + (1,) * (q.ndim - 1))
    return e4m3_decode(q) * s
