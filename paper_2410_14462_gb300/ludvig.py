"""Thin ctypes binding of libludvig (include/ludvig.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Torch tensors are passed by data pointer together with the current
CUDA stream.  There is no fallback: if ``libludvig.so`` is missing or fails to
load, or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libludvig.so")

F32 = 0
BF16 = 1
ERR_ARG = 1
MAX_BATCH_SLOTS = 32          # LUDVIG_MAX_BATCH_SLOTS

STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_TIMEOUT", 5: "ERR_INTERNAL",
          6: "ERR_UNSUPPORTED"}

# function name -> (restype, argtypes); mirrors include/ludvig.h
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_F = ctypes.c_float
SIGNATURES = {
    "ludvig_abi_version": (_I32, []),
    "ludvig_last_error": (ctypes.c_char_p, []),
    "ludvig_scene_create": (_I32, [_P, _P, _P, _P, _I64, _P, _P, ctypes.POINTER(_P)]),
    "ludvig_sync": (_I32, [_P]),
    "ludvig_scene_destroy": (_I32, [_P]),
    "ludvig_scene_size": (_I64, [_P]),
    "ludvig_scene_workspace_bytes": (_I64, [_P]),
    "ludvig_uplift_accumulate": (_I32, [_P, _P, _I32, _I32, _I32, _P, _I32, _I32, _P, _P, _P]),
    "ludvig_uplift_finalize": (_I32, [_I64, _I32, _P, _P, _P, _P, _P]),
    "ludvig_uplift": (_I32, [_P, _P, _I32, _I32, _I32, _P, _I32, _I32, _P, _P, _P]),
    "ludvig_uplift_batch": (_I32, [_P, _I32, _I32, _P, _P]),
    "ludvig_batch_release_workspaces": (_I32, []),
    "ludvig_batch_last_plan": (_I32, [_P, _I32]),
    "ludvig_batch_forget_tuning": (_I32, []),
    "ludvig_fp8_quantize": (_I32, [_P, _I32, _I32, _I64, _P, _P, _P]),
    "ludvig_uplift_fp8": (_I32, [_P, _P, _I32, _I32, _I32, _P, _P, _I32, _P, _P, _P]),
    "ludvig_uplift_host": (_I32, [_P, _P, _I32, _I32, _I32, _P, _I32, _I32, _P, _P, _P]),
    "ludvig_render": (_I32, [_P, _P, _I32, _I32, _I32, _P, _I32, _P, _P]),
    "ludvig_beta_select": (_I32, [_P, _P, _I64, _P, _P]),
    "ludvig_relevancy": (_I32, [_P, _I64, _I32, _P, _I32, _I32, _F, _P, _P]),
    "ludvig_graph_build_rbf": (_I32, [_P, _I32, _P, _I32, _P, ctypes.POINTER(_P)]),
    "ludvig_graph_feature_scale": (_I32, [_P, ctypes.POINTER(_F)]),
    "ludvig_graph_reweight": (_I32, [_P, _F, _P, _F, _I32, _P]),
    "ludvig_unary_anchor": (_I32, [_P, _P, _I32, _P, _F, _P, _P]),
    "ludvig_topfrac_positive": (_I32, [_P, _P, _I32, _P, _P]),
    "ludvig_reach_weight": (_I32, [_P, _P, _I32, _I32, _P, _P, _P]),
    "ludvig_scene_subset": (_I32, [_P, _P, _I64, _P, ctypes.POINTER(_P)]),
    "ludvig_set_option": (_I32, [_I32, _I64]),
    "ludvig_get_option": (_I64, [_I32]),
    "ludvig_trace_enable": (_I32, [_I32]),
    "ludvig_trace_read": (_I32, [_P, _I32]),
    "ludvig_debug_project": (_I32, [_P, _P, _I32, _I32, _P, _P, _P]),
    "ludvig_debug_tile_lists": (_I32, [_P, _P, _I32, _I32, _I32, _P, _P, _I64, ctypes.POINTER(_I64), _P]),
    "ludvig_debug_transmittance": (_I32, [_P, _P, _I32, _I32, _P, _P, _P]),
    "ludvig_debug_mma_bf16": (_I32, [_P, _P, _I32, _P, _P]),
    "ludvig_debug_wait_timeout": (_I32, [_I64, ctypes.POINTER(_I64), _P]),
    "ludvig_debug_scene_timeout": (_I32, [_P, _I64, _P]),
    "ludvig_knn": (_I32, [_P, _I32, _P, _P]),
    "ludvig_graph_build": (_I32, [_P, _I32, _P, _I32, _F, _F, _I32, _P, ctypes.POINTER(_P)]),
    "ludvig_graph_destroy": (_I32, [_P]),
    "ludvig_graph_nnz": (_I64, [_P]),
    "ludvig_graph_workspace_bytes": (_I64, [_P]),
    "ludvig_graph_export": (_I32, [_P, _P, _P, _P, _P]),
    "ludvig_diffuse": (_I32, [_P, _P, _I32, _I32, _P, _P]),
    "ludvig_diffuse_noalloc": (_I32, [_P, _P, _I32, _I32, _P, _P]),
}

_lib = None
_lock = threading.Lock()


class LudvigError(RuntimeError):
    pass


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libludvig.so (raises if it is missing: no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise LudvigError(f"{path} not found: build it with "
                                  "`python -m paper_2410_14462_gb300.build`")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        msg = load().ludvig_last_error().decode(errors="replace")
        raise LudvigError(f"{what}: {STATUS.get(rc, rc)}: {msg}")


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t: torch.Tensor, dtype=None, name="tensor"):
    if not t.is_cuda:
        raise LudvigError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise LudvigError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise LudvigError(f"{name} must be {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


class CameraArray(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


def cameras_struct(params: np.ndarray):
    """[V,16] float32 (R, t, fx, fy, cx, cy) -> ludvig_camera[V] (host memory)."""
    p = np.ascontiguousarray(params, dtype=np.float32).reshape(-1, 16)
    arr = (CameraArray * max(1, p.shape[0]))()
    ctypes.memmove(arr, p.ctypes.data, p.nbytes)
    return arr, p.shape[0]


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.bfloat16:
        return BF16
    raise LudvigError(f"features must be float32 or bfloat16, got {t.dtype}")


class SceneOpts(ctypes.Structure):
    """ludvig_scene_opts."""
    _fields_ = [("scales_are_linear", ctypes.c_int32)]


class Scene:
    """A device-resident Gaussian scene (ludvig_scene_create).  scales are
    linear standard deviations unless log_scales is set."""

    def __init__(self, means, scales, quats, opacity, stream=None, log_scales=False):
        L = load()
        dev = torch.device("cuda")
        t = [torch.as_tensor(a, dtype=torch.float32).to(dev).contiguous()
             for a in (means, scales, quats, opacity)]
        self.n = int(t[0].shape[0])
        h = ctypes.c_void_p()
        opts = SceneOpts(0 if log_scales else 1)
        _check(L.ludvig_scene_create(_dev(t[0]), _dev(t[1]), _dev(t[2]), _dev(t[3]), self.n,
                                     ctypes.byref(opts), _stream(stream), ctypes.byref(h)),
               "ludvig_scene_create")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        self._h = h

    @classmethod
    def from_inputs(cls, scene, stream=None):
        return cls(scene.means, scene.scales, scene.quats, scene.opacity, stream)

    @classmethod
    def _wrap(cls, handle, n):
        obj = cls.__new__(cls)
        obj._h = handle
        obj.n = int(n)
        return obj

    def subset(self, idx: torch.Tensor, stream=None) -> "Scene":
        """A new scene of Gaussians idx (int32 CUDA tensor), ludvig_scene_subset."""
        h = ctypes.c_void_p()
        _check(load().ludvig_scene_subset(self._h, _dev(idx, torch.int32, "idx"), int(idx.numel()),
                                          _stream(stream), ctypes.byref(h)), "ludvig_scene_subset")
        return Scene._wrap(h, idx.numel())

    @property
    def handle(self):
        return self._h

    def sync(self):
        """ludvig_sync: wait for and complete the scene's last asynchronous uplift."""
        _check(load().ludvig_sync(self._h), "ludvig_sync")

    def workspace_bytes(self) -> int:
        """ludvig_scene_workspace_bytes: device bytes of the scene's workspace."""
        return int(load().ludvig_scene_workspace_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ludvig_scene_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def uplift(scene: Scene, cams_params, width, height, feats: torch.Tensor, out=None, beta=None,
           stream=None, sync=True):
    """f = D^-1 W^T F on the device.  feats: [V,H,W,D] float32/bfloat16 CUDA tensor.
    With sync (the default) the call ends with ludvig_sync, so out/beta are
    final on return; otherwise call scene.sync() before using them."""
    L = load()
    cams, nv = cameras_struct(cams_params)
    d = int(feats.shape[-1])
    if out is None:
        out = torch.empty((scene.n, d), dtype=torch.float32, device=feats.device)
    if beta is None:
        beta = torch.empty((scene.n,), dtype=torch.float32, device=feats.device)
    _check(L.ludvig_uplift(scene.handle, cams, nv, width, height, _dev(feats, name="feats"),
                           _dtype_code(feats), d, _dev(out, torch.float32, "out"),
                           _dev(beta, torch.float32, "beta"), _stream(stream)), "ludvig_uplift")
    if sync:
        scene.sync()
    return out, beta


class UpliftJob(ctypes.Structure):
    """ludvig_uplift_job: the arguments of one ludvig_uplift call."""
    _fields_ = [("scene", ctypes.c_void_p), ("cams", ctypes.c_void_p), ("n_views", ctypes.c_int32),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("feats", ctypes.c_void_p),
                ("dtype", ctypes.c_int32), ("d", ctypes.c_int32), ("out", ctypes.c_void_p),
                ("beta", ctypes.c_void_p)]


def uplift_batch(jobs, slots: int = 6, stream=None, raise_on_error: bool = True):
    """ludvig_uplift_batch over jobs given as (scene, cams_params, width, height,
    feats[V,H,W,D], out or None, beta or None); outputs left as None are
    allocated here.  Returns [(out, beta)] in job order and the per-job
    status codes."""
    L = load()
    arr = (UpliftJob * max(1, len(jobs)))()
    keep, results = [], []
    for k, (scene, cams_params, width, height, feats, out, beta) in enumerate(jobs):
        cams, nv = cameras_struct(cams_params)
        d = int(feats.shape[-1])
        if out is None:
            out = torch.empty((scene.n, d), dtype=torch.float32, device=feats.device)
        if beta is None:
            beta = torch.empty((scene.n,), dtype=torch.float32, device=feats.device)
        keep.append(cams)
        results.append((out, beta))
        arr[k] = UpliftJob(scene.handle.value, ctypes.addressof(cams), nv, width, height,
                           _dev(feats, name="feats").value, _dtype_code(feats), d,
                           _dev(out, torch.float32, "out").value, _dev(beta, torch.float32, "beta").value)
    status = (ctypes.c_int32 * max(1, len(jobs)))()
    rc = L.ludvig_uplift_batch(arr, len(jobs), int(slots), status, _stream(stream))
    if raise_on_error:
        _check(rc, "ludvig_uplift_batch")
    return results, [int(status[k]) for k in range(len(jobs))]


def fp8_quantize(feats: torch.Tensor, q=None, scales=None, stream=None):
    """ludvig_fp8_quantize: per-view absmax scale and E4M3 codes of feats
    [V, ...] (float32 or bfloat16 CUDA tensor).  Returns (q uint8 of the same
    shape, scales [V] float32)."""
    V = int(feats.shape[0])
    ve = int(feats[0].numel()) if V else 0
    if q is None:
        q = torch.empty(feats.shape, dtype=torch.uint8, device=feats.device)
    if scales is None:
        scales = torch.empty((V,), dtype=torch.float32, device=feats.device)
    _check(load().ludvig_fp8_quantize(_dev(feats, name="feats"), _dtype_code(feats), V, ve,
                                      _dev(q, torch.uint8, "q"), _dev(scales, torch.float32, "scales"),
                                      _stream(stream)), "ludvig_fp8_quantize")
    return q, scales


def uplift_fp8(scene: Scene, cams_params, width, height, q: torch.Tensor, scales: torch.Tensor, out=None,
               beta=None, stream=None, sync=True):
    """ludvig_uplift_fp8: uplift of E4M3 features q [V,H,W,D] (uint8) with
    per-view scales [V]."""
    cams, nv = cameras_struct(cams_params)
    d = int(q.shape[-1])
    if out is None:
        out = torch.empty((scene.n, d), dtype=torch.float32, device=q.device)
    if beta is None:
        beta = torch.empty((scene.n,), dtype=torch.float32, device=q.device)
    _check(load().ludvig_uplift_fp8(scene.handle, cams, nv, width, height, _dev(q, torch.uint8, "q"),
                                    _dev(scales, torch.float32, "scales"), d, _dev(out, torch.float32, "out"),
                                    _dev(beta, torch.float32, "beta"), _stream(stream)), "ludvig_uplift_fp8")
    if sync:
        scene.sync()
    return out, beta


def batch_release_workspaces():
    """ludvig_batch_release_workspaces: free the batch executor's idle pooled
    workspaces and contexts."""
    _check(load().ludvig_batch_release_workspaces(), "ludvig_batch_release_workspaces")


class BatchClass(ctypes.Structure):
    """ludvig_batch_class: one class of the last batch."""
    _fields_ = [(name, ctypes.c_int32) for name in
                ("dtype", "d", "width", "height", "jobs", "views", "groups", "group_mb", "tuned", "redone",
                 "workspace_mb")] + [("ms", ctypes.c_float)]


def batch_last_plan() -> list[dict]:
    """ludvig_batch_last_plan: the classes of the last ludvig_uplift_batch
    call (the last entry, groups = -1, counts the jobs run as single calls)."""
    L = load()
    n = int(L.ludvig_batch_last_plan(None, 0))
    arr = (BatchClass * max(1, n))()
    n = int(L.ludvig_batch_last_plan(arr, n))
    return [{f: (float if f == "ms" else int)(getattr(arr[k], f)) for f, _ in BatchClass._fields_}
            for k in range(n)]


def batch_forget_tuning():
    """ludvig_batch_forget_tuning: the next batch times its classes again."""
    _check(load().ludvig_batch_forget_tuning(), "ludvig_batch_forget_tuning")


def uplift_accumulate(scene: Scene, cams_params, width, height, feats, num, den, stream=None, sync=True):
    L = load()
    cams, nv = cameras_struct(cams_params)
    _check(L.ludvig_uplift_accumulate(scene.handle, cams, nv, width, height, _dev(feats, name="feats"),
                                      _dtype_code(feats), int(feats.shape[-1]),
                                      _dev(num, torch.float32, "num"), _dev(den, torch.float32, "den"),
                                      _stream(stream)), "ludvig_uplift_accumulate")
    if sync:
        scene.sync()


def uplift_finalize(num, den, out=None, beta=None, stream=None):
    L = load()
    n, d = num.shape
    out = num if out is None else out
    _check(L.ludvig_uplift_finalize(n, d, _dev(num), _dev(den), _dev(out),
                                    None if beta is None else _dev(beta), _stream(stream)),
           "ludvig_uplift_finalize")
    return out


def uplift_host(scene: Scene, cams_params, width, height, feats: torch.Tensor, out=None, beta=None, stream=None):
    """The same uplift from host (CPU, ideally pinned) features into host
    outputs: out [N, D] and beta [N] float32 CPU tensors (pinned ones are
    copied at the full link rate), allocated pinned here when not given;
    returns (out, beta)."""
    L = load()
    if feats.is_cuda or not feats.is_contiguous():
        raise LudvigError("feats must be a contiguous CPU tensor")
    cams, nv = cameras_struct(cams_params)
    d = int(feats.shape[-1])
    if out is None:
        out = torch.empty((scene.n, d), dtype=torch.float32, pin_memory=True)
    if beta is None:
        beta = torch.empty((scene.n,), dtype=torch.float32, pin_memory=True)
    for t, shape, name in ((out, (scene.n, d), "out"), (beta, (scene.n,), "beta")):
        if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or tuple(t.shape) != shape:
            raise LudvigError(f"{name} must be a contiguous float32 CPU tensor of shape {shape}")
    _check(L.ludvig_uplift_host(scene.handle, cams, nv, width, height, ctypes.c_void_p(feats.data_ptr()),
                                _dtype_code(feats), d, ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(beta.data_ptr()), _stream(stream)), "ludvig_uplift_host")
    return out, beta


def render(scene: Scene, cams_params, width, height, f: torch.Tensor, out=None, stream=None):
    """F_hat = W f (Eq. 4) on the device.  f: [N,D] float32 CUDA tensor; returns
    (or fills) out [V,H,W,D] float32."""
    L = load()
    cams, nv = cameras_struct(cams_params)
    if f.dim() != 2 or f.shape[0] != scene.n:
        raise LudvigError(f"f must be [{scene.n}, d], got {tuple(f.shape)}")
    d = int(f.shape[1])
    if out is None:
        out = torch.empty((nv, height, width, d), dtype=torch.float32, device=f.device)
    _check(L.ludvig_render(scene.handle, cams, nv, width, height, _dev(f, torch.float32, "f"), d,
                           _dev(out, torch.float32, "out"), _stream(stream)), "ludvig_render")
    return out


def beta_select(scene: Scene, beta: torch.Tensor, keep: int, stream=None) -> torch.Tensor:
    """Indices (ascending, int32) of the `keep` Gaussians with the largest beta
    (ties to the lower index): Gaussian filtering, Sec. 3.2."""
    kept = torch.empty((int(keep),), dtype=torch.int32, device=beta.device)
    _check(load().ludvig_beta_select(scene.handle, _dev(beta, torch.float32, "beta"), int(keep),
                                     _dev(kept, torch.int32, "kept"), _stream(stream)), "ludvig_beta_select")
    return kept


def topfrac_positive(scene: Scene, u: torch.Tensor, percent: int = 10, stream=None) -> torch.Tensor:
    """g_0 = u on the top `percent` % of the positive entries (ludvig_topfrac_positive)."""
    g0 = torch.empty_like(u)
    _check(load().ludvig_topfrac_positive(scene.handle, _dev(u, torch.float32, "u"), int(percent),
                                          _dev(g0, torch.float32, "g0"), _stream(stream)), "ludvig_topfrac_positive")
    return g0


def relevancy(feats: torch.Tensor, phi_queries: torch.Tensor, phi_canon: torch.Tensor, temperature: float = 10.0,
              out=None, stream=None) -> torch.Tensor:
    """LERF relevancy r [n, q] of features [n, d] to query embeddings [q, d]
    against canonical-phrase embeddings [k, d] (ludvig_relevancy)."""
    n, d = feats.shape
    phi = torch.cat([phi_queries, phi_canon]).to(torch.float32).contiguous()
    nq = int(phi_queries.shape[0])
    if out is None:
        out = torch.empty((n, nq), dtype=torch.float32, device=feats.device)
    _check(load().ludvig_relevancy(_dev(feats, torch.float32, "feats"), int(n), int(d), _dev(phi), nq,
                                   int(phi_canon.shape[0]), float(temperature), _dev(out, torch.float32, "r"),
                                   _stream(stream)), "ludvig_relevancy")
    return out


OPT_F32_TENSOR_CORES = 0
OPT_COUNT_NORMALISE = 1
OPT_FAULT_ALLOC = 2
OPT_FAULT_LAUNCH = 3
OPT_AGG_CONFIG = 4
OPT_GROUP_MB = 5
OPT_BATCH_TUNE = 6
OPT_BATCH_PACK = 7
OPT_AGG_SMS = 8


def set_option(option: int, value: int):
    _check(load().ludvig_set_option(option, int(value)), "ludvig_set_option")


def get_option(option: int) -> int:
    return int(load().ludvig_get_option(option))


STAGES = ["project", "depth_sort", "bin", "tile_sort", "composite", "normalise", "knn", "graph", "diffuse",
          "weights", "aggregate", "render", "render_product", "filter", "relevancy"]


class TraceStruct(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 16), ("calls", ctypes.c_int64 * 16),
                ("kernel_launches", ctypes.c_int64)]


def trace_enable(on: bool = True):
    _check(load().ludvig_trace_enable(int(on)), "ludvig_trace_enable")


def trace_read(reset: bool = True) -> dict:
    """Per-stage device milliseconds, interval counts and the kernel launch count."""
    t = TraceStruct()
    _check(load().ludvig_trace_read(ctypes.byref(t), int(reset)), "ludvig_trace_read")
    return {"ms": {s: t.ms[i] for i, s in enumerate(STAGES)},
            "calls": {s: t.calls[i] for i, s in enumerate(STAGES)},
            "kernel_launches": int(t.kernel_launches)}


def debug_project(scene: Scene, cam_params, width, height, stream=None):
    L = load()
    cams, _ = cameras_struct(cam_params)
    rec = torch.zeros((scene.n, 8), dtype=torch.float32, device="cuda")
    rect = torch.zeros((scene.n, 4), dtype=torch.int32, device="cuda")
    _check(L.ludvig_debug_project(scene.handle, cams, width, height, _dev(rec), _dev(rect), _stream(stream)),
           "ludvig_debug_project")
    return rec, rect


def debug_tile_lists(scene: Scene, cam_params, width, height, pruned=False, stream=None):
    L = load()
    cams, _ = cameras_struct(cam_params)
    ntiles = ((width + 15) // 16) * ((height + 15) // 16)
    ranges = torch.zeros((ntiles, 2), dtype=torch.int64, device="cuda")
    total = ctypes.c_int64(0)
    _check(L.ludvig_debug_tile_lists(scene.handle, cams, width, height, int(pruned), _dev(ranges), None, 0,
                                     ctypes.byref(total), _stream(stream)), "ludvig_debug_tile_lists")
    lst = torch.zeros((max(1, total.value),), dtype=torch.int32, device="cuda")
    _check(L.ludvig_debug_tile_lists(scene.handle, cams, width, height, int(pruned), _dev(ranges), _dev(lst),
                                     lst.numel(), ctypes.byref(total), _stream(stream)), "ludvig_debug_tile_lists")
    return ranges, lst[: total.value]


def debug_transmittance(scene: Scene, cam_params, width, height, stream=None):
    L = load()
    cams, _ = cameras_struct(cam_params)
    t = torch.empty((height, width), dtype=torch.float32, device="cuda")
    c = torch.empty((height, width), dtype=torch.int32, device="cuda")
    _check(L.ludvig_debug_transmittance(scene.handle, cams, width, height, _dev(t), _dev(c), _stream(stream)),
           "ludvig_debug_transmittance")
    return t, c


def debug_mma_bf16(a: torch.Tensor, f: torch.Tensor, stream=None):
    """out[128,d] = a[128,256] @ f[256,d] through the uplift's tensor-core path."""
    L = load()
    d = int(f.shape[-1])
    out = torch.zeros((128, d), dtype=torch.float32, device="cuda")
    _check(L.ludvig_debug_mma_bf16(_dev(a, torch.bfloat16, "a"), _dev(f, torch.bfloat16, "f"), d, _dev(out),
                                   _stream(stream)), "ludvig_debug_mma_bf16")
    return out


def knn(scene: Scene, k: int, stream=None):
    L = load()
    nbr = torch.empty((scene.n, k), dtype=torch.int32, device="cuda")
    _check(L.ludvig_knn(scene.handle, k, _dev(nbr), _stream(stream)), "ludvig_knn")
    return nbr


class Graph:
    """Diffusion graph on the device (ludvig_graph_build)."""

    def __init__(self, scene: Scene, k: int, feats: torch.Tensor, spatial_h: float = 0.01,
                 binarize: float = 0.0, row_normalize: bool = True, stream=None):
        L = load()
        h = ctypes.c_void_p()
        _check(L.ludvig_graph_build(scene.handle, k, _dev(feats, torch.float32, "feats"), int(feats.shape[1]),
                                    spatial_h, binarize, int(row_normalize), _stream(stream), ctypes.byref(h)),
               "ludvig_graph_build")
        self._h = h
        self.n = scene.n

    @classmethod
    def rbf(cls, scene: Scene, k: int, feats: torch.Tensor, stream=None) -> "Graph":
        """ludvig_graph_build_rbf: the union kNN graph with each edge's squared
        normalised-feature distance and the median edge distance s_f."""
        L = load()
        h = ctypes.c_void_p()
        _check(L.ludvig_graph_build_rbf(scene.handle, k, _dev(feats, torch.float32, "feats"), int(feats.shape[1]),
                                        _stream(stream), ctypes.byref(h)), "ludvig_graph_build_rbf")
        obj = cls.__new__(cls)
        obj._h = h
        obj.n = scene.n
        return obj

    @property
    def feature_scale(self) -> float:
        v = ctypes.c_float()
        _check(load().ludvig_graph_feature_scale(self._h, ctypes.byref(v)), "ludvig_graph_feature_scale")
        return float(v.value)

    def reweight(self, bandwidth: float, unary=None, binarize: float = 0.0, row_normalize: bool = False,
                 stream=None):
        _check(load().ludvig_graph_reweight(self._h, float(bandwidth),
                                            None if unary is None else _dev(unary, torch.float32, "unary"),
                                            float(binarize), int(row_normalize), _stream(stream)),
               "ludvig_graph_reweight")

    def unary_anchor(self, feats: torch.Tensor, g0: torch.Tensor, bandwidth: float, out=None, stream=None):
        if out is None:
            out = torch.empty((self.n,), dtype=torch.float32, device=feats.device)
        _check(load().ludvig_unary_anchor(self._h, _dev(feats, torch.float32, "feats"), int(feats.shape[1]),
                                          _dev(g0, torch.float32, "g0"), float(bandwidth),
                                          _dev(out, torch.float32, "unary"), _stream(stream)), "ludvig_unary_anchor")
        return out

    def reach_weight(self, g0: torch.Tensor, steps: int, unary=None, out=None, stream=None):
        g0 = g0.contiguous()
        dx = 1 if g0.dim() == 1 else int(g0.shape[1])
        if out is None:
            out = torch.empty_like(g0)
        _check(load().ludvig_reach_weight(self._h, _dev(g0, torch.float32, "g0"), dx, int(steps),
                                          None if unary is None else _dev(unary, torch.float32, "unary"),
                                          _dev(out, torch.float32, "h"), _stream(stream)), "ludvig_reach_weight")
        return out

    @property
    def nnz(self) -> int:
        return int(load().ludvig_graph_nnz(self._h))

    def workspace_bytes(self) -> int:
        """ludvig_graph_workspace_bytes: device bytes of the graph's workspace."""
        return int(load().ludvig_graph_workspace_bytes(self._h))

    def export(self, stream=None):
        L = load()
        rp = torch.empty((self.n + 1,), dtype=torch.int64, device="cuda")
        col = torch.empty((max(1, self.nnz),), dtype=torch.int32, device="cuda")
        val = torch.empty((max(1, self.nnz),), dtype=torch.float32, device="cuda")
        _check(L.ludvig_graph_export(self._h, _dev(rp), _dev(col), _dev(val), _stream(stream)),
               "ludvig_graph_export")
        return rp, col[: self.nnz], val[: self.nnz]

    def _diffusion_args(self, x0: torch.Tensor, out):
        """The C entry points cannot see buffer sizes: x0 must be [n] or
        [n, dx] and out the same shape, both contiguous float32 on the GPU."""
        if x0.dim() not in (1, 2) or int(x0.shape[0]) != self.n:
            raise LudvigError(f"x0 must be [{self.n}] or [{self.n}, dx], got {tuple(x0.shape)}")
        if out is not None and tuple(out.shape) != tuple(x0.shape):
            raise LudvigError(f"out must have the shape of x0 {tuple(x0.shape)}, got {tuple(out.shape)}")
        return 1 if x0.dim() == 1 else int(x0.shape[1])

    def diffuse(self, x0: torch.Tensor, iters: int, out=None, stream=None):
        L = load()
        x0 = x0.contiguous()
        dx = self._diffusion_args(x0, out)
        if out is None:
            out = torch.empty_like(x0)
        _check(L.ludvig_diffuse(self._h, _dev(x0, torch.float32, "x0"), dx, iters,
                                _dev(out, torch.float32, "out"), _stream(stream)), "ludvig_diffuse")
        return out

    def diffuse_noalloc(self, x0: torch.Tensor, iters: int, out: torch.Tensor, stream=None):
        """ludvig_diffuse_noalloc: the same diffusion with the library's static
        scratch; `out` must be supplied (nothing is allocated)."""
        L = load()
        x0 = x0.contiguous()
        dx = self._diffusion_args(x0, out)
        _check(L.ludvig_diffuse_noalloc(self._h, _dev(x0, torch.float32, "x0"), dx, iters,
                                        _dev(out, torch.float32, "out"), _stream(stream)),
               "ludvig_diffuse_noalloc")
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ludvig_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
