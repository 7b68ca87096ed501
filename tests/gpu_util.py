"""Helpers shared by the GPU parity tests (not collected as tests)."""
import numpy as np
import torch


def rel_l2(got, ref, mask=None):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    if mask is not None:
        got, ref = got[mask], ref[mask]
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (den if den > 0 else 1.0))


def device_features(wl, views, dtype=torch.float32):
    """[V,H,W,D] on the GPU, generated view by view."""
    return torch.stack([wl.features(v, device="cuda", dtype=dtype) for v in views]).contiguous()
