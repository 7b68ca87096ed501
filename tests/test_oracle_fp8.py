"""Pins of the oracle's FP8-E4M3 storage (the OCP 8-bit format: bias 7, 3
mantissa bits, max 448, no infinities): every code decodes as torch's
float8_e4m3fn does; encoding agrees with torch's conversion on random values
and on every tie between neighbouring codes (round to nearest even);
hand-derived codes; and the per-view absmax quantiser keeps the view's
largest magnitude at 448 with the format's relative error bound."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
if not hasattr(torch, "float8_e4m3fn"):
    pytest.skip("torch without float8_e4m3fn", allow_module_level=True)


def _torch_decode(codes):
    return torch.from_numpy(np.asarray(codes, np.uint8).copy()).view(torch.float8_e4m3fn).to(torch.float64).numpy()


def _torch_encode(x):
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.float8_e4m3fn).view(torch.uint8).numpy()


def test_decode_every_code():
    codes = np.arange(256, dtype=np.uint8)
    got, ref = oracle.e4m3_decode(codes), _torch_decode(codes)
    assert np.array_equal(np.isnan(got), np.isnan(ref)) and np.isnan(got).sum() == 2
    assert np.array_equal(got[~np.isnan(got)], ref[~np.isnan(ref)])
    assert oracle.e4m3_decode(0x7E) == 448.0 and oracle.e4m3_decode(0x01) == 2.0 ** -9


def test_encode_hand_values():
    # ties: 1.0625 between 1 and 1.125 -> even 1.0; 1.1875 -> even 1.25;
    # 15 2^-10 between 7 and 8 quanta of 2^-9 -> 8; 232 between 224 and 240 -> 224
    cases = [(1.0, 0x38), (448.0, 0x7E), (2.0 ** -9, 0x01), (2.0 ** -10, 0x00), (3 * 2.0 ** -10, 0x02),
             (-2.0, 0xC0), (500.0, 0x7E), (-1e9, 0xFE), (0.0, 0x00), (-0.0, 0x80), (1.0625, 0x38),
             (1.1875, 0x3A), (2.0 ** -6, 0x08), (7 * 2.0 ** -9, 0x07), (15 * 2.0 ** -10, 0x08),
             (240.0, 0x77), (232.0, 0x76)]
    for x, c in cases:
        assert oracle.e4m3_encode(np.float32(x)) == c, (x, hex(int(oracle.e4m3_encode(np.float32(x)))), hex(c))
    assert oracle.e4m3_encode(np.float32("nan")) == 0x7F


def test_encode_matches_torch_on_random_values_and_ties():
    rng = np.random.default_rng(0)
    x = rng.normal(size=200_000) * rng.choice([1e-4, 1e-2, 1.0, 30.0, 300.0], 200_000)
    x = np.concatenate([x, rng.uniform(-448, 448, 50_000)])
    pos = oracle.e4m3_decode(np.arange(0x7F, dtype=np.uint8))          # 0 .. 448 ascending
    ties = (pos[:-1] + pos[1:]) / 2
    x = np.concatenate([x, pos, ties, -ties]).astype(np.float32)
    x = x[np.abs(x) <= 448]
    assert np.array_equal(oracle.e4m3_encode(x), _torch_encode(x))


def test_per_view_quantiser():
    rng = np.random.default_rng(1)
    views = rng.normal(size=(3, 7, 9, 5)).astype(np.float32) * np.array([1e-3, 1.0, 50.0], np.float32)[:, None, None, None]
    views = np.concatenate([views, np.zeros((1, 7, 9, 5), np.float32)])
    q, s = oracle.fp8_quantize(views)
    assert q.dtype == np.uint8 and q.shape == views.shape and s.dtype == np.float32
    for v in range(3):
        amax = np.abs(views[v]).max()
        assert s[v] == np.float32(amax) / np.float32(448)
        assert q[v].reshape(-1)[np.argmax(np.abs(views[v]))] & 0x7F == 0x7E      # the largest sits at 448
    assert s[3] == 1 and (q[3] == 0).all()
    x = oracle.fp8_dequantize(q, s)
    y = views.astype(np.float64)
    big = np.abs(y / s.reshape(-1, 1, 1, 1)) >= 2.0 ** -6
    assert (np.abs(x - y)[big] <= 2.0 ** -4 * np.abs(y)[big] * (1 + 1e-6)).all()       # half a mantissa step
    small = ~big
    assert (np.abs(x - y)[small] <= 2.0 ** -10 * np.broadcast_to(s.reshape(-1, 1, 1, 1), y.shape)[small] * 1.000001).all()
