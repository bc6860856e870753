"""Oracle pins: storage formats and brick extraction (brick commit).

The oracle's own float16 / bfloat16 / fp8-e4m3 encoders and decoders are
checked against library conversions (numpy float16, torch bfloat16 and
float8_e4m3fn), all round-to-nearest-even."""
import numpy as np
import pytest
import torch

from paper_2407_00179_b300 import inputs


def _probe_values(seed=0, n=20000, scale=1.0):
    g = np.random.default_rng(seed)
    v = np.concatenate([
        g.uniform(-1, 1, n) * scale,
        g.normal(0, 1, n) * scale,
        np.exp(g.uniform(-30, 10, n)) * np.sign(g.uniform(-1, 1, n)),
        [0.0, -0.0, 1.0, 0.5, 65504.0, 65519.0, 6.1e-5, 5.96e-8, 2.98e-8, 1e-10],
    ])
    return v.astype(np.float32)


def test_f16_matches_numpy(orc):
    v = _probe_values()
    v = v[np.abs(v) < 65520]
    ours = orc.quantize(v, orc.F16)
    ref = v.astype(np.float16).view(np.uint16)
    np.testing.assert_array_equal(ours, ref)
    back = orc.dequantize(ours, orc.F16)
    np.testing.assert_array_equal(back, ref.view(np.float16).astype(np.float64))


def test_f16_overflow_to_inf(orc):
    v = np.array([65520.0, 1e6, -1e6], np.float32)
    with np.errstate(over="ignore"):
        ref = v.astype(np.float16).view(np.uint16)
    np.testing.assert_array_equal(orc.quantize(v, orc.F16), ref)


def test_bf16_matches_torch(orc):
    v = _probe_values(1)
    ours = orc.quantize(v, orc.BF16)
    ref = torch.from_numpy(v).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(ours, ref)
    back = orc.dequantize(ours, orc.BF16)
    np.testing.assert_array_equal(back, torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy())


def test_fp8_matches_torch_in_range(orc):
    v = _probe_values(2, scale=100.0)
    v = v[np.abs(v) <= 448.0]
    ours = orc.quantize(v, orc.FP8)
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    np.testing.assert_array_equal(ours, ref)


def test_fp8_decode_all_codes(orc):
    codes = np.arange(256, dtype=np.uint8)
    ours = orc.dequantize(codes, orc.FP8)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    finite = np.isfinite(ref)
    np.testing.assert_array_equal(ours[finite], ref[finite])
    assert np.all(np.isnan(ours[~finite]))
    assert ours[0x7E] == 448.0 and ours[0x01] == 2.0 ** -9


def test_fp8_saturates(orc):
    v = np.array([448.0, 460.0, 1000.0, -5000.0, 464.0], np.float32)
    q = orc.quantize(v, orc.FP8)
    np.testing.assert_array_equal(orc.dequantize(q, orc.FP8), [448.0, 448.0, 448.0, -448.0, 448.0])


def test_fp8_scale_maps_max_to_448(orc):
    g = np.random.default_rng(3)
    v = g.uniform(0, 0.7, 1000).astype(np.float32)
    v[17] = 0.83
    s = orc.brick_scale(v, orc.FP8)
    assert s == np.float32(np.float32(0.83) / np.float32(448.0))
    q = orc.quantize(v, orc.FP8, s)
    d = orc.dequantize(q, orc.FP8, float(s))
    # e4m3 has 3 fraction bits: relative error <= 2^-4 for normal values
    big = np.abs(v) > 2.0 ** -6 * s
    assert np.all(np.abs(d[big] - v[big]) <= 2.0 ** -4 * np.abs(v[big]) + 1e-12)
    assert orc.brick_scale(v, orc.F16) == 1.0


def test_stored_box_and_extract(orc):
    dims = (11, 7, 5)
    f = np.arange(11 * 7 * 5, dtype=np.float32).reshape(5, 7, 11)
    # interior rank: owned [3, 8) in x -> stored nodes 2..8
    s_lo, s_n = orc.stored_box(dims, (3, 0, 2), (8, 7, 5))
    assert list(s_lo) == [2, 0, 1] and list(s_n) == [7, 7, 4]
    b = orc.extract_brick(f, (3, 0, 2), (8, 7, 5))
    np.testing.assert_array_equal(b, f[1:5, 0:7, 2:9])
    # a rank owning everything stores everything
    s_lo, s_n = orc.stored_box(dims, (0, 0, 0), dims)
    assert list(s_lo) == [0, 0, 0] and list(s_n) == list(dims)


def test_partitions_tile_the_volume():
    dims = (37, 29, 23)
    for part in (inputs.regular_partition(dims, (2, 3, 2)), inputs.kd_partition(dims, 11, seed=4)):
        cover = np.zeros((dims[2], dims[1], dims[0]), np.int32)
        for lo, hi in zip(part.lo, part.hi):
            assert np.all(hi > lo)
            cover[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += 1
        assert np.all(cover == 1)
