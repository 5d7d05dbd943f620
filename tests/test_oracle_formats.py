"""Pins of the oracle's BF16 and E4M3 codecs against PyTorch's conversions
(independent library routines) and the format definitions."""
import numpy as np
import pytest
import torch

import oracle as O


def test_bf16_decode_all_codes():
    codes = np.arange(1 << 16, dtype=np.uint16)
    ref = torch.from_numpy(codes.view(np.int16)).view(torch.bfloat16).float().numpy()
    got = O.bf16_value(codes)
    fin = np.isfinite(ref)
    assert np.array_equal(got[fin], ref[fin].astype(np.float64))
    assert np.array_equal(np.isnan(got), np.isnan(ref))


def test_bf16_encode_matches_torch_and_ties_to_even():
    rng = np.random.default_rng(0)
    x = np.concatenate([
        rng.standard_normal(200000).astype(np.float32),
        (rng.standard_normal(20000) * 1e30).astype(np.float32),
        (rng.standard_normal(20000) * 1e-38).astype(np.float32),
        np.array([0.0, -0.0, np.inf, -np.inf, 3.4028235e38], np.float32),
    ])
    # exact halfway points between adjacent BF16 values, both parities
    hi = rng.integers(0, 0x7F00, 5000).astype(np.uint32) << 16
    ties = (hi | 0x8000).view(np.float32)
    x = np.concatenate([x, ties, -ties])
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(O.bf16_bits(x), ref)
    # a tie rounds to the even upper half
    t = np.array([np.frombuffer(np.uint32(0x3F808000).tobytes(), np.float32)[0]], np.float32)
    assert O.bf16_bits(t)[0] == 0x3F80
    t = np.array([np.frombuffer(np.uint32(0x3F818000).tobytes(), np.float32)[0]], np.float32)
    assert O.bf16_bits(t)[0] == 0x3F82


def _e4m3_all():
    return np.array([O.lib().orc_e4m3_decode(c) for c in range(256)])


def test_e4m3_decode_all_codes():
    codes = np.arange(256, dtype=np.uint8)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).float().numpy().astype(np.float64)
    got = O.e4m3_value(codes)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    fin = ~np.isnan(ref)
    assert np.array_equal(got[fin], ref[fin])
    assert np.nanmax(got) == 448.0 and got[0x7E] == 448.0 and got[1] == 2.0 ** -9


def test_e4m3_encode_matches_torch_in_range():
    rng = np.random.default_rng(1)
    x = np.concatenate([
        (rng.standard_normal(200000) * 40).astype(np.float32),
        (rng.standard_normal(50000) * 0.01).astype(np.float32),
        rng.uniform(-448, 448, 50000).astype(np.float32),
        np.array([0.0, -0.0, 448.0, -448.0, 2.0 ** -9, 2.0 ** -10, 3 * 2.0 ** -11], np.float32),
    ])
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(O.e4m3_bits(x), ref)


def test_e4m3_ties_to_even_and_saturation():
    vals = _e4m3_all()
    pos = np.sort(np.unique(vals[(vals >= 0) & np.isfinite(vals)]))
    mids = ((pos[:-1] + pos[1:]) / 2).astype(np.float32)
    got = O.e4m3_value(O.e4m3_bits(mids))
    for lo, hi, g in zip(pos[:-1], pos[1:], got):
        clo = int(np.where(vals == lo)[0][0]) & 0x7F
        chi = int(np.where(vals == hi)[0][0]) & 0x7F
        assert g == (lo if clo % 2 == 0 else hi) and (clo % 2) != (chi % 2)
    big = np.array([448.0, 460.0, 464.0, 1e6, np.inf, -1e9, -np.inf], np.float32)
    assert list(O.e4m3_value(O.e4m3_bits(big))) == [448, 448, 448, 448, 448, -448, -448]
    assert O.e4m3_bits(np.array([np.nan], np.float32))[0] & 0x7F == 0x7F


def test_row_quantisation():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((6, 300)).astype(np.float32)
    x[3] = 0.0
    q, s = O.quant_rows_e4m3(x)
    assert s[3] == 1.0 and not q[3].any()
    for r in (0, 1, 2, 4, 5):
        amax = np.abs(x[r]).max()
        assert s[r] == np.float32(amax) / np.float32(448.0)
        j = int(np.argmax(np.abs(x[r])))
        assert O.e4m3_value(q[r, j:j + 1])[0] == np.sign(x[r, j]) * 448.0
        deq = O.e4m3_value(q[r]) * s[r]
        big = np.abs(x[r]) > s[r] * 2.0 ** -6
        rel = np.abs(deq[big] - x[r][big]) / np.abs(x[r][big])
        assert rel.max() <= 2.0 ** -4 * 1.0001  # half a spacing of 3 mantissa bits
