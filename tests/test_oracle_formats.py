"""Pins for the oracle-side storage-format definitions (oracle/formats.py).

Checked against library conversions (torch bfloat16 / float8_e4m3fn) and
against the formats' stated exact ranges.
"""
import numpy as np
import pytest
import torch

from oracle import formats


def test_u8_overflow_roundtrip():
    rng = np.random.default_rng(0)
    V = rng.integers(0, 2000, size=(50, 33))
    small = rng.integers(0, 255, size=V.shape)
    V = np.where(rng.random(V.shape) < 0.7, small, V)
    plane, ptr, col, add = formats.pack_u8_overflow(V)
    assert plane.dtype == np.uint8 and plane.max() <= 255
    assert ptr[0] == 0 and ptr[-1] == col.shape[0]
    assert (formats.unpack_u8_overflow(plane, ptr, col, add) == V).all()
    for i in range(V.shape[0]):
        cs = col[ptr[i]:ptr[i + 1]]
        assert (np.diff(cs.astype(int)) > 0).all()


def test_u8_overflow_boundaries():
    V = np.array([[254, 255, 256, 255 + 65535]])
    plane, ptr, col, add = formats.pack_u8_overflow(V)
    assert plane.tolist() == [[254, 255, 255, 255]]
    assert col.tolist() == [2, 3] and add.tolist() == [1, 65535]
    with pytest.raises(ValueError):
        formats.pack_u8_overflow(np.array([[255 + 65536]]))


def test_bf16_matches_library_rounding():
    v = np.concatenate([np.arange(0, 70000), np.array([2.0 ** 20 + 3, 123456789.0])])
    ours = formats.bf16_bits(v)
    lib = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert (ours == lib).all()
    assert (formats.bf16_decode(ours) == formats.bf16_round(v)).all()
    ints = np.arange(0, 257)
    assert (formats.bf16_round(ints) == ints).all()          # exact up to 256
    assert formats.bf16_round(257) == 256 and formats.bf16_round(259) == 260


def test_e4m3_decode_matches_library():
    codes = np.arange(256, dtype=np.uint8)
    lib = torch.tensor(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    ours = formats.e4m3_decode(codes)
    both_nan = np.isnan(lib) & np.isnan(ours)
    assert (both_nan | (lib == ours)).all()
    assert formats.E4M3_MAX == 448.0


def test_e4m3_encode_matches_library_rounding():
    rng = np.random.default_rng(3)
    v = np.concatenate([np.arange(0, 448.25, 0.25), rng.uniform(0, 448, 5000)])
    ours = formats.e4m3_encode(v)
    lib = torch.tensor(v, dtype=torch.float64).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert (ours == lib).all()


def test_e4m3_exact_integers_and_row_scale():
    ints = np.arange(0, 17)
    assert (formats.e4m3_decode(formats.e4m3_encode(ints)) == ints).all()
    assert formats.e4m3_decode(formats.e4m3_encode(np.array([17.0])))[0] == 16.0  # tie -> even
    V = np.array([[0, 3, 448], [0, 449, 1], [1000, 2, 0], [0, 0, 0]], float)
    codes, e = formats.pack_e4m3(V)
    assert e.tolist() == [0, 1, 2, 0]
    back = formats.unpack_e4m3(codes, e)
    assert back[0].tolist() == [0, 3, 448]
    assert back[3].tolist() == [0, 0, 0]
    assert np.all(np.abs(back - V) <= np.maximum(V, 1) * 2.0 ** -4)
