"""Pins for the oracle's number formats, RNG and direction table.

Each check compares the oracle with something outside itself: numpy's and
torch's own float16 / float8_e4m3fn conversions (library routines), the
published splitmix64 test vector, and hand-derived bit patterns.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle as O


def _f16_grid_midpoints():
    # every positive finite f16 value and the midpoint to its successor
    codes = np.arange(0, 0x7C00, dtype=np.uint16)
    vals = codes.view(np.float16).astype(np.float32)
    mids = ((vals[:-1].astype(np.float64) + vals[1:].astype(np.float64)) / 2).astype(np.float32)
    return vals, mids


def test_f16_encode_matches_numpy_rne():
    rng = np.random.default_rng(1)
    bits = rng.integers(0, 2**32, size=60_000, dtype=np.uint64).astype(np.uint32)
    x = bits.view(np.float32)
    x = x[np.isfinite(x) & (np.abs(x) < 60000)]
    vals, mids = _f16_grid_midpoints()
    pick = rng.choice(len(mids), size=20_000, replace=False)
    x = np.concatenate([x, mids[pick], -mids[pick], vals[pick], np.float32([0.0, -0.0, 65504, 65519, 1e-8])])
    got = O.f32_to_f16(x)
    want = x.astype(np.float16).view(np.uint16)
    assert np.array_equal(got, want)


def test_f16_overflow_and_specials():
    got = O.f32_to_f16(np.float32([65520.0, 1e6, -1e6, np.inf]))
    assert got.tolist() == [0x7C00, 0x7C00, 0xFC00, 0x7C00]


def test_f16_decode_all_codes():
    codes = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    got = O.f16_to_f32(codes)
    want = codes.view(np.float16).astype(np.float32)
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan], want[~nan])


def test_e4m3_decode_all_codes_matches_torch():
    codes = np.arange(256, dtype=np.uint8)
    got = O.e4m3_to_f32(codes)
    want = torch.from_numpy(codes).view(torch.float8_e4m3fn).float().numpy()
    nan = np.isnan(want)
    assert nan.sum() == 2  # S.1111.111 only
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan], want[~nan])
    assert got[0x7E] == 448.0 and got[0x01] == 2.0 ** -9


def test_e4m3_encode_matches_torch_in_range():
    rng = np.random.default_rng(2)
    grid = np.sort(np.unique(np.abs(O.e4m3_to_f32(np.arange(0, 0x7F, dtype=np.uint8)))))
    mids = ((grid[:-1].astype(np.float64) + grid[1:]) / 2).astype(np.float32)
    x = np.concatenate([rng.uniform(-448, 448, 20_000).astype(np.float32),
                        (rng.standard_normal(20_000) * 0.05).astype(np.float32),
                        mids, -mids, grid, np.nextafter(mids, np.float32(0)), np.nextafter(mids, np.float32(1e9))])
    got = O.f32_to_e4m3(x)
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(got, want)


def test_e4m3_saturates():
    got = O.f32_to_e4m3(np.float32([448.0, 449.0, 464.0, 1e30, -500.0, np.inf, np.nan]))
    assert got.tolist() == [0x7E, 0x7E, 0x7E, 0x7E, 0xFE, 0x7E, 0x7F]


def test_encode_f16_integer_data_is_exact():
    rng = np.random.default_rng(3)
    X = rng.integers(0, 256, size=(300, 128)).astype(np.float32)
    X[0] = 0.0  # all-zero vector: scale 1
    codes, scales = O.encode(X, O.F16)
    assert scales[0] == 1.0
    e = np.log2(scales[1:])
    assert np.array_equal(e, np.round(e))  # powers of two
    mx = np.abs(X[1:]).max(axis=1) / scales[1:]
    assert ((mx >= 2**14) & (mx < 2**15)).all()
    assert np.array_equal(O.decode(codes, scales, O.F16), X)


def test_f16_stored_value_is_an_exact_product():
    """An FP16 row's stored value s * h (s a power of two) is exact in FP32
    for rows whose largest |x| is at least 2^-88, across magnitudes: so
    q - s * h rounded once (one fused multiply-add, as the kernel forms it)
    equals q minus the rounded stored value, as the oracle forms it."""
    rng = np.random.default_rng(8)
    mags = 2.0 ** rng.uniform(-88, 100, size=(400, 1))
    X = (rng.standard_normal((400, 64)) * mags).astype(np.float32)
    X[:5, 10:] = 0.0
    codes, scales = O.encode(X, O.F16)
    h = O.decode(codes, np.ones_like(scales), O.F16).astype(np.float64)
    exact = scales[:, None].astype(np.float64) * h
    stored = O.decode(codes, scales, O.F16)
    assert np.array_equal(stored.astype(np.float64), exact)
    Q = (rng.standard_normal((400, 64)) * mags).astype(np.float32)
    two_step = (Q - stored).astype(np.float32)                      # rn(q - rn(s h))
    fused = (Q.astype(np.float64) - exact).astype(np.float32)       # rn(q - s h): q - s h is exact in FP64 here
    assert np.array_equal(two_step, fused)


def test_encode_e4m3_error_bound():
    rng = np.random.default_rng(4)
    X = (rng.standard_normal((200, 96)) * rng.uniform(0.1, 50, (200, 1))).astype(np.float32)
    codes, scales = O.encode(X, O.E4M3)
    np.testing.assert_allclose(scales, np.abs(X).max(axis=1) / np.float32(448), rtol=1e-7)
    Xd = O.decode(codes, scales, O.E4M3).astype(np.float64)
    # 3 mantissa bits: half an ulp is 2^-4 relative in the normal range, and
    # 2^-10 * scale absolute below it (subnormal spacing 2^-9)
    err = np.abs(Xd - X)
    bound = np.maximum(np.abs(X) * 2.0 ** -4, scales[:, None].astype(np.float64) * 2.0 ** -10) * (1 + 1e-6)
    assert (err <= bound).all()
    assert (np.abs(Xd).max(axis=1) <= 448 * scales * (1 + 1e-6)).all()


def test_splitmix64_published_vector():
    # splitmix64 seeded with 1234567: the published first five outputs
    golden = 0x9E3779B97F4A7C15
    s = 1234567
    got = [O.splitmix64((s + i * golden) & (2**64 - 1)) for i in range(5)]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]
    assert O.splitmix64(0) == 0xE220A8397B1DCDAF


def test_dir_table_hand_derived(golden_dir):
    fx = json.load(open(os.path.join(golden_dir, "dir_bits_40d.json")))
    d = 40
    xu = np.zeros(d, np.float32)
    xv = np.array([1.0 if i % 3 == 0 else (0.0 if i % 3 == 1 else -1.0) for i in range(d)], np.float32)
    Xs = np.stack([xu, xv])
    G = np.array([[1, O.INVALID], [0, 0]], dtype=np.uint32)
    D = O.dir_table(Xs, G)
    assert D.shape == (2, 2, 2)
    assert [hex(int(w)) for w in D[0, 0]] == fx["u_to_v"]
    assert D[0, 1].tolist() == [0, 0]
    assert [hex(int(w)) for w in D[1, 0]] == fx["v_to_u"]


def test_dir_table_popcount_identity():
    # matching sign bits between q-x_u and x_v-x_u count coordinates where
    # both point the same way; with the reversed edge the roles swap
    rng = np.random.default_rng(5)
    X = rng.standard_normal((50, 70)).astype(np.float32)
    G = np.array([[(i + 1) % 50, (i + 7) % 50] for i in range(50)], dtype=np.uint32)
    D = O.dir_table(X, G)
    for u in range(50):
        for j, v in enumerate(G[u]):
            ones = sum(bin(int(w)).count("1") for w in D[u, j])
            assert ones == int((X[v] > X[u]).sum())
