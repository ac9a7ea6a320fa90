"""Pins of the quantisation oracle (oracle/quant.py): the rounding it restates
agrees with torch's own float32 -> bfloat16 / float8_e4m3fn conversions, and
the per-element error bound holds for every code, found by brute force over all
65,536 BF16 bit patterns and all 256 E4M3 codes. The lower bound it implies is
never above the exact distance."""
import numpy as np
import pytest

from oracle import quant as Q

torch = pytest.importorskip("torch")


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(200000).astype(np.float32) * 10.0 ** rng.integers(-30, 30, 200000),
                        np.array([0.0, -0.0, 1e-40, -3e-39, 65504.0, 3.3e38], np.float32)]).astype(np.float32)
    ours = Q.bf16_round(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ours.view(np.uint32), ref.view(np.uint32))


def test_bf16_bound_every_code():
    # every finite BF16 value v: the float32 inputs that round to v lie within
    # half the gap to each neighbour; the bound must cover both half-gaps
    bits = np.arange(65536, dtype=np.uint32) << 16
    v = bits.view(np.float32).astype(np.float64)
    fin = np.isfinite(v) & (v >= 0)
    vals = np.unique(v[fin])
    gaps = np.diff(vals)
    half_lo = np.concatenate([[gaps[0]], gaps]) / 2       # to the neighbour below (0's own subnormal gap)
    half_hi = np.concatenate([gaps, [gaps[-1]]]) / 2
    worst = np.maximum(half_lo, half_hi)
    assert np.all(worst <= Q.bf16_bound(vals))


def test_bf16_bound_random_inputs():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(500000) * 10.0 ** rng.integers(-40, 38, 500000)).astype(np.float32)
    x = x[np.isfinite(x)]
    xh = Q.bf16_round(x)
    ok = np.isfinite(xh)
    assert np.all(np.abs(x[ok].astype(np.float64) - xh[ok]) <= Q.bf16_bound(xh[ok]))


def test_e4m3_table_and_rounding_match_torch():
    codes = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).to(torch.float32).numpy()
    ours = Q.e4m3_values()
    both_nan = np.isnan(codes) & np.isnan(ours)
    assert np.all(both_nan | (codes == ours))
    rng = np.random.default_rng(2)
    v = np.concatenate([rng.uniform(-448, 448, 100000), rng.uniform(-1, 1, 100000) * 2.0 ** -6,
                        Q._SORTED, (Q._SORTED[1:] + Q._SORTED[:-1]) / 2]).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    assert np.array_equal(Q.e4m3_round(v.astype(np.float64)).astype(np.float32), ref)


def test_e4m3_bound_every_code():
    vals = Q._SORTED[Q._SORTED >= 0]
    gaps = np.diff(vals)
    half_lo = np.concatenate([[gaps[0]], gaps]) / 2
    half_hi = np.concatenate([gaps, [0.0]]) / 2             # 448 is the top: inputs are clamped there
    worst = np.maximum(half_lo, half_hi)
    assert np.all(worst <= Q.e4m3_bound(vals))


def test_lower_bound_below_exact_distance():
    rng = np.random.default_rng(3)
    x = (rng.standard_normal((2000, 64)) * rng.uniform(0.01, 30, 64)).astype(np.float32)
    q = (rng.standard_normal((10, 64)) * 5).astype(np.float32)
    xh = Q.bf16_round(x)
    e = Q.bf16_bound(xh)
    s = Q.fp8_scales(x)
    c = Q.e4m3_round(x / s)
    x8 = c * s
    e8 = Q.e4m3_bound(c) * s
    for qq in q.astype(np.float64):
        exact = ((x.astype(np.float64) - qq) ** 2).sum(axis=1)
        assert np.all(Q.lower_bound_l2(qq, xh, e) <= exact)
        assert np.all(Q.lower_bound_l2(qq, x8, e8) <= exact)
        # and the bound is not vacuous
        assert np.mean(Q.lower_bound_l2(qq, xh, e) / exact) > 0.9
