"""Element-wise quantisation to BF16 / FP8-E4M3 and its error bound.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper stores float32 and names compression of PDX dimensions as future
work (Sec. 8). The low-precision scan stores x_hat = quantised x and prunes
with a lower bound of the distance. Its correctness rests on one per-element
fact: |x - x_hat| <= e(x_hat). This module restates the two formats from
their definitions and the bound, so that tests can pin the bound by brute
force over every code:

* BF16: 1 sign, 8 exponent, 7 fraction bits. Round to nearest, ties to even,
  from float32. A normal x_hat = m * 2^E with 1 <= m < 2 has spacing 2^(E-7),
  so |x - x_hat| <= 2^(E-8) <= |x_hat| * 2^-8. Below the smallest normal the
  spacing is 2^-133, and the bound is 2^-134.
* FP8 E4M3 (no infinities, max 448): 1 sign, 4 exponent (bias 7),
  3 fraction bits. The element is c = round(x / s_j) with the per-dimension
  scale s_j = max_i |x_ij| / 448, so |x / s_j| <= 448 and nothing saturates.
  A normal code has spacing 2^(E-3), so |x/s - c| <= |c| * 2^-4. Subnormal
  codes (|c| < 2^-6) have spacing 2^-9 and error at most 2^-10. So
  |x - s c| <= s * max(|c| 2^-4, 2^-10). The float32 divide x / s and the
  product s * c add relative errors of at most 2^-24 each, and the bound used
  in the kernels is widened by a factor (1 + 2^-20).
"""
from __future__ import annotations

import numpy as np

FP8_MAX = 448.0
SLACK = 1.0 + 2.0 ** -20


# ---------------------------------------------------------------- BF16
def bf16_round(x):
    """float32 -> nearest BF16 (ties to even), returned as float32."""
    x = np.ascontiguousarray(x, np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    return np.where(np.isnan(x), x, out)


def bf16_bound(xh):
    """Upper bound on |x - x_hat| given the BF16 value x_hat."""
    xh = np.abs(np.asarray(xh, np.float64))
    return np.maximum(xh * 2.0 ** -8, 2.0 ** -134) * SLACK


# ---------------------------------------------------------------- FP8 E4M3
def e4m3_values():
    """All 256 codes -> float64 value (NaN for the two NaN codes)."""
    vals = np.empty(256)
    for b in range(256):
        s = -1.0 if b & 0x80 else 1.0
        e = (b >> 3) & 0xF
        f = b & 0x7
        if e == 0xF and f == 0x7:
            vals[b] = np.nan
        elif e == 0:
            vals[b] = s * (f / 8.0) * 2.0 ** -6
        else:
            vals[b] = s * (1.0 + f / 8.0) * 2.0 ** (e - 7)
    return vals


_E4M3 = e4m3_values()
_FINITE = np.isfinite(_E4M3)
_SORTED = np.sort(np.unique(_E4M3[_FINITE]))


def e4m3_round(v):
    """Nearest E4M3 value (ties: even code, i.e. even fraction), saturating at
    +-448 (inputs beyond are clamped first)."""
    v = np.clip(np.asarray(v, np.float64), -FP8_MAX, FP8_MAX)
    idx = np.searchsorted(_SORTED, v)
    idx = np.clip(idx, 1, len(_SORTED) - 1)
    lo, hi = _SORTED[idx - 1], _SORTED[idx]
    dlo, dhi = v - lo, hi - v
    pick_hi = dhi < dlo
    tie = dhi == dlo
    # tie: choose the value with an even fraction field
    def even(val):
        code = np.array([_code_of(x) for x in np.atleast_1d(val)])
        return (code & 1) == 0
    if np.any(tie):
        he = even(hi[tie])
        pick_hi = pick_hi.copy()
        pick_hi[tie] = he
    return np.where(pick_hi, hi, lo)


_VAL2CODE = {}
for _b in range(256):
    if np.isfinite(_E4M3[_b]) and not (_E4M3[_b] == 0 and _b & 0x80):
        _VAL2CODE.setdefault(float(_E4M3[_b]), _b)


def _code_of(val):
    return _VAL2CODE[float(val)]


def e4m3_bound(c):
    """Upper bound on |x/s - c| for the E4M3 value c."""
    c = np.abs(np.asarray(c, np.float64))
    return np.maximum(c * 2.0 ** -4, 2.0 ** -10) * SLACK


def fp8_scales(x):
    """Per-dimension scale s_j = max_i |x_ij| / 448 (1 where a column is 0)."""
    m = np.abs(np.asarray(x, np.float64)).max(axis=0)
    return np.where(m > 0, m / FP8_MAX, 1.0)


def lower_bound_l2(q, xh, e):
    """sum_j max(0, |q_j - x_hat_j| - e_j)^2: a lower bound of ||q - x||^2
    whenever |x_j - x_hat_j| <= e_j for all j."""
    t = np.maximum(0.0, np.abs(np.asarray(q, np.float64) - np.asarray(xh, np.float64)) - e)
    return (t * t).sum(axis=-1)
