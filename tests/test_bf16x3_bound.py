"""The error bound of the split-BF16 parity test follows from the arithmetic.

The GPU test (test_gpu_bf16x3.py) compares one split-BF16 step with the
binary64 oracle step against
    |dy_i| <= c0 dt (3 2^-18 + 3 Np 2^-24) sum_j |J_ij b_j| + r_i.
Here the arithmetic that bound was derived from is emulated on the CPU:
- J and b split into BF16 parts rounded to nearest even (hi = bf16(v),
  lo = bf16(v - hi));
- the products J_hi b_hi, J_lo b_hi and J_hi b_lo, each exact in binary32;
- the 3 Np products summed in binary32, and the binary32 update in the
  Methods order.
The same bound must hold, so the tolerance is a consequence of the
arithmetic, not a fit to a measurement.  The emulation is test code: neither
the oracle nor the library uses it.
"""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_bf16x3 import _one_step_bound


def _bf16(v):
    # round binary32 to the nearest BF16 (8 significant bits), ties to even
    b = np.ascontiguousarray(v, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _split(v):
    hi = _bf16(v)
    return hi, _bf16(np.float32(v) - hi)  # v - hi is exact in binary32


def _force_bf16x3(J, b, Np):
    Jh, Jl = _split(J)
    bh, bl = _split(b)
    R, n = b.shape
    acc = np.zeros((R, n), np.float32)
    for j in range(n):
        for u, w in ((bh, Jh), (bh, Jl), (bl, Jh)):
            acc = acc + np.outer(u[:, j], w[:, j])  # exact products, rounded sums
    # the zero-padded columns up to Np add exact zeros
    assert acc.dtype == np.float32 and Np >= n
    return acc


def _update_f32(x, y, f, pk, c0, dt, q, g):
    f32 = np.float32
    yt = y + (f32(c0) * f - f32(pk) * x) * f32(dt)
    xt = x + f32(q) * yt
    hit = np.abs(xt) > 1
    x1 = np.where(hit, np.sign(xt), xt).astype(np.float32)
    y1 = (np.where(hit, f32(0), yt) + f32(g) * y).astype(np.float32)
    return x1, y1


def _bf16_rounding_is_nearest_even():
    v = np.array([1.0, 1.00390625, 1.005859375, 1.0078125, -3.0e-5], np.float32)
    hi = _bf16(v)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: to even (1); 1 + 1.5 2^-8 rounds up
    np.testing.assert_array_equal(hi[:4], np.float32([1.0, 1.0, 1.0078125, 1.0078125]))
    assert abs(hi[4] - v[4]) <= 2.0**-9 * abs(v[4])


@pytest.mark.parametrize("form,n,R", [(0, 300, 16), (1, 300, 16), (0, 130, 9)])
def test_emulated_split_bf16_step_is_within_the_bound(form, n, R):
    _bf16_rounding_is_nearest_even()
    J = synth.sk_gauss(n, 21)
    rng = np.random.default_rng(5 + n)
    x0 = rng.uniform(-1, 1, (R, n)).astype(np.float32)
    y0 = rng.uniform(-1, 1, (R, n)).astype(np.float32)
    steps, k, dt, gamma = 100, 37, 1.1, 0.5
    c0 = oracle.c0_from_c1(J, 0.9 if form == 0 else 0.7)
    pk = oracle.pump_factor(1.0, k, steps)
    Np = (n + 127) // 128 * 128
    b = x0 if form == 0 else np.where(x0 >= 0, 1.0, -1.0).astype(np.float32)
    f = _force_bf16x3(J, b, Np)
    x1, y1 = _update_f32(x0, y0, f, pk, c0, dt, dt, gamma * dt)
    xr, yr, fr = oracle.step(J, x0, y0, form, pk, c0, dt, dt, gamma * dt, "f64")
    bound = _one_step_bound(J, x0, y0, fr, pk, c0, dt, dt, gamma * dt, Np, form == 1)
    yt = y0 + (c0 * fr - pk * x0) * dt
    xt = x0 + dt * yt
    ok = np.abs(np.abs(xt) - 1.0) > dt * bound
    assert ok.mean() > 0.95
    dy = np.abs(y1.astype(np.float64) - yr)
    dx = np.abs(x1.astype(np.float64) - xr)
    assert np.all(dy[ok] <= bound[ok]), np.max(dy[ok] / bound[ok])
    assert np.all(dx[ok] <= dt * bound[ok] + 2.0**-20)
    # the split is not a no-op: a plain BF16 force (hi parts only) breaks the bound
    Jh, _ = _split(J)
    bh, _ = _split(b)
    f_hi = (bh.astype(np.float64) @ Jh.astype(np.float64).T).astype(np.float32)
    _, y_hi = _update_f32(x0, y0, f_hi, pk, c0, dt, dt, gamma * dt)
    assert np.any(np.abs(y_hi.astype(np.float64) - yr)[ok] > bound[ok])
