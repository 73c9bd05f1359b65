"""The Nose-Hoover tolerance of the GPU kernels follows from their arithmetic.

The kernels form S = sum_i y_i^2 of Eq. (eq_NH) from momenta rounded to
multiples of 2^-24 (the oracle's test double restates that sum); the oracle
proper forms the exact sum rounded once.  After one step from the seeded
state both have the same momenta, and xi_1 = xi0 + (dt/M)(S - N T) differs
only through S.  tests/test_gpu_nose_hoover.py bounds that difference by
  (dt/M) (2^-24 sum|y_i| + N 2^-50 + 2^-52 S + 2^-51 (S + N T))
      + 2^-51 (|(dt/M)(S - N T)| + |xi_1|).
Here, on the CPU, the oracle with the test double stands in for the kernels:
the bound holds, is used by a real difference (every replica's xi differs in
its last bits), and stays far below the step xi takes.
"""
import numpy as np
import pytest

import oracle
import synth


def _bound(y, n, h, NT, xi):
    y64 = y.astype(np.float64)
    S = (y64 * y64).sum(axis=1)
    D = 2.0**-24 * np.abs(y64).sum(axis=1) + n * 2.0**-50 + 2.0**-52 * S
    return h * (D + 2.0**-51 * (S + NT)) + 2.0**-51 * (np.abs(h * (S - NT)) + np.abs(xi))


@pytest.mark.parametrize("kind,form,n", [("pm1", 1, 300), ("gauss", 0, 257), ("pm1", 1, 1000)])
def test_one_step_xi_of_the_quantised_sum_is_within_the_stated_bound(kind, form, n):
    J = synth.sk_pm1(n, 70 + n) if kind == "pm1" else synth.sk_gauss(n, 70 + n)
    R = 64
    NH = dict(nh_T=0.3, nh_M=20.0 * n, nh_xi0=-0.05)
    c0 = oracle.c0_from_c1(J, 0.7 if form == 1 else 0.9)
    plain = oracle.run(J, oracle.make_params(form, c0, 1.1, 0.0, eval_every=0, nose_hoover=True,
                                             **NH), 1, 9, range(R), "f32")
    quant = oracle.run(J, oracle.make_params(form, c0, 1.1, 0.0, eval_every=0, nose_hoover=True,
                                             nh_sum_q24=True, **NH), 1, 9, range(R), "f32")
    np.testing.assert_array_equal(plain["x"], quant["x"])
    np.testing.assert_array_equal(plain["y"], quant["y"])
    h = 1.1 / NH["nh_M"]
    bound = _bound(plain["y"], n, h, n * NH["nh_T"], quant["xi"])
    dev = np.abs(plain["xi"] - quant["xi"])
    assert np.all(dev <= bound)
    assert np.count_nonzero(dev) > R // 2          # the two sums do differ
    step = np.abs(plain["xi"] - NH["nh_xi0"])
    assert np.median(bound) < 1e-3 * np.median(step)
