"""GPU parity of the split-BF16 tensor-core path (general couplings).

The force is J_hi x_hi + J_lo x_hi + J_hi x_lo with BF16 parts and FP32
accumulation, so trajectories are not bit-exact; the bound below is derived
from that arithmetic.  With hi = bf16(v) and lo = bf16(v - hi) (8 significant
bits each), |v - hi - lo| <= 2^-18 |v|, so the dropped part of each product
J_ij x_j is at most 3 * 2^-18 |J_ij x_j|; summing K = 3 Np products in FP32
adds at most K * 2^-24 of sum_j |J_ij x_j|.  One step then differs from the
binary64 oracle by
    |dy_i| <= c0 dt (3 * 2^-18 + 3 Np 2^-24) sum_j |J_ij x_j| + r_i
where r_i = 2^-20 (|y_i| + |c0 f_i dt| + |p x_i dt| + |g y_i|) covers the
binary32 rounding of the update itself (six operations).  Spins whose
unclamped position lies within q * bound of a wall are not compared (the wall
decision may go either way within the bound).
"""
import numpy as np
import pytest

import oracle
import paper_2203_08361_gb300 as hsb
import synth

pytestmark = pytest.mark.gpu


def _one_step_bound(J, x, y, f_ref, pk, c0, dt, q, g, Np, discrete):
    Jd = J.astype(np.float64)
    op = np.ones_like(x, dtype=np.float64) if discrete else np.abs(x.astype(np.float64))
    absJx = op @ np.abs(Jd).T  # [R, N]: sum_j |J_ij b_j|, b = x or sgn(x)
    eps = 3 * 2.0**-18 + 3 * Np * 2.0**-24
    r = 2.0**-20 * (np.abs(y) + np.abs(c0 * f_ref * dt) + np.abs(pk * x * dt) + np.abs(g * y))
    return c0 * dt * eps * absJx + r


@pytest.mark.parametrize("form,n,R", [("ballistic", 2000, 64), ("discrete", 2000, 64),
                                      ("ballistic", 300, 130)])
def test_one_step_error_within_derived_bound(form, n, R):
    J = synth.sk_gauss(n, 21)
    rng = np.random.default_rng(5)
    x0 = rng.uniform(-1, 1, (R, n)).astype(np.float32)
    y0 = rng.uniform(-1, 1, (R, n)).astype(np.float32)
    steps, k = 100, 37
    c1 = 0.9 if form == "ballistic" else 0.7
    gamma = 0.5
    c0 = oracle.c0_from_c1(J, c1)
    p = hsb.params(form, "bf16x3", c1=c1, dt=1.1, gamma=gamma)
    with hsb.Solver(J) as s:
        x1, y1 = s.advance(p, steps, k, k + 1, x0, y0)
    pk = oracle.pump_factor(1.0, k, steps)
    fcode = 0 if form == "ballistic" else 1
    xr, yr, fr = oracle.step(J, x0, y0, fcode, pk, c0, 1.1, 1.1, gamma * 1.1, "f64")
    Np = (n + 127) // 128 * 128
    bound = _one_step_bound(J, x0, y0, fr, pk, c0, 1.1, 1.1, gamma * 1.1, Np, fcode == 1)
    # unclamped position of the oracle step, to skip ambiguous wall decisions
    yt = y0 + (c0 * fr - pk * x0) * 1.1
    xt = x0 + 1.1 * yt
    ambiguous = np.abs(np.abs(xt) - 1.0) <= 1.1 * bound
    dy = np.abs(y1.astype(np.float64) - yr)
    dx = np.abs(x1.astype(np.float64) - xr)
    ok = ~ambiguous
    assert ok.mean() > 0.95
    assert np.all(dy[ok] <= bound[ok]), f"max dy/bound {np.max(dy[ok] / bound[ok])}"
    assert np.all(dx[ok] <= 1.1 * bound[ok] + 2.0**-20)
    print(f"\n{form} N={n}: max |dy| = {dy[ok].max():.3e}, max |dy|/bound = "
          f"{np.max(dy[ok] / bound[ok]):.3e}, ambiguous walls {ambiguous.sum()}")


def test_bf16x3_run_is_deterministic_and_independent_of_R():
    J = synth.sk_gauss(500, 2)
    p = hsb.params("ballistic", "bf16x3", c1=0.9, dt=1.1, gamma=0.5, eval_every=50)
    with hsb.Solver(J) as s:
        sa, ea = s.run(p, 256, 300, 4)
        xa, _ = s.get_state(256)
        sb, eb = s.run(p, 256, 300, 4)
        xb, _ = s.get_state(256)
    np.testing.assert_array_equal(sa, sb)
    np.testing.assert_array_equal(ea, eb)
    np.testing.assert_array_equal(xa, xb)


def test_bf16x3_full_size_gaussian_workload_statistics():
    # HbSB on an N = 2000 Gaussian SK instance, R = 1024, 5000 steps, dt 1.1,
    # c1 0.9, gamma 0.5: the split-BF16 tensor-core path against the plain
    # FP32 path (bit-exact to the binary32 oracle) on the same seeds.  The
    # dynamics are chaotic, so the comparison is of the best-energy
    # distributions; every returned energy is the binary64 energy of the
    # returned spins (checked on sampled replicas against the oracle).
    J = synth.sk_gauss(2000, 2)
    R, steps, seed = 1024, 5000, 3
    pb = hsb.params("ballistic", "bf16x3", c1=0.9, dt=1.1, gamma=0.5, eval_every=100)
    pf = hsb.params("ballistic", "fp32", c1=0.9, dt=1.1, gamma=0.5, eval_every=100)
    with hsb.Solver(J) as s:
        sb, eb = s.run(pb, R, steps, seed)
        sf, ef = s.run(pf, R, steps, seed)
    for r in (0, 511, 1023):
        assert oracle.ising_energy(J, sb[r]) == pytest.approx(eb[r], rel=1e-12)
    mb, mf = eb.mean(), ef.mean()
    sd = np.sqrt((eb.var() + ef.var()) / R)
    print(f"\nmean best E: bf16x3 {mb:.2f}, fp32 {mf:.2f} (std err {sd:.2f}); "
          f"min {eb.min():.2f} / {ef.min():.2f}")
    assert abs(mb - mf) < 5 * sd + 1e-3 * abs(mf)
    # plausibility for Gaussian SK: E / N^1.5 near the ground state ~ -0.76
    assert -0.80 < eb.min() / 2000**1.5 < -0.70
