"""GPU parity of the CTA-pair FP8 kernel (schedule 4) against the CPU oracle.

The pair kernel forms the force transposed (F^T = S^T J, replicas as the MMA's
M dimension) with each pair of CTAs holding 256 replicas x 128 spins.  Positions, momenta, best spins and best energies equal the
binary32 oracle bit for bit (the FP8 products are exact integers).  Sizes span
several spin blocks and replica pairs with ragged tails: N one past and one
short of a 128-spin block, R one past a 128-replica block (the second block
of the pair then holds padding only), N = 2, N = 2048 and N = 3000.
"""
import numpy as np
import pytest

import oracle
import paper_2203_08361_gb300 as hsb
import synth

pytestmark = pytest.mark.gpu


def _oparams(J, ev, c1=0.7, dt=1.1, gamma=0.06):
    return oracle.make_params(1, oracle.c0_from_c1(J, c1), dt, gamma, eval_every=ev)


def _check(J, p, R, steps, seed, ev, rows=None):
    with hsb.Solver(J) as s:
        spins, energy = s.run(p, R, steps, seed)
        x, y = s.get_state(R)
    sel = range(R) if rows is None else rows
    ref = oracle.run(J, _oparams(J, ev), steps, seed, sel, "f32")
    idx = list(sel)
    np.testing.assert_array_equal(x[idx], ref["x"])
    np.testing.assert_array_equal(y[idx], ref["y"])
    np.testing.assert_array_equal(spins[idx], ref["best_s"])
    np.testing.assert_array_equal(energy[idx], ref["best_e"])


@pytest.mark.parametrize("n,R", [(128, 256), (300, 200), (257, 130), (2, 129), (700, 500),
                                 (1100, 256), (2048, 256), (1999, 512), (129, 511), (3000, 256)])
def test_pair_schedule_bit_exact(n, R):
    J = synth.sk_pm1(n, 1000 + n)
    steps, seed, ev = 150, 7, 40
    p = hsb.params("discrete", "fp8", c1=0.7, dt=1.1, gamma=0.06, eval_every=ev,
                   schedule="pair")
    _check(J, p, R, steps, seed, ev)


@pytest.mark.parametrize("n,R,steps,ev", [
    (129, 129, 1, 0),     # one step, final evaluation only
    (129, 200, 37, 0),    # final evaluation only (the 700-spin protocol)
    (200, 256, 30, 100),  # evaluation cadence longer than the run
    (256, 129, 64, 1),    # evaluation at every step
])
def test_pair_schedule_edge_cases(n, R, steps, ev):
    J = synth.sk_pm1(n, 500 + n)
    p = hsb.params("discrete", "fp8", c1=0.7, dt=1.1, gamma=0.06, eval_every=ev,
                   schedule="pair")
    _check(J, p, R, steps, 21, ev)


def test_pair_schedule_diluted_couplings():
    n, R, steps, seed, ev = 500, 256, 120, 4, 30
    J = synth.sk_pm1(n, 8)
    rng = np.random.default_rng(8 + 99)
    keep = np.triu(rng.random((n, n)) >= 0.5, 1)
    keep = keep | keep.T
    J = np.where(keep, J, np.float32(0.0)).astype(np.float32)
    p = hsb.params("discrete", "fp8", c1=0.7, dt=1.1, gamma=0.06, eval_every=ev,
                   schedule="pair")
    _check(J, p, R, steps, seed, ev)


def test_pair_schedule_one_step_split_runs_and_device_advance():
    n, R, steps = 260, 200, 50
    J = synth.sk_pm1(n, 4)
    rng = np.random.default_rng(0)
    x0 = rng.uniform(-1, 1, (R, n)).astype(np.float32)
    y0 = rng.uniform(-1, 1, (R, n)).astype(np.float32)
    p = hsb.params("discrete", "fp8", c1=0.7, dt=1.1, gamma=0.06, schedule="pair")
    c0 = oracle.c0_from_c1(J, 0.7)
    with hsb.Solver(J) as s:
        x1, y1 = s.advance(p, steps, 10, 11, x0, y0)
        xr, yr, _ = oracle.step(J, x0, y0, 1, oracle.pump_factor(1.0, 10, steps), c0, 1.1,
                                1.0 * 1.1, 0.06 * 1.1, "f32")
        np.testing.assert_array_equal(x1, xr)
        np.testing.assert_array_equal(y1, yr)
        xa, ya = s.advance(p, steps, 0, steps, x0, y0)
        xb, yb = s.advance(p, steps, 0, 17, x0, y0)
        xb, yb = s.advance(p, steps, 17, steps, xb, yb)
        np.testing.assert_array_equal(xa, xb)
        np.testing.assert_array_equal(ya, yb)
        # the device-resident continuation (the bench's loop timing) equals
        # the host round trip
        s.run(p, R, steps, 3)
        xs, ys = s.get_state(R)
        s.advance_device(p, R, 2 * steps, steps, 2 * steps)
        s.synchronize()
        xd, yd = s.get_state(R)
        xh, yh = s.advance(p, 2 * steps, steps, 2 * steps, xs, ys)
        np.testing.assert_array_equal(xd, xh)
        np.testing.assert_array_equal(yd, yh)


def test_pair_schedule_equals_the_other_fp8_schedules_at_full_size():
    # N = 2000, R = 1024 (the benchmark's workload), 300 steps: the pair
    # kernel, the one-CTA persistent kernel and the per-step kernel agree
    J = synth.sk_pm1(2000, 1)
    R, steps, seed = 1024, 300, 3
    out = {}
    with hsb.Solver(J) as s:
        for sched in ("pair", "persistent", "per_step"):
            p = hsb.params("discrete", "fp8", c1=0.7, dt=1.1, gamma=0.06, eval_every=100,
                           schedule=sched)
            sp, en = s.run(p, R, steps, seed)
            x, y = s.get_state(R)
            out[sched] = (sp, en, x, y)
    for sched in ("persistent", "per_step"):
        for a, b in zip(out["pair"], out[sched]):
            np.testing.assert_array_equal(a, b)


def test_pair_schedule_is_refused_where_it_does_not_apply():
    J = synth.sk_pm1(300, 3)
    with hsb.Solver(J) as s:
        for R, kw in ((128, {}),                       # one 128-replica block: no pair
                      (256, {"trace_every": 1}),
                      (256, {"thermostat": "nose_hoover", "nh_T": 0.3, "nh_M": 6000.0})):
            with pytest.raises(hsb.HsbError) as e:
                s.run(hsb.params("discrete", "fp8", schedule="pair", **kw), R, 10, 0)
            assert e.value.status == hsb.HSB_E_UNSUPPORTED
    with hsb.Solver(synth.sk_pm1(4200, 0)) as s:   # more K chunks than poller lanes
        with pytest.raises(hsb.HsbError) as e:
            s.run(hsb.params("discrete", "fp8", schedule="pair"), 256, 4, 0)
        assert e.value.status == hsb.HSB_E_UNSUPPORTED
