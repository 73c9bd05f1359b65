"""GPU parity of Nose-Hoover SB (Eqs. eq_NH1, eq_NH) against the CPU oracle.

The friction -xi_r y replaces the constant heating term; xi_r advances after
each step from S_r = sum_i y_i^2.  The oracle forms S by its definition: the
exact sum of the exact squares of the binary32 momenta, rounded once to
binary64.  The CUDA kernels form it from momenta rounded to multiples of
2^-24 (squares exact in 64-bit integers, an exact 128-bit sum, one rounding),
which does not depend on the order of the terms and differs from the exact
sum by at most 2^-24 sum_i |y_i| + N 2^-50.  So:
  - one step from the seeded state: positions, momenta, spins and energies
    equal the oracle's bit for bit, and xi(t_1) is within the bound that
    distance implies;
  - whole runs (the trajectories are chaotic, so a last-bit difference in xi
    grows): positions, momenta, xi, best spins and energies equal, bit for
    bit, the oracle run with the test double of the kernels' sum
    (nh_sum_q24), whose own pins fix it to its definition.
Runs on plain FP32 (any couplings) and on both FP8 schedules (+/-1
couplings): the persistent kernel, whose tiles exchange their sums of q^2
through a second set of flags each step, and the one-launch-per-step kernel
with a separate xi update, with ragged spin and replica tails.
"""
import numpy as np
import pytest

import oracle
import paper_2203_08361_gb300 as hsb
import synth

pytestmark = pytest.mark.gpu



def _nh(n):
    # M of order 20 N: the increments dt (S - N T) / M stay of order
    # dt (T_inst - T) / 20, so xi settles instead of driving |1 - xi dt| past 1
    return dict(nh_T=0.3, nh_M=20.0 * n, nh_xi0=-0.05)


def _nh_oracle(J, form, c1, dt, eval_every, trace_every=0, q24=True, **nh):
    # q24=True: S from the test double of the kernels' sum (whole runs);
    # q24=False: the plain definition (the oracle proper)
    c0 = oracle.c0_from_c1(J, c1)
    return oracle.make_params(form, c0, dt, 0.0, eval_every=eval_every, trace_every=trace_every,
                              nose_hoover=True, nh_sum_q24=q24, **nh)


@pytest.mark.parametrize("kind,form,prec,schedule,n,R", [
    ("pm1", "discrete", "fp8", "persistent", 1000, 300),
    ("pm1", "discrete", "fp8", "per_step", 257, 130),
    ("pm1", "discrete", "fp32", "auto", 300, 130),
    ("gauss", "ballistic", "fp32", "auto", 300, 130),
])
def test_nose_hoover_one_step_against_the_plain_definition(kind, form, prec, schedule, n, R):
    # One step from the seeded state: the update uses xi0, so x, y and the
    # evaluated spins and energies equal the plain oracle's bit for bit; xi_1
    # = xi0 + (dt/M)(S - N T) differs only through S.  The kernels' S lies
    # within D = 2^-24 sum |y_i| + N 2^-50 of the exact sum before its one
    # rounding, and the oracle's is the exact sum rounded once; the binary64
    # operations after it add at most an ulp each.
    J = synth.sk_pm1(n, 70 + n) if kind == "pm1" else synth.sk_gauss(n, 70 + n)
    fcode = 0 if form == "ballistic" else 1
    c1 = 0.7 if form == "discrete" else 0.9
    NH = _nh(n)
    p = hsb.params(form, prec, c1=c1, dt=1.1, eval_every=0, schedule=schedule,
                   thermostat="nose_hoover", **NH)
    with hsb.Solver(J) as s:
        spins, energy = s.run(p, R, 1, 9)
        x, y = s.get_state(R)
        xi = s.get_xi(R)
    ref = oracle.run(J, _nh_oracle(J, fcode, c1, 1.1, 0, q24=False, **NH), 1, 9, range(R),
                     "f32")
    np.testing.assert_array_equal(x, ref["x"])
    np.testing.assert_array_equal(y, ref["y"])
    np.testing.assert_array_equal(spins, ref["best_s"])
    if kind == "pm1":
        np.testing.assert_array_equal(energy, ref["best_e"])
    else:
        np.testing.assert_allclose(energy, ref["best_e"], rtol=1e-12, atol=1e-9)
    h = 1.1 / NH["nh_M"]
    NT = n * NH["nh_T"]
    y64 = ref["y"].astype(np.float64)
    S = (y64 * y64).sum(axis=1)
    D = 2.0**-24 * np.abs(y64).sum(axis=1) + n * 2.0**-50 + 2.0**-52 * S
    bound = h * (D + 2.0**-51 * (S + NT)) + 2.0**-51 * (np.abs(h * (S - NT)) + np.abs(xi))
    dev = np.abs(xi - ref["xi"])
    assert np.all(dev <= bound), (dev.max(), bound.min())
    # the bound is far below the step xi takes, so it tells a wrong S apart
    step = np.abs(ref["xi"] - NH["nh_xi0"])
    assert np.median(bound) < 1e-3 * np.median(step)


@pytest.mark.parametrize("kind,form,prec,schedule,n,R", [
    ("pm1", "discrete", "fp8", "persistent", 1000, 300),
    ("pm1", "discrete", "fp8", "persistent", 257, 130),
    ("pm1", "discrete", "fp8", "persistent", 4000, 256),
    ("pm1", "discrete", "fp8", "per_step", 1000, 300),
    ("pm1", "discrete", "fp8", "per_step", 257, 130),
    ("pm1", "discrete", "fp32", "auto", 300, 130),
    ("gauss", "ballistic", "fp32", "auto", 300, 130),
    ("gauss", "discrete", "fp32", "auto", 200, 40),
])
def test_nose_hoover_bit_exact(kind, form, prec, schedule, n, R):
    J = synth.sk_pm1(n, 40 + n) if kind == "pm1" else synth.sk_gauss(n, 40 + n)
    fcode = 0 if form == "ballistic" else 1
    c1 = 0.7 if form == "discrete" else 0.9
    steps, seed, ev, te = 200, 12, 50, 10
    NH = _nh(n)
    p = hsb.params(form, prec, c1=c1, dt=1.1, eval_every=ev, trace_every=te,
                   schedule=schedule, thermostat="nose_hoover", **NH)
    with hsb.Solver(J) as s:
        spins, energy = s.run(p, R, steps, seed)
        x, y = s.get_state(R)
        xi = s.get_xi(R)
        tr = s.get_trace()
        launches = s.run_stats()
    if schedule == "persistent":
        assert launches == 5  # init, xi init, the step loop, best selection, trace
    ref = oracle.run(J, _nh_oracle(J, fcode, c1, 1.1, ev, te, **NH), steps, seed, range(R),
                     "f32", want_trace=te > 0)
    np.testing.assert_array_equal(xi, ref["xi"])
    np.testing.assert_array_equal(x, ref["x"])
    np.testing.assert_array_equal(y, ref["y"])
    np.testing.assert_array_equal(spins, ref["best_s"])
    if kind == "pm1":
        np.testing.assert_array_equal(energy, ref["best_e"])
    else:
        np.testing.assert_allclose(energy, ref["best_e"], rtol=1e-12, atol=1e-9)
    # the thermostat acts: xi moved away from xi0 in every replica
    assert np.all(xi != NH["nh_xi0"])
    if te == 0:
        return
    # trace: minimum / mean energy and mean T_inst at t_k, k = 0, 10, ...;
    # exact integers for +/-1 couplings, binary32 force sums otherwise
    rt = 0.0 if kind == "pm1" else 1e-5
    np.testing.assert_allclose(tr[:, 0], ref["trace_e"].min(axis=0), rtol=rt, atol=1e-9)
    np.testing.assert_allclose(tr[:, 1], ref["trace_e"].mean(axis=0), rtol=max(rt, 1e-12),
                               atol=1e-9)
    np.testing.assert_allclose(tr[:, 2], ref["trace_t"].mean(axis=0), rtol=1e-6)


@pytest.mark.parametrize("prec,schedule", [("fp8", "persistent"), ("fp8", "per_step"),
                                           ("fp32", "per_step")])
def test_nose_hoover_large_mass_equals_constant_heating(prec, schedule):
    # With M = 1e300 the xi increments vanish below binary64 resolution, so a
    # run with xi0 = -gamma is the constant-gamma run, bit for bit.
    J = synth.sk_pm1(500, 5)
    R, steps, seed = 200, 150, 3
    heat = hsb.params("discrete", prec, c1=0.7, dt=1.1, gamma=0.06, eval_every=30,
                      schedule=schedule)
    nh = hsb.params("discrete", prec, c1=0.7, dt=1.1, eval_every=30, schedule=schedule,
                    thermostat="nose_hoover", nh_T=0.3, nh_M=1e300, nh_xi0=-0.06)
    with hsb.Solver(J) as s:
        sa, ea = s.run(heat, R, steps, seed)
        xa, ya = s.get_state(R)
        sb, eb = s.run(nh, R, steps, seed)
        xb, yb = s.get_state(R)
        xi = s.get_xi(R)
    np.testing.assert_array_equal(sa, sb)
    np.testing.assert_array_equal(ea, eb)
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(ya, yb)
    np.testing.assert_array_equal(xi, np.full(R, -0.06))


def test_nose_hoover_argument_checks():
    J = synth.sk_pm1(256, 1)
    G = synth.sk_gauss(256, 1)
    nh = dict(thermostat="nose_hoover", **_nh(256))
    with hsb.Solver(J) as s:
        with pytest.raises(hsb.HsbError) as e:
            s.run(hsb.params("discrete", "fp8", schedule="resident", **nh), 128, 10, 0)
        assert e.value.status == hsb.HSB_E_UNSUPPORTED
        with pytest.raises(hsb.HsbError) as e:
            s.run(hsb.params("discrete", "fp8", thermostat="nose_hoover", nh_M=0.0), 128, 10, 0)
        assert e.value.status == hsb.HSB_E_INVAL
        with pytest.raises(hsb.HsbError) as e:
            s.run(hsb.params("discrete", "fp8", thermostat=2), 128, 10, 0)
        assert e.value.status == hsb.HSB_E_INVAL
        x0 = np.zeros((4, 256), np.float32)
        with pytest.raises(hsb.HsbError) as e:
            s.advance(hsb.params("discrete", "fp32", **nh), 10, 0, 5, x0, x0)
        assert e.value.status == hsb.HSB_E_UNSUPPORTED
        # xi exists only after a Nose-Hoover run, for its replica count
        s.run(hsb.params("discrete", "fp8", gamma=0.06), 128, 10, 0)
        with pytest.raises(hsb.HsbError):
            s.get_xi(128)
        s.run(hsb.params("discrete", "fp8", **nh), 128, 10, 0)
        assert s.get_xi(128).shape == (128,)
        with pytest.raises(hsb.HsbError):
            s.get_xi(64)
    with hsb.Solver(G) as s:
        with pytest.raises(hsb.HsbError) as e:
            s.run(hsb.params("ballistic", "bf16x3", **nh), 128, 10, 0)
        assert e.value.status == hsb.HSB_E_UNSUPPORTED
        # AUTO picks plain FP32 for general couplings under the thermostat
        s.run(hsb.params("ballistic", "auto", **nh), 128, 10, 0)
        assert s.get_xi(128).shape == (128,)


def test_nose_hoover_full_size_workload_sampled_replicas():
    # the benchmarked Nose-Hoover workload (N = 2000, R = 1024, 2000 steps,
    # T = 0.3, M = 40000, xi0 = -0.05, persistent FP8) in its launch
    # configuration: replicas 0 and 1023 equal the oracle bit for bit,
    # spins, best energy, final state and xi
    J = synth.sk_pm1(2000, 1)
    R, steps, seed = 1024, 2000, 1000
    nh = dict(nh_T=0.3, nh_M=40000.0, nh_xi0=-0.05)
    p = hsb.params("discrete", "fp8", c1=0.7, dt=1.1, eval_every=100,
                   thermostat="nose_hoover", **nh)
    with hsb.Solver(J) as s:
        spins, energy = s.run(p, R, steps, seed)
        x, y = s.get_state(R)
        xi = s.get_xi(R)
    rows = [0, 1023]
    ref = oracle.run(J, _nh_oracle(J, 1, 0.7, 1.1, 100, **nh), steps, seed, rows, "f32")
    np.testing.assert_array_equal(spins[rows], ref["best_s"])
    np.testing.assert_array_equal(energy[rows], ref["best_e"])
    np.testing.assert_array_equal(x[rows], ref["x"])
    np.testing.assert_array_equal(y[rows], ref["y"])
    np.testing.assert_array_equal(xi[rows], ref["xi"])
