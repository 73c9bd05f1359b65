"""GPU parity of the FP4 path (packed e2m1 J and sgn(x), tcgen05 kind::mxf4
with unit UE8M0 block scales, FP32 accumulation), on the persistent kernel
(the automatic choice where its grid fits) and one launch per step.

The products of +/-1 and 0 codes are exact, the per-instruction partial sums
are integers below 2^24, so the force equals the FP8 path's and the binary32
oracle's: positions, momenta, best spins, best energies, the per-step trace
and the Nose-Hoover friction all match bit for bit.  The FP4 tile holds 192
replicas, so the sizes here put replica tails on both sides of 192-row tile
edges, and N values whose K padding (N rounded up to 256 in e2m1 values)
exceeds the 128-spin padding of the other paths.
"""
import numpy as np
import pytest

import oracle
import paper_2203_08361_gb300 as hsb
import synth

pytestmark = pytest.mark.gpu


def _op(J, ev, c1=0.7, dt=1.1, gamma=0.06, **kw):
    return oracle.make_params(1, oracle.c0_from_c1(J, c1), dt, gamma, eval_every=ev, **kw)


def _run(s, prec, R, steps, seed, **kw):
    p = hsb.params("discrete", prec, c1=0.7, dt=1.1, gamma=0.06, **kw)
    sp, en = s.run(p, R, steps, seed)
    x, y = s.get_state(R)
    return sp, en, x, y


@pytest.mark.parametrize("n,R", [(300, 191), (300, 192), (300, 193), (513, 385), (130, 577),
                                 (256, 200), (2, 200)])
def test_fp4_ragged_replica_tiles_bit_exact(n, R):
    J = synth.sk_pm1(n, 40 + n)
    steps, seed, ev = 90, 5, 30
    with hsb.Solver(J) as s:
        sp, en, x, y = _run(s, "fp4", R, steps, seed, eval_every=ev)
    ref = oracle.run(J, _op(J, ev), steps, seed, range(R), "f32")
    np.testing.assert_array_equal(x, ref["x"])
    np.testing.assert_array_equal(y, ref["y"])
    np.testing.assert_array_equal(sp, ref["best_s"])
    np.testing.assert_array_equal(en, ref["best_e"])


def test_fp4_equals_fp8_at_full_size_and_sampled_replicas_match_the_oracle():
    # N = 2000, R = 1024 (the benchmark's workload), 300 steps: FP4 on the
    # persistent kernel and one launch per step, FP8 on both
    J = synth.sk_pm1(2000, 1)
    R, steps, seed = 1024, 300, 3
    with hsb.Solver(J) as s:
        a = _run(s, "fp4", R, steps, seed, eval_every=100, schedule="persistent")
        others = [_run(s, "fp4", R, steps, seed, eval_every=100, schedule="per_step"),
                  _run(s, "fp8", R, steps, seed, eval_every=100, schedule="per_step"),
                  _run(s, "fp8", R, steps, seed, eval_every=100, schedule="persistent")]
    for b in others:
        for u, v in zip(a, b):
            np.testing.assert_array_equal(u, v)
    rows = [0, 191, 192, 1023]
    ref = oracle.run(J, _op(J, 100), steps, seed, rows, "f32")
    np.testing.assert_array_equal(a[2][rows], ref["x"])
    np.testing.assert_array_equal(a[3][rows], ref["y"])
    np.testing.assert_array_equal(a[0][rows], ref["best_s"])
    np.testing.assert_array_equal(a[1][rows], ref["best_e"])


def test_fp4_large_instance_with_trace_equals_fp8():
    # N = 16384, R = 4096 (the large streamed instance), 12 steps with the
    # per-step trace.  The FP8 sign operand (67 MB) is walked in two replica
    # bands, the FP4 one (34 MB) in one: all replicas agree, and replicas at
    # both ends of each band match the oracle.
    J = synth.sk_pm1(16384, 3)
    R, steps, seed = 4096, 12, 2
    with hsb.Solver(J) as s:
        a = _run(s, "fp4", R, steps, seed, eval_every=5, trace_every=1)
        ta = s.get_trace()
        b = _run(s, "fp8", R, steps, seed, eval_every=5, trace_every=1, schedule="per_step")
        tb = s.get_trace()
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    np.testing.assert_array_equal(ta, tb)
    rows = [0, 2047, 2048, 4095]
    ref = oracle.run(J, _op(J, 5), steps, seed, rows, "f32", nthreads=0)
    np.testing.assert_array_equal(a[2][rows], ref["x"])
    np.testing.assert_array_equal(a[3][rows], ref["y"])
    np.testing.assert_array_equal(a[0][rows], ref["best_s"])
    np.testing.assert_array_equal(a[1][rows], ref["best_e"])


@pytest.mark.parametrize("n,R", [(700, 256), (2000, 1024), (257, 129)])
def test_fp4_persistent_trace_equals_fp8(n, R):
    J = synth.sk_pm1(n, 12)
    steps, seed = 120, 6
    with hsb.Solver(J) as s:
        a = _run(s, "fp4", R, steps, seed, eval_every=30, trace_every=1, schedule="persistent")
        ta = s.get_trace()
        b = _run(s, "fp8", R, steps, seed, eval_every=30, trace_every=1, schedule="persistent")
        tb = s.get_trace()
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    np.testing.assert_array_equal(ta, tb)


def test_fp4_nose_hoover_equals_fp8():
    J = synth.sk_pm1(700, 6)
    R, steps, seed = 256, 200, 8
    nh = dict(thermostat="nose_hoover", nh_T=0.3, nh_M=6000.0, nh_xi0=-0.05)
    with hsb.Solver(J) as s:
        a = _run(s, "fp4", R, steps, seed, eval_every=50, **nh)
        xa = s.get_xi(R)
        b = _run(s, "fp8", R, steps, seed, eval_every=50, schedule="per_step", **nh)
        xb = s.get_xi(R)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    np.testing.assert_array_equal(xa, xb)


def test_fp4_device_run_advance_and_set_couplings():
    n, R, steps = 400, 200, 60
    J = synth.sk_pm1(n, 9)
    p = hsb.params("discrete", "fp4", c1=0.7, dt=1.1, gamma=0.06, eval_every=20)
    with hsb.Solver(J) as s:
        # device continuation equals the host round trip
        s.run(p, R, steps, 3)
        xs, ys = s.get_state(R)
        s.advance_device(p, R, 2 * steps, steps, 2 * steps)
        s.synchronize()
        xd, yd = s.get_state(R)
        xh, yh = s.advance(p, 2 * steps, steps, 2 * steps, xs, ys)
        np.testing.assert_array_equal(xd, xh)
        np.testing.assert_array_equal(yd, yh)
        # new +/-1 couplings: the packed J is rebuilt
        J2 = synth.sk_pm1(n, 10)
        s.set_couplings(J2)
        sp, en = s.run(p, R, steps, 4)
        x, y = s.get_state(R)
        ref = oracle.run(J2, _op(J2, 20), steps, 4, range(R), "f32")
        np.testing.assert_array_equal(x, ref["x"])
        np.testing.assert_array_equal(en, ref["best_e"])
        # Gaussian couplings: FP4 no longer applies
        s.set_couplings(synth.sk_gauss(n, 11))
        with pytest.raises(hsb.HsbError) as e:
            s.run(p, R, steps, 4)
        assert e.value.status == hsb.HSB_E_UNSUPPORTED


def test_fp4_is_refused_where_it_does_not_apply():
    J = synth.sk_pm1(300, 3)
    with hsb.Solver(J) as s:
        for form, kw in (("ballistic", {}), ("discrete", {"schedule": "resident"}),
                         ("discrete", {"schedule": "pair"})):
            with pytest.raises(hsb.HsbError) as e:
                s.run(hsb.params(form, "fp4", **kw), 256, 10, 0)
            assert e.value.status == hsb.HSB_E_UNSUPPORTED
    with hsb.Solver(synth.sk_pm1(4200, 0)) as s:  # 33 row blocks: no persistent grid
        with pytest.raises(hsb.HsbError) as e:
            s.run(hsb.params("discrete", "fp4", schedule="persistent"), 128, 4, 0)
        assert e.value.status == hsb.HSB_E_UNSUPPORTED
    with hsb.Solver(synth.sk_gauss(300, 3)) as s:
        with pytest.raises(hsb.HsbError) as e:
            s.run(hsb.params("discrete", "fp4"), 64, 10, 0)
        assert e.value.status == hsb.HSB_E_UNSUPPORTED
