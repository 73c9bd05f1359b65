"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle.

Discrete form with +/-1 couplings (FP8 and FP4 tensor cores, plain FP32): positions,
momenta, best spins and best energies equal the binary32 oracle bit for bit.
Plain FP32 for every form and coupling type: bit for bit as well (both sides
form the force with fused multiply-adds over j ascending).  Sizes span several
128 x 128 tiles with ragged spin and replica tails; the full-size workload
(N = 2000, R = 1024, 2000 steps, in the launch configuration the benchmark
times) is checked on sampled replicas.
"""
import numpy as np
import pytest

import oracle
import paper_2203_08361_gb300 as hsb
import synth

pytestmark = pytest.mark.gpu


def _oparams(J, form, c1, dt, gamma, eval_every, L=1.0, c0=None):
    c0 = oracle.c0_from_c1(J, c1) if c0 is None else c0
    return oracle.make_params(form, c0, dt, gamma, eval_every=eval_every, init_half_width=L)


def _assert_same(got_x, got_y, spins, energy, ref, rows=None):
    sel = slice(None) if rows is None else rows
    np.testing.assert_array_equal(got_x[sel], ref["x"])
    np.testing.assert_array_equal(got_y[sel], ref["y"])
    np.testing.assert_array_equal(spins[sel], ref["best_s"])
    np.testing.assert_array_equal(energy[sel], ref["best_e"])


@pytest.mark.parametrize("prec,schedule", [("fp8", "persistent"), ("fp8", "resident"),
                                           ("fp8", "per_step"), ("fp4", "per_step"), ("fp4", "persistent"),
                                           ("fp32", "auto")])
@pytest.mark.parametrize("n,R", [(128, 128), (300, 40), (257, 130), (2, 3), (700, 300),
                                 (1100, 130), (2048, 128)])
def test_discrete_pm1_bit_exact(prec, schedule, n, R):
    J = synth.sk_pm1(n, 1000 + n)
    steps, seed, ev = 150, 7, 40
    p = hsb.params("discrete", prec, c1=0.7, dt=1.1, gamma=0.06, eval_every=ev,
                   schedule=schedule)
    with hsb.Solver(J) as s:
        spins, energy = s.run(p, R, steps, seed)
        x, y = s.get_state(R)
        assert s.run_stats() >= 3
    ref = oracle.run(J, _oparams(J, 1, 0.7, 1.1, 0.06, ev), steps, seed, range(R), "f32")
    _assert_same(x, y, spins, energy, ref)


@pytest.mark.parametrize("form,gamma,c1", [("ballistic", 0.5, 0.9), ("discrete", 0.06, 0.7)])
def test_fp32_gaussian_bit_exact(form, gamma, c1):
    n, R, steps, seed, ev = 200, 50, 120, 3, 30
    J = synth.sk_gauss(n, 9)
    fcode = 0 if form == "ballistic" else 1
    p = hsb.params(form, "fp32", c1=c1, dt=1.1, gamma=gamma, eval_every=ev)
    with hsb.Solver(J) as s:
        spins, energy = s.run(p, R, steps, seed)
        x, y = s.get_state(R)
    ref = oracle.run(J, _oparams(J, fcode, c1, 1.1, gamma, ev), steps, seed, range(R), "f32")
    np.testing.assert_array_equal(x, ref["x"])
    np.testing.assert_array_equal(y, ref["y"])
    np.testing.assert_array_equal(spins, ref["best_s"])
    # binary64 energies of the same spins, summed in another order
    np.testing.assert_allclose(energy, ref["best_e"], rtol=1e-12, atol=1e-9)


def test_small_ballistic_pm1_workload_fp32():
    # HbSB on one +/-1 SK instance, N = 100, R = 64, x0, y0 in [-0.1, 0.1],
    # a0 = 1, c0 = 0.5 / sqrt(N) (sigma_J = 1), dt = 1, 2000 steps.
    n, R, steps, seed = 100, 64, 2000, 0
    J = synth.sk_pm1(n, 0)
    c0 = 0.5 / np.sqrt(n)
    p = hsb.params("ballistic", "fp32", c0=c0, dt=1.0, gamma=0.5, init_half_width=0.1,
                   eval_every=100)
    with hsb.Solver(J) as s:
        spins, energy = s.run(p, R, steps, seed)
        x, y = s.get_state(R)
    ref = oracle.run(J, _oparams(J, 0, 0, 1.0, 0.5, 100, L=0.1, c0=c0), steps, seed, range(R),
                     "f32")
    _assert_same(x, y, spins, energy, ref)
    e0 = oracle.run(J, _oparams(J, 0, 0, 1.0, 0.5, 100, L=0.1, c0=c0), steps, seed, range(R),
                    "f64")["best_e"]
    # binary32 and binary64 trajectories differ, their best energies stay close
    assert abs(np.mean(energy) - np.mean(e0)) < 0.05 * abs(np.mean(e0))


@pytest.mark.parametrize("prec,schedule", [("fp8", "persistent"), ("fp8", "resident"),
                                           ("fp8", "per_step"), ("fp4", "per_step"), ("fp4", "persistent"),
                                           ("fp32", "auto")])
def test_one_step_and_split_runs(prec, schedule):
    n, R, steps = 260, 70, 50
    J = synth.sk_pm1(n, 4)
    rng = np.random.default_rng(0)
    x0 = rng.uniform(-1, 1, (R, n)).astype(np.float32)
    y0 = rng.uniform(-1, 1, (R, n)).astype(np.float32)
    p = hsb.params("discrete", prec, c1=0.7, dt=1.1, gamma=0.06, schedule=schedule)
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


@pytest.mark.parametrize("prec", ["fp8", "fp4"])
@pytest.mark.parametrize("n", [2000, 16384])
def test_fp8_force_is_the_exact_integer_product(n, prec):
    # With a0 = 2^-40, c0 = 1, dt = 2^-20 and y = 0, one step leaves
    # y' = fl(fl(f - p x) dt) with |p x| < 2^-60, so round(y'/dt) = f, the force.
    # Replica 0 has x = 2^-30 J[0, :] (x_0 = 0 counts as +1), so f_0 = N - 1.
    J = synth.sk_pm1(n, 77)
    R = 2
    rng = np.random.default_rng(1)
    x0 = (rng.choice([-1.0, 1.0], size=(R, n)) * 2.0**-30).astype(np.float32)
    x0[0] = (J[0] * 2.0**-30).astype(np.float32)
    y0 = np.zeros((R, n), np.float32)
    p = hsb.params("discrete", prec, a0=2.0**-40, c0=1.0, dt=2.0**-20, gamma=0.0)
    with hsb.Solver(J) as s:
        x1, y1 = s.advance(p, 4, 0, 1, x0, y0)
    f = np.rint(y1.astype(np.float64) / 2.0**-20).astype(np.int64)
    s_ = np.where(x0 >= 0, 1, -1).astype(np.float32)
    # float32 sums of +/-1 terms below 2^24 are exact in any order
    want = np.rint(s_ @ J.T).astype(np.int64)
    np.testing.assert_array_equal(f, want)
    assert f[0, 0] == n - 1


def _config2():
    J = synth.sk_pm1(2000, 1)
    p = hsb.params("discrete", "fp8", c1=0.7, dt=1.1, gamma=0.06, init_half_width=1.0,
                   eval_every=100)
    return J, p


def test_full_size_discrete_workload_sampled_replicas():
    # N = 2000 +/-1 SK, R = 1024, 2000 steps, FP8 (the benchmark's workload and
    # launch configuration); replicas 0, 1, 513 and 1023 against the oracle.
    J, p = _config2()
    R, steps, seed = 1024, 2000, 1
    with hsb.Solver(J) as s:
        spins, energy = s.run(p, R, steps, seed)
        x, y = s.get_state(R)
        spins2, energy2 = s.run(p, R, steps, seed)
        np.testing.assert_array_equal(spins, spins2)
        np.testing.assert_array_equal(energy, energy2)
    rows = [0, 1, 513, 1023]
    ref = oracle.run(J, _oparams(J, 1, 0.7, 1.1, 0.06, 100), steps, seed, rows, "f32")
    _assert_same(x, y, spins, energy, ref, rows=rows)
    # plausibility for SK N = 2000: E / N^1.5 near -0.7 (ground state ~ -0.763)
    assert -0.78 < energy.min() / 2000**1.5 < -0.70


def test_full_size_fp8_equals_fp32_and_is_independent_of_R():
    J, p = _config2()
    steps, seed = 400, 2
    with hsb.Solver(J) as s:
        sa, ea = s.run(p, 1024, steps, seed)
        xa, ya = s.get_state(1024)
        p32 = hsb.params("discrete", "fp32", c1=0.7, dt=1.1, gamma=0.06, eval_every=100)
        sb, eb = s.run(p32, 1024, steps, seed)
        xb, yb = s.get_state(1024)
        pps = hsb.params("discrete", "fp8", c1=0.7, dt=1.1, gamma=0.06, eval_every=100,
                         schedule="per_step")
        sd, ed = s.run(pps, 1024, steps, seed)
        xd, yd = s.get_state(1024)
        pst = hsb.params("discrete", "fp8", c1=0.7, dt=1.1, gamma=0.06, eval_every=100,
                         schedule="resident")
        sg, eg = s.run(pst, 1024, steps, seed)
        xg, yg = s.get_state(1024)
        sc, ec = s.run(p, 8, steps, seed)
    for other_s, other_e, other_x, other_y in ((sb, eb, xb, yb), (sd, ed, xd, yd),
                                               (sg, eg, xg, yg)):
        np.testing.assert_array_equal(sa, other_s)
        np.testing.assert_array_equal(ea, other_e)
        np.testing.assert_array_equal(xa, other_x)
        np.testing.assert_array_equal(ya, other_y)
    np.testing.assert_array_equal(sa[:8], sc)
    np.testing.assert_array_equal(ea[:8], ec)


def test_run_device_set_couplings_and_advance_device():
    torch = pytest.importorskip("torch")
    n, R, steps = 300, 64, 100
    J1, J2 = synth.sk_pm1(n, 1), synth.sk_pm1(n, 2)
    p = hsb.params("discrete", "fp8", eval_every=25)
    with hsb.Solver(J1) as s:
        st = torch.cuda.Stream()
        s.set_stream(st.cuda_stream)
        spins = torch.empty((R, n), dtype=torch.int8, device="cuda")
        energy = torch.empty(R, dtype=torch.float64, device="cuda")
        s.run_device(p, R, steps, 5, spins.data_ptr(), energy.data_ptr())
        s.synchronize()
        hs, he = s.run(p, R, steps, 5)
        np.testing.assert_array_equal(spins.cpu().numpy(), hs)
        np.testing.assert_array_equal(energy.cpu().numpy(), he)
        # continuing on the device equals continuing on the host
        xs, ys = s.get_state(R)
        s.advance_device(p, R, 2 * steps, steps, 2 * steps)
        s.synchronize()
        xd, yd = s.get_state(R)
        xh, yh = s.advance(p, 2 * steps, steps, 2 * steps, xs, ys)
        np.testing.assert_array_equal(xd, xh)
        np.testing.assert_array_equal(yd, yh)
        s.set_couplings(J2)
        s2, e2 = s.run(p, R, steps, 5)
    with hsb.Solver(J2) as t:
        s3, e3 = t.run(p, R, steps, 5)
    np.testing.assert_array_equal(s2, s3)
    np.testing.assert_array_equal(e2, e3)


def test_unsupported_precision_and_argument_errors():
    G = synth.sk_gauss(64, 0)
    with hsb.Solver(G) as s:
        with pytest.raises(hsb.HsbError) as e:
            s.run(hsb.params("discrete", "fp8"), 4, 10, 0)
        assert e.value.status == 7
        with pytest.raises(hsb.HsbError) as e:
            s.run(hsb.params("discrete", "fp32"), 0, 10, 0)
        assert e.value.status == 1
    J = synth.sk_pm1(64, 0)
    with hsb.Solver(J) as s:
        with pytest.raises(hsb.HsbError) as e:
            s.run(hsb.params("ballistic", "fp8"), 4, 10, 0)
        assert e.value.status == 7
        # the per-step trace runs on the persistent and per-step schedules,
        # not on the resident-J one
        with pytest.raises(hsb.HsbError) as e:
            s.run(hsb.params("discrete", "fp8", trace_every=1, schedule="resident"), 4, 10, 0)
        assert e.value.status == 7
    # J held on chip needs N <= 2048
    with hsb.Solver(synth.sk_pm1(2100, 0)) as s:
        with pytest.raises(hsb.HsbError) as e:
            s.run(hsb.params("discrete", "fp8", schedule="resident"), 128, 4, 0)
        assert e.value.status == 7


def test_best_energy_bounded_by_ground_state():
    n = 16
    J = synth.sk_pm1(n, 31)
    e0, _ = oracle.brute_force(J)
    with hsb.Solver(J) as s:
        spins, energy = s.run(hsb.params("discrete", "fp8", eval_every=10), 256, 300, 3)
    assert np.all(energy >= e0)
    assert energy.min() == e0
    for r in range(0, 256, 37):
        assert oracle.ising_energy(J, spins[r]) == energy[r]


def _dilute_pm1(n, seed, p_zero=0.5):
    # +/-1 couplings with about half of the pairs removed (J_ij = 0): still
    # the FP8 path (0 is exact in e4m3), exact integer forces
    J = synth.sk_pm1(n, seed)
    rng = np.random.default_rng(seed + 99)
    keep = np.triu(rng.random((n, n)) >= p_zero, 1)
    keep = keep | keep.T
    return np.where(keep, J, np.float32(0.0)).astype(np.float32)


@pytest.mark.parametrize("prec,schedule", [("fp8", "persistent"), ("fp8", "per_step"),
                                           ("fp4", "per_step"), ("fp4", "persistent"), ("fp32", "auto")])
@pytest.mark.parametrize("n,R,steps,ev", [
    (129, 1, 1, 0),       # one replica, one step, final evaluation only
    (129, 1, 37, 0),      # final evaluation only (the 700-spin protocol)
    (200, 5, 30, 100),    # evaluation cadence longer than the run
    (256, 129, 64, 1),    # evaluation at every step
])
def test_edge_cases_bit_exact(prec, schedule, n, R, steps, ev):
    J = synth.sk_pm1(n, 500 + n)
    seed = 21
    p = hsb.params("discrete", prec, c1=0.7, dt=1.1, gamma=0.06, eval_every=ev,
                   schedule=schedule)
    with hsb.Solver(J) as s:
        spins, energy = s.run(p, R, steps, seed)
        x, y = s.get_state(R)
    ref = oracle.run(J, _oparams(J, 1, 0.7, 1.1, 0.06, ev), steps, seed, range(R), "f32")
    _assert_same(x, y, spins, energy, ref)


@pytest.mark.parametrize("prec,schedule", [("fp8", "persistent"), ("fp8", "per_step"),
                                           ("fp4", "per_step"), ("fp4", "persistent"), ("fp32", "auto")])
def test_diluted_couplings_bit_exact(prec, schedule):
    n, R, steps, seed, ev = 500, 70, 120, 4, 30
    J = _dilute_pm1(n, 8)
    assert 0.4 < np.mean(J == 0) < 0.6
    p = hsb.params("discrete", prec, c1=0.7, dt=1.1, gamma=0.06, eval_every=ev,
                   schedule=schedule)
    with hsb.Solver(J) as s:
        spins, energy = s.run(p, R, steps, seed)
        x, y = s.get_state(R)
    # c0 = c1 / (sqrt(N) sigma_J), sigma_J < 1 for diluted couplings
    ref = oracle.run(J, _oparams(J, 1, 0.7, 1.1, 0.06, ev), steps, seed, range(R), "f32")
    _assert_same(x, y, spins, energy, ref)


@pytest.mark.parametrize("n", [6000, 6500])
def test_general_couplings_final_energy_fixed_point_and_large_n(n):
    # the final binary64 energies of general couplings: fixed point up to
    # N of about 6300, one block per replica beyond; both within 1e-12 of the
    # oracle's binary64 sum of the returned spins
    J = synth.sk_gauss(n, 31)
    R, steps, seed = 32, 3, 2
    p = hsb.params("ballistic", "fp32", c1=0.9, dt=1.1, gamma=0.5, eval_every=0)
    with hsb.Solver(J) as s:
        spins, energy = s.run(p, R, steps, seed)
    for r in (0, 17, 31):
        assert energy[r] == pytest.approx(oracle.ising_energy(J, spins[r]), rel=1e-12)


def test_auto_schedule_falls_back_when_the_persistent_grid_does_not_fit():
    # N = 1024, R = 4096: 8 x 32 = 256 tiles of 128 x 128, more than the
    # co-resident grid of one CTA per SM, so AUTO runs one launch per step;
    # sampled replicas equal the oracle bit for bit and the run equals the
    # explicit per-step schedule
    n, R, steps, seed, ev = 1024, 4096, 30, 13, 10
    J = synth.sk_pm1(n, 77)
    p = hsb.params("discrete", "fp8", c1=0.7, dt=1.1, gamma=0.06, eval_every=ev)
    ps = hsb.params("discrete", "fp8", c1=0.7, dt=1.1, gamma=0.06, eval_every=ev,
                    schedule="per_step")
    with hsb.Solver(J) as s:
        spins, energy = s.run(p, R, steps, seed)
        assert s.run_stats() > steps  # one launch per step at least
        x, y = s.get_state(R)
        spins2, energy2 = s.run(ps, R, steps, seed)
        with pytest.raises(hsb.HsbError) as e:
            s.run(hsb.params("discrete", "fp8", schedule="persistent"), R, steps, seed)
        assert e.value.status == hsb.HSB_E_UNSUPPORTED
    np.testing.assert_array_equal(spins, spins2)
    np.testing.assert_array_equal(energy, energy2)
    rows = [0, 1, 2047, 4095]
    ref = oracle.run(J, _oparams(J, 1, 0.7, 1.1, 0.06, ev), steps, seed, rows, "f32")
    _assert_same(x, y, spins, energy, ref, rows=rows)


def test_set_couplings_across_coupling_classes():
    # one handle serving instances of different kinds: +/-1 (FP8), Gaussian
    # (BF16x3 and FP32, exact fixed-point final energies), +/-1 again; every
    # run equals a run on a fresh handle of the same instance
    n, R, steps, seed = 256, 128, 60, 3
    Ja, Jg, Jb = synth.sk_pm1(n, 4), synth.sk_gauss(n, 4), synth.sk_pm1(n, 5)
    pd = hsb.params("discrete", "auto", c1=0.7, dt=1.1, gamma=0.06, eval_every=20)
    pb = hsb.params("ballistic", "auto", c1=0.9, dt=1.1, gamma=0.5, eval_every=20)
    pf = hsb.params("ballistic", "fp32", c1=0.9, dt=1.1, gamma=0.5, eval_every=20)
    seq = [(Ja, pd), (Jg, pb), (Jg, pf), (Jb, pd), (Ja, pd)]
    got = []
    with hsb.Solver(Ja) as s:
        for J, p in seq:
            s.set_couplings(J)
            got.append(s.run(p, R, steps, seed))
    for (J, p), (sp, en) in zip(seq, got):
        with hsb.Solver(J) as t:
            sp2, en2 = t.run(p, R, steps, seed)
        np.testing.assert_array_equal(sp, sp2)
        np.testing.assert_array_equal(en, en2)
    # the cut values follow the current instance's sum of couplings
    with hsb.Solver(Ja) as s:
        s.set_couplings(Jg)
        c = s.cut_values(np.array([-10.0]))
    assert c[0] == pytest.approx(5.0 - 0.25 * float(Jg.astype(np.float64).sum()), rel=1e-15)
