"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: values worked
out by hand from the Methods equations (tests/golden), the MAX-CUT identity of
Eq. (eq_Cut), exhaustive enumeration, published SplitMix64 outputs, the
conserved quadratic form of the symplectic-Euler map (per eigenmode of J), the
closed-form linear map of the heated update without walls, the gamma = 0
reduction to plain bSB / dSB and the wall invariants.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


# ------------------------------------------------------------------ RNG ----

def test_splitmix64_published_outputs():
    # First four outputs of SplitMix64 seeded with 0, as published with the
    # generator's reference implementation (Steele, Lea & Flood 2014 / Vigna).
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [oracle.splitmix64(0, n) for n in (1, 2, 3, 4)] == want


def test_init_values_open_interval_and_grid():
    x, y = oracle.init_values(7, 0, range(4), 500, 1.0)
    for a in (x, y):
        assert np.all(np.abs(a) < 1.0)
        # L = 1: values are odd multiples of 2^-24
        k = a.astype(np.float64) * 2.0**24
        assert np.all(k == np.round(k))
        assert np.all(np.mod(np.round(k), 2) == 1)
    x2, _ = oracle.init_values(7, 0, range(2), 500, 0.1)
    assert np.all(np.abs(x2) < 0.1)


def test_init_values_uniform():
    scipy_stats = pytest.importorskip("scipy.stats")
    x, y = oracle.init_values(11, 3, range(8), 1000, 1.0)
    v = np.concatenate([x.ravel(), y.ravel()]).astype(np.float64)
    res = scipy_stats.kstest(v, "uniform", args=(-1.0, 2.0))
    assert res.pvalue > 1e-3
    # different streams (seed, instance, replica, component) differ
    x3, _ = oracle.init_values(11, 4, range(1), 1000, 1.0)
    assert not np.array_equal(x3[0], x[0])
    assert not np.array_equal(x[0], y[0])


# --------------------------------------------------------------- energy ----

def test_energy_hand_values_and_cut_identity():
    g = _golden("worked_steps.json")["energies"]
    for case in g["cases"]:
        J = np.array(case["J"], np.float32)
        for s, e, c in zip(case["states"], case["E"], case["C"]):
            s = np.array(s, np.int8)
            assert oracle.ising_energy(J, s) == e
            assert oracle.cut_value(J, s) == c
        e0, _ = oracle.brute_force(J)
        assert e0 == case["E_ground"]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_energy_equals_cut_relation(seed):
    # Eq. (eq_Cut): C = -E/2 - (1/4) sum_ij J_ij, with C counted edge by edge.
    J = synth.sk_gauss(9, seed)
    rng = np.random.default_rng(seed)
    for _ in range(5):
        s = rng.choice(np.array([-1, 1], np.int8), size=9)
        cut = 0.0
        for i in range(9):
            for j in range(9):
                if s[i] != s[j]:
                    cut += -float(J[i, j]) / 2.0  # w_ij counted from both ends, halved
        E = oracle.ising_energy(J, s)
        assert E == pytest.approx(-2.0 * (cut + 0.25 * float(J.astype(np.float64).sum())), abs=1e-9)
        assert oracle.cut_value(J, s) == pytest.approx(cut, abs=1e-9)


def test_energy_single_flip_identity():
    # Flipping spin i changes E by 2 s_i h_i with the local field h_i = sum_j J_ij s_j.
    J = synth.sk_pm1(15, 4)
    rng = np.random.default_rng(4)
    s = rng.choice(np.array([-1, 1], np.int8), size=15)
    E = oracle.ising_energy(J, s)
    for i in range(15):
        h = float(J[i].astype(np.float64) @ s.astype(np.float64))
        t = s.copy()
        t[i] = -t[i]
        assert oracle.ising_energy(J, t) - E == 2.0 * s[i] * h


@pytest.mark.parametrize("n,seed", [(6, 0), (9, 1), (11, 2)])
def test_brute_force_matches_python_enumeration(n, seed):
    J = synth.sk_pm1(n, seed)
    best = math.inf
    for bits in itertools.product((1, -1), repeat=n):
        s = np.array(bits, np.float64)
        # number of unsatisfied bonds form: E = sum_{i<j} -J_ij s_i s_j
        e = 0.0
        for i in range(n):
            for j in range(i + 1, n):
                e -= float(J[i, j]) * s[i] * s[j]
        best = min(best, e)
    e0, s0 = oracle.brute_force(J)
    assert e0 == best
    assert oracle.ising_energy(J, s0) == e0


# ---------------------------------------------------------- worked steps ---

@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_worked_steps(precision):
    g = _golden("worked_steps.json")
    for case in g["cases"]:
        J = np.array(case["J"], np.float32)
        x1, y1, f = oracle.step(J, case["x"], case["y"], case["form"], case["pk"], case["c0"],
                                case["dt"], case["q"], case["g"], precision)
        tol = case.get("tolerance", 0.0)
        if precision == "f32" and tol:
            tol = 1e-6
        np.testing.assert_allclose(f[0], case["f"], rtol=0, atol=tol, err_msg=case["name"])
        np.testing.assert_allclose(x1[0], case["x_next"], rtol=0, atol=tol, err_msg=case["name"])
        np.testing.assert_allclose(y1[0], case["y_next"], rtol=0, atol=tol, err_msg=case["name"])


def _round_f32(q):
    """The binary32 value nearest to the rational q, ties to even."""
    from fractions import Fraction
    x = np.float32(float(q))  # within one binary32 ulp of q
    cands = [np.nextafter(x, np.float32(-np.inf)), x, np.nextafter(x, np.float32(np.inf))]
    return min(cands, key=lambda c: (abs(Fraction(float(c)) - q),
                                     int(np.array(c, np.float32).view(np.uint32)) & 1))


def test_binary32_force_is_one_rounding_per_term_j_ascending():
    # The binary32 reading of f_i = sum_j J_ij b_j (Eq. eq_fb): acc <- the
    # binary32 value nearest to J_ij b_j + acc (a fused multiply-add), j
    # ascending.  Checked against exact rational arithmetic.
    from fractions import Fraction as F
    n, R = 24, 2
    J = synth.sk_gauss(n, 7)
    x = np.random.default_rng(7).uniform(-1, 1, (R, n)).astype(np.float32)
    _, _, f = oracle.step(J, x, np.zeros_like(x), 0, 0.0, 1.0, 1.0, 0.0, 0.0, "f32")
    differs = False
    for r in range(R):
        for i in range(n):
            acc = two = np.float32(0)
            for j in range(n):
                acc = _round_f32(F(float(J[i, j])) * F(float(x[r, j])) + F(float(acc)))
                two = np.float32(two + np.float32(J[i, j] * x[r, j]))  # two roundings
            assert f[r, i] == acc, (r, i)
            differs |= bool(two != acc)
    assert differs  # the two readings are told apart on this input


def test_binary32_update_rounds_each_operation_in_the_stated_order():
    # The binary32 reading of one update (Methods, Eqs. eq_SyEuY, eq_SyEuX,
    # eq_WallX, eq_WallY, eq_EuHeat): u = c0 f, v = p x, w = u - v,
    # y~ = y + w dt, x~ = x + q y~, the walls, y' = y~~ + g y, every operation
    # rounded once to binary32.  Checked against exact rational arithmetic.
    from fractions import Fraction as F

    def r32(v):
        return F(float(_round_f32(v)))

    n, R = 16, 4
    J = synth.sk_gauss(n, 9)
    rng = np.random.default_rng(9)
    x = rng.uniform(-0.9, 0.9, (R, n)).astype(np.float32)
    y = rng.uniform(-0.5, 0.5, (R, n)).astype(np.float32)
    pk, c0, dt, q, g = 0.7, 0.37, 0.45, 0.45, 0.03
    x1, y1, f = oracle.step(J, x, y, 0, pk, c0, dt, q, g, "f32")
    P, C0, DT, Q, G = (F(float(np.float32(v))) for v in (pk, c0, dt, q, g))
    differs, walls = False, 0
    for r in range(R):
        for i in range(n):
            x0, y0, fi = F(float(x[r, i])), F(float(y[r, i])), F(float(f[r, i]))
            u, v = r32(C0 * fi), r32(P * x0)
            w = r32(u - v)
            yt = r32(y0 + r32(w * DT))
            xt = r32(x0 + r32(Q * yt))
            if abs(xt) > 1:
                xn, ytt = F(1 if xt > 0 else -1), F(0)
                walls += 1
            else:
                xn, ytt = xt, yt
            yn = r32(ytt + r32(G * y0))
            assert (F(float(x1[r, i])), F(float(y1[r, i]))) == (xn, yn), (r, i)
            # an algebraically equal order, u dt - v dt, rounds differently
            differs |= r32(y0 + r32(r32(u * DT) - r32(v * DT))) != yt
    assert differs and walls > 0


# ------------------------------------------------------- dynamics pins ----

def _modes(J):
    lam, V = np.linalg.eigh(J.astype(np.float64))
    return lam, V


def test_quadratic_form_conserved_per_eigenmode():
    # gamma = 0, constant p, no wall hit: in eigenmode m of J the update is the
    # symplectic Euler map of a harmonic oscillator with P_m = (p - c0 lam_m) dt
    # and q = a0 dt, which conserves P x^2 + q y^2 - P q x y exactly.
    n = 8
    J = synth.sk_pm1(n, 5)
    lam, V = _modes(J)
    p, c0, dt, a0 = 1.0, 0.03, 0.5, 1.0
    q = a0 * dt
    P = (p - c0 * lam) * dt
    assert np.all(P > 0) and np.all(P * q < 4)
    rng = np.random.default_rng(0)
    x = rng.uniform(-0.01, 0.01, n)
    y = rng.uniform(-0.01, 0.01, n)

    def Q(x, y):
        xm, ym = V.T @ x, V.T @ y
        return P * xm**2 + q * ym**2 - P * q * xm * ym

    q0 = Q(x, y)
    for _ in range(300):
        x, y, _ = oracle.step(J, x, y, 0, p, c0, dt, q, 0.0, "f64")
        x, y = x[0], y[0]
        assert np.max(np.abs(x)) < 1.0
    np.testing.assert_allclose(Q(x, y), q0, rtol=1e-11, atol=0)
    # A sign error on the force would make P_m = (p + c0 lam_m) dt: not conserved.
    Pw = (p + c0 * lam) * dt
    xm, ym = V.T @ x, V.T @ y
    assert not np.allclose(Pw * xm**2 + q * ym**2 - Pw * q * xm * ym, q0, rtol=1e-6)


def test_heated_update_is_linear_map_per_eigenmode():
    # Without walls, one heated step maps each eigenmode (x_m, y_m) by
    # [[1 - q P_m, q], [-P_m, 1 + g]] with g = gamma dt (Eqs. eq_SyEuY,
    # eq_SyEuX, eq_EuHeat).
    n = 7
    J = synth.sk_gauss(n, 3)
    lam, V = _modes(J)
    p, c0, dt, a0, gamma = 0.8, 0.05, 0.7, 1.0, 0.3
    q, g = a0 * dt, gamma * dt
    rng = np.random.default_rng(1)
    x = rng.uniform(-1e-3, 1e-3, n)
    y = rng.uniform(-1e-3, 1e-3, n)
    xm, ym = V.T @ x, V.T @ y
    steps = 25
    for _ in range(steps):
        x, y, _ = oracle.step(J, x, y, 0, p, c0, dt, q, g, "f64")
        x, y = x[0], y[0]
    assert np.max(np.abs(x)) < 1.0
    for m in range(n):
        Pm = (p - c0 * lam[m]) * dt
        M = np.array([[1 - q * Pm, q], [-Pm, 1 + g]])
        want = np.linalg.matrix_power(M, steps) @ np.array([xm[m], ym[m]])
        got = np.array([V[:, m] @ x, V[:, m] @ y])
        np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-15)


def test_two_spin_normal_modes():
    # N = 2, J12 = 1: u = x1 + x2 and v = x1 - x2 decouple with
    # P_u = (p - c0) dt and P_v = (p + c0) dt (eigenvalues +1 and -1 of J).
    J = np.array([[0, 1], [1, 0]], np.float32)
    p, c0, dt, gamma = 0.6, 0.2, 0.9, 0.1
    q, g = dt, gamma * dt
    x = np.array([0.01, -0.003])
    y = np.array([-0.002, 0.004])
    u0 = np.array([x[0] + x[1], y[0] + y[1]])
    v0 = np.array([x[0] - x[1], y[0] - y[1]])
    steps = 12
    for _ in range(steps):
        x, y, _ = oracle.step(J, x, y, 0, p, c0, dt, q, g, "f64")
        x, y = x[0], y[0]
    for P, m0, got in (((p - c0) * dt, u0, [x[0] + x[1], y[0] + y[1]]),
                       ((p + c0) * dt, v0, [x[0] - x[1], y[0] - y[1]])):
        M = np.array([[1 - q * P, q], [-P, 1 + g]])
        np.testing.assert_allclose(got, np.linalg.matrix_power(M, steps) @ m0, rtol=1e-10)


def test_heating_uses_momentum_before_the_step():
    # Eq. (eq_EuHeat): y(t_{k+1}) = y~~ + gamma y(t_k) dt; the heated and the
    # plain (gamma = 0) step from the same state differ in y by g*y(t_k) only.
    J = synth.sk_gauss(10, 8)
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, (3, 10))
    y = rng.uniform(-1, 1, (3, 10))
    args = (0, 0.4, 0.3, 1.1, 1.1)
    xh, yh, _ = oracle.step(J, x, y, *args, 0.25, precision="f64")
    xp, yp, _ = oracle.step(J, x, y, *args, 0.0, precision="f64")
    np.testing.assert_array_equal(xh, xp)
    np.testing.assert_allclose(yh - yp, 0.25 * y, rtol=1e-12, atol=1e-15)


def _plain_sb_f32(J, x, y, steps, c0, dt, a0, form):
    """Plain bSB / dSB (no heating) as in Goto et al. 2021, written with numpy
    float32 element-wise operations; the discrete force of +/-1 couplings is an
    exact integer product."""
    x = x.astype(np.float32).copy()
    y = y.astype(np.float32).copy()
    c0 = np.float32(c0)
    dtf = np.float32(dt)
    q = np.float32(a0 * dt)
    Ji = J.astype(np.int64)
    for k in range(steps):
        pk = np.float32(a0 - (a0 * k) / steps)
        if form == 1:
            s = np.where(x >= 0, 1, -1).astype(np.int64)
            f = (s @ Ji.T).astype(np.float32)
        else:
            raise NotImplementedError
        ynew = y + (c0 * f - pk * x) * dtf
        xnew = x + q * ynew
        hit = np.abs(xnew) > 1
        xnew = np.where(hit, np.sign(xnew), xnew).astype(np.float32)
        ynew = np.where(hit, np.float32(0), ynew).astype(np.float32)
        x, y = xnew, ynew
    return x, y


@pytest.mark.parametrize("a0,steps", [(1.0, 150), (0.73, 5)])
def test_gamma_zero_reduces_to_plain_dsb_bit_exact(a0, steps):
    # a0 != 1 also fixes q = a0 dt and p_k as binary64 values rounded once
    # (with a0 = 0.73 and dt = 1.1, rounding a0 and dt first gives another q;
    # after 5 steps most spins are still inside the walls, which erase it)
    n, reps = 40, [0, 3, 9]
    J = synth.sk_pm1(n, 12)
    c0 = oracle.c0_from_c1(J, 0.6)
    prm = oracle.make_params(1, c0, 1.1, 0.0, a0=a0, eval_every=0)
    out = oracle.run(J, prm, steps, 77, reps, "f32")
    x0, y0 = oracle.init_values(77, 0, reps, n, 1.0)
    xp, yp = _plain_sb_f32(J, x0, y0, steps, c0, 1.1, a0, 1)
    np.testing.assert_array_equal(out["x"], xp)
    np.testing.assert_array_equal(out["y"], yp)


def test_gamma_zero_reduces_to_plain_bsb_f64():
    # Plain bSB in binary64 with Python loops in the same summation order.
    n, steps = 6, 60
    J = synth.sk_gauss(n, 13)
    c0, dt, a0 = 0.3, 0.7, 1.0
    prm = oracle.make_params(0, c0, dt, 0.0, eval_every=0)
    out = oracle.run(J, prm, steps, 5, [2], "f64")
    x0, y0 = oracle.init_values(5, 0, [2], n, 1.0)
    x = [float(v) for v in x0[0]]
    y = [float(v) for v in y0[0]]
    Jd = J.astype(np.float64)
    for k in range(steps):
        pk = a0 - (a0 * k) / steps
        f = []
        for i in range(n):
            acc = 0.0
            for j in range(n):
                acc = acc + float(Jd[i, j]) * x[j]
            f.append(acc)
        for i in range(n):
            yt = y[i] + (c0 * f[i] - pk * x[i]) * dt
            xt = x[i] + (a0 * dt) * yt
            if abs(xt) > 1:
                x[i], y[i] = math.copysign(1.0, xt), 0.0
            else:
                x[i], y[i] = xt, yt
    np.testing.assert_array_equal(out["x"][0], np.array(x))
    np.testing.assert_array_equal(out["y"][0], np.array(y))


def test_wall_invariants_along_a_trajectory():
    n = 30
    J = synth.sk_pm1(n, 21)
    c0 = oracle.c0_from_c1(J, 0.9)
    dt, a0, gamma = 1.1, 1.0, 0.5
    q, g = a0 * dt, gamma * dt
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, (2, n))
    y = rng.uniform(-1, 1, (2, n))
    steps, clamps = 200, 0
    for k in range(steps):
        pk = oracle.pump_factor(a0, k, steps)
        x1, y1, f = oracle.step(J, x, y, 0, pk, c0, dt, q, g, "f64")
        assert np.all(np.abs(x1) <= 1.0)
        # recompute the unclamped position to find the clamped spins
        yt = y + (c0 * f - pk * x) * dt
        xt = x + q * yt
        hit = np.abs(xt) > 1
        clamps += int(hit.sum())
        assert np.all(np.abs(x1[hit]) == 1.0)
        assert np.all(np.sign(x1[hit]) == np.sign(xt[hit]))
        np.testing.assert_allclose(y1[hit], g * y[hit], rtol=0, atol=0)
        x, y = x1, y1
    assert clamps > 0


# -------------------------------------------------------- run protocol ----

def test_replica_independence_and_determinism():
    n, steps = 50, 300
    J = synth.sk_pm1(n, 2)
    c0 = oracle.c0_from_c1(J, 0.7)
    prm = oracle.make_params(1, c0, 1.1, 0.06, eval_every=50)
    a = oracle.run(J, prm, steps, 123, range(6), "f32", nthreads=1)
    b = oracle.run(J, prm, steps, 123, [4, 1], "f32", nthreads=2)
    c = oracle.run(J, prm, steps, 123, range(6), "f32", nthreads=4)
    for key in ("x", "y", "best_s", "best_e"):
        np.testing.assert_array_equal(a[key][[4, 1]], b[key])
        np.testing.assert_array_equal(a[key], c[key])
    d = oracle.run(J, prm, steps, 124, range(6), "f32")
    assert not np.array_equal(a["x"], d["x"])


def test_int_force_shortcut_equals_plain_sum():
    n, steps = 64, 120
    J = synth.sk_pm1(n, 6)
    c0 = oracle.c0_from_c1(J, 0.7)
    for prec in ("f32", "f64"):
        fast = oracle.run(J, oracle.make_params(1, c0, 1.1, 0.06, eval_every=20), steps, 9,
                          range(4), prec)
        slow = oracle.run(J, oracle.make_params(1, c0, 1.1, 0.06, eval_every=20,
                                                force_plain_sum=True), steps, 9, range(4), prec)
        for key in ("x", "y", "best_s", "best_e"):
            np.testing.assert_array_equal(fast[key], slow[key])


def test_best_tracking_and_eval_cadence():
    n, steps, ev = 40, 400, 100
    J = synth.sk_pm1(n, 3)
    c0 = oracle.c0_from_c1(J, 0.7)
    prm = oracle.make_params(1, c0, 1.1, 0.06, eval_every=ev)
    out = oracle.run(J, prm, steps, 3, range(5), "f32", want_trace=True)
    tr = out["e_trace"]
    assert tr.shape == (5, 4)  # t = 100, 200, 300, 400
    np.testing.assert_array_equal(out["best_e"], tr.min(axis=1))
    for r in range(5):
        assert oracle.ising_energy(J, out["best_s"][r]) == out["best_e"][r]
        # the final evaluation is sgn(x(t_Ns))
        s_fin = np.where(out["x"][r] >= 0, 1, -1).astype(np.int8)
        assert oracle.ising_energy(J, s_fin) == tr[r, -1]
    last = oracle.run(J, oracle.make_params(1, c0, 1.1, 0.06, eval_every=0), steps, 3,
                      range(5), "f32")
    np.testing.assert_array_equal(last["best_e"], tr[:, -1])


def test_best_state_ties_keep_the_earliest_evaluation():
    # J = 0: every evaluation has E = 0 while the spins keep turning (the
    # pumped oscillator of each x_i), so a new best needing a strictly lower
    # energy keeps the spins of the first evaluation step t = eval_every.
    n, steps, ev, a0, dt, c0 = 16, 300, 50, 1.0, 0.5, 0.3
    J = np.zeros((n, n), np.float32)
    out = oracle.run(J, oracle.make_params(1, c0, dt, 0.0, a0=a0, eval_every=ev), steps, 5,
                     range(4), "f64")
    x, y = oracle.init_values(5, 0, range(4), n, 1.0)
    for k in range(ev):
        x, y, _ = oracle.step(J, x, y, 1, oracle.pump_factor(a0, k, steps), c0, dt, a0 * dt,
                              0.0, "f64")
    s_first = np.where(x >= 0, 1, -1).astype(np.int8)
    s_last = np.where(out["x"] >= 0, 1, -1).astype(np.int8)
    assert np.any(s_first != s_last)
    np.testing.assert_array_equal(out["best_e"], 0.0)
    np.testing.assert_array_equal(out["best_s"], s_first)


@pytest.mark.parametrize("form,gamma", [(1, 0.06), (0, 0.5)])
def test_small_instances_reach_brute_force_ground_state(form, gamma):
    n = 14
    J = synth.sk_pm1(n, 30)
    e0, _ = oracle.brute_force(J)
    c0 = oracle.c0_from_c1(J, 0.7 if form else 0.9)
    prm = oracle.make_params(form, c0, 1.1, gamma, eval_every=10)
    out = oracle.run(J, prm, 300, 1, range(32), "f64")
    assert np.all(out["best_e"] >= e0)
    assert out["best_e"].min() == e0


def test_pump_schedule_and_c0():
    assert oracle.pump_factor(1.0, 0, 2000) == 1.0
    assert oracle.pump_factor(1.0, 1000, 2000) == 0.5
    assert oracle.pump_factor(1.0, 1999, 2000) == pytest.approx(1 / 2000, rel=1e-12)
    J = synth.sk_pm1(100, 0)
    assert oracle.sigma_j(J) == 1.0
    assert oracle.c0_from_c1(J, 0.5) == 0.5 / 10.0
    G = synth.sk_gauss(300, 0)
    s = oracle.sigma_j(G)
    assert 0.9 < s < 1.1


def test_trace_energy_and_instantaneous_temperature():
    # Eq. (eq_TInst): T_inst = (1/N) sum_i y_i^2; at t_0 it is the mean square
    # of the initial momenta; traced energies at evaluation times equal the
    # evaluation energies.
    n, steps = 40, 120
    J = synth.sk_pm1(n, 8)
    c0 = oracle.c0_from_c1(J, 0.7)
    prm = oracle.make_params(1, c0, 1.1, 0.06, eval_every=30, trace_every=10)
    out = oracle.run(J, prm, steps, 4, range(3), "f64", want_trace=True)
    assert out["trace_e"].shape == (3, 12)
    _, y0 = oracle.init_values(4, 0, range(3), n, 1.0)
    np.testing.assert_allclose(out["trace_t"][:, 0], (y0.astype(np.float64) ** 2).mean(axis=1),
                               rtol=1e-14)
    x0, _ = oracle.init_values(4, 0, range(3), n, 1.0)
    for r in range(3):
        s0 = np.where(x0[r] >= 0, 1, -1).astype(np.int8)
        assert out["trace_e"][r, 0] == oracle.ising_energy(J, s0)
    # evaluations at t = 30, 60, 90 are traced at indices 3, 6, 9
    np.testing.assert_array_equal(out["trace_e"][:, [3, 6, 9]], out["e_trace"][:, :3])
    # a period that does not divide N_s: the traced times are k = 0, 10, ..., 120 < 125
    # (the count is checked first: the trace buffers are sized by it)
    assert oracle.num_traced(125, 10) == len(range(0, 125, 10)) == 13
    assert oracle.num_traced(120, 10) == 12 and oracle.num_traced(5, 1) == 5
    prm = oracle.make_params(1, c0, 1.1, 0.06, eval_every=120, trace_every=10)
    out = oracle.run(J, prm, 125, 4, range(3), "f64", want_trace=True)
    assert out["trace_e"].shape == (3, 13)
    np.testing.assert_array_equal(out["trace_e"][:, 12], out["e_trace"][:, 0])


# ------------------------------------------------------- Nose-Hoover SB ----
# Eqs. (eq_NH1), (eq_NH): the friction -xi y_i replaces the heating term and
# xi follows (sum_i y_i^2 - N T) / M.

@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_nose_hoover_large_mass_is_constant_heating(form, prec):
    # The paper: large M makes xi nearly constant, and xi = -gamma is heated
    # SB.  With M = 1e300 the xi increments vanish below binary64 resolution,
    # so the run equals the constant-gamma run bit for bit and xi stays xi0.
    J = synth.sk_pm1(48, 3)
    c0 = oracle.c0_from_c1(J, 0.7)
    # with gamma = 0.05 and dt = 1.1, rounding gamma and dt before their
    # product gives another binary32 g: both runs must take fl32(gamma dt)
    gamma = 0.05
    heat = oracle.make_params(form, c0, 1.1, gamma, eval_every=20)
    nh = oracle.make_params(form, c0, 1.1, 0.0, eval_every=20, nose_hoover=True, nh_T=0.3,
                            nh_M=1e300, nh_xi0=-gamma)
    a = oracle.run(J, heat, 150, 5, range(4), prec)
    b = oracle.run(J, nh, 150, 5, range(4), prec)
    for key in ("best_e", "best_s", "x", "y"):
        np.testing.assert_array_equal(a[key], b[key])
    np.testing.assert_array_equal(b["xi"], np.full(4, -gamma))


def _thermostat_only(n, T, M, xi0, dt, steps, seed=11, trace=False):
    # J = 0 and a0 = 0: no force, no pump and x fixed, so only y and xi move:
    # y' = (1 - xi dt) y, the discrete form of y' = -xi y.
    J = np.zeros((n, n), np.float32)
    prm = oracle.make_params(0, 1.0, dt, 0.0, a0=0.0, eval_every=0, nose_hoover=True,
                             nh_T=T, nh_M=M, nh_xi0=xi0, trace_every=1 if trace else 0)
    return oracle.run(J, prm, steps, seed, [0], "f64", want_trace=trace)


def test_nose_hoover_heats_below_and_cools_above_the_temperature():
    # T_inst < T drives xi negative and T_inst up (heating); T_inst > T drives
    # xi positive and T_inst down (cooling).  The initial T_inst of U(-1, 1)
    # momenta is about 1/3.
    n = 64
    for T, sign in ((1.0, -1.0), (0.05, 1.0)):
        out = _thermostat_only(n, T, 2.0, 0.0, 0.05, 40, trace=True)
        xi1 = _thermostat_only(n, T, 2.0, 0.0, 0.05, 1)["xi"][0]
        assert np.sign(xi1) == sign
        t_inst = out["trace_t"][0]
        # step 0 runs with xi_0 = 0: no friction yet, T_inst(t_1) = T_inst(t_0)
        assert t_inst[1] == t_inst[0]
        if sign < 0:
            assert t_inst[10] > t_inst[2] > t_inst[1]
        else:
            assert t_inst[10] < t_inst[2] < t_inst[1]


def test_nose_hoover_force_free_invariant_and_mean_temperature():
    # Without force, S = sum_i y_i^2 and xi obey dS/dt = -2 xi S and
    # dxi/dt = (S - N T) / M, which conserve H = M xi^2 + S - N T ln S (dH/dt
    # = 2 M xi xi' + S' - N T S'/S = 2 xi (S - N T) - 2 xi (S - N T) = 0), and
    # the time average of xi' vanishes over a bounded orbit, so the mean of
    # T_inst is T.  The discrete map conserves H up to O(dt).  A wrong sign
    # of the friction or of the xi equation turns the orbit into growth or
    # decay of H.
    n, T, M, dt = 6, 0.5, 5.0, 0.01
    steps = 1200   # about two periods (2 pi / sqrt(2 N T / M) = 5.7 time units)
    ks = list(range(0, steps, 40))
    tr = _thermostat_only(n, T, M, 0.0, dt, steps, trace=True)["trace_t"][0]
    S = n * tr[ks]
    xi = np.array([0.0] + [_thermostat_only(n, T, M, 0.0, dt, k)["xi"][0] for k in ks[1:]])
    H = M * xi ** 2 + S - n * T * np.log(S)
    h_min = n * T - n * T * math.log(n * T)          # at S = N T, xi = 0
    swing = H[0] - h_min
    assert swing > 0.05                                # a real orbit
    assert np.max(np.abs(H - H[0])) < 0.02 * swing
    assert xi.min() < -0.5 * math.sqrt(swing / M)      # xi swings both ways
    assert xi.max() > 0.5 * math.sqrt(swing / M)
    # mean of T_inst over the run: sum_k (S_k - N T) = M (xi_K - xi_0) / dt
    long = _thermostat_only(n, T, M, 0.0, dt, 20000, trace=True)
    assert abs(long["trace_t"][0].mean() - T) < 0.01 * T


@pytest.mark.parametrize("xi0", [0.25, -0.25])
def test_nose_hoover_xi_reads_the_updated_momenta(xi0):
    # Discrete Eq. (eq_NH): xi_{k+1} takes S = sum_i y_i^2 at t_{k+1}, after
    # the momentum update.  Force-free and unpumped (J = 0, a0 = 0), one step
    # only scales y by 1 - xi0 dt.  With N T = S(t_0), a xi read from the old
    # momenta would not move; read from the new ones it moves against xi0 by
    # (dt / M) ((1 - xi0 dt)^2 - 1) S(t_0), up to the rounding of S.
    n, dt, M = 64, 0.5, 7.0  # dt / M not a power of two: its products round
    J = np.zeros((n, n), np.float32)
    x0, y0 = oracle.init_values(11, 0, [0], n, 1.0)
    S0 = oracle.kinetic_sum(y0[0], "f64")
    prm = oracle.make_params(0, 0.0, dt, 0.0, a0=0.0, eval_every=0, nose_hoover=True,
                             nh_T=S0 / n, nh_M=M, nh_xi0=xi0)
    out = oracle.run(J, prm, 1, 11, [0], "f64")
    np.testing.assert_array_equal(out["x"][0], x0[0])
    np.testing.assert_array_equal(out["y"][0], y0[0].astype(np.float64) * (1.0 - xi0 * dt))
    want = xi0 + dt / M * ((1.0 - xi0 * dt) ** 2 - 1.0) * S0
    assert abs(want - xi0) > 0.1
    assert out["xi"][0] == pytest.approx(want, abs=1e-6)
    # and in binary64 exactly xi0 + (dt / M) (S(t_1) - N T), rounded in that order
    S1 = oracle.kinetic_sum(out["y"][0], "f64")
    assert out["xi"][0] == xi0 + (dt / M) * (S1 - n * (S0 / n))


def test_kinetic_sum_binary32_is_the_exact_sum_of_squares_rounded_once():
    # S of Eq. (eq_NH) for binary32 momenta: the exact sum of the exact
    # squares, rounded once to binary64.  Reference: Python's exact rationals
    # (float() of a Fraction is correctly rounded, ties to even).
    from fractions import Fraction
    rng = np.random.default_rng(4)
    t = 2.0 ** -27   # t^2 = 2^-54: two of them put 1 + 2^-53 on a tie
    cases = [
        rng.uniform(-1, 1, 1000).astype(np.float32),
        # tiny, subnormal and large momenta, zeros of both signs
        np.float32([2.0**-24, 3 * 2.0**-26, 2.0**-25, 1e-12, 7e-8, -2.0**-40, 0.0, -0.0,
                    255.9, 1e-40, -3e-45, 2.0**-149]),
        np.concatenate([rng.uniform(-1, 1, 300), rng.uniform(-1e-6, 1e-6, 300),
                        rng.uniform(-1e-30, 1e-30, 50),
                        rng.uniform(-200, 200, 40)]).astype(np.float32),
        np.float32([1.0] * 70000),              # carries across 64-bit limbs
        np.float32([1.0, t, t]),                # a tie: rounds to even (1.0)
        np.float32([1.0, t, t, 2.0**-80]),      # just above the tie: rounds up
        np.float32([1.0, t, t, t]),             # 1 + 1.5 2^-53: rounds up
        np.float32([3e38, -3e38, 1e-45]),       # the largest binary32 magnitudes
        np.float32([1e-40, -3e-45, 2.0**-149, 5e-39]),   # subnormals alone
        np.float32([]),
    ]
    for y in cases:
        exact = sum((Fraction(float(v)) ** 2 for v in y), Fraction(0))
        want = float(exact)
        assert oracle.kinetic_sum(y, "f32") == want
        assert oracle.kinetic_sum(y[::-1].copy(), "f32") == want   # order-free
    assert oracle.kinetic_sum(np.float32([1.0, t, t]), "f32") == 1.0
    assert oracle.kinetic_sum(np.float32([1.0, t, t, 2.0**-80]), "f32") == 1.0 + 2.0**-52


def test_kinetic_sum_binary64_is_the_plain_sum_in_ascending_order():
    # For binary64 momenta S is the plain binary64 sum, i ascending, one
    # rounding per square and per addition.  Three squares of 2^-54 before
    # 1.0 add up to 1.5 2^-53 first and then round 1 + 1.5 2^-53 up; after
    # 1.0 each is lost to rounding.  Squares and partial sums that are exact
    # give the exact sum; otherwise the error stays within the bound of a
    # sum of N rounded terms.
    from fractions import Fraction
    t = 2.0 ** -27
    assert oracle.kinetic_sum(np.array([t, t, t, 1.0]), "f64") == 1.0 + 2.0 ** -52
    assert oracle.kinetic_sum(np.array([1.0, t, t, t]), "f64") == 1.0
    ints = np.arange(-40.0, 41.0)
    assert oracle.kinetic_sum(ints, "f64") == float(np.sum(ints.astype(np.int64) ** 2))
    rng = np.random.default_rng(5)
    y = rng.standard_normal(5000)
    exact = sum((Fraction(float(v)) ** 2 for v in y), Fraction(0))
    got = oracle.kinetic_sum(y, "f64")
    assert abs(Fraction(got) - exact) <= exact * len(y) * Fraction(2, 2**53)


def test_kinetic_sum_q24_test_double_is_its_fixed_point_definition():
    # The test double of the CUDA kernels' sum: each y_i rounded to the
    # nearest multiple of 2^-24, the squares summed exactly, 2^-48 times the
    # total rounded once.  Reference: Python's exact rationals (round() to
    # nearest even, float() correctly rounded).  It stays within
    # 2^-24 sum |y_i| + N 2^-50 of the plain sum before its final rounding.
    from fractions import Fraction
    rng = np.random.default_rng(4)
    cases = [
        rng.uniform(-1, 1, 1000).astype(np.float32),
        np.float32([2.0**-24, 3 * 2.0**-26, 2.0**-25, 3 * 2.0**-25, 1e-12, 7e-8, -2.0**-40,
                    0.0, -0.0, 255.9]),
        np.concatenate([rng.uniform(-1, 1, 300), rng.uniform(-1e-6, 1e-6, 300),
                        rng.uniform(-200, 200, 40)]).astype(np.float32),
        np.float32([1.0] * 70000),    # the 128-bit sum carries past 2^64
    ]
    for y in cases:
        units = sum(round(Fraction(float(v)) * 2**24) ** 2 for v in y)
        want = float(Fraction(units, 2**48))
        assert oracle.kinetic_sum(y, q24=True) == want
        assert oracle.kinetic_sum(y[::-1].copy(), q24=True) == want
        exact = sum(Fraction(float(v)) ** 2 for v in y)
        bound = sum(abs(Fraction(float(v))) for v in y) * Fraction(1, 2**24) \
            + Fraction(len(y), 2**50) + abs(exact) * Fraction(1, 2**53)
        assert abs(Fraction(want) - exact) <= bound
