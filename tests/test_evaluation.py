"""Trial statistics of the evaluation harness (Results: P and step-to-solution
S = N_s log(0.01) / log(1 - P)), checked against closed forms."""
import math

import numpy as np
import pytest

from paper_2203_08361_gb300 import evaluation as ev


def test_step_to_solution_closed_forms():
    # log(0.01) / log(0.1) = 2 and log(0.01) / log(0.5) = log2(100)
    assert ev.step_to_solution(0.9, 100) == pytest.approx(200.0, rel=1e-15)
    assert ev.step_to_solution(0.5, 100) == pytest.approx(100 * math.log2(100.0), rel=1e-14)
    # one run succeeds with probability >= 0.99: S = N_s; continuous at 0.99
    assert ev.step_to_solution(0.99, 700) == 700.0
    assert ev.step_to_solution(1.0, 700) == 700.0
    assert ev.step_to_solution(0.98999999, 700) == pytest.approx(700.0, rel=1e-5)
    assert ev.step_to_solution(0.0, 50) == math.inf
    # fewer successes need more steps
    ps = np.linspace(0.01, 0.98, 50)
    s = [ev.step_to_solution(float(p), 100) for p in ps]
    assert all(a > b for a, b in zip(s, s[1:]))
    with pytest.raises(ValueError):
        ev.step_to_solution(1.5, 10)
    with pytest.raises(ValueError):
        ev.step_to_solution(0.5, 0)


def test_success_probability_counts_trials_at_or_below_target():
    e = np.array([-10.0, -12.0, -12.0, -11.0, -9.0])
    assert ev.success_probability(e, -12.0) == pytest.approx(0.4)
    assert ev.success_probability(e, -11.0) == pytest.approx(0.6)
    assert ev.success_probability(e, -13.0) == 0.0
    assert ev.success_probability(e, -11.5, tol=0.6) == pytest.approx(0.6)
    with pytest.raises(ValueError):
        ev.success_probability([], 0.0)


def test_grid_points_cover_the_product_last_name_fastest():
    g = {"dt": [0.5, 1.1], "gamma": [0.0, 0.06, 0.1]}
    pts = ev.grid_points(g)
    assert len(pts) == 6
    assert pts[0] == {"dt": 0.5, "gamma": 0.0} and pts[1] == {"dt": 0.5, "gamma": 0.06}
    assert pts[-1] == {"dt": 1.1, "gamma": 0.1}
    assert ev.grid_points({"c1": [0.7]}) == [{"c1": 0.7}]
    with pytest.raises(ValueError):
        ev.grid_points({"dt": []})


class _OracleSolver:
    """Test double of hsb.Solver for the harness's host logic: runs the
    binary32 oracle (only tests may) and the cut identity of Eq. (eq_Cut)."""

    def __init__(self, J):
        import oracle
        self.oracle = oracle
        self.J = np.asarray(J, np.float32)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def run(self, p, R, steps, seed):
        c0 = self.oracle.c0_from_c1(self.J, p.c1)
        op = self.oracle.make_params(p.form, c0, p.dt, p.gamma, eval_every=p.eval_every)
        out = self.oracle.run(self.J, op, steps, seed, range(R), "f32")
        return out["best_s"], out["best_e"]

    def cut_values(self, energy):
        return -0.5 * np.asarray(energy) - 0.25 * float(self.J.astype(np.float64).sum())


def test_evaluate_and_sweep_statistics_on_the_host(monkeypatch):
    import oracle
    import synth
    monkeypatch.setattr(ev, "Solver", _OracleSolver)
    J = synth.sk_pm1(12, 3)
    e0, s0 = oracle.brute_force(J)
    stats = ev.evaluate(J, "discrete", [10, 40], 24, 5, e0, prec="fp32", c1=0.7, dt=1.1,
                        gamma=0.06, eval_every=10)
    for st in stats:
        c0 = oracle.c0_from_c1(J, 0.7)
        ref = oracle.run(J, oracle.make_params(1, c0, 1.1, 0.06, eval_every=10), st.steps, 5,
                         range(24), "f32")
        cuts = np.array([oracle.cut_value(J, s) for s in ref["best_s"]])
        assert st.trials == 24
        assert st.mean_cut == pytest.approx(cuts.mean(), rel=1e-12)
        assert st.max_cut == pytest.approx(cuts.max(), rel=1e-12)
        assert st.min_energy == ref["best_e"].min()
        assert st.p == ev.success_probability(ref["best_e"], e0)
        assert st.step_to_solution == ev.step_to_solution(st.p, st.steps)
    pts = ev.sweep(J, "discrete", {"gamma": [0.0, 0.06], "dt": [0.9]}, 20, 16, 2, e0,
                   prec="fp32", c1=0.7, eval_every=10)
    assert [pt.params for pt in pts] == [{"gamma": 0.0, "dt": 0.9}, {"gamma": 0.06, "dt": 0.9}]
    assert all(0.0 <= pt.stats.p <= 1.0 for pt in pts)
