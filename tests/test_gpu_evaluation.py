"""MAX-CUT values (Eq. (eq_Cut), hsb_cut_values) against the oracle's cut
function, and the trial statistics of the evaluation harness against the same
statistics of oracle runs on the same seeds."""
import numpy as np
import pytest

import oracle
import paper_2203_08361_gb300 as hsb
import synth
from paper_2203_08361_gb300 import evaluation as ev

pytestmark = pytest.mark.gpu


def test_cut_values_pm1_exact():
    J = synth.sk_pm1(300, 17)
    p = hsb.params("discrete", "fp8", c1=0.7, dt=1.1, gamma=0.06, eval_every=40)
    with hsb.Solver(J) as s:
        spins, energy = s.run(p, 40, 200, 3)
        cut = s.cut_values(energy)
    for r in range(40):
        assert cut[r] == oracle.cut_value(J, spins[r])


def test_cut_values_gaussian():
    J = synth.sk_gauss(200, 5)
    p = hsb.params("ballistic", "fp32", c1=0.9, dt=1.1, gamma=0.5, eval_every=50)
    with hsb.Solver(J) as s:
        spins, energy = s.run(p, 16, 200, 4)
        cut = s.cut_values(energy)
    for r in range(16):
        assert cut[r] == pytest.approx(oracle.cut_value(J, spins[r]), rel=1e-12, abs=1e-9)


def test_harness_statistics_match_oracle_trials():
    # 16-spin SK instance: the target is the brute-force ground energy; the
    # plain FP32 path is bit-exact against the binary32 oracle, so P and S of
    # the GPU trials equal those of oracle trials on the same seeds
    J = synth.sk_pm1(16, 8)
    e0 = float(oracle.brute_force(J)[0])
    trials, seed = 64, 11
    kw = dict(prec="fp32", c1=0.7, dt=1.1, gamma=0.06, eval_every=20)
    stats = ev.evaluate(J, "discrete", [20, 80], trials, seed, e0, **kw)
    c0 = oracle.c0_from_c1(J, 0.7)
    for st in stats:
        op = oracle.make_params(1, c0, 1.1, 0.06, eval_every=20)
        ref = oracle.run(J, op, st.steps, seed, range(trials), "f32")
        p_ref = ev.success_probability(ref["best_e"], e0)
        assert st.p == p_ref
        assert st.step_to_solution == ev.step_to_solution(p_ref, st.steps)
        assert st.min_energy == float(np.min(ref["best_e"])) >= e0
    assert stats[-1].p > 0.0  # the ground state is found within 80 steps


def test_parameter_sweep_matches_oracle_trials():
    # the paper's gamma / dt scan at fixed N_s on a 16-spin instance: every
    # grid point's P equals that of oracle trials with the same parameters
    J = synth.sk_pm1(16, 8)
    e0 = float(oracle.brute_force(J)[0])
    trials, seed, steps = 48, 3, 40
    grid = {"dt": [0.5, 1.1], "gamma": [0.0, 0.06]}
    pts = ev.sweep(J, "discrete", grid, steps, trials, seed, e0, prec="fp32", c1=0.7,
                   eval_every=20)
    assert [pt.params for pt in pts] == ev.grid_points(grid)
    c0 = oracle.c0_from_c1(J, 0.7)
    for pt in pts:
        op = oracle.make_params(1, c0, pt.params["dt"], pt.params["gamma"], eval_every=20)
        ref = oracle.run(J, op, steps, seed, range(trials), "f32")
        assert pt.stats.p == ev.success_probability(ref["best_e"], e0)
        assert pt.stats.min_energy == float(np.min(ref["best_e"]))
