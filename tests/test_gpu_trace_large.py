"""The per-step trace and the large-instance workload on the GPU.

Trace: at t_k (k = m * trace_every) the minimum and mean Ising energy over
replicas (Eq. eq_Ising) and the mean instantaneous temperature T_inst =
(1/N) sum_i y_i^2 (Eq. eq_TInst).  For +/-1 couplings and the discrete form
the energies are exact integers and must equal the oracle's; T_inst is a
binary32 sum of squares per 128-spin block added in binary64, compared to the
oracle's binary64 value within 1e-6 relative.

Large instance: N = 16384 +/-1 SK (FP8 couplings 268 MB, beyond the 126 MB L2),
R = 4096, FP8 on the one-launch-per-step schedule; sampled replicas are checked
bit for bit against the oracle.
"""
import numpy as np
import pytest

import oracle
import paper_2203_08361_gb300 as hsb
import synth

pytestmark = pytest.mark.gpu


def _oracle_trace(J, c1, steps, seed, reps, trace_every, eval_every=0):
    c0 = oracle.c0_from_c1(J, c1)
    op = oracle.make_params(1, c0, 1.1, 0.06, eval_every=eval_every, trace_every=trace_every)
    return oracle.run(J, op, steps, seed, reps, "f32", nthreads=0)


@pytest.mark.parametrize("prec,schedule", [("fp8", "persistent"), ("fp8", "per_step"),
                                           ("fp32", "auto")])
def test_trace_matches_oracle(prec, schedule):
    n, R, steps, te = 300, 40, 100, 10
    J = synth.sk_pm1(n, 17)
    p = hsb.params("discrete", prec, c1=0.7, dt=1.1, gamma=0.06, eval_every=25, trace_every=te,
                   schedule=schedule)
    with hsb.Solver(J) as s:
        spins, energy = s.run(p, R, steps, 6)
        tr = s.get_trace()
        tc = s.trace_cut()
        x, y = s.get_state(R)
        if schedule == "persistent":
            assert s.run_stats() == 4  # init, step loop, best selection, trace entries
    ref = _oracle_trace(J, 0.7, steps, 6, range(R), te, eval_every=25)
    assert tr.shape == (steps // te, 3)
    # instantaneous cut values (Eq. eq_Cut, w = -J): C_r = -E_r/2 - sum(J)/4
    # per replica, so the trace's maximum and mean cut follow from the
    # oracle's per-replica energies
    c_ref = -0.5 * ref["trace_e"] - 0.25 * float(J.astype(np.float64).sum())
    np.testing.assert_allclose(tc[:, 0], c_ref.max(axis=0), rtol=1e-15)
    np.testing.assert_allclose(tc[:, 1], c_ref.mean(axis=0), rtol=1e-12)
    np.testing.assert_array_equal(tc[:, 2], tr[:, 2])
    np.testing.assert_array_equal(tr[:, 0], ref["trace_e"].min(axis=0))
    np.testing.assert_array_equal(tr[:, 1], ref["trace_e"].mean(axis=0))
    np.testing.assert_allclose(tr[:, 2], ref["trace_t"].mean(axis=0), rtol=1e-6)
    # the trace does not change the trajectory
    np.testing.assert_array_equal(x, ref["x"])
    np.testing.assert_array_equal(energy, ref["best_e"])


def test_large_instance_fp8_sampled_replicas_and_trace():
    n, steps, seed = 16384, 40, 11
    J = synth.sk_pm1(n, 3)
    p = hsb.params("discrete", "fp8", c1=0.7, dt=1.1, gamma=0.06, eval_every=0, trace_every=1)
    with hsb.Solver(J) as s:
        spins, energy = s.run(p, 4096, steps, seed)
        x_all, _ = s.get_state(4096)
        tr_all = s.get_trace()
        spins2, energy2 = s.run(p, 2, steps, seed)
        x2, y2 = s.get_state(2)
        tr2 = s.get_trace()
    # replica independence at full size
    np.testing.assert_array_equal(x_all[:2], x2)
    np.testing.assert_array_equal(spins[:2], spins2)
    # two replicas against the oracle, bit for bit, with their trace
    ref = _oracle_trace(J, 0.7, steps, seed, [0, 1], 1)
    np.testing.assert_array_equal(x2, ref["x"])
    np.testing.assert_array_equal(y2, ref["y"])
    np.testing.assert_array_equal(energy2, ref["best_e"])
    np.testing.assert_array_equal(tr2[:, 0], ref["trace_e"].min(axis=0))
    np.testing.assert_array_equal(tr2[:, 1], ref["trace_e"].mean(axis=0))
    np.testing.assert_allclose(tr2[:, 2], ref["trace_t"].mean(axis=0), rtol=1e-6)
    # full trace: integer energies, min <= mean, T_inst of U(-1,1) momenta ~ 1/3 at t_0
    assert tr_all.shape == (steps, 3)
    assert np.all(tr_all[:, 0] == np.round(tr_all[:, 0]))
    assert np.all(tr_all[:, 0] <= tr_all[:, 1])
    assert abs(tr_all[0, 2] - 1.0 / 3.0) < 1e-3


def test_persistent_trace_every_step_full_size_sampled():
    # the paper's per-step trace (Fig. 2) at N = 2000, R = 1024 on the
    # persistent kernel: the trace entries of two replicas' runs equal the
    # oracle's, and the full trace is that of the per-step schedule
    n, R, steps, seed = 2000, 1024, 60, 4
    J = synth.sk_pm1(n, 1)
    kw = dict(c1=0.7, dt=1.1, gamma=0.06, eval_every=20, trace_every=1)
    with hsb.Solver(J) as s:
        s.run(hsb.params("discrete", "fp8", schedule="persistent", **kw), R, steps, seed)
        tr_p = s.get_trace()
        s.run(hsb.params("discrete", "fp8", schedule="per_step", **kw), R, steps, seed)
        tr_s = s.get_trace()
        s.run(hsb.params("discrete", "fp8", schedule="persistent", **kw), 2, steps, seed)
        tr2 = s.get_trace()
    assert tr_p.shape == (steps, 3)
    np.testing.assert_array_equal(tr_p[:, :2], tr_s[:, :2])   # exact integer energies
    np.testing.assert_allclose(tr_p[:, 2], tr_s[:, 2], rtol=1e-6)
    ref = _oracle_trace(J, 0.7, steps, seed, [0, 1], 1, eval_every=20)
    np.testing.assert_array_equal(tr2[:, 0], ref["trace_e"].min(axis=0))
    np.testing.assert_array_equal(tr2[:, 1], ref["trace_e"].mean(axis=0))
    np.testing.assert_allclose(tr2[:, 2], ref["trace_t"].mean(axis=0), rtol=1e-6)


def test_persistent_trace_beyond_one_launch_of_entries():
    # more traced steps than one launch of the batched reduction takes
    # (65535 entries): N = 128, two replicas, 70000 steps, trace every step
    n, R, steps, seed = 128, 2, 70000, 8
    J = synth.sk_pm1(n, 9)
    p = hsb.params("discrete", "fp8", c1=0.7, dt=1.1, gamma=0.06, eval_every=0, trace_every=1,
                   schedule="persistent")
    with hsb.Solver(J) as s:
        s.run(p, R, steps, seed)
        tr = s.get_trace()
        assert s.run_stats() == 3 + 2
    ref = _oracle_trace(J, 0.7, steps, seed, range(R), 1, eval_every=0)
    assert tr.shape == (steps, 3)
    np.testing.assert_array_equal(tr[:, 0], ref["trace_e"].min(axis=0))
    np.testing.assert_array_equal(tr[:, 1], ref["trace_e"].mean(axis=0))
    # late in this long run the momenta decay below 2^-63, where their binary32
    # squares underflow (the oracle squares in binary64): an absolute floor
    np.testing.assert_allclose(tr[:, 2], ref["trace_t"].mean(axis=0), rtol=1e-6, atol=1e-30)
