"""Batched heated discrete SB over many instances of uneven size (FP8 or packed
FP4 e2m1 operands, one launch): every instance's best spins and energies must
equal those of a separate run of the same instance (same random stream), and
the oracle's on sampled instances; the FP4 batch equals the FP8 batch."""
import numpy as np
import pytest

import oracle
import paper_2203_08361_gb300 as hsb
import synth

pytestmark = pytest.mark.gpu


def _batch_vs_single(sizes, R, steps, ev, seed, check_oracle=(), oracle_rows=None,
                     prec="fp8"):
    Js = [synth.sk_pm1(n, 500 + b) for b, n in enumerate(sizes)]
    solvers = [hsb.Solver(J) for J in Js]
    p = hsb.params("discrete", prec, c1=0.7, dt=1.1, gamma=0.06, eval_every=ev)
    try:
        out = hsb.run_batch([s.h for s in solvers], p, R, steps, seed)
        for b, s in enumerate(solvers):
            pb = hsb.params("discrete", prec, c1=0.7, dt=1.1, gamma=0.06, eval_every=ev,
                            instance=b)
            spins, energy = s.run(pb, R, steps, seed)
            np.testing.assert_array_equal(out[b][0], spins, err_msg=f"instance {b}")
            np.testing.assert_array_equal(out[b][1], energy, err_msg=f"instance {b}")
        for b in check_oracle:
            J = Js[b]
            op = oracle.make_params(1, oracle.c0_from_c1(J, 0.7), 1.1, 0.06, eval_every=ev,
                                    instance=b)
            rows = list(range(R)) if oracle_rows is None else list(oracle_rows)
            ref = oracle.run(J, op, steps, seed, rows, "f32", nthreads=0)
            np.testing.assert_array_equal(out[b][0][rows], ref["best_s"])
            np.testing.assert_array_equal(out[b][1][rows], ref["best_e"])
    finally:
        for s in solvers:
            s.close()
    return out


@pytest.mark.parametrize("prec", ["fp8", "fp4"])
def test_batch_small_uneven_instances(prec):
    # ragged sizes (one 128-row block up to several, odd block counts; in FP4
    # K paddings beyond the 128-spin padding) and R
    _batch_vs_single([100, 128, 257, 300, 511, 700, 129, 2, 640], 40, 150, 30, 3,
                     check_oracle=(0, 2, 7), prec=prec)


@pytest.mark.parametrize("R", [1, 64, 96, 200])
def test_batch_fp4_replica_widths(R):
    # one accumulator per buffer up to 224 replica columns, K split over two
    # MMA warps up to 96
    _batch_vs_single([300, 1000, 513], R, 60, 20, 6, check_oracle=(0,), prec="fp4")


def test_batch_more_instances_than_ctas_per_cta_reuse():
    # 400 small instances: every CTA takes several instances in turn
    sizes = [int(v) for v in synth.batch_sizes(400, 7, lo=2, hi=260)]
    _batch_vs_single(sizes, 32, 60, 20, 5, check_oracle=(0, 399))


def test_batch_uneven_workload_full_size():
    # 256 SK instances, N uniform in [100, 2000], R = 64, 2000 steps, eval every
    # 100: one batched launch against 256 separate runs; the smallest and the
    # largest instance against the oracle on replicas at both ends
    sizes = [int(v) for v in synth.batch_sizes(256, 4)]
    _batch_vs_single(sizes, 64, 2000, 100, 9,
                     check_oracle=(sizes.index(min(sizes)), sizes.index(max(sizes))),
                     oracle_rows=(0, 1, 62, 63))


def test_batch_fp4_equals_fp8_on_the_uneven_workload():
    # 256 SK instances, N uniform in [100, 2000], R = 64, 300 steps: the FP4
    # batch equals the FP8 batch for every instance
    sizes = [int(v) for v in synth.batch_sizes(256, 4)]
    Js = [synth.sk_pm1(n, 500 + b) for b, n in enumerate(sizes)]
    solvers = [hsb.Solver(J) for J in Js]
    try:
        hs = [s.h for s in solvers]
        out = {}
        for prec in ("fp8", "fp4"):
            p = hsb.params("discrete", prec, c1=0.7, dt=1.1, gamma=0.06, eval_every=100)
            out[prec] = hsb.run_batch(hs, p, 64, 300, 9)
        for b in range(len(sizes)):
            np.testing.assert_array_equal(out["fp8"][b][0], out["fp4"][b][0], err_msg=f"{b}")
            np.testing.assert_array_equal(out["fp8"][b][1], out["fp4"][b][1], err_msg=f"{b}")
    finally:
        for s in solvers:
            s.close()


@pytest.mark.parametrize("kind", ["gauss", "nose_hoover"])
def test_batch_of_other_instances_runs_them_one_after_another(kind):
    # instances the batched FP8 kernel does not take (general couplings, the
    # Nose-Hoover thermostat) run one after another with instance = b: the
    # same results as separate runs
    sizes = [150, 300, 77]
    R, steps, seed = 40, 60, 9
    if kind == "gauss":
        Js = [synth.sk_gauss(n, 600 + b) for b, n in enumerate(sizes)]
        kw = dict(form="ballistic", prec="auto", c1=0.9, dt=1.1, gamma=0.5, eval_every=20)
    else:
        Js = [synth.sk_pm1(n, 600 + b) for b, n in enumerate(sizes)]
        kw = dict(form="discrete", prec="auto", c1=0.7, dt=1.1, eval_every=20,
                  thermostat="nose_hoover", nh_T=0.3, nh_M=20.0 * max(sizes), nh_xi0=-0.05)
    solvers = [hsb.Solver(J) for J in Js]
    try:
        out = hsb.run_batch([s.h for s in solvers], hsb.params(**kw), R, steps, seed)
        for b, s in enumerate(solvers):
            spins, energy = s.run(hsb.params(instance=b, **kw), R, steps, seed)
            np.testing.assert_array_equal(out[b][0], spins)
            np.testing.assert_array_equal(out[b][1], energy)
    finally:
        for s in solvers:
            s.close()
