"""Failure detection on the GPU without a GPU fault.

Every spin-wait of the persistent kernels (mbarrier waits, the flag pollers)
gives up after a wall-clock budget (about 2 s), raises the CTA's abort flag
and the error word, waits (bounded) for the copies and MMAs it issued, frees
tensor memory and returns.  The test hook makes one
tile skip the publication of its sign operand: the other tiles' waits run
out, the run returns HSB_E_TIMEOUT, and the handle and the context stay
usable: the next run on the same handle equals a run before the failure.
Allocation failure is injected on the host (a cap on one device allocation):
the call returns HSB_E_NOMEM and the handle recovers once the cap is lifted.
"""
import time

import numpy as np
import pytest

import paper_2203_08361_gb300 as hsb
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("schedule", ["persistent", "pair"])
def test_dropped_publication_times_out_and_the_handle_stays_usable(schedule):
    J = synth.sk_pm1(512, 7)
    R, steps, seed = 256, 40, 5
    p = hsb.params("discrete", "fp8", c1=0.7, dt=1.1, gamma=0.06, eval_every=10,
                   schedule=schedule)
    with hsb.Solver(J) as s:
        s1, e1 = s.run(p, R, steps, seed)
        hsb.debug_drop_publication(s.h, 1)
        t0 = time.monotonic()
        with pytest.raises(hsb.HsbError) as e:
            s.run(p, R, steps, seed)
        waited = time.monotonic() - t0
        assert e.value.status == hsb.HSB_E_TIMEOUT
        assert 1.0 < waited < 60.0
        s2, e2 = s.run(p, R, steps, seed)
        with pytest.raises(hsb.HsbError) as e:
            hsb.debug_drop_publication(s.h, 4)   # N = 512: row blocks 0..3
        assert e.value.status == hsb.HSB_E_INVAL
    np.testing.assert_array_equal(s1, s2)
    np.testing.assert_array_equal(e1, e2)
    # a new handle on the same device works as well
    with hsb.Solver(J) as s:
        s3, e3 = s.run(p, R, steps, seed)
    np.testing.assert_array_equal(s1, s3)


def test_allocation_failure_is_reported_and_the_handle_recovers():
    # Host-side fault injection: a cap on one device allocation makes the
    # library's allocations fail as they do on a full device.
    J = synth.sk_pm1(256, 5)
    p = hsb.params("discrete", "fp8", eval_every=10)
    with hsb.Solver(J) as s:
        s_ref, e_ref = s.run(p, 128, 50, 3)
        try:
            hsb.debug_alloc_cap(1 << 20)
            with pytest.raises(hsb.HsbError) as e:
                s.run(p, 4096, 50, 3)                  # x alone takes 4 MiB
            assert e.value.status == hsb.HSB_E_NOMEM
            with pytest.raises(hsb.HsbError) as e:
                hsb.create(synth.sk_pm1(1024, 1))      # J takes 4 MiB
            assert e.value.status == hsb.HSB_E_NOMEM
        finally:
            hsb.debug_alloc_cap(0)
        s1, e1 = s.run(p, 128, 50, 3)
        s2, e2 = s.run(p, 4096, 50, 3)
    np.testing.assert_array_equal(s1, s_ref)
    np.testing.assert_array_equal(e1, e_ref)
    # replica r depends on (seed, r) only: the first 128 of the larger run agree
    np.testing.assert_array_equal(s2[:128], s_ref)
    np.testing.assert_array_equal(e2[:128], e_ref)
