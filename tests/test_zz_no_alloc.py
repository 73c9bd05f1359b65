"""hsb_run_fp32_noalloc, the entry point that allocates nothing (it works in a
fixed scratch array the library holds), for callers that cannot allocate
device memory on demand: against hsb_run on the plain FP32 path, two calls in
a row, each on a different instance, must give the same best spins and
energies (exact integers for +/-1 couplings; for general couplings the
no-alloc path sums the final energies in binary64 and hsb_run in exact fixed
point, so they agree to 1e-12 relative), and both equal the binary32 oracle.
A call made while every device allocation of the library is capped at one
byte succeeds: it allocates nothing.  This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
import paper_2203_08361_gb300 as hsb
import synth

pytestmark = pytest.mark.gpu


def _noalloc(torch, J, p, R, steps, seed, stream):
    n = J.shape[0]
    dJ = torch.from_numpy(J).to("cuda")
    spins = torch.empty((R, n), dtype=torch.int8, device="cuda")
    energy = torch.empty(R, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        hsb.run_fp32_noalloc(dJ.data_ptr(), n, p, R, steps, seed, spins.data_ptr(),
                             energy.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return spins.cpu().numpy(), energy.cpu().numpy()


def test_no_alloc_run_matches_hsb_run_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    cases = [
        # +/-1 couplings, discrete form, ragged N and R
        (synth.sk_pm1(300, 3), "discrete", 0.7 / np.sqrt(300), 0.06, 100, 150, 40),
        # Gaussian couplings, ballistic form
        (synth.sk_gauss(200, 4), "ballistic", 0.9 / np.sqrt(200), 0.5, 64, 120, 30),
    ]
    for J, form, c0, gamma, R, steps, ev in cases:
        p = hsb.params(form, "fp32", c0=c0, dt=1.1, gamma=gamma, eval_every=ev)
        with hsb.Solver(J) as s:
            want_s, want_e = s.run(p, R, steps, 9)
        got_s, got_e = _noalloc(torch, J, p, R, steps, 9, stream)
        np.testing.assert_array_equal(got_s, want_s)
        exact = bool(np.all(np.isin(J, (-1.0, 0.0, 1.0))))
        np.testing.assert_allclose(got_e, want_e, rtol=0 if exact else 1e-12, atol=0)
        # and the binary32 oracle on sampled replicas
        rows = [0, 1, R - 1]
        op = oracle.make_params(0 if form == "ballistic" else 1, c0, 1.1, gamma, eval_every=ev)
        ref = oracle.run(J, op, steps, 9, rows, "f32")
        np.testing.assert_array_equal(got_s[rows], ref["best_s"])
        np.testing.assert_allclose(got_e[rows], ref["best_e"], rtol=0 if exact else 1e-12,
                                   atol=0)


def test_no_alloc_run_allocates_nothing():
    # every device allocation the library makes goes through one wrapper that
    # honours the cap; with the cap at one byte the call still succeeds
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    J = synth.sk_pm1(256, 8)
    p = hsb.params("discrete", "fp32", c0=0.7 / 16.0, dt=1.1, gamma=0.06, eval_every=20)
    want_s, want_e = _noalloc(torch, J, p, 64, 60, 2, stream)  # set-up before the cap
    dJ = torch.from_numpy(J).to("cuda")
    spins = torch.empty((64, 256), dtype=torch.int8, device="cuda")
    energy = torch.empty(64, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    try:
        hsb.debug_alloc_cap(1)
        with torch.cuda.stream(stream):
            hsb.run_fp32_noalloc(dJ.data_ptr(), 256, p, 64, 60, 2, spins.data_ptr(),
                                 energy.data_ptr(), stream.cuda_stream)
        stream.synchronize()
    finally:
        hsb.debug_alloc_cap(0)
    np.testing.assert_array_equal(spins.cpu().numpy(), want_s)
    np.testing.assert_array_equal(energy.cpu().numpy(), want_e)


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    J = synth.sk_pm1(600, 1)
    dJ = torch.from_numpy(J).to("cuda")
    spins = torch.empty((4, 600), dtype=torch.int8, device="cuda")
    energy = torch.empty(4, dtype=torch.float64, device="cuda")
    p = hsb.params("discrete", "fp32", c0=0.03)
    with pytest.raises(hsb.HsbError) as e:
        hsb.run_fp32_noalloc(dJ.data_ptr(), 600, p, 4, 10, 0, spins.data_ptr(),
                             energy.data_ptr())
    assert e.value.status == 1
    assert "512" in str(e.value)
