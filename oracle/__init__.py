"""CPU oracle for heated simulated bifurcation (TEST INFRASTRUCTURE ONLY).

Plain, slow C (``hsb_oracle.c``) loaded through ctypes.  Only the tests, the
smoke check and the benchmark's CPU-baseline / reference legs may import this
package; the CUDA library never does, and this package never imports the CUDA
library.  What it computes and the readings it takes of the paper are stated
in the header of ``hsb_oracle.c``.

Parity status of each function (what pins it, in tests/test_oracle_pins.py):
  ising_energy     -- cut-value identity Eq. (eq_Cut), hand-derived fixtures,
                      single-flip identity, brute force
  brute_force      -- independent Python enumeration, hand-derived fixtures
  init_values      -- published SplitMix64 output vectors, range/uniformity
  step / run       -- hand-derived worked steps (tests/golden), the binary32
                      force as a chain of correctly rounded fused multiply-adds
                      and the binary32 update as one rounding per operation in
                      the stated order (exact rational arithmetic), gamma = 0
                      reduction to plain bSB/dSB, wall invariants, conserved
                      quadratic form per eigenmode, linear heating map, N = 2
                      normal modes, replica independence, determinism,
                      ties keep the earliest evaluation (J = 0), the traced
                      times k = m*trace_every < Ns (ragged count)
  kinetic_sum      -- binary32: exact rational arithmetic (Python fractions:
                      the exact sum of squares rounded once), subnormal,
                      tiny and large momenta, order independence;
                      binary64: exact sums of exactly representable squares,
                      the i-ascending order (an input whose two orders
                      round differently), the error bound of a sum of N
                      terms
  kinetic_sum q24  -- (test double of the CUDA kernels' sum) exact rational
                      arithmetic of its own definition, within its stated
                      distance of the plain sum
  run, Nose-Hoover -- large-M reduction to constant heating gamma = -xi0,
                      the conserved quantity M xi^2 + S - N T ln S of the
                      force-free thermostat, time average of T_inst equal to
                      T, the heating / cooling direction of xi, xi read
                      from the momenta after the update (one force-free step)

The pins are themselves checked: tests/test_oracle_mutants.py plants one
plausible mistake at a time in a copy of the C source (a dropped term, a wrong
sign or index, an operand at the wrong time, an off-by-one) and every such
copy fails at least one pin.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "hsb_oracle.c"), os.path.join(_HERE, "hsb_oracle_impl.h")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# gcc flags: no contraction into fused multiply-add (arm64 gcc contracts by
# default in GNU mode), no fast-math, OpenMP only over independent replicas.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
          "-fno-fast-math", "-fopenmp"]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc); returns its path."""
    newest = max(os.path.getmtime(p) for p in _SRC)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC[0], "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    """Mirror of oracle_params in hsb_oracle.c."""
    _fields_ = [
        ("form", C.c_int),
        ("eval_every", C.c_int),
        ("a0", C.c_double),
        ("c0", C.c_double),
        ("dt", C.c_double),
        ("gamma", C.c_double),
        ("init_half_width", C.c_double),
        ("instance", C.c_uint32),
        ("force_plain_sum", C.c_int),
        ("trace_every", C.c_int),
        ("thermostat", C.c_int),
        ("nh_T", C.c_double),
        ("nh_M", C.c_double),
        ("nh_xi0", C.c_double),
        ("nh_sum", C.c_int),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # HSB_ORACLE_LIB names another compiled copy of this source to load
        # instead (the planted-mistake test runs the pins against such copies).
        lib = C.CDLL(os.environ.get("HSB_ORACLE_LIB") or build())
        P = C.c_void_p
        lib.oracle_splitmix64.restype = C.c_uint64
        lib.oracle_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        lib.oracle_init_value.restype = C.c_float
        lib.oracle_init_value.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                          C.c_int, C.c_double]
        lib.oracle_ising_energy.restype = C.c_double
        lib.oracle_ising_energy.argtypes = [P, C.c_int, P]
        lib.oracle_cut_value.restype = C.c_double
        lib.oracle_cut_value.argtypes = [P, C.c_int, P]
        lib.oracle_brute_force.restype = C.c_int
        lib.oracle_brute_force.argtypes = [P, C.c_int, P, P]
        lib.oracle_sigma_j.restype = C.c_double
        lib.oracle_sigma_j.argtypes = [P, C.c_int]
        lib.oracle_c0.restype = C.c_double
        lib.oracle_c0.argtypes = [P, C.c_int, C.c_double]
        lib.oracle_pump_factor.restype = C.c_double
        lib.oracle_pump_factor.argtypes = [C.c_double, C.c_int, C.c_int]
        lib.oracle_num_evals.restype = C.c_int
        lib.oracle_num_evals.argtypes = [C.c_int, C.c_int]
        lib.oracle_num_traced.restype = C.c_int
        lib.oracle_num_traced.argtypes = [C.c_int, C.c_int]
        lib.oracle_is_pm1.restype = C.c_int
        lib.oracle_is_pm1.argtypes = [P, C.c_int]
        for sfx in ("f64", "f32"):
            for name in (f"oracle_kinetic_sum_{sfx}", f"oracle_kinetic_sum_q24_{sfx}"):
                ks = getattr(lib, name)
                ks.restype = C.c_double
                ks.argtypes = [P, C.c_int]
        for sfx, real in (("f64", C.c_double), ("f32", C.c_float)):
            st = getattr(lib, f"oracle_step_{sfx}")
            st.restype = C.c_int
            st.argtypes = [P, C.c_int, C.c_int, P, P, C.c_int, real, real, real, real, real, P]
            rn = getattr(lib, f"oracle_run_{sfx}")
            rn.restype = C.c_int
            rn.argtypes = [P, C.c_int, C.POINTER(Params), C.c_int, C.c_uint64, C.c_int, P, P, P,
                           P, P, P, P, P, P, C.c_int]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _coupling(J) -> np.ndarray:
    J = np.ascontiguousarray(J, dtype=np.float32)
    if J.ndim != 2 or J.shape[0] != J.shape[1]:
        raise ValueError("J must be square")
    return J


def _real(precision: str):
    if precision == "f64":
        return np.float64
    if precision == "f32":
        return np.float32
    raise ValueError("precision is 'f64' or 'f32'")


# ---------------------------------------------------------------- helpers --

def splitmix64(state: int, n: int) -> int:
    """Output number n (n >= 1) of SplitMix64 started from `state`."""
    return int(_load().oracle_splitmix64(state & (2**64 - 1), n & (2**64 - 1)))


def init_value(seed: int, instance: int, r: int, i: int, comp: int, half_width: float) -> float:
    return float(_load().oracle_init_value(seed, instance, r, i, comp, half_width))


def init_values(seed: int, instance: int, reps, n: int, half_width: float):
    """x0, y0 as float32 [len(reps), n] from the counter-based generator."""
    lib = _load()
    reps = list(reps)
    x = np.empty((len(reps), n), np.float32)
    y = np.empty((len(reps), n), np.float32)
    for a, r in enumerate(reps):
        for i in range(n):
            x[a, i] = lib.oracle_init_value(seed, instance, r, i, 0, half_width)
            y[a, i] = lib.oracle_init_value(seed, instance, r, i, 1, half_width)
    return x, y


def ising_energy(J, s) -> float:
    J = _coupling(J)
    s = np.ascontiguousarray(s, dtype=np.int8)
    return float(_load().oracle_ising_energy(_ptr(J), J.shape[0], _ptr(s)))


def cut_value(J, s) -> float:
    J = _coupling(J)
    s = np.ascontiguousarray(s, dtype=np.int8)
    return float(_load().oracle_cut_value(_ptr(J), J.shape[0], _ptr(s)))


def brute_force(J):
    """(minimum energy, first minimising state) over all 2^N states, N <= 24."""
    J = _coupling(J)
    n = J.shape[0]
    e = C.c_double()
    s = np.empty(n, np.int8)
    rc = _load().oracle_brute_force(_ptr(J), n, C.byref(e), _ptr(s))
    if rc != 0:
        raise ValueError(f"oracle_brute_force failed ({rc})")
    return float(e.value), s


def sigma_j(J) -> float:
    J = _coupling(J)
    return float(_load().oracle_sigma_j(_ptr(J), J.shape[0]))


def c0_from_c1(J, c1: float) -> float:
    J = _coupling(J)
    return float(_load().oracle_c0(_ptr(J), J.shape[0], c1))


def pump_factor(a0: float, k: int, steps: int) -> float:
    """p_k = a0 - a(t_k), binary64."""
    return float(_load().oracle_pump_factor(a0, k, steps))


def num_evals(steps: int, eval_every: int) -> int:
    return int(_load().oracle_num_evals(steps, eval_every))


def kinetic_sum(y, precision: str = "f32", q24: bool = False) -> float:
    """S = sum_i y_i^2 of Eq. (eq_NH) by its definition: for binary32
    momenta the exact sum of the exact squares rounded once to binary64, for
    binary64 momenta the binary64 sum (i ascending).  q24=True gives instead
    the test double of the CUDA kernels' sum (each y_i rounded to a multiple
    of 2^-24, squares summed exactly, one rounding)."""
    real = _real(precision)
    y = np.ascontiguousarray(y, dtype=real).ravel()
    name = f"oracle_kinetic_sum_q24_{precision}" if q24 else f"oracle_kinetic_sum_{precision}"
    fn = getattr(_load(), name)
    return float(fn(_ptr(y), int(y.shape[0])))


def is_pm1(J) -> bool:
    J = _coupling(J)
    return bool(_load().oracle_is_pm1(_ptr(J), J.shape[0]))


def step(J, x, y, form: int, pk: float, c0: float, dt: float, q: float, g: float,
         precision: str = "f64"):
    """One time step for state x, y [nrep, N]; returns (x', y', f).

    The constants are rounded to the working precision by this wrapper (one
    rounding from the given binary64 values).
    """
    J = _coupling(J)
    real = _real(precision)
    x = np.array(x, dtype=real, order="C", copy=True)
    y = np.array(y, dtype=real, order="C", copy=True)
    if x.ndim == 1:
        x = x[None, :]
        y = y[None, :]
    nrep, n = x.shape
    if n != J.shape[0] or y.shape != x.shape:
        raise ValueError("state shape mismatch")
    f = np.empty_like(x)
    fn = getattr(_load(), f"oracle_step_{precision}")
    rc = fn(_ptr(J), n, nrep, _ptr(x), _ptr(y), form, real(pk), real(c0), real(dt), real(q),
            real(g), _ptr(f))
    if rc != 0:
        raise RuntimeError(f"oracle_step failed ({rc})")
    return x, y, f


def make_params(form: int, c0: float, dt: float, gamma: float, a0: float = 1.0,
                init_half_width: float = 1.0, eval_every: int = 100, instance: int = 0,
                force_plain_sum: bool = False, trace_every: int = 0,
                nose_hoover: bool = False, nh_T: float = 0.0, nh_M: float = 1.0,
                nh_xi0: float = 0.0, nh_sum_q24: bool = False) -> Params:
    """Run parameters; nose_hoover=True replaces the constant heating gamma by
    the dynamic xi of Eqs. (eq_NH1), (eq_NH) with temperature nh_T, mass nh_M
    and xi(t_0) = nh_xi0.  nh_sum_q24=True forms S with the test double of
    the CUDA kernels' 2^-24 fixed-point sum instead of the plain definition."""
    return Params(form=int(form), eval_every=int(eval_every), a0=float(a0), c0=float(c0),
                  dt=float(dt), gamma=float(gamma), init_half_width=float(init_half_width),
                  instance=int(instance), force_plain_sum=int(bool(force_plain_sum)),
                  trace_every=int(trace_every), thermostat=1 if nose_hoover else 0,
                  nh_T=float(nh_T), nh_M=float(nh_M), nh_xi0=float(nh_xi0),
                  nh_sum=1 if nh_sum_q24 else 0)


def num_traced(steps: int, trace_every: int) -> int:
    return int(_load().oracle_num_traced(steps, trace_every))


def run(J, params: Params, steps: int, seed: int, reps, precision: str = "f64",
        nthreads: int = 0, want_trace: bool = False):
    """Whole run for the replica indices `reps`.

    Returns dict(best_e [nrep] float64, best_s [nrep, N] int8, x, y [nrep, N]
    in the working precision, e_trace [nrep, n_evals] or None, trace_e /
    trace_t [nrep, n_traced] or None, xi [nrep] float64: the Nose-Hoover
    variable after the last step).
    """
    J = _coupling(J)
    real = _real(precision)
    n = J.shape[0]
    reps = np.ascontiguousarray(np.asarray(list(reps), dtype=np.int32))
    nrep = reps.shape[0]
    best_s = np.zeros((nrep, n), np.int8)
    best_e = np.zeros(nrep, np.float64)
    x = np.zeros((nrep, n), real)
    y = np.zeros((nrep, n), real)
    ne = num_evals(steps, params.eval_every)
    trace = np.zeros((nrep, ne), np.float64) if want_trace else None
    nt = num_traced(steps, params.trace_every)
    tr_e = np.zeros((nrep, nt), np.float64) if nt else None
    tr_t = np.zeros((nrep, nt), np.float64) if nt else None
    xi = np.zeros(nrep, np.float64)
    fn = getattr(_load(), f"oracle_run_{precision}")
    rc = fn(_ptr(J), n, C.byref(params), int(steps), C.c_uint64(seed & (2**64 - 1)), nrep,
            _ptr(reps), _ptr(best_s), _ptr(best_e), _ptr(x), _ptr(y),
            _ptr(trace) if trace is not None else None,
            _ptr(tr_e) if tr_e is not None else None,
            _ptr(tr_t) if tr_t is not None else None, _ptr(xi), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_run failed ({rc})")
    return {"best_e": best_e, "best_s": best_s, "x": x, "y": y, "e_trace": trace,
            "trace_e": tr_e, "trace_t": tr_t, "xi": xi}
