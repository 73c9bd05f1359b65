"""Python binding of libhsb, the GB300 heated simulated bifurcation library.

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI of include/hsb.h.  The functions carry the names of
the C entry points without the ``hsb_`` prefix (``create``, ``run``,
``run_device``, ``get_state``, ``advance``, ``set_stream``, ``synchronize``,
``destroy``).  There is no CPU fallback: when libhsb.so has not been built, or
no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhsb.so")

HSB_BALLISTIC, HSB_DISCRETE = 0, 1
HSB_PREC_AUTO, HSB_PREC_FP32, HSB_PREC_FP8, HSB_PREC_BF16X3, HSB_PREC_FP4 = 0, 1, 2, 3, 4
HSB_E_INVAL, HSB_E_NOMEM, HSB_E_TIMEOUT, HSB_E_UNSUPPORTED = 1, 4, 6, 7
HSB_HEAT_CONSTANT, HSB_HEAT_NOSE_HOOVER = 0, 1
STATUS = {0: "HSB_OK", 1: "HSB_E_INVAL", 2: "HSB_E_ASYM", 3: "HSB_E_DIAG", 4: "HSB_E_NOMEM",
          5: "HSB_E_CUDA", 6: "HSB_E_TIMEOUT", 7: "HSB_E_UNSUPPORTED", 8: "HSB_E_NODEVICE"}
PREC = {"auto": HSB_PREC_AUTO, "fp32": HSB_PREC_FP32, "fp8": HSB_PREC_FP8,
        "bf16x3": HSB_PREC_BF16X3, "fp4": HSB_PREC_FP4}
FORM = {"ballistic": HSB_BALLISTIC, "discrete": HSB_DISCRETE}
SCHEDULE = {"auto": 0, "persistent": 1, "per_step": 2, "resident": 3, "pair": 4}
THERMOSTAT = {"constant": HSB_HEAT_CONSTANT, "nose_hoover": HSB_HEAT_NOSE_HOOVER}

# Every symbol include/hsb.h declares.
EXPORTS = ["hsb_params_default", "hsb_version", "hsb_create", "hsb_destroy", "hsb_set_stream",
           "hsb_info", "hsb_run", "hsb_run_device", "hsb_get_state", "hsb_advance",
           "hsb_advance_device", "hsb_set_couplings", "hsb_run_stats", "hsb_synchronize",
           "hsb_run_fp32_noalloc", "hsb_get_trace", "hsb_run_batch", "hsb_cut_values",
           "hsb_get_xi", "hsb_debug_drop_publication", "hsb_debug_alloc_cap",
           "hsb_last_error"]


class HsbError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Params(C.Structure):
    """Mirror of hsb_params (include/hsb.h)."""
    _fields_ = [
        ("form", C.c_int),
        ("prec", C.c_int),
        ("a0", C.c_double),
        ("c1", C.c_double),
        ("c0", C.c_double),
        ("dt", C.c_double),
        ("gamma", C.c_double),
        ("init_half_width", C.c_double),
        ("eval_every", C.c_int),
        ("trace_every", C.c_int),
        ("instance", C.c_uint32),
        ("schedule", C.c_int),
        ("thermostat", C.c_int),
        ("reserved0", C.c_int),
        ("nh_T", C.c_double),
        ("nh_M", C.c_double),
        ("nh_xi0", C.c_double),
        ("reserved", C.c_uint32 * 2),
    ]


_lock = threading.Lock()
_lib = None


def load():
    """Loads libhsb.so (built in-tree by __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = C.CDLL(LIB_PATH)
        P, I, H = C.c_void_p, C.c_int, C.c_void_p
        lib.hsb_version.restype = I
        lib.hsb_version.argtypes = []
        lib.hsb_last_error.restype = C.c_char_p
        lib.hsb_last_error.argtypes = []
        lib.hsb_params_default.restype = I
        lib.hsb_params_default.argtypes = [C.POINTER(Params)]
        lib.hsb_create.restype = I
        lib.hsb_create.argtypes = [P, I, C.POINTER(H)]
        lib.hsb_destroy.restype = None
        lib.hsb_destroy.argtypes = [H]
        lib.hsb_set_stream.restype = I
        lib.hsb_set_stream.argtypes = [H, P]
        lib.hsb_info.restype = I
        lib.hsb_info.argtypes = [H, C.POINTER(I), C.POINTER(I)]
        lib.hsb_cut_values.restype = I
        lib.hsb_cut_values.argtypes = [H, I, P, P]
        lib.hsb_run.restype = I
        lib.hsb_run.argtypes = [H, C.POINTER(Params), I, I, C.c_uint64, P, P]
        lib.hsb_run_device.restype = I
        lib.hsb_run_device.argtypes = [H, C.POINTER(Params), I, I, C.c_uint64, P, P]
        lib.hsb_get_state.restype = I
        lib.hsb_get_state.argtypes = [H, P, P]
        lib.hsb_advance.restype = I
        lib.hsb_advance.argtypes = [H, C.POINTER(Params), I, I, I, I, P, P]
        lib.hsb_advance_device.restype = I
        lib.hsb_advance_device.argtypes = [H, C.POINTER(Params), I, I, I, I]
        lib.hsb_set_couplings.restype = I
        lib.hsb_set_couplings.argtypes = [H, P]
        lib.hsb_run_stats.restype = I
        lib.hsb_run_stats.argtypes = [H, C.POINTER(C.c_longlong)]
        lib.hsb_synchronize.restype = I
        lib.hsb_synchronize.argtypes = [H]
        lib.hsb_run_batch.restype = I
        lib.hsb_run_batch.argtypes = [P, I, C.POINTER(Params), I, I, C.c_uint64, P, P]
        lib.hsb_get_trace.restype = I
        lib.hsb_get_trace.argtypes = [H, P, C.c_size_t, C.POINTER(C.c_size_t)]
        lib.hsb_get_xi.restype = I
        lib.hsb_get_xi.argtypes = [H, I, P]
        lib.hsb_debug_drop_publication.restype = I
        lib.hsb_debug_drop_publication.argtypes = [H, I]
        lib.hsb_debug_alloc_cap.restype = I
        lib.hsb_debug_alloc_cap.argtypes = [C.c_size_t]
        lib.hsb_run_fp32_noalloc.restype = I
        lib.hsb_run_fp32_noalloc.argtypes = [P, I, C.POINTER(Params), I, I, C.c_uint64, P, P, P]
        _lib = lib
        return lib


def _check(status: int):
    if status != 0:
        msg = load().hsb_last_error().decode(errors="replace")
        raise HsbError(status, msg)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def version() -> int:
    return int(load().hsb_version())


def params(form="discrete", prec="auto", **kw) -> Params:
    """hsb_params from the library defaults, with overrides by field name."""
    p = Params()
    _check(load().hsb_params_default(C.byref(p)))
    p.form = FORM[form] if isinstance(form, str) else int(form)
    p.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    if isinstance(kw.get("schedule"), str):
        kw["schedule"] = SCHEDULE[kw["schedule"]]
    if isinstance(kw.get("thermostat"), str):
        kw["thermostat"] = THERMOSTAT[kw["thermostat"]]
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(f"hsb_params has no field {k!r}")
        setattr(p, k, v)
    return p


def create(J: np.ndarray) -> int:
    """hsb_create: J is copied to the current CUDA device; returns the handle."""
    J = np.ascontiguousarray(J, dtype=np.float32)
    if J.ndim != 2 or J.shape[0] != J.shape[1]:
        raise ValueError("J must be a square matrix")
    h = C.c_void_p()
    _check(load().hsb_create(_ptr(J), J.shape[0], C.byref(h)))
    return h.value


def destroy(h: int) -> None:
    load().hsb_destroy(C.c_void_p(h))


def set_stream(h: int, stream_ptr: int | None) -> None:
    _check(load().hsb_set_stream(C.c_void_p(h), C.c_void_p(stream_ptr or 0)))


def info(h: int):
    n, pm1 = C.c_int(), C.c_int()
    _check(load().hsb_info(C.c_void_p(h), C.byref(n), C.byref(pm1)))
    return n.value, bool(pm1.value)


def cut_values(h: int, best_energy: np.ndarray) -> np.ndarray:
    """hsb_cut_values: MAX-CUT values (weights w = -J) of the given energies."""
    e = np.ascontiguousarray(best_energy, dtype=np.float64)
    cut = np.empty_like(e)
    _check(load().hsb_cut_values(C.c_void_p(h), int(e.shape[0]), _ptr(e), _ptr(cut)))
    return cut


def run(h: int, p: Params, R: int, steps: int, seed: int):
    """hsb_run with host outputs: (best_spins int8 [R, N], best_energy float64 [R])."""
    n, _ = info(h)
    spins = np.empty((R, n), np.int8)
    energy = np.empty(R, np.float64)
    _check(load().hsb_run(C.c_void_p(h), C.byref(p), int(R), int(steps),
                          C.c_uint64(seed & (2**64 - 1)), _ptr(spins), _ptr(energy)))
    return spins, energy


def run_device(h: int, p: Params, R: int, steps: int, seed: int, spins_ptr: int,
               energy_ptr: int) -> None:
    """hsb_run_device: outputs are device pointers (e.g. torch tensor data_ptr())."""
    _check(load().hsb_run_device(C.c_void_p(h), C.byref(p), int(R), int(steps),
                                 C.c_uint64(seed & (2**64 - 1)), C.c_void_p(spins_ptr),
                                 C.c_void_p(energy_ptr)))


def get_state(h: int, R: int):
    n, _ = info(h)
    x = np.empty((R, n), np.float32)
    y = np.empty((R, n), np.float32)
    _check(load().hsb_get_state(C.c_void_p(h), _ptr(x), _ptr(y)))
    return x, y


def advance(h: int, p: Params, steps: int, k_begin: int, k_end: int, x: np.ndarray,
            y: np.ndarray):
    """hsb_advance on copies of x, y (float32 [R, N]); returns the new (x, y)."""
    x = np.array(x, dtype=np.float32, order="C", copy=True)
    y = np.array(y, dtype=np.float32, order="C", copy=True)
    if x.ndim != 2 or x.shape != y.shape:
        raise ValueError("x and y must be [R, N]")
    _check(load().hsb_advance(C.c_void_p(h), C.byref(p), x.shape[0], int(steps), int(k_begin),
                              int(k_end), _ptr(x), _ptr(y)))
    return x, y


def advance_device(h: int, p: Params, R: int, steps: int, k_begin: int, k_end: int) -> None:
    """hsb_advance_device: continue the device-resident state (queued, no copies)."""
    _check(load().hsb_advance_device(C.c_void_p(h), C.byref(p), int(R), int(steps),
                                     int(k_begin), int(k_end)))


def set_couplings(h: int, J: np.ndarray) -> None:
    """hsb_set_couplings: new instance of the same N for an existing handle."""
    J = np.ascontiguousarray(J, dtype=np.float32)
    _check(load().hsb_set_couplings(C.c_void_p(h), _ptr(J)))


def run_batch(handles, p: Params, R: int, steps: int, seed: int):
    """hsb_run_batch: list of (best_spins int8 [R, N_b], best_energy float64 [R])."""
    count = len(handles)
    ns = [info(h)[0] for h in handles]
    spins = [np.empty((R, n), np.int8) for n in ns]
    energy = [np.empty(R, np.float64) for _ in ns]
    harr = (C.c_void_p * count)(*handles)
    sarr = (C.c_void_p * count)(*[a.ctypes.data for a in spins])
    earr = (C.c_void_p * count)(*[a.ctypes.data for a in energy])
    _check(load().hsb_run_batch(harr, count, C.byref(p), int(R), int(steps),
                                C.c_uint64(seed & (2**64 - 1)), sarr, earr))
    return list(zip(spins, energy))


def get_trace(h: int):
    """hsb_get_trace: float64 [n, 3] = (min E, mean E, mean T_inst) per traced time."""
    n = C.c_size_t()
    _check(load().hsb_get_trace(C.c_void_p(h), None, 0, C.byref(n)))
    buf = np.zeros((n.value, 3), np.float64)
    if n.value:
        _check(load().hsb_get_trace(C.c_void_p(h), _ptr(buf), n.value, C.byref(n)))
    return buf


def trace_cut(h: int):
    """The trace as cut values (the paper's instantaneous C and T_inst at every
    traced step): float64 [n, 3] = (max C, mean C, mean T_inst).  C = -E/2 -
    1/4 sum_ij J_ij (Eq. eq_Cut, w = -J) is affine in E with a negative slope,
    so the maximum cut is the cut of the minimum energy and the mean cut the
    cut of the mean energy."""
    tr = get_trace(h)
    if tr.shape[0] == 0:
        return tr
    return np.stack([cut_values(h, tr[:, 0]), cut_values(h, tr[:, 1]), tr[:, 2]], axis=1)


def get_xi(h: int, R: int):
    """hsb_get_xi: float64 [R], the Nose-Hoover xi of each replica after the last run."""
    xi = np.zeros(int(R), np.float64)
    _check(load().hsb_get_xi(C.c_void_p(h), int(R), _ptr(xi)))
    return xi


def debug_drop_publication(h: int, row_block: int) -> None:
    """hsb_debug_drop_publication: the next persistent FP8 run drops one tile's
    publication, so its bounded device waits expire (failure-detection tests)."""
    _check(load().hsb_debug_drop_publication(C.c_void_p(h), int(row_block)))


def debug_alloc_cap(nbytes: int) -> None:
    """hsb_debug_alloc_cap: device allocations of more than nbytes bytes fail
    with HSB_E_NOMEM from now on (process-wide; 0 removes the cap)."""
    _check(load().hsb_debug_alloc_cap(int(nbytes)))


def run_stats(h: int) -> int:
    """Kernels queued by the last run on the handle."""
    n = C.c_longlong()
    _check(load().hsb_run_stats(C.c_void_p(h), C.byref(n)))
    return int(n.value)


def run_fp32_noalloc(J_ptr: int, N: int, p: Params, R: int, steps: int, seed: int,
                     spins_ptr: int, energy_ptr: int, stream_ptr: int | None = None) -> None:
    """hsb_run_fp32_noalloc: device couplings and outputs, fixed scratch, no allocation."""
    _check(load().hsb_run_fp32_noalloc(C.c_void_p(J_ptr), int(N), C.byref(p), int(R),
                                       int(steps), C.c_uint64(seed & (2**64 - 1)),
                                       C.c_void_p(spins_ptr), C.c_void_p(energy_ptr),
                                       C.c_void_p(stream_ptr or 0)))


def synchronize(h: int) -> None:
    _check(load().hsb_synchronize(C.c_void_p(h)))


class Solver:
    """Owns one handle; thin convenience over the functions above."""

    def __init__(self, J: np.ndarray):
        self.n = int(np.asarray(J).shape[0])
        self.h = create(J)

    def run(self, p: Params, R: int, steps: int, seed: int):
        return run(self.h, p, R, steps, seed)

    def run_device(self, p, R, steps, seed, spins_ptr, energy_ptr):
        return run_device(self.h, p, R, steps, seed, spins_ptr, energy_ptr)

    def get_state(self, R: int):
        return get_state(self.h, R)

    def cut_values(self, best_energy):
        return cut_values(self.h, best_energy)

    def advance(self, p, steps, k_begin, k_end, x, y):
        return advance(self.h, p, steps, k_begin, k_end, x, y)

    def advance_device(self, p, R, steps, k_begin, k_end):
        return advance_device(self.h, p, R, steps, k_begin, k_end)

    def set_couplings(self, J):
        set_couplings(self.h, J)

    def run_stats(self):
        return run_stats(self.h)

    def get_trace(self):
        return get_trace(self.h)

    def get_xi(self, R: int):
        return get_xi(self.h, R)

    def trace_cut(self):
        return trace_cut(self.h)

    def set_stream(self, stream_ptr):
        set_stream(self.h, stream_ptr)

    def synchronize(self):
        synchronize(self.h)

    def close(self):
        if self.h:
            destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
