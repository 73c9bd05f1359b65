"""Planted mistakes in the CPU oracle are caught by its pins.

Each mutant is a copy of the oracle's C source with one plausible mistake
planted by a textual substitution: a dropped term or factor, a wrong sign, a
wrong index, an operand taken at the wrong time, an off-by-one.  The copy is
compiled with the oracle's own flags, the pin suite (test_oracle_pins.py) runs
against it in a child process, and at least one pin must fail.  The unmodified
source goes through the same harness first, so a broken harness cannot pass
for a caught mutant.

Not planted: changes that are no mistake for the inputs the method takes
(transposing J, which is symmetric; enumerating half of the states in the
brute force, which the global spin flip makes equivalent), and changes of
a reading the paper leaves open in the same way for the pins as for the
CUDA path (the instance stream offset of the generator).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")
IMPL = "hsb_oracle_impl.h"
MAIN = "hsb_oracle.c"

# (name, file, exact text, replacement); the text occurs once in the file.
MUTANTS = [
    # ---- force, Eqs. (eq_fb), (eq_fd)
    ("sgn of zero is -1", IMPL,
     "return x >= (REAL)0 ? (REAL)1 : (REAL)-1;",
     "return x > (REAL)0 ? (REAL)1 : (REAL)-1;"),
    ("binary64 force term subtracted", IMPL,
     "return acc + t;", "return acc - t;"),
    ("binary32 force fma operands swapped", IMPL,
     "fmaf((float)jv, (float)b, (float)acc)", "fmaf((float)jv, (float)acc, (float)b)"),
    ("binary32 force term rounded twice", IMPL,
     "return (REAL)fmaf((float)jv, (float)b, (float)acc);",
     "return (REAL)((float)acc + (float)jv * (float)b);"),
    ("integer force uses the row's own spin", IMPL,
     "acc += (int32_t)row[j] * (int32_t)stmp[j];",
     "acc += (int32_t)row[j] * (int32_t)stmp[i];"),
    ("ballistic force uses the row's own position", IMPL,
     "REAL b = form == 1 ? SFX(sgn)(x[j]) : x[j];",
     "REAL b = form == 1 ? SFX(sgn)(x[j]) : x[i];"),
    ("ballistic force takes the sign", IMPL,
     "REAL b = form == 1 ? SFX(sgn)(x[j]) : x[j];",
     "REAL b = SFX(sgn)(x[j]);"),
    ("binary64 force term without the state", IMPL,
     "REAL t = jv * b;", "REAL t = jv;"),
    ("integer couplings copied with the wrong sign", IMPL,
     "Jint[e] = (int8_t)J[e];", "Jint[e] = (int8_t)-J[e];"),
    # ---- symplectic Euler step, Eqs. (eq_SyEuY), (eq_SyEuX)
    ("c0 dropped from the force term", IMPL,
     "REAL u = c0 * f[i];", "REAL u = f[i];"),
    ("pump term dropped", IMPL,
     "REAL w = u - v;", "REAL w = u;"),
    ("pump term with the wrong sign", IMPL,
     "REAL w = u - v;", "REAL w = u + v;"),
    ("dt dropped from the momentum update", IMPL,
     "REAL wd = w * dt;", "REAL wd = w;"),
    ("momentum step as u dt - v dt", IMPL,
     "REAL wd = w * dt;", "REAL wd = u * dt - v * dt;"),
    ("a0 dt rounded twice", IMPL,
     "const REAL q = (REAL)(p->a0 * p->dt);", "const REAL q = (REAL)p->a0 * (REAL)p->dt;"),
    ("gamma dt rounded twice", IMPL,
     "const REAL g = (REAL)(p->gamma * p->dt);", "const REAL g = (REAL)p->gamma * (REAL)p->dt;"),
    ("xi dt rounded twice", IMPL,
     "const REAL gk = (REAL)(-xi * p->dt);", "const REAL gk = -(REAL)xi * (REAL)p->dt;"),
    ("p_k formed in binary32", IMPL,
     "pk[k] = (REAL)oracle_pump_factor(p->a0, k, steps);",
     "pk[k] = (REAL)p->a0 - (REAL)p->a0 * (REAL)k / (REAL)steps;"),
    ("position advanced with the old momentum", IMPL,
     "REAL qy = q * yt;", "REAL qy = q * y0;"),
    # ---- inelastic walls, Eqs. (eq_WallX), (eq_WallY)
    ("momentum kept at the upper wall", IMPL,
     "xn = (REAL)1;\n            ytt = (REAL)0;",
     "xn = (REAL)1;\n            ytt = yt;"),
    ("lower wall at +1", IMPL,
     "xn = (REAL)-1;", "xn = (REAL)1;"),
    # ---- heating, Eq. (eq_EuHeat)
    ("heating with the momentum after the step", IMPL,
     "REAL gy = g * y0;", "REAL gy = g * yt;"),
    ("heating with the wrong sign", IMPL,
     "y[i] = ytt + gy;", "y[i] = ytt - gy;"),
    ("heating term dropped", IMPL,
     "y[i] = ytt + gy;", "y[i] = ytt;"),
    # ---- Nose-Hoover, Eqs. (eq_NH1), (eq_NH)
    ("kinetic sum truncated instead of rounded", IMPL,
     "fabs(nearbyint((double)y[i] * 0x1p24))", "fabs(trunc((double)y[i] * 0x1p24))"),
    ("kinetic sum scaled by 2^-24", IMPL,
     "return (double)acc * 0x1p-48;", "return (double)acc * 0x1p-24;"),
    ("thermostat variable moves the wrong way", IMPL,
     "xi = xi + nh_h * (s2 - nh_NT);", "xi = xi - nh_h * (s2 - nh_NT);"),
    ("thermostat step as h S - h N T", IMPL,
     "xi = xi + nh_h * (s2 - nh_NT);", "xi = xi + (nh_h * s2 - nh_h * nh_NT);"),
    ("friction with the wrong sign", IMPL,
     "const REAL gk = (REAL)(-xi * p->dt);", "const REAL gk = (REAL)(xi * p->dt);"),
    ("xi reads the momenta before the update", IMPL,
     "SFX(update)(N, x, y, f, c0, pk[k], dt, q, gk);\n                    /* xi_{k+1} from the updated momenta, Eq. (eq_NH) */\n                    const double s2 = p->nh_sum == 1 ? SFX(oracle_kinetic_sum_q24)(y, N)\n                                                     : SFX(oracle_kinetic_sum)(y, N);",
     "const double s2 = p->nh_sum == 1 ? SFX(oracle_kinetic_sum_q24)(y, N)\n                                                     : SFX(oracle_kinetic_sum)(y, N);\n                    SFX(update)(N, x, y, f, c0, pk[k], dt, q, gk);"),
    ("Nose-Hoover runs take the kernels' quantised sum", IMPL,
     "const double s2 = p->nh_sum == 1 ?", "const double s2 = p->nh_sum != 1 ?"),
    ("binary64 kinetic sum in descending order", IMPL,
     "for (int i = 0; i < N; ++i) {\n            const double v = (double)y[i];",
     "for (int i = N - 1; i >= 0; --i) {\n            const double v = (double)y[i];"),
    ("exact square sum drops subnormal momenta", MAIN,
     "        if (sh < 0) {\n            sq >>= -sh;\n            sh = 0;\n        }",
     "        if (sh < 0)\n            continue;"),
    ("exact square sum truncated, not rounded", MAIN,
     "if (round && (sticky || (sig & 1u))) {", "if (0) {"),
    ("exact square sum rounds ties up", MAIN,
     "if (round && (sticky || (sig & 1u))) {", "if (round) {"),
    ("exact square sum drops the carry between limbs", MAIN,
     "        carry = c1 | c2;", "        carry = 0;"),
    ("N dropped from N T", IMPL,
     "const double nh_NT = (double)N * p->nh_T;", "const double nh_NT = p->nh_T;"),
    ("thermostat step M / dt in place of dt / M", IMPL,
     "const double nh_h = p->dt / p->nh_M;", "const double nh_h = p->nh_M / p->dt;"),
    # ---- trace, Eq. (eq_TInst), and the best-state bookkeeping
    ("instantaneous temperature not divided by N", IMPL,
     "trace_t[at] = t2 / (double)N;", "trace_t[at] = t2;"),
    ("instantaneous temperature from the positions", IMPL,
     "t2 += (double)y[i] * (double)y[i];", "t2 += (double)x[i] * (double)x[i];"),
    ("final step not evaluated", IMPL,
     "int is_eval = (k == steps) || (", "int is_eval = ("),
    ("best state is the last of equal energies", IMPL,
     "if (e < best) {", "if (e <= best) {"),
    ("evaluation cadence shifted by one step", IMPL,
     "k % p->eval_every == 0);", "k % p->eval_every == 1);"),
    # ---- energy and cut, Eqs. (eq_Ising), (eq_Cut)
    ("energy without the factor 1/2", MAIN,
     "return -0.5 * acc;", "return -acc;"),
    ("energy with s_i twice", MAIN,
     "acc += (double)J[(size_t)i * N + j] * (double)s[i] * (double)s[j];",
     "acc += (double)J[(size_t)i * N + j] * (double)s[i] * (double)s[i];"),
    ("cut with w = J instead of -J", MAIN,
     "acc += -(double)J[(size_t)i * N + j]", "acc += (double)J[(size_t)i * N + j]"),
    ("cut value counted from both ends", MAIN,
     "return 0.5 * acc;", "return acc;"),
    ("brute force reads one bit for every spin", MAIN,
     "s[i] = ((b >> i) & 1u) ? -1 : 1;", "s[i] = ((b >> 0) & 1u) ? -1 : 1;"),
    # ---- scale and pumping schedule
    ("sigma_J over N^2 pairs", MAIN,
     "sqrt(acc / ((double)N * (double)(N - 1)))", "sqrt(acc / ((double)N * (double)N))"),
    ("c0 with N in place of sqrt(N)", MAIN,
     "c1 / (sqrt((double)N) * oracle_sigma_j(J, N))", "c1 / ((double)N * oracle_sigma_j(J, N))"),
    ("pump factor a(t) in place of a0 - a(t)", MAIN,
     "return a0 - t;", "return t;"),
    ("pump a(t) without the factor a0", MAIN,
     "double t = a0 * (double)k;", "double t = (double)k;"),
    ("pump schedule over Ns - 1 steps", MAIN,
     "t = t / (double)steps;", "t = t / (double)(steps - 1);"),
    ("traced count off by one", MAIN,
     "return trace_every > 0 ? (steps - 1) / trace_every + 1 : 0;",
     "return trace_every > 0 ? steps / trace_every : 0;"),
    ("evaluation count off by one", MAIN,
     "return (eval_every > 0 ? (steps - 1) / eval_every : 0) + 1;",
     "return (eval_every > 0 ? steps / eval_every : 0) + 1;"),
    # ---- counter-based generator
    ("SplitMix64 second shift 28", MAIN,
     "z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;", "z = (z ^ (z >> 28)) * 0x94D049BB133111EBULL;"),
    ("x and y streams overlap", MAIN,
     "2u * (uint64_t)i + (uint64_t)(comp & 1)", "(uint64_t)i + (uint64_t)(comp & 1)"),
    ("initial values over twice the width", MAIN,
     "(float)(half_width / 16777216.0)", "(float)(half_width / 8388608.0)"),
    ("initial values on the closed interval", MAIN,
     "(float)(2.0 * (double)m + 1.0 - 16777216.0)", "(float)(2.0 * (double)m - 16777216.0)"),
]


def _compile(src_dir, dst_dir, edit=None):
    os.makedirs(dst_dir)
    for f in (MAIN, IMPL):
        shutil.copy(os.path.join(src_dir, f), dst_dir)
    if edit is not None:
        fname, old, new = edit
        path = os.path.join(dst_dir, fname)
        with open(path) as fh:
            text = fh.read()
        assert text.count(old) == 1, f"{old!r} occurs {text.count(old)} times in {fname}"
        with open(path, "w") as fh:
            fh.write(text.replace(old, new))
    lib = os.path.join(dst_dir, "liboracle.so")
    subprocess.run(["gcc", *oracle.CFLAGS, "-o", lib, os.path.join(dst_dir, MAIN), "-lm"],
                   check=True, cwd=dst_dir, capture_output=True)
    return lib


def _run_pins(lib):
    env = dict(os.environ, HSB_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    proc = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           "-m", "not gpu", PINS],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return proc.returncode, proc.stdout[-2000:]


def test_mutant_texts_are_distinct():
    assert len({(f, old, new) for _, f, old, new in MUTANTS}) == len(MUTANTS)
    assert len({name for name, *_ in MUTANTS}) == len(MUTANTS)


@pytest.mark.timeout(900)
def test_every_planted_mistake_fails_a_pin(tmp_path):
    src = os.path.dirname(os.path.abspath(oracle.__file__))
    rc, out = _run_pins(_compile(src, str(tmp_path / "control")))
    assert rc == 0, "the unmodified oracle must pass its pins through this harness:\n" + out

    def one(k):
        name, fname, old, new = MUTANTS[k]
        lib = _compile(src, str(tmp_path / f"m{k:02d}"), (fname, old, new))
        return name, *_run_pins(lib)

    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with cf.ThreadPoolExecutor(workers) as pool:
        results = list(pool.map(one, range(len(MUTANTS))))
    # pytest exits 1 when a test failed; anything else (0: all passed, 2-5:
    # harness trouble, < 0: a crash) does not count as caught.
    survivors = [(name, rc, out) for name, rc, out in results if rc != 1]
    assert not survivors, "planted mistakes the pins did not catch:\n" + "\n".join(
        f"  {name}: pytest exit {rc}\n{out[-400:]}" for name, rc, out in survivors)
