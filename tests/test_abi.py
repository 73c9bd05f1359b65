"""The C ABI library loads and exports every symbol include/hsb.h declares;
host-side validation and the no-device behaviour need no GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2203_08361_gb300 as hsb
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "hsb.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"HSB_API[^;(]*?\b(hsb_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    lib = hsb.load()
    declared = _declared()
    assert declared == sorted(hsb.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_version_and_defaults():
    assert hsb.version() == 2
    p = hsb.params()
    assert (p.form, p.prec) == (hsb.HSB_DISCRETE, hsb.HSB_PREC_AUTO)
    # the paper's tuned HdSB settings (Fig. 1 caption), a0 = 1 (Results)
    assert (p.a0, p.c1, p.dt, p.gamma, p.init_half_width, p.eval_every) == \
        (1.0, 0.7, 1.1, 0.06, 1.0, 100)
    # constant heating by default; Nose-Hoover fields at their documented offsets
    assert (p.thermostat, p.nh_T, p.nh_M, p.nh_xi0) == (0, 0.0, 1.0, 0.0)
    assert (hsb.Params.thermostat.offset, hsb.Params.nh_T.offset) == (72, 80)
    assert C.sizeof(hsb.Params) == 112


def test_create_validates_couplings_on_the_host():
    J = synth.sk_pm1(8, 0)
    bad = J.copy()
    bad[0, 1] = -bad[0, 1]
    with pytest.raises(hsb.HsbError) as e:
        hsb.create(bad)
    assert e.value.status == 2  # HSB_E_ASYM
    bad = J.copy()
    bad[3, 3] = 1.0
    with pytest.raises(hsb.HsbError) as e:
        hsb.create(bad)
    assert e.value.status == 3  # HSB_E_DIAG
    with pytest.raises(hsb.HsbError) as e:
        hsb.create(np.zeros((1, 1), np.float32))
    assert e.value.status == 1  # HSB_E_INVAL
    with pytest.raises(hsb.HsbError) as e:
        hsb.create(np.zeros((5, 5), np.float32))
    assert e.value.status == 1  # all zero
    bad = synth.sk_gauss(8, 0)
    bad[2, 5] = bad[5, 2] = np.inf  # symmetric, but not a finite coupling
    with pytest.raises(hsb.HsbError) as e:
        hsb.create(bad)
    assert e.value.status == 1 and "infinite" in str(e.value)


@pytest.mark.parametrize("n", [63, 64, 65, 200, 301])
def test_symmetry_check_covers_every_pair(n):
    # the host check walks 64 x 64 block pairs of the upper triangle: a single
    # broken pair anywhere (inside a block, across block edges, last row and
    # column, or a NaN) is found and named
    rng = np.random.default_rng(n)
    J = synth.sk_gauss(n, 1)
    pairs = [(0, 1), (0, n - 1), (n - 2, n - 1), (62 % (n - 1), 63 % n)]
    pairs += [tuple(sorted(rng.choice(n, 2, replace=False))) for _ in range(20)]
    for i, j in pairs:
        if i == j:
            continue
        for lower in (False, True):
            bad = J.copy()
            a, b = (j, i) if lower else (i, j)
            bad[a, b] = np.nextafter(bad[a, b], np.float32(np.inf))
            with pytest.raises(hsb.HsbError) as e:
                hsb.create(bad)
            assert e.value.status == 2, (i, j, lower)
            assert f"J[{min(i, j)}][{max(i, j)}]" in str(e.value)
    bad = J.copy()
    bad[n // 2, n // 3] = bad[n // 3, n // 2] = np.nan
    with pytest.raises(hsb.HsbError) as e:
        hsb.create(bad)
    assert e.value.status == 2


def test_no_cpu_fallback_without_a_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(hsb.HsbError) as e:
        hsb.create(synth.sk_pm1(8, 0))
    assert e.value.status == 8  # HSB_E_NODEVICE


def test_header_is_plain_c_and_matches_the_binding_layout(tmp_path):
    # include/hsb.h is a C ABI: it compiles as strict C11, and its parameter struct
    # has the size and offsets the ctypes mirror uses
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    checks = [f"_Static_assert(sizeof(hsb_params) == {C.sizeof(hsb.Params)}, \"size\");"]
    for name, _ in hsb.Params._fields_:
        off = getattr(hsb.Params, name).offset
        checks.append(f"_Static_assert(offsetof(hsb_params, {name}) == {off}, \"{name}\");")
    # and its enumerators have the values the binding passes and decodes
    consts = {name: code for code, name in hsb.STATUS.items()}
    consts.update({n: getattr(hsb, n) for n in (
        "HSB_BALLISTIC", "HSB_DISCRETE", "HSB_PREC_AUTO", "HSB_PREC_FP32", "HSB_PREC_FP8",
        "HSB_PREC_BF16X3", "HSB_HEAT_CONSTANT", "HSB_HEAT_NOSE_HOOVER")})
    for name, v in consts.items():
        checks.append(f"_Static_assert({name} == {v}, \"{name}\");")
    src = tmp_path / "abi_check.c"
    src.write_text("#include <stddef.h>\n#include \"hsb.h\"\n" + "\n".join(checks) +
                   "\nint main(void) { return 0; }\n")
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-pedantic", "-I", inc, "-c",
                        str(src), "-o", str(tmp_path / "abi_check.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    # and C++ clients include it as is (extern "C" linkage, no C-only syntax)
    gxx = shutil.which("g++")
    if gxx is not None:
        cxx = tmp_path / "abi_check.cpp"
        cxx.write_text("#include \"hsb.h\"\nint main() { hsb_params p; "
                       "return hsb_params_default(&p) == HSB_OK ? 0 : 1; }\n")
        r = subprocess.run([gxx, "-std=c++17", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                            inc, "-c", str(cxx), "-o", str(tmp_path / "abi_check_cxx.o")],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_a_c_program_links_and_calls_the_library(tmp_path):
    # A plain C11 client, linked against libhsb.so with nothing else: the
    # defaults, the host validation with its message, and hsb_create on valid
    # couplings (HSB_E_NODEVICE without a device, a handle otherwise).
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    hsb.load()
    libdir = os.path.dirname(hsb.LIB_PATH)
    src = tmp_path / "client.c"
    src.write_text(r"""
#include <stdio.h>
#include "hsb.h"
int main(void)
{
    hsb_params p;
    if (hsb_version() != HSB_API_VERSION || hsb_params_default(&p) != HSB_OK)
        return 10;
    if (p.form != HSB_DISCRETE || p.prec != HSB_PREC_AUTO || p.dt != 1.1)
        return 11;
    float bad[9] = {0, 1, -1, 1, 0, 1, -1, 2, 0}; /* J[1][2] = 1, J[2][1] = 2 */
    hsb_handle h = (hsb_handle)&p;
    if (hsb_create(bad, 3, &h) != HSB_E_ASYM || h != NULL)
        return 12;
    printf("asym: %s\n", hsb_last_error());
    if (hsb_create(bad, 1, &h) != HSB_E_INVAL)
        return 13;
    float J[9] = {0, 1, -1, 1, 0, 1, -1, 1, 0};
    hsb_status s = hsb_create(J, 3, &h);
    printf("create: %d\n", (int)s);
    if (s == HSB_OK)
        hsb_destroy(h);
    return 0;
}
""")
    exe = tmp_path / "client"
    inc = os.path.join(ROOT, "include")
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-pedantic", "-I", inc, str(src),
                        "-L", libdir, "-lhsb", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert "J[1][2]" in r.stdout
    torch = pytest.importorskip("torch")
    want = 0 if torch.cuda.is_available() else 8  # HSB_OK or HSB_E_NODEVICE
    assert f"create: {want}" in r.stdout


@pytest.mark.gpu
def test_a_c_program_runs_the_library_and_advances_a_worked_step(tmp_path):
    # A plain C11 client on a device: hsb_run on the antiferromagnetic
    # triangle (J = -1 on every pair), whose energies Eq. (eq_Ising) gives by
    # hand (tests/golden/worked_steps.json: 3 with no pair cut, -1 otherwise);
    # and hsb_advance over the hand-derived two-spin discrete step of the
    # same file (k = 0, so p_0 = a0; c0 = dt = 1/2, gamma dt = 1/8): the
    # positions and momenta it prints must be the worked values exactly.
    import json
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    hsb.load()
    libdir = os.path.dirname(hsb.LIB_PATH)
    with open(os.path.join(ROOT, "tests", "golden", "worked_steps.json")) as fh:
        golden = json.load(fh)
    step = next(c for c in golden["cases"] if c["name"] == "dsb_n2_no_wall")
    tri = next(c for c in golden["energies"]["cases"] if c["name"] == "antiferro_triangle")
    src = tmp_path / "runner.c"
    src.write_text(r"""
#include <stdio.h>
#include "hsb.h"
int main(void)
{
    float J[9] = {0, -1, -1, -1, 0, -1, -1, -1, 0};
    hsb_handle h;
    if (hsb_create(J, 3, &h) != HSB_OK)
        return 10;
    hsb_params p;
    hsb_params_default(&p);
    p.eval_every = 5;
    enum { R = 8 };
    int8_t spins[R * 3];
    double energy[R];
    if (hsb_run(h, &p, R, 60, 7, spins, energy) != HSB_OK)
        return 11;
    for (int r = 0; r < R; ++r)
        printf("run %d %d %d %.17g\n", spins[3 * r], spins[3 * r + 1], spins[3 * r + 2],
               energy[r]);
    hsb_destroy(h);

    float J2[4] = {0, 1, 1, 0};
    if (hsb_create(J2, 2, &h) != HSB_OK)
        return 12;
    hsb_params_default(&p);
    p.form = HSB_DISCRETE;
    p.prec = HSB_PREC_FP32;
    p.a0 = 1.0;
    p.c0 = 0.5;
    p.dt = 0.5;
    p.gamma = 0.25;
    float x[2] = {0.5f, -0.25f}, y[2] = {0.125f, 0.0f};
    if (hsb_advance(h, &p, 1, 4, 0, 1, x, y) != HSB_OK)
        return 13;
    printf("step %.9g %.9g %.9g %.9g\n", x[0], x[1], y[0], y[1]);
    hsb_destroy(h);
    return 0;
}
""")
    exe = tmp_path / "runner"
    inc = os.path.join(ROOT, "include")
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-pedantic", "-I", inc, str(src),
                        "-L", libdir, "-lhsb", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    lines = r.stdout.split("\n")
    runs = [ln.split()[1:] for ln in lines if ln.startswith("run ")]
    assert len(runs) == 8
    hand = {tuple(s): e for s, e in zip(tri["states"], tri["E"])}
    for fields in runs:
        s = tuple(int(v) for v in fields[:3])
        e = float(fields[3])
        # the energy of a state and of its global flip are equal
        key = s if s in hand else tuple(-v for v in s)
        assert e == hand[key], (s, e)
        assert e == tri["E_ground"]  # 60 heated steps find a frustrated ground state
    got = [float(v) for v in next(ln for ln in lines if ln.startswith("step ")).split()[1:]]
    assert got == step["x_next"] + step["y_next"]
