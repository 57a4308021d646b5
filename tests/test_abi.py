"""The C-ABI library (no GPU needed): it loads, exports every function that
the headers under include/ declare, and rejects invalid arguments
before touching the device."""
import ctypes as C
import os
import re

import pytest

import paper_1409_6948_gb300 as P
from paper_1409_6948_gb300 import ecmc as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        with open(os.path.join(ROOT, "include", fn)) as f:
            src = f.read()
        names += re.findall(r"^ECMC_API\s+[\w\s\*]+?\b(ecmc3?_\w+)\s*\(", src, re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ecmc_create", "ecmc_sweep", "ecmc_positions", "ecmc_pressure",
                     "ecmc_destroy", "ecmc_set_stream", "ecmc_set_param", "ecmc_gr"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = C.CDLL(P.ecmc.library_path() if os.path.exists(P.ecmc.library_path()) else
                 E._build.build())
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(E._SIGS)


def test_version_and_messages():
    assert "sm_103a" in P.version()
    lib = P.load()
    for code in range(-9, 1):
        assert lib.ecmc_strerror(code).decode()


@pytest.mark.parametrize("args", [
    (255, 16.9, 1.0, 2, 2, 4.0, 1),      # N not a perfect square
    (256, 16.9, 1.0, 3, 2, 4.0, 1),      # odd number of cells
    (256, 16.9, 1.0, 0, 2, 4.0, 1),      # no cells
    (256, 16.9, 1.0, 18, 18, 4.0, 1),    # cell side below sigma
    (256, 15.0, 1.0, 2, 2, 4.0, 1),      # lattice spacing below sigma
    (256, 16.9, 1.0, 2, 2, -1.0, 1),     # negative displacement
    (256, -1.0, 1.0, 2, 2, 4.0, 1),      # negative box
])
def test_invalid_arguments_are_rejected_before_device_work(args):
    lib = P.load()
    h = C.c_void_p()
    rc = lib.ecmc_create(C.byref(h), *[C.c_int64(args[0]), C.c_double(args[1]),
                                       C.c_double(args[2]), C.c_int(args[3]), C.c_int(args[4]),
                                       C.c_double(args[5]), C.c_uint64(args[6])])
    assert rc == E.ERR_ARG and not h.value


@pytest.mark.parametrize("args", [
    (0, 10.0, 1.0, 2, 1.0, 1),           # no spheres
    (63, 10.0, 1.0, 2, 1.0, 1),          # N not a perfect cube
    (64, 10.0, 1.0, 3, 1.0, 1),          # odd cells per side
    (64, 10.0, 1.0, 12, 1.0, 1),         # cell side below sigma
    (1000, 9.0, 1.0, 2, 1.0, 1),         # cubic lattice spacing below sigma
    (64, 10.0, 1.0, 2, -1.0, 1),         # negative displacement
    (64, -1.0, 1.0, 2, 1.0, 1),          # negative box
])
def test_invalid_three_dimensional_arguments_are_rejected(args):
    lib = P.load()
    h = C.c_void_p()
    N, L, sigma, cells, ell, seed = args
    rc = lib.ecmc3_create(C.byref(h), N, L, sigma, cells, ell, seed)
    assert rc == E.ERR_ARG and not h.value


@pytest.mark.parametrize("args", [
    (0, 10.0, 1.0, 2, 1.0, 1),           # no disks
    (63, 10.0, 1.0, 2, 1.0, 1),          # N not a perfect square
    (64, 10.0, 1.0, 3, 1.0, 1),          # odd number of stripes
    (64, 10.0, 1.0, 12, 1.0, 1),         # stripe width below sigma
    (144, 11.0, 1.0, 2, 1.0, 1),         # square lattice spacing below sigma
    (64, 10.0, 1.0, 2, -1.0, 1),         # negative displacement
    (64, float("inf"), 1.0, 2, 1.0, 1),  # infinite box
])
def test_invalid_stripe_arguments_are_rejected(args):
    lib = P.load()
    h = C.c_void_p()
    N, L, sigma, stripes, ell, seed = args
    rc = lib.ecmc_stripes_create(C.byref(h), N, L, sigma, stripes, ell, seed)
    assert rc == E.ERR_ARG and not h.value
    assert lib.ecmc_stripes_create(None, 64, 10.0, 1.0, 2, 1.0, 1) == E.ERR_ARG


def test_null_handle_calls_fail_cleanly():
    lib = P.load()
    assert lib.ecmc_sweep(None, 1) == E.ERR_ARG
    assert lib.ecmc_destroy(None) == 0
    d = C.c_double()
    assert lib.ecmc_pressure(None, C.byref(d), None) == E.ERR_ARG
    assert lib.ecmc3_sweep(None, 1) == E.ERR_ARG
    assert lib.ecmc3_destroy(None) == 0
    assert lib.ecmc3_pressure(None, C.byref(d), None) == E.ERR_ARG
    assert lib.ecmc_stripes_sweep(None, 1) == E.ERR_ARG
    assert lib.ecmc_stripes_destroy(None) == 0
    assert lib.ecmc_stripes_pressure(None, C.byref(d), None) == E.ERR_ARG
    assert lib.ecmc_stripes_set_param(None, 1, 1.0) == E.ERR_ARG


def test_noalloc_rejects_invalid_arguments_before_device_work():
    # the allocation-free sweep shares the handle path's argument checks; each
    # of these returns before any CUDA call, so the pointer is never used
    lib = P.load()
    fake = C.c_void_p(256)
    L = 131600.0
    cases = [
        # cells_x * cells_y above 2^26 (the int cell count would overflow)
        (1000, L, 1.0, 131584, 130562, 8.0, 1, 0, 1),
        (256, 16.9, 1.0, 3, 2, 4.0, 1, 0, 1),      # odd cells
        (256, 16.9, 1.0, 2, 2, 4.0, 0, 0, 1),      # n_m < 1
        (256, 16.9, 1.0, 2, 2, 4.0, 1, -1, 1),     # t0 < 0
        (256, 16.9, 1.0, 2, 2, 4.0, 1, 0, -1),     # n_sweeps < 0
        (256, 16.9, 1.0, 18, 18, 4.0, 1, 0, 1),    # cell side below sigma
        (0, 16.9, 1.0, 2, 2, 4.0, 1, 0, 1),        # N < 1
    ]
    for (N, Lb, sig, cx, cy, ell, nm, t0, ns) in cases:
        rc = lib.ecmc_sweep_noalloc(fake, N, Lb, sig, cx, cy, ell, nm, 1, 0, t0, ns, None)
        assert rc == E.ERR_ARG, (N, cx, cy, nm, t0, ns, rc)
    assert lib.ecmc_sweep_noalloc(None, 256, 16.9, 1.0, 2, 2, 4.0, 1, 1, 0, 0, 1,
                                  None) == E.ERR_ARG


@pytest.mark.parametrize("N,eta", [(1048576, 0.72), (262144, 0.70), (4096, 0.60), (65536, 0.708),
                                   (4194304, 0.716)])
def test_suggested_parameters_follow_the_papers_strategy(N, eta):
    # Sec. 4: N / (eta n) > 100 for the largest such n; ell from eq. criterion;
    # n_m from eq. nm (host arithmetic only, no device needed)
    import math
    import ecmc_workloads as W
    L = W.box_side(N, eta)
    d = E.suggest_parameters(N, L)
    n = d["cells_x"] ** 2 / 4.0
    assert d["cells_x"] % 2 == 0 and d["cells_x"] == d["cells_y"]
    assert N / (eta * n) > 100.0
    n_next = (d["cells_x"] + 2) ** 2 / 4.0
    assert N / (eta * n_next) <= 100.0
    lam = (W.ETA_HCP - eta) / (2 * W.ETA_HCP)
    assert d["ell"] == pytest.approx(lam * math.sqrt(N / (eta * n)), rel=1e-12)
    assert d["ell"] > 10 * lam
    assert d["n_m"] == max(1, int(math.floor(N / (4 * n) * lam / d["ell"] + 0.5)))


def test_headers_compile_as_plain_c():
    # the boundary is a C ABI: every header must compile as C99 on its own,
    # and every declared function must be referable from C
    import shutil
    import subprocess
    import tempfile

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    names = declared_functions()
    headers = sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    src = "".join('#include "%s"\n' % f for f in headers)
    src += "typedef void (*fn)(void);\n"
    src += "fn refs[] = {%s};\n" % ", ".join("(fn)&%s" % n for n in names)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "use.c")
        with open(path, "w") as f:
            f.write(src)
        r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                            "-fsyntax-only", "-I", os.path.join(ROOT, "include"), path],
                           capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def header_constants():
    out = {}
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as f:
                for m in re.finditer(r"^#define\s+(ECMC\w*)\s+(-?\d+)\b", f.read(), re.M):
                    out[m.group(1)] = int(m.group(2))
    return out


def test_binding_constants_equal_the_headers():
    # ECMC_X -> X, ECMC3_PARAM_X -> PARAM3_X, ECMC_STRIPES_PARAM_X -> PARAM_STRIPES_X
    consts = header_constants()
    assert len(consts) > 40
    for name, value in consts.items():
        if name.startswith("ECMC3_PARAM_"):
            py = "PARAM3_" + name[len("ECMC3_PARAM_"):]
        elif name.startswith("ECMC_STRIPES_PARAM_"):
            py = "PARAM_STRIPES_" + name[len("ECMC_STRIPES_PARAM_"):]
        else:
            py = name[len("ECMC_"):]
        assert getattr(E, py) == value, (name, py)


def test_binding_structs_match_the_c_layout():
    # sizes and field offsets as the C compiler lays the header's structs out
    import shutil
    import subprocess
    import tempfile

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {"ecmc_counters_t": E.Counters, "ecmc_timing_t": E.Timing,
               "ecmc_tune_result_t": E.TuneResult, "ecmc_replica_desc_t": E.ReplicaDesc,
               "ecmc_geom_trial_t": E.GeomTrial}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ecmc.h"', 'int main(void) {']
    for cname, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append('printf("ecmc_chain_rec_t %zu\\n", sizeof(ecmc_chain_rec_t));')
    for f in E.CHAIN_REC.names:
        lines.append('printf("ecmc_chain_rec_t.%s %%zu\\n", offsetof(ecmc_chain_rec_t, %s));'
                     % (f, f))
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines))
        r = subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    c = dict(ln.rsplit(" ", 1) for ln in out.splitlines())
    for cname, cls in structs.items():
        assert int(c[cname]) == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(c[cname + "." + f]) == getattr(cls, f).offset, (cname, f)
    assert int(c["ecmc_chain_rec_t"]) == E.CHAIN_REC.itemsize
    for f in E.CHAIN_REC.names:
        assert int(c["ecmc_chain_rec_t." + f]) == E.CHAIN_REC.fields[f][1], f
