"""The benchmark's reference arm (`bench.py --impl reference`, the oracle timed
on the host cores) needs no GPU: its JSON line keeps the contract, and under
a multi-rank launch only rank 0 works and prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(env_extra, *args):
    env = dict(os.environ)
    env.update(env_extra)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", *args], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=300)
    return r.returncode, r.stdout


def test_reference_arm_prints_one_contract_line():
    rc, out = run({}, "--workload", "small", "--steps", "2", "--warmup", "3")
    assert rc == 0
    lines = [ln for ln in out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["unit"] == "events/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_other_ranks_exit_without_work():
    rc, out = run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"},
                  "--workload", "small", "--steps", "2", "--warmup", "3")
    assert rc == 0 and out.strip() == ""


def _reference_run_loads(*args):
    # run the reference arm in a fresh interpreter and report whether the
    # product package or its library was loaded on the way
    code = ("import runpy, sys\n"
            "sys.argv = ['bench.py', '--impl', 'reference'] + %r\n"
            "try:\n"
            "    runpy.run_path('bench.py', run_name='__main__')\n"
            "except SystemExit:\n"
            "    pass\n"
            "maps = open('/proc/self/maps').read()\n"
            "print('PACKAGE', 'paper_1409_6948_gb300' in sys.modules)\n"
            "print('LIBECMC', 'libecmc' in maps)\n"
            "print('LIBORACLE', 'liboracle' in maps)\n" % (list(args),))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    lines = dict(ln.split() for ln in r.stdout.splitlines() if ln.startswith(("PACKAGE",
                                                                               "LIBECMC",
                                                                               "LIBORACLE")))
    return lines


def test_reference_arm_runs_without_the_product_library():
    # the default workload picks its cells and ell by the paper's strategy;
    # the reference arm takes that choice from the oracle
    got = _reference_run_loads("--steps", "1", "--warmup", "3", "--melt", "0")
    assert got == {"PACKAGE": "False", "LIBECMC": "False", "LIBORACLE": "True"}
    got = _reference_run_loads("--workload", "eos", "--steps", "2", "--warmup", "3")
    assert got == {"PACKAGE": "False", "LIBECMC": "False", "LIBORACLE": "True"}
