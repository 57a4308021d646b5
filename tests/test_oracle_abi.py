"""The oracle's ctypes mirrors have the C layout of the oracle's structs
(sizes and field offsets as gcc lays them out), so every argument reaches
the C code as written."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_structs_match_the_c_layout():
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {"orc_params": oracle.Params, "orc3_params": oracle.Params3,
               "orc_stats": oracle.Stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ecmc_oracle.h"',
             '#include "ecmc_oracle3.h"', '#include "ecmc_oracle_stripes.h"', 'int main(void) {']
    for cname, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append('printf("orc_chain_rec %zu\\n", sizeof(orc_chain_rec));')
    for f in oracle.CHAIN_REC.names:
        lines.append('printf("orc_chain_rec.%s %%zu\\n", offsetof(orc_chain_rec, %s));' % (f, f))
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as fh:
            fh.write("\n".join(lines))
        r = subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "oracle"), src, "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    c = dict(ln.rsplit(" ", 1) for ln in out.splitlines())
    for cname, cls in structs.items():
        assert int(c[cname]) == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(c[cname + "." + f]) == getattr(cls, f).offset, (cname, f)
    assert int(c["orc_chain_rec"]) == oracle.CHAIN_REC.itemsize
    for f in oracle.CHAIN_REC.names:
        assert int(c["orc_chain_rec." + f]) == oracle.CHAIN_REC.fields[f][1], f
