"""The C ABI from plain C99: the header compiles with -std=c99 -pedantic -Werror (no C++
constructs leak into it) and a C program linked against the library parses DIMACS and
runs Algorithm 1 on the host (no GPU).  The expected figures follow from the instance:
x3 = x1 AND x2 in Tseitin form plus the unit clause x3 gives 3 variables, 2 primary
inputs, 1 output, 1 gate on 1 cone level; the CNF costs sum(len - 1) + (clauses - 1)
= 4 + 3 = 7 two-input operations, the circuit 1 gate + (outputs - 1) = 1 (Fig. 5)."""
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
PKG = ROOT / "paper_2502_08673_b300"


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c99_program_against_the_library(tmp_path):
    from paper_2502_08673_b300 import build
    lib = build.build()
    exe = tmp_path / "abi_from_c"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", str(ROOT / "include"),
                    str(ROOT / "tests" / "c" / "abi_from_c.c"), "-L", str(lib.parent), "-lsatsampler",
                    f"-Wl,-rpath,{lib.parent}", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert out == ["3", "2", "1", "1", "1", "7", "1"]


@pytest.mark.gpu
@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c99_sampler_end_to_end(gpu, tmp_path):
    """The whole sampler from a C program: every returned assignment satisfies the CNF
    (oracle check) and no assignment repeats."""
    import numpy as np
    import oracle
    from paper_2502_08673_b300 import build
    from workloads import planted_3sat
    lib = build.build()
    exe = tmp_path / "sample_from_c"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", str(ROOT / "include"),
                    str(ROOT / "tests" / "c" / "sample_from_c.c"), "-L", str(lib.parent), "-lsatsampler",
                    f"-Wl,-rpath,{lib.parent}", "-o", str(exe)], check=True)
    text = planted_3sat(50, 200, 1).dimacs()
    cnf_path, out_path = tmp_path / "in.cnf", tmp_path / "out.txt"
    cnf_path.write_text(text)
    subprocess.run([str(exe), str(cnf_path), str(out_path)], check=True)
    lines = out_path.read_text().split("\n")
    n_vars, n = (int(x) for x in lines[0].split())
    rows = [[int(h, 16) for h in ln.split()] for ln in lines[1:1 + n]]
    assert n_vars == 50 and n == len(rows) > 0
    assign = np.zeros((n, n_vars + 1), np.uint8)
    for i, r in enumerate(rows):
        for v in range(1, n_vars + 1):
            assign[i, v] = (r[(v - 1) // 64] >> ((v - 1) % 64)) & 1
    nv, cl = oracle.parse_dimacs(text)
    assert oracle.cnf_check(nv, cl, assign).all()
    assert len({tuple(r) for r in rows}) == n
