"""The C ABI from a plain C program (tests/c/consumer.c, compiled with gcc against
include/adscl.h and the in-tree libadscl.so): its results equal those of the same calls through
the Python binding bit for bit."""
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ad():
    from paper_1706_07413_b300 import adscl
    adscl.load()
    return adscl


def test_c_program_matches_python_binding(ad, tmp_path):
    from paper_1706_07413_b300 import build
    exe = tmp_path / "consumer"
    libdir = os.path.dirname(build.LIB)
    subprocess.run(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "consumer.c"), "-L", libdir, "-ladscl",
                    "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    lines = out.stdout.strip().splitlines()
    # the same calls through the Python binding
    B, K, J, S = 3, 6, 16, 3
    a = np.array([[0.1 * (b + 1) / (1.0 + k * k) for k in range(K)] for b in range(B)])
    s = ad.Solver([257, 513, 1025], ko_sigma=0.5, collapse_threshold=1.0 / 128.0, out_dt=0.25)
    s.set_initial_modes(a)
    th, qh, _ = s.track(0.0, 0.25, S, J, ad.PREC_FP64)
    tr, tc, m, st = s.evolve(0.5)
    for b in range(B):
        f = lines[b].split()
        assert int(f[0]) == b and int(f[1]) == st[b]
        assert float(f[2]) == tr[b] and float(f[3]) == m[b]
        assert [float(x) for x in f[4:7]] == list(qh[S - 1, b])
    Pi = s.get_state(0)[1]
    acc = 0.0
    for i, v in enumerate(Pi.tolist()):   # the C program's order of summation
        acc += v * (i + 1)
    assert lines[B] == "checksum %.17g" % acc
