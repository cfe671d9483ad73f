"""The plain C client (tests/c_client/kc_count.c) on the GPU: its output equals
the oracle's result."""
import os
import subprocess

import numpy as np
import pytest

import synth
import paper_1712_03254_gb300 as kc

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_client_matches_oracle(oracle_mod, tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = kc.build()
    exe = tmp_path / "kc_count"
    subprocess.run(["gcc", "-std=c99", "-O2", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_client", "kc_count.c"), "-o", str(exe),
                    "-L", os.path.dirname(lib), "-l:" + os.path.basename(lib),
                    "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    w = synth.tiny(scale=0.05)
    rs = w.samples[0]
    text = "\n".join(rs.read(r) for r in range(rs.n_reads)) + "\n"
    out = subprocess.run([str(exe), "31", "24", "2"], input=text, capture_output=True, text=True, check=True,
                         timeout=300).stdout
    rows = [line.split("\t") for line in out.splitlines()]
    keys = np.array([int(a) for a, _ in rows], dtype=np.uint64)
    counts = np.array([int(b) for _, b in rows], dtype=np.uint32)
    ok, oc = oracle_mod.count(w).result()
    assert keys.size > 100
    assert np.array_equal(keys, ok) and np.array_equal(counts, oc[:, 0])
