"""The index-checked build (compiled with -DLQ_BOUNDS): in a child process
that loads liblqdd_checked.so, the hopping kernels K1 and K2 (FP64, FP32,
df64, BF16), the full operator, the layout kernels, the clover build, the SAP
smoother, the batched hop in every launch form and the fermion-force kernels
run on 2^4 to 8^4 lattices; every index check must pass, every canary around
the caller's fields must be intact, and the operators must still match the
oracle.  compute-sanitizer is not available on these GPUs, so these checks
stand in for its out-of-bounds detection."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_index_checks_and_canaries_clean():
    from paper_2407_08092_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, LQ_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_child.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    rep = json.loads(r.stdout.strip().splitlines()[-1])
    assert rep["checked"] == 1, rep
    assert rep["violations"] == 0 and rep["status"] == 0, rep
    assert rep["bad_canaries"] == [], rep
    assert rep["failed"] == [], rep
