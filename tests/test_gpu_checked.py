"""The checked library (libfgl_checked.so, built with FGL_CHECKED): the
traversal kernels compare every node and triangle index with the scene's
record counts before reading it and report FGL_ERR_DEVICE instead of
reading out of range -- the debugging stand-in for a memory checker.  On the
workloads of tests/checked_cases.py it must report no error and return
results bitwise equal to the production library's.  It runs in a child
process (FGL_CHECKED=1), since a process loads one of the two libraries."""

import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
fgl = pytest.importorskip("paper_2509_17390_gb300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = """
import sys
import numpy as np
import torch
import paper_2509_17390_gb300 as fgl
from checked_cases import run_cases
assert fgl.lib()._name.endswith("libfgl_checked.so"), fgl.lib()._name
np.savez(sys.argv[1], **run_cases(fgl, torch))
"""


def test_checked_library_reports_nothing_and_matches(tmp_path):
    from paper_2509_17390_gb300 import build_native
    from checked_cases import run_cases
    build_native.build(checked=True)
    path = str(tmp_path / "checked.npz")
    path_dirs = [ROOT, os.path.join(ROOT, "tests"), os.environ.get("PYTHONPATH", "")]
    env = dict(os.environ, FGL_CHECKED="1", PYTHONPATH=os.pathsep.join(path_dirs))
    r = subprocess.run([sys.executable, "-c", CHILD, path], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert fgl.lib()._name.endswith("libfgl.so")
    prod = run_cases(fgl, torch)
    chk = np.load(path)
    assert sorted(chk.files) == sorted(prod)
    for k in prod:
        assert np.array_equal(prod[k], chk[k]), k
    assert int(chk["lbvh_overflow"][0]) == 0
    assert (prod["inst_fused_k"] >= 0).sum() > 100 and (prod["plain8_tri"] >= 0).mean() > 0.5
