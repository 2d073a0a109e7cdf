"""The smoother autotuner's choices kept across processes: with
AMR_SWEEP_TUNE_FILE set, the first process times the candidates and appends
its choices to the file; a later process reads them and times nothing (the
way a profiler run reproduces the plain run's launch shapes), and both
processes solve to the same bits."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
from paper_1812_03689_gb300 import amrmg
import hierarchies
H = amrmg.Hierarchy(32, 2, boxes=hierarchies.nested_centred(32), precision="mixed")
rng = np.random.default_rng(4)
for l in range(H.nlevels):
    H.set(l, "rho", rng.normal(size=H.shape(l)) * (H.mask(l) > 0))
H.solve(eps=1e-30, max_iter=2)
np.save({out!r}, np.concatenate([H.get(l, "phi").ravel() for l in range(H.nlevels)]))
"""


def run_child(tmp_path, tune, tag):
    out = str(tmp_path / f"phi_{tag}.npy")
    env = dict(os.environ, AMR_SWEEP_TUNE_FILE=tune, AMR_SWEEP_LOG="1",
               PYTHONPATH=os.path.join(ROOT, "tests") + os.pathsep + ROOT)
    env.pop("AMR_SWEEP", None)
    p = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, out=out)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return p.stderr, np.load(out)


def test_tune_file_written_then_reused(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_03689_gb300 import build
    build.build()
    tune = str(tmp_path / "tune.txt")
    err1, phi1 = run_child(tmp_path, tune, "first")
    assert "sweep-tune" in err1                      # candidates timed
    lines = [l.split() for l in open(tune).read().splitlines() if l.strip()]
    assert lines and all(len(l) == 4 for l in lines)
    assert all(l[0] == "4" for l in lines)           # FP32 smoothing (mixed form)
    err2, phi2 = run_child(tmp_path, tune, "second")
    assert "sweep-tune" not in err2                  # choices read, nothing timed
    assert np.array_equal(phi1, phi2)
