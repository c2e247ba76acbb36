"""The library built with its device bounds checks (LF_CHECKED: every
data-dependent index of the traversal, the k-buffer hit codes and the ray
queues is checked; a failed check reports LF_ERR_BOUNDS, prints the index
and skips the access) runs the parity, gradient, edge-case, cross-state and
serving scenarios clean: no check fires and the results still match the
oracle.  compute-sanitizer is not available to this project, so this is the
memory-safety check of the kernels.  The scenarios run in a child process
that loads the checked build through LIGHTFUSE_LIB."""
import os
import re
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCENARIOS = [
    "tests/test_gpu_parity.py::test_c1_primary_gbuffer_parity",
    "tests/test_gpu_parity.py::test_c1_shaded_parity",
    "tests/test_gpu_parity.py::test_c2_one_bounce_parity_on_pixel_subset",
    "tests/test_gpu_parity.py::test_refit_matches_rebuild_bitwise",
    "tests/test_gpu_parity.py::test_c3_gradient_parity",
    "tests/test_gpu_edge_cases.py",
    "tests/test_gpu_state.py",
    "tests/test_gpu_serving.py::test_served_frames_equal_alone_and_plain_loop",
]


def test_checked_build_runs_the_scenarios_clean():
    from paper_2608_29269_b300.build import CHECKED_LIB, build_checked
    build_checked()
    env = dict(os.environ, LIGHTFUSE_LIB=CHECKED_LIB)
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider", *SCENARIOS]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    out = r.stdout + r.stderr
    assert "bounds check failed" not in out and "LF_ERR_BOUNDS" not in out, out[-4000:]
    assert r.returncode == 0, out[-4000:]
    m = re.search(r"(\d+) passed", out)
    print("checked build:", m.group(0) if m else out[-300:])
    assert m and int(m.group(1)) >= 15, out[-2000:]  # every scenario ran
