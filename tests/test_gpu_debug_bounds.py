"""The index-checking build (-DFLAME_DEBUG_BOUNDS, libflame_debug.so).

It checks every computed global-memory index of the step passes, the
standalone FFT passes and flame_state_from_field against the extent of its
array before the access, skips a failing access and reports it through the
handle's status words (FLAME_EBOUNDS).  It stands in for a memory checker.

- The reporting path is seen through flame_debug_bounds_probe, which runs one
  check with no memory access at all: nothing out of range is ever touched.
- A selection of the GPU parity tests (tiny grids from 16 x 32 up to the
  4096 x 8192 benchmark grid, both precisions, every integrator, forcing,
  the per-step record with the area, ensembles, the fused column pass, the
  warp-local pass B variant, the standalone FFTs, host-buffer steps) runs again in a child process against
  the index-checking library: each must still match the oracle, and no
  handle may end with a failed check (conftest's autouse fixture).
- The normal library has no checks: the probe answers FLAME_EUNSUPPORTED.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# tests re-run under the index checks (pytest -k expression over the files below)
CHILD_FILES = ["tests/test_gpu_step.py", "tests/test_gpu_schemes.py", "tests/test_gpu_fft.py",
               "tests/test_diagnostics.py"]
CHILD_SELECT = ("one_step_identical_input or linear_and_nonlinear_only or fp32_full_size_one_step "
                "or batch_equals_individual or batch_of_compile_time_grids or fused_multi_step "
                "or state_from_field or heun_step_matches or fp64_short_line or host_buffers "
                "or if_step_matches or forcing_matches or multi_step_graphs "
                "or r2c_c2r_parity or device_record or warp_local_rows")


def _debug_env():
    env = dict(os.environ)
    env["FLAME_DEBUG_BOUNDS"] = "1"
    return env


@pytest.fixture(scope="module")
def debug_lib():
    from paper_0911_2889_gb300 import build
    return build.build_library(debug=True)


PROBE = r"""
import torch
from paper_0911_2889_gb300 import flame
assert flame.debug_bounds() and flame.library_path().endswith("libflame_debug.so")
f = flame.Flame(16, 32, prec="fp64")
flame.flame_debug_bounds_probe(f.h, 2, 3)      # in range: nothing recorded
f.sync_status()
flame.flame_debug_bounds_probe(f.h, 5, 3)      # out of range: recorded, no access
flame.flame_debug_bounds_probe(f.h, -1, 3)     # a second failure keeps the first record
try:
    f.sync_status()
except flame.FlameError as e:
    assert e.status == flame.FLAME_EBOUNDS, e
    msg = str(e)
    assert "site 17" in msg and "index 5" in msg and "[0, 3)" in msg, msg
else:
    raise SystemExit("no FLAME_EBOUNDS")
f.sync_status()                                # read and cleared
flame.flame_debug_bounds_probe(f.h, 7, 7)
f.close()
assert flame.bounds_failures and "index 7" in flame.bounds_failures[0], flame.bounds_failures
print("probe ok")
"""


@pytest.mark.gpu
def test_probe_reports_an_index_outside_its_array(debug_lib):
    r = subprocess.run([sys.executable, "-c", PROBE], cwd=ROOT, env=_debug_env(), capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and "probe ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]


@pytest.mark.gpu
def test_parity_suite_runs_clean_under_index_checks(debug_lib):
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           "-k", CHILD_SELECT, *CHILD_FILES]
    r = subprocess.run(cmd, cwd=ROOT, env=_debug_env(), capture_output=True, text=True, timeout=3000)
    tail = r.stdout[-4000:] + r.stderr[-2000:]
    assert r.returncode == 0, tail
    assert " passed" in tail and "failed" not in tail, tail


@pytest.mark.gpu
def test_normal_build_has_no_checks(fl):
    if fl.debug_bounds():
        pytest.skip("this process runs the index-checking library")
    f = fl.Flame(16, 32, prec="fp64")
    with pytest.raises(fl.FlameError) as e:
        fl.flame_debug_bounds_probe(f.h, 5, 3)
    assert e.value.status == fl.FLAME_EUNSUPPORTED
    f.sync_status()
    f.close()
