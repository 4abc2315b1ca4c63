"""The host-checked build (libdmas_checked.so: the library compiled with
DMAS_CHECKED, every shared- and global-memory index of the beamform,
every-order and envelope kernels tested before its access; a failed test sets
the error word, which dmas_plan_check reports as DMAS_EBOUNDS, and skips the
access).

The parity cases most likely to push an index past its buffer (frames of 1 to
257 samples, ragged direction groups and time tiles, several microphone
staging passes, wide delay spreads, interpolation fractions at the ends of
[0, 1), the every-order pass and mixed batches) run again in a child pytest
process that loads the checked library; every plan.check() in them must come
back clean, and their images must still match the oracle.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHECKED = os.path.join(ROOT, "paper_2511_09165_b300", "_lib", "libdmas_checked.so")

SELECTION = [
    ("test_gpu_parity.py", "short_frames or several_staging_passes or ragged_tiles or "
                           "microphone_chunks or weights_near_the_ends or every_order or "
                           "single_mic or order_above or zero_frame or newton_girard or "
                           "wide_tile"),
    ("test_gpu_orders.py", ""),
    ("test_gpu_serving.py", "bitwise or tile_cap"),
    ("test_zz_no_alloc.py", ""),
]


@pytest.mark.parametrize("path,expr", SELECTION, ids=[p for p, _ in SELECTION])
def test_parity_cases_under_the_host_checked_build(path, expr):
    assert os.path.exists(CHECKED), "build it with python -m paper_2511_09165_b300.build --both"
    env = dict(os.environ, DMAS_LIBRARY="checked")
    cmd = [sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-m", "gpu",
           os.path.join(ROOT, "tests", path)]
    if expr:
        cmd += ["-k", expr]
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    tail = (res.stdout + res.stderr)[-3000:]
    assert res.returncode == 0, tail
    assert " passed" in res.stdout and "failed" not in res.stdout, tail


def test_checked_library_is_the_one_loaded_in_the_child():
    code = ("import paper_2511_09165_b300 as dm; lib = dm.load_library(); "
            "print(lib._name)")
    env = dict(os.environ, DMAS_LIBRARY="checked")
    res = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    assert res.stdout.strip().endswith("libdmas_checked.so")
