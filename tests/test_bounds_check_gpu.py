"""The parity cases again, through the bounds-checked build of the library.

libhr2_bounds.so is the same source compiled with HR2_BOUNDS_CHECK=1: before
the prep, forward and binning kernels read a record row, a table or operand
block, a row of the instrument operator or an output row, they check its
index against the buffer it lies in; a failed check sets a bit of the
batch's error word (reported as HR2_EBOUNDS by hr2_stream_check, which every
parity case calls) and skips the access.  Running the small and
maximum-size parity cases through it shows that none of those indices
leaves its buffer.  The library is loaded in a child process (a process
holds one build of the library).
"""
import os
import re
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = ("tiny_grids or maximum_sizes or mixed_absorber_counts or uneven_three_setups or stage_variants or "
         "launch_shapes or absorber_counts_level_gridded or low_wavenumbers or cia_only")


def test_parity_cases_pass_under_index_checks():
    from paper_1910_01070_b300 import build
    lib = build.build(bounds_check=True)
    env = dict(os.environ, HR2_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_parity_gpu.py"), "-q",
                        "-m", "gpu", "-p", "no:cacheprovider", "-k", CASES], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1800)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    m = re.search(r"(\d+) passed", tail)
    assert m and int(m.group(1)) >= 20 and "failed" not in tail, tail


def test_streamed_operand_cases_pass_under_index_checks():
    """The streamed operand's cases: the forward kernel's operand reads through each group's
    setup view (tile range and ring) checked against the view's bounds."""
    from paper_1910_01070_b300 import build
    lib = build.build(bounds_check=True)
    env = dict(os.environ, HR2_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_stream_operand_gpu.py"), "-q",
                        "-m", "gpu", "-p", "no:cacheprovider"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1800)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    m = re.search(r"(\d+) passed", tail)
    assert m and int(m.group(1)) >= 4 and "failed" not in tail, tail
