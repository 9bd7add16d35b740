"""The bounds-checked debug build (libsfhad_debug.so, -DSFH_DEBUG).

Its kernels address global and shared memory through checked pointers: an
index outside its buffer latches SFH_EBOUNDS and the access is not made.  This
test builds it, checks that its self-test sees the checks act (a read and a
write outside a pointer's extent, kept inside the allocation so that nothing
could go wrong even unchecked), and runs the small-case parity tests of every
kernel family against it in a child process (SFH_LIB_VARIANT=debug): a
correct kernel must pass them with no index ever leaving its buffer, since
any such index would turn its status into SFH_EBOUNDS.  The release library
must report that it has no checks.
"""
import os
import subprocess
import sys

import pytest
import torch

from paper_2306_11665_gb300 import _abi as A

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# small-case parity and edge-case tests of the volume (all precisions and
# kernels), VJP, surface, modal and serving paths, and the metric-range errors
SELECTION = [
    ("tests/test_gpu_volume.py",
     "parity_small or edge_cases or rough_states or domain_error or host_entry_point or bound_metric"),
    ("tests/test_gpu_vjp.py", "parity_small"),
    ("tests/test_gpu_surface.py", "parity_small or errors_and_domain"),
    ("tests/test_gpu_chandrashekar.py", "parity_small_all_modes or vjp_parity"),
    ("tests/test_gpu_modal.py", "all_modes or uncollocated or unaligned or modal_vjp_parity"),
    ("tests/test_gpu_serve.py", "alone_equals_in_the_mix or chandrashekar_requests"),
    ("tests/test_gpu_metric_range.py", ""),
]


def _env():
    env = dict(os.environ)
    env["SFH_LIB_VARIANT"] = "debug"
    return env


def test_release_library_has_no_checks():
    from paper_2306_11665_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    if A.LIB_VARIANT == "debug":
        pytest.skip("this process runs the debug library")
    assert A.sfh_build_flags() & A.SFH_BUILD_DEBUG == 0
    assert A.sfh_selftest_bounds() == A.SFH_EUNSUPPORTED


def test_debug_build_self_test_and_small_parity():
    from paper_2306_11665_gb300 import build
    path = build.build(debug=True)
    assert os.path.basename(path) == "libsfhad_debug.so"
    probe = ("from paper_2306_11665_gb300 import _abi as A\n"
             "assert A.LIB_PATH.endswith('libsfhad_debug.so'), A.LIB_PATH\n"
             "assert A.sfh_build_flags() & A.SFH_BUILD_DEBUG\n"
             "assert A.sfh_selftest_bounds() == A.SFH_OK\n"
             "print('debug build self-test ok')\n")
    r = subprocess.run([sys.executable, "-c", probe], cwd=ROOT, env=_env(), capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    for f, k in SELECTION:
        cmd = [sys.executable, "-m", "pytest", f, "-m", "gpu", "-q", "-x", "-p", "no:cacheprovider"]
        if k:
            cmd += ["-k", k]
        r = subprocess.run(cmd, cwd=ROOT, env=_env(), capture_output=True, text=True, timeout=1800)
        tail = (r.stdout + r.stderr)[-3000:]
        assert r.returncode == 0, f"{f} on the debug build:\n{tail}"
        assert " passed" in r.stdout and "error" not in r.stdout.splitlines()[-1], tail
