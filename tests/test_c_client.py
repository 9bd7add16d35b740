"""The C ABI from plain C: tests/c_client/sfh_client.c is compiled with gcc
(C99, -Wall -Wextra -Werror -pedantic) against include/sfhad.h and linked to
libsfhad.so; its host-only calls run here, its FP64 residual on a GPU is
checked against the oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2306_11665_gb300 import inputs as I
from tests._helpers import ROOT, have_gpu, rel_err_per_var

SRC = os.path.join(ROOT, "tests", "c_client", "sfh_client.c")


def _cuda_root():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    from paper_2306_11665_gb300 import build
    lib = build.build()
    cuda = _cuda_root()
    exe = str(tmp_path_factory.mktemp("c_client") / "sfh_client")
    libdir = os.path.dirname(lib)
    cudalib = os.path.join(cuda, "lib64")
    if not os.path.exists(os.path.join(cudalib, "libcudart.so")):
        import glob
        cands = glob.glob(os.path.join(cuda, "targets", "*", "lib", "libcudart.so"))
        assert cands, "libcudart.so not found under the CUDA toolkit"
        cudalib = os.path.dirname(cands[0])
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-O1", SRC, "-o", exe,
           "-I", os.path.join(ROOT, "include"), "-isystem", os.path.join(cuda, "include"),
           "-L", libdir, "-l:libsfhad.so", f"-Wl,-rpath,{libdir}",
           "-L", cudalib, "-lcudart", f"-Wl,-rpath,{cudalib}"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    return exe


def test_host_calls_from_c(client):
    res = subprocess.run([client, "tables"], capture_output=True, text=True, timeout=60)
    assert res.returncode == 0, res.stderr
    out = dict(line.split(" ", 1) for line in res.stdout.strip().splitlines())
    xi, w, D, Q1 = (np.asarray(a) for a in _oracle_op1d(4, 0))
    vals = [float(x) for x in out["gll4"].split()[1:4]] + [float(x) for x in out["gll4"].split()[5:7]]
    assert np.allclose(vals, [xi[0], xi[1], xi[2], w[0], w[1]], rtol=0, atol=1e-15)
    V = O.basis_1d(3, 1, O.BASIS_LEGENDRE)
    leg = out["leg3"].split()
    assert abs(float(leg[1]) - V[0, 0]) < 1e-15 and abs(float(leg[3]) - V[1, 1]) < 1e-15
    assert out["bad_create"] == "1 msg"      # SFH_EINVAL with a message
    assert out["bad_basis"] == "1"


def _oracle_op1d(p, kind):
    n = p + 1
    xi, w, D, Q1 = np.zeros(n), np.zeros(n), np.zeros(n * n), np.zeros(n * n)
    O._check(O._load().orc_op1d(p, kind, O._p(xi), O._p(w), O._p(D), O._p(Q1)))
    return xi, w, D, Q1


@pytest.mark.gpu
def test_fp64_residual_from_c(client, tmp_path):
    assert have_gpu(), "GPU tests need a CUDA device"
    d, p, kind = 3, 3, 1
    u, Ja = I.workload(d, p, kind, 2)
    fu, fj, fr = (str(tmp_path / n) for n in ("u.bin", "Ja.bin", "r.bin"))
    np.ascontiguousarray(u).tofile(fu)
    np.ascontiguousarray(Ja).tofile(fj)
    res = subprocess.run([client, "residual", str(d), str(p), str(kind), str(u.shape[0]), fu, fj, fr],
                         capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stderr
    r = np.fromfile(fr, dtype=np.float64).reshape(u.shape)
    assert rel_err_per_var(r, O.volume_sf(d, p, kind, O.FLUX_EULER, u, Ja)) <= 1e-12
