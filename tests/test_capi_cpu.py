"""The C-ABI library on the CPU: it loads, exports every symbol the header
declares, computes its operator tables on the host (checked against the
oracle's independent construction) and rejects bad arguments before touching
a device."""
import ctypes

import numpy as np
import pytest

import oracle as O
from tests._helpers import header_functions


@pytest.fixture(scope="module")
def A():
    from paper_2306_11665_gb300 import build
    build.build()
    from paper_2306_11665_gb300 import _abi
    return _abi


def test_exports_every_header_symbol(A):
    names = header_functions()
    assert len(names) >= 16
    lib = ctypes.CDLL(A.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    # and the binding wraps each of them under the same name
    for n in names:
        assert hasattr(A, n), n


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("p", range(1, 9))
def test_operator_tables_vs_oracle(A, kind, p):
    xi, w, D, Q1 = A.sfh_operator_tables(p, kind)
    oxi, ow, oD, oQ1 = O.op1d(p, kind)
    assert np.abs(xi - oxi).max() < 2e-16
    assert np.abs(w - ow).max() < 1e-15
    assert np.abs(D - oD).max() < 1e-14 * max(1, np.abs(oD).max())
    assert np.abs(Q1 - oQ1).max() < 1e-15 * max(1, np.abs(oQ1).max())
    # exact symmetry of the node set
    assert np.array_equal(xi, -xi[::-1])


def test_bad_arguments_rejected(A):
    with pytest.raises(A.SfhError) as e:
        A.sfh_create(4, 3, 0, 6, 1)
    assert e.value.status == A.SFH_EINVAL
    for args in [(3, 0, 0, 5, 1), (3, 9, 0, 5, 1), (3, 3, 2, 5, 1), (3, 3, 0, 4, 1), (2, 3, 0, 2, 0), (3, 3, 0, 5, 7),
                 (3, 3, 0, 4, 2), (2, 3, 0, 1, 2), (3, 3, 0, 5, 3)]:
        with pytest.raises(A.SfhError) as e:
            A.sfh_create(*args)
        assert e.value.status == A.SFH_EINVAL, args
        assert A.sfh_last_error()
    with pytest.raises(A.SfhError) as e:
        A.sfh_volume_residual(0, 10, 1, 1, 1, 0, 0)
    assert e.value.status == A.SFH_EINVAL
    with pytest.raises(A.SfhError) as e:
        A.sfh_operator_tables(0, 0)
    assert e.value.status == A.SFH_EINVAL
    # the bound-metric entry points check their arguments before any CUDA call
    with pytest.raises(A.SfhError) as e:
        A.sfh_bind_metric(0, 10, 8)
    assert e.value.status == A.SFH_EINVAL
    with pytest.raises(A.SfhError) as e:
        A.sfh_volume_residual_host_bound(0, 10, 8, 8, A.SFH_FP32_KAHAN)
    assert e.value.status == A.SFH_EINVAL


def test_no_device_is_reported_not_crashed(A):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    for flux in (A.SFH_FLUX_EULER_RANOCHA, A.SFH_FLUX_EULER_CHANDRASHEKAR):
        with pytest.raises(A.SfhError) as e:
            A.sfh_create(3, 4, 0, 5, flux)
        assert e.value.status in (A.SFH_EUNSUPPORTED, A.SFH_ECUDA)


def test_basis_table_matches_the_oracle(A):
    """The library's modal basis tables (host code, no device) against the
    oracle's: orthonormal Legendre and the two Lagrange bases on both
    cubature node sets."""
    import oracle as O
    for p in (1, 4, 8):
        for kind in (0, 1):
            for basis in (A.SFH_BASIS_LEGENDRE, A.SFH_BASIS_LAGRANGE_GLL, A.SFH_BASIS_LAGRANGE_GAUSS):
                V = A.sfh_basis_table(p, kind, basis)
                assert np.abs(V - O.basis_1d(p, kind, basis)).max() <= 1e-14, (p, kind, basis)
    with pytest.raises(A.SfhError) as e:
        A.sfh_basis_table(4, 0, 3)
    assert e.value.status == A.SFH_EINVAL


@pytest.mark.parametrize("n_elem", [1 << 62, (1 << 63) - 1, 1 << 40, 1 << 24])
@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_refuses_huge_element_counts_before_any_device_call(A, n_elem, prec):
    """The allocation-free entry point caps the element count before any
    product with it (a byte count that wraps would otherwise pass the size
    check): the refusal is SFH_EINVAL with the cap in the message, and it comes
    before any CUDA call (on this machine without a GPU a CUDA call would give
    another status)."""
    u = np.zeros(16)
    Ja = np.zeros(16)
    r = np.zeros(16)
    st = A.lib().sfh_volume_residual_host_noalloc(3, 4, 0, A.SFH_FLUX_EULER_RANOCHA, n_elem, u.ctypes.data,
                                                   Ja.ctypes.data, r.ctypes.data, prec, None)
    assert st == A.SFH_EINVAL
    msg = A.sfh_last_error()
    assert "at most" in msg and "elements" in msg


def test_struct_layouts_match_the_header(A, tmp_path):
    """The ctypes structures of the binding have the C header's sizes and
    field offsets (compiled with the host C compiler, no GPU involved)."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    structs = {"sfh_request": A.Request, "sfh_result": A.Result, "sfh_server_opts": A.ServerOpts,
               "sfh_serve_stats_t": A.ServeStats}
    # C names of the fields the binding renames (lambda is a Python keyword)
    cname = {"lambda_": "lambda"}
    lines = ["#include <stddef.h>", "#include <stdio.h>", "#include \"sfhad.h\"", "int main(void) {"]
    for cs, py in structs.items():
        lines.append(f'    printf("{cs} %zu\\n", sizeof({cs}));')
        for f, _ in py._fields_:
            c = cname.get(f, f)
            lines.append(f'    printf("{cs}.{f} %zu\\n", offsetof({cs}, {c}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.splitlines())
    for cs, py in structs.items():
        assert int(got[cs]) == ctypes.sizeof(py), cs
        for f, _ in py._fields_:
            assert int(got[f"{cs}.{f}"]) == getattr(py, f).offset, (cs, f)
