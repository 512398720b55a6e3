"""C-ABI checks that need no GPU: the library builds, loads, exports every
entry point declared in include/spfd.h, and rejects invalid arguments before
touching the device."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def spfd():
    from paper_2010_12879_gb300 import build as b
    b.build()
    import paper_2010_12879_gb300 as m
    m.lib()
    return m


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(spfd_[a-z_0-9]+)\s*\(", text))
    return names


def test_exports_every_declared_symbol(spfd):
    declared = _declared()
    assert declared, "no declarations found"
    assert declared == set(spfd.EXPORTS)
    L = spfd.lib()
    for name in declared:
        assert hasattr(L, name), name


def test_opts_default(spfd):
    o = spfd.spfd_opts_default()
    assert o.tol == 1e-8 and o.maxit == 200 and o.nu_pre == 1 and o.nu_post == 1
    assert o.precision == spfd.SPFD_FP64 and o.coarse_max == 512


def _raw_build(spfd, sigma, nx, ny, nz, h, out=True):
    L = spfd.lib()
    handle = ctypes.c_void_p()
    st = L.spfd_build(ctypes.c_void_p(sigma), nx, ny, nz, h, None, None,
                      ctypes.byref(handle) if out else None)
    return st, handle.value


@pytest.mark.parametrize("args", [
    (0, 4, 4, 4, 2e-3),            # null sigma
    (8, 0, 4, 4, 2e-3),            # zero dims
    (8, 4, -1, 4, 2e-3),
    (8, 4, 4, 4, 0.0),             # h <= 0
    (8, 4, 4, 4, float("nan")),
    (8, 4000, 4000, 4000, 2e-3),   # > 2^31 nodes
])
def test_build_rejects_invalid_arguments(spfd, args):
    st, h = _raw_build(spfd, *args)
    assert st == spfd.SPFD_EINVAL and h is None
    assert spfd.spfd_last_error()


def test_build_rejects_null_out(spfd):
    st, _ = _raw_build(spfd, 8, 4, 4, 4, 2e-3, out=False)
    assert st == spfd.SPFD_EINVAL


def test_null_context_calls(spfd):
    L = spfd.lib()
    info = spfd.SpfdInfo()
    assert L.spfd_solve(None, ctypes.c_void_p(8), 1e-8, ctypes.c_void_p(8), ctypes.byref(info)) == spfd.SPFD_EINVAL
    assert L.spfd_solve_host(None, ctypes.c_void_p(8), 1e-8, ctypes.c_void_p(8), None) == spfd.SPFD_EINVAL
    assert L.spfd_efield(None, ctypes.c_void_p(8), ctypes.c_void_p(8), 1.0, ctypes.c_void_p(8)) == spfd.SPFD_EINVAL
    assert L.spfd_get_info(None, ctypes.byref(info)) == spfd.SPFD_EINVAL
    L.spfd_destroy(None)  # no-op


@pytest.mark.parametrize("args", [
    (0, 8, 4, 4, 4, 2, 2),          # null b
    (8, 0, 4, 4, 4, 2, 2),          # null a
    (8, 1 << 20, 0, 4, 4, 2, 2),    # zero dims
    (8, 1 << 20, 4, 4, 4, 5, 2),    # root line outside (j0 > ny)
    (8, 1 << 20, 4, 4, 4, 2, -1),   # root line outside (k0 < 0)
    (8, 16, 4, 4, 4, 2, 2),         # a overlaps b
])
def test_tree_cotree_rejects_invalid_arguments(spfd, args):
    """Checked on the host before any launch (no GPU needed)."""
    b, a, nx, ny, nz, j0, k0 = args
    st = spfd.lib().spfd_tree_cotree(ctypes.c_void_p(b), nx, ny, nz, j0, k0, None,
                                     ctypes.c_void_p(a))
    assert st == spfd.SPFD_EINVAL
    assert spfd.spfd_last_error()


@pytest.mark.parametrize("args", [
    (0, 8, 4, 4, 4, 2e-3, 1.0),          # null sigma
    (8, 8, 0, 4, 4, 2e-3, 1.0),          # zero dims
    (8, 8, 4000, 4000, 4000, 2e-3, 1.0), # > 2^31 nodes
    (8, 8, 4, 4, 4, 2e-3, float("inf")), # omega not finite
])
def test_pipeline_host_rejects_invalid_arguments(spfd, args):
    """Checked on the host before any device work (no GPU needed)."""
    sig, a, nx, ny, nz, h, omega = args
    st = spfd.lib().spfd_pipeline_host(ctypes.c_void_p(sig), ctypes.c_void_p(a), nx, ny, nz,
                                       h, 1e-8, omega, None, None, ctypes.c_void_p(8),
                                       ctypes.c_void_p(8), None)
    assert st == spfd.SPFD_EINVAL
    assert spfd.spfd_last_error()


def test_invalid_options_rejected(spfd):
    L = spfd.lib()
    o = spfd.spfd_opts_default()
    o.maxit = 0
    handle = ctypes.c_void_p()
    st = L.spfd_build(ctypes.c_void_p(8), 4, 4, 4, 2e-3, ctypes.byref(o), None, ctypes.byref(handle))
    assert st == spfd.SPFD_EINVAL


@pytest.mark.parametrize("degree", [0, 9, -1])
def test_chebyshev_degree_out_of_range_rejected(spfd, degree):
    """The Chebyshev smoother takes degrees 1..8; others are an error
    (checked before any device work)."""
    L = spfd.lib()
    o = spfd.spfd_opts_default()
    o.smoother = spfd.SPFD_SMOOTHER_CHEBYSHEV
    o.cheb_degree = degree
    handle = ctypes.c_void_p()
    st = L.spfd_build(ctypes.c_void_p(8), 4, 4, 4, 2e-3, ctypes.byref(o), None, ctypes.byref(handle))
    assert st == spfd.SPFD_EINVAL and not handle.value
    assert "cheb_degree" in spfd.spfd_last_error()


def test_unknown_smoother_rejected(spfd):
    L = spfd.lib()
    o = spfd.spfd_opts_default()
    o.smoother = 7
    handle = ctypes.c_void_p()
    st = L.spfd_build(ctypes.c_void_p(8), 4, 4, 4, 2e-3, ctypes.byref(o), None, ctypes.byref(handle))
    assert st == spfd.SPFD_EINVAL and not handle.value


def test_without_gpu_build_reports_cuda_error(spfd):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, h = _raw_build(spfd, 8, 4, 4, 4, 2e-3)
    assert st == spfd.SPFD_ECUDA and h is None


def test_struct_layouts_match_header(spfd, tmp_path):
    """The ctypes structures of the binding have the size and field offsets
    of the C structures in include/spfd.h, as a C compiler lays them out
    (a field added on one side only would shift every later field)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"spfd_opts": spfd.SpfdOpts, "spfd_info": spfd.SpfdInfo,
               "spfd_kernel_stat": spfd.SpfdKernelStat, "spfd_tune_entry": spfd.SpfdTuneEntry}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "spfd.h"',
             "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for ln in out.split("\n"):
        if ln:
            cname, key, val = ln.split()
            got[(cname, key)] = int(val)
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert got[(cname, field)] == getattr(cls, field).offset, (cname, field)


def test_constants_match_header(spfd):
    """Every SPFD_* enumerator of include/spfd.h has the binding's value."""
    text = open(os.path.join(ROOT, "include", "spfd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    found = dict((k, int(v)) for k, v in re.findall(r"\b(SPFD_[A-Z0-9_]+)\s*=\s*(\d+)", text))
    assert len(found) >= 10
    for name, value in found.items():
        assert getattr(spfd, name) == value, name
