"""The allocation-free residual entry point, called through the C ABI.

``spfd_residual_noalloc`` is for callers that cannot allocate device memory
while they check a solution: processes whose device memory another allocator
has reserved up front, or loops that must stay out of the allocator.  Its
result must agree with the relative residual the CPU oracle computes for the
same potential from its own right-hand side and matrix, and with what
``spfd_solve`` reports, within the tolerance the parity tests use for
residuals; it must do so on two calls in a row, because every call reuses the
same fixed device scratch array; and repeated calls must not take device
memory.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

from spfd_inputs import (body_phantom, loop_potential, random_phantom,
                         sphere_phantom, uniform_b_landau)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_12879_gb300 import build as b
    b.build()
    import paper_2010_12879_gb300 as spfd
    return torch, spfd


def _case(name):
    if name == "sphere":
        ph = sphere_phantom()
        return ph, uniform_b_landau(ph.dims, ph.h, ph.origin)
    if name == "body16":
        ph = body_phantom(32, 20, 112, h=16e-3)
        return ph, loop_potential(ph.dims, ph.h, ph.origin)
    rng = np.random.default_rng(31)
    ph = random_phantom(23, 11, 14, rng, air_fraction=0.5)
    nx, ny, nz = ph.dims
    return ph, rng.normal(size=(3, nz + 1, ny + 1, nx + 1)) * 1e-9


def _oracle_rel_res(ph, a, psi_host):
    """||b - A psi|| / ||b|| over the oracle's unknowns, b = -G^T M a
    unprojected (Eq. 3), from the oracle's assembled system."""
    import oracle
    sys_ = oracle.assemble(ph.sigma, ph.h)
    b = oracle.rhs(sys_, a)
    r = b - oracle.matvec(sys_, sys_.gather(psi_host))
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def _call(spfd, sig, ad, psi, dims, h, stream):
    nx, ny, nz = dims
    out = ctypes.c_double(-1.0)
    status = spfd.lib().spfd_residual_noalloc(
        ctypes.c_void_p(sig.data_ptr()), ctypes.c_void_p(ad.data_ptr()),
        ctypes.c_void_p(psi.data_ptr()), nx, ny, nz, h,
        ctypes.c_void_p(stream), ctypes.byref(out))
    assert status == spfd.SPFD_OK, spfd.spfd_last_error()
    return out.value


@pytest.mark.parametrize("name", ["sphere", "body16", "random"])
def test_noalloc_residual_matches_oracle_and_solver_report(env, name):
    torch, spfd = env
    ph, a = _case(name)
    sig = torch.from_numpy(ph.sigma).cuda()
    ad = torch.from_numpy(a).cuda()
    with spfd.Solver(sig, ph.h) as S:
        psi, info, st = S.solve(ad, 1e-10)
    assert st == spfd.SPFD_OK
    ref_solver = info["rel_res_true"]
    ref_oracle = _oracle_rel_res(ph, a, psi.cpu().numpy())
    stream = torch.cuda.current_stream().cuda_stream
    values = [_call(spfd, sig, ad, psi, ph.dims, ph.h, stream) for _ in range(2)]
    for v in values:
        assert abs(v - ref_oracle) <= 1e-3 * ref_oracle + 1e-14, (v, ref_oracle)
        assert abs(v - ref_solver) <= 1e-3 * ref_solver + 1e-14, (v, ref_solver)
    assert values[0] == values[1]


def test_noalloc_takes_no_device_memory(env):
    """After the first call (which loads the library's module on this device
    and looks up the scratch array), further calls leave the device's free
    memory unchanged."""
    torch, spfd = env
    ph, a = _case("body16")
    sig = torch.from_numpy(ph.sigma).cuda()
    ad = torch.from_numpy(a).cuda()
    psi = torch.zeros(tuple(d + 1 for d in ph.dims[::-1]), dtype=torch.float64,
                      device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    first = _call(spfd, sig, ad, psi, ph.dims, ph.h, stream)
    assert first == pytest.approx(1.0, rel=1e-12)  # psi = 0: r = b
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(4):
        assert _call(spfd, sig, ad, psi, ph.dims, ph.h, stream) == first
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0, (free0, free1)


def test_noalloc_rejects_grids_beyond_its_scratch(env):
    torch, spfd = env
    L = spfd.lib()
    out = ctypes.c_double(0.0)
    dummy = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    status = L.spfd_residual_noalloc(dummy, dummy, dummy, 599, 599, 599, 2e-3,
                                     None, ctypes.byref(out))
    assert status == spfd.SPFD_EINVAL
    assert "134217728" in spfd.spfd_last_error()
