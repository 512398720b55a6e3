"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle.

Tolerances (readings of Sec. II-A and the parity bar):
* Psi: ||Psi_gpu - Psi_oracle||_2 / ||Psi_oracle||_2 <= 1e-9 after
  per-component mean removal, the oracle solving to 1e-13 relative residual
  and the GPU to the same 1e-13 on the small grids (1e-12 on the 8 mm body):
  where |E| sits at the floor below, the bar is an absolute 1e-13 of the
  field scale, which a 1e-12 solve meets only by chance of its iteration
  path;
* |E|: max over conducting voxels of |dE| / max(E_oracle, 1e-6 max E_oracle)
  <= 1e-7, where the 1e-6 floor is taken of the larger of max E_oracle and
  the source field scale omega/h max|a| (so that fields which vanish
  identically are not compared noise against noise).
"""

import numpy as np
import pytest

from spfd_inputs import (loop_potential, random_phantom, sphere_phantom,
                         uniform_b_landau, uniform_b_symmetric)
from spfd_inputs import body_phantom

pytestmark = pytest.mark.gpu

OMEGA = 2 * np.pi * 85e3
PSI_TOL = 1e-9
E_TOL = 1e-7


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_12879_gb300 import build as b
    b.build()
    return torch


@pytest.fixture(scope="module")
def spfd(torch_cuda):
    import paper_2010_12879_gb300 as m
    return m


def _dev(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _gpu_solve(torch, spfd, ph, a, tol=1e-12, **opts):
    sig = _dev(torch, ph.sigma)
    ad = _dev(torch, a)
    with spfd.Solver(sig, ph.h, **opts) as S:
        psi, info, st = S.solve(ad, tol)
        E = S.efield(ad, psi, OMEGA)
        torch.cuda.synchronize()
        return psi.cpu().numpy(), E.cpu().numpy(), info, st


def _compare(oracle, ph, a, psi_g, E_g, tol_psi=PSI_TOL, tol_e=E_TOL):
    psi_r, info_r, sys = oracle.solve(ph.sigma, ph.h, a, tol=1e-13)
    assert info_r["converged"]
    g = oracle.project(sys, sys.gather(psi_g))
    r = sys.gather(psi_r)
    # removed nodes are exactly zero on the GPU side
    full = psi_g.reshape(-1).copy()
    full[sys.nodes] = 0.0
    assert np.all(full == 0.0)
    nr = np.linalg.norm(r)
    err = np.linalg.norm(g - r) / nr if nr > 0 else np.linalg.norm(g)
    assert err <= tol_psi, f"psi rel L2 error {err:.3e}"
    E_r = oracle.efield(ph.sigma, a, psi_r, ph.h, OMEGA)
    m = ph.sigma > 0
    if m.any():
        # floor: 1e-6 of the field scale, the larger of max |E| and the
        # source scale omega/h*max|a| (fields that vanish identically, e.g. a
        # lone voxel, otherwise compare rounding noise with rounding noise)
        floor = 1e-6 * max(E_r[m].max(), OMEGA / ph.h * np.abs(a).max())
        e_err = (np.abs(E_g - E_r)[m] / np.maximum(E_r[m], floor)).max()
        assert e_err <= tol_e, f"|E| max rel error {e_err:.3e}"
    assert np.all(E_g[~m] == 0.0)
    return err


@pytest.mark.parametrize("gauge", ["symmetric", "landau"])
def test_sphere_parity(torch_cuda, spfd, oracle_mod, gauge):
    """The 32^3 sphere (R = 28 mm, h = 2 mm) in a uniform 27 uT field, both gauges."""
    ph = sphere_phantom()
    f = uniform_b_symmetric if gauge == "symmetric" else uniform_b_landau
    a = f(ph.dims, ph.h, ph.origin, 27e-6)
    psi, E, info, st = _gpu_solve(torch_cuda, spfd, ph, a, tol=1e-13)
    assert st == spfd.SPFD_OK and info["converged"] and info["rel_res_true"] <= 1e-13
    assert info["n_dof"] == 13469 and info["n_comp"] == 1
    _compare(oracle_mod, ph, a, psi, E)


@pytest.mark.parametrize("gauge", ["symmetric", "landau"])
def test_sphere_mixed_precision(torch_cuda, spfd, oracle_mod, gauge):
    """The same sphere and source through the mixed form (FP32
    V-cycle with BF16 level-0 conductances and FP32 accumulation inside FP64
    refinement).  Solved to 1e-13 it meets the FP64 parity bars; solved to
    the 1e-8 target its errors against the FP64 oracle stay at the level of
    that target (<= 1e-6 in Psi and in |E|)."""
    ph = sphere_phantom()
    f = uniform_b_symmetric if gauge == "symmetric" else uniform_b_landau
    a = f(ph.dims, ph.h, ph.origin, 27e-6)
    psi, E, info, st = _gpu_solve(torch_cuda, spfd, ph, a, tol=1e-13,
                                  precision=spfd.SPFD_MIXED)
    assert st == spfd.SPFD_OK and info["rel_res_true"] <= 1e-13 and info["outer_iters"] >= 2
    _compare(oracle_mod, ph, a, psi, E)
    psi, E, info, st = _gpu_solve(torch_cuda, spfd, ph, a, tol=1e-8,
                                  precision=spfd.SPFD_MIXED)
    assert st == spfd.SPFD_OK and info["rel_res_true"] <= 1e-8
    _compare(oracle_mod, ph, a, psi, E, tol_psi=1e-6, tol_e=1e-6)


@pytest.mark.parametrize("seed,dims,air", [
    (1, (21, 13, 17), 0.3),    # ragged tails on every axis, several bricks
    (2, (9, 30, 11), 0.6),     # many components
    (3, (40, 7, 5), 0.0),      # no air
    (4, (1, 1, 1), 0.0),       # one voxel
])
def test_random_phantom_parity(torch_cuda, spfd, oracle_mod, seed, dims, air):
    rng = np.random.default_rng(seed)
    ph = random_phantom(*dims, rng, air_fraction=air)
    nx, ny, nz = dims
    a = rng.normal(size=(3, nz + 1, ny + 1, nx + 1)) * 1e-9
    psi, E, info, st = _gpu_solve(torch_cuda, spfd, ph, a, tol=1e-13)
    assert st == spfd.SPFD_OK and info["rel_res_true"] <= 1e-13
    sys = oracle_mod.assemble(ph.sigma, ph.h)
    assert info["n_dof"] == sys.n and info["n_comp"] == sys.ncomp
    _compare(oracle_mod, ph, a, psi, E)


def test_coarse_level_with_more_bricks_than_fine(torch_cuda, spfd, oracle_mod):
    """64 separate 6^3-voxel blobs, one inside each odd-indexed 8^3-node
    brick of a 64^3 grid: each such brick has two coarse parent bricks per
    axis, so level 1 holds 125 bricks against level 0's 64 and is coarsened
    once more (64 components, ~22k unknowns)."""
    from types import SimpleNamespace
    n = 64
    rng = np.random.default_rng(5)
    sigma = np.zeros((n, n, n))
    for bz in (1, 3, 5, 7):
        for by in (1, 3, 5, 7):
            for bx in (1, 3, 5, 7):
                sigma[8 * bz + 1:8 * bz + 7, 8 * by + 1:8 * by + 7, 8 * bx + 1:8 * bx + 7] = \
                    rng.uniform(0.05, 1.0, size=(6, 6, 6))
    ph = SimpleNamespace(sigma=sigma, h=2e-3)
    a = rng.normal(size=(3, n + 1, n + 1, n + 1)) * 1e-9
    psi, E, info, st = _gpu_solve(torch_cuda, spfd, ph, a, tol=1e-13)
    assert st == spfd.SPFD_OK and info["rel_res_true"] <= 1e-13
    assert info["n_comp"] == 64 and info["n_levels"] >= 3
    _compare(oracle_mod, ph, a, psi, E)


def test_body_8mm_parity(torch_cuda, spfd, oracle_mod):
    """The body phantom at 8 mm (64 x 40 x 224 voxels, ~159k unknowns): many
    bricks, 40 tissue labels with 100x contrast, loop source."""
    ph = body_phantom(64, 40, 224, h=8e-3)
    a = loop_potential(ph.dims, ph.h, ph.origin)
    psi, E, info, st = _gpu_solve(torch_cuda, spfd, ph, a)
    assert st == spfd.SPFD_OK and info["rel_res_true"] <= 1e-12
    assert info["n_levels"] >= 3
    _compare(oracle_mod, ph, a, psi, E)


@pytest.mark.parametrize("dims", [(19, 10, 12), (150, 6, 5)])
def test_efield_kernel_matches_oracle_on_given_psi(torch_cuda, spfd, oracle_mod, dims):
    """|E| kernel alone: same (a, Psi) in, oracle's Eq. 1 evaluation out.
    Both evaluate each edge term as (a_e + Psi_head) - Psi_tail, add the four
    edges of an axis in the same order and contract no multiply-add, so the
    results are identical bit for bit.  (150, 6, 5) spans several warps and
    two blocks per row."""
    rng = np.random.default_rng(9)
    ph = random_phantom(*dims, rng, air_fraction=0.4)
    nx, ny, nz = ph.dims
    a = rng.normal(size=(3, nz + 1, ny + 1, nx + 1))
    psi = rng.normal(size=(nz + 1, ny + 1, nx + 1))
    torch = torch_cuda
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        E = S.efield(_dev(torch, a), _dev(torch, psi), OMEGA).cpu().numpy()
    E_r = oracle_mod.efield(ph.sigma, a, psi, ph.h, OMEGA)
    np.testing.assert_array_equal(E, E_r)


def test_all_air_grid(torch_cuda, spfd):
    torch = torch_cuda
    sigma = torch.zeros((5, 6, 7), dtype=torch.float64, device="cuda")
    a = torch.ones((3, 6, 7, 8), dtype=torch.float64, device="cuda")
    with spfd.Solver(sigma, 2e-3) as S:
        psi, info, st = S.solve(a, 1e-8)
        E = S.efield(a, psi, OMEGA)
    assert st == spfd.SPFD_OK and info["n_dof"] == 0
    assert torch.count_nonzero(psi).item() == 0 and torch.count_nonzero(E).item() == 0


def test_zero_source(torch_cuda, spfd):
    torch = torch_cuda
    ph = sphere_phantom(12, 2e-3, 0.008)
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        a = torch.zeros((3,) + S.node_shape, dtype=torch.float64, device="cuda")
        psi, info, st = S.solve(a, 1e-8)
    assert st == spfd.SPFD_OK and info["converged"]
    assert torch.count_nonzero(psi).item() == 0


def test_maxit_reports_not_converged(torch_cuda, spfd):
    torch = torch_cuda
    ph = sphere_phantom()
    a = uniform_b_landau(ph.dims, ph.h, ph.origin)
    with spfd.Solver(_dev(torch, ph.sigma), ph.h, maxit=2) as S:
        psi, info, st = S.solve(_dev(torch, a), 1e-12)
    assert st == spfd.SPFD_ENOTCONVERGED
    assert info["iters"] == 2 and not info["converged"] and info["rel_res_true"] > 1e-12
    assert torch.isfinite(psi).all()


@pytest.mark.parametrize("bad", [float("nan"), -1.0, float("inf")])
def test_invalid_sigma(torch_cuda, spfd, bad):
    torch = torch_cuda
    s = np.full((4, 4, 4), 0.3)
    s[2, 1, 3] = bad
    with pytest.raises(spfd.SpfdError) as e:
        spfd.Solver(_dev(torch, s), 2e-3)
    assert e.value.status == spfd.SPFD_EINVAL


def test_non_finite_source_rejected(torch_cuda, spfd):
    torch = torch_cuda
    ph = sphere_phantom(12, 2e-3, 0.008)
    a = uniform_b_landau(ph.dims, ph.h, ph.origin)
    a[0, 6, 6, 6] = np.nan  # an edge inside the sphere
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        with pytest.raises(spfd.SpfdError) as e:
            S.solve(_dev(torch, a), 1e-8)
        assert e.value.status == spfd.SPFD_EINVAL
        # the context stays usable
        psi, info, st = S.solve(_dev(torch, uniform_b_landau(ph.dims, ph.h, ph.origin)), 1e-8)
        assert st == spfd.SPFD_OK


def test_injected_allocation_failure_leaks_nothing(torch_cuda, spfd, monkeypatch):
    torch = torch_cuda
    ph = sphere_phantom()
    sig = _dev(torch, ph.sigma)
    torch.cuda.synchronize()
    spfd.spfd_release_cached_memory()
    free0, _ = torch.cuda.mem_get_info()
    for k in (1, 3, 7, 15, 40):
        monkeypatch.setenv("SPFD_FAIL_ALLOC_AT", str(k))
        with pytest.raises(spfd.SpfdError) as e:
            spfd.Solver(sig, ph.h)
        assert e.value.status == spfd.SPFD_ENOMEM
    monkeypatch.delenv("SPFD_FAIL_ALLOC_AT")
    torch.cuda.synchronize()
    # blocks of the failed builds went to the library's cache: hand them back
    assert spfd.spfd_release_cached_memory() > 0
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 < 8 << 20
    with spfd.Solver(sig, ph.h) as S:
        assert S.info()["n_dof"] == 13469


def test_host_array_entry_point(torch_cuda, spfd, oracle_mod):
    torch = torch_cuda
    ph = sphere_phantom()
    a = uniform_b_landau(ph.dims, ph.h, ph.origin)
    a_h = torch.from_numpy(a).pin_memory()
    psi_h = torch.empty(tuple(s + 1 for s in ph.sigma.shape), dtype=torch.float64).pin_memory()
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        info, st = S.solve_host(a_h, psi_h, 1e-12)
        psi_d, _, _ = S.solve(_dev(torch, a), 1e-12)
    assert st == spfd.SPFD_OK
    np.testing.assert_array_equal(psi_h.numpy(), psi_d.cpu().numpy())


@pytest.mark.parametrize("pinned", [True, False])
def test_host_pipeline_entry_point(torch_cuda, spfd, oracle_mod, pinned):
    """spfd_pipeline_host (host sigma and a in, host Psi and |E| out, the
    rows of a pulled selectively when the device can read the host memory,
    else copied whole) gives the device path's results bit for bit and the
    oracle's within the parity bar, on the 16 mm body (several bricks, air
    rows of a that are never read) and the sphere."""
    torch = torch_cuda
    for ph in (body_phantom(32, 20, 112, h=16e-3), sphere_phantom()):
        a = loop_potential(ph.dims, ph.h, ph.origin)
        nz, ny, nx = ph.sigma.shape
        if pinned:
            sig_h = torch.from_numpy(ph.sigma).pin_memory()
            a_h = torch.from_numpy(a).pin_memory()
            psi_h = torch.empty((nz + 1, ny + 1, nx + 1), dtype=torch.float64).pin_memory()
            E_h = torch.empty((nz, ny, nx), dtype=torch.float64).pin_memory()
        else:
            sig_h, a_h = ph.sigma.copy(), a.copy()
            psi_h = np.full((nz + 1, ny + 1, nx + 1), np.nan)
            E_h = np.full((nz, ny, nx), np.nan)
        st, info = spfd.pipeline_host(sig_h, a_h, ph.h, 1e-13, OMEGA, psi_h, E_h)
        assert st == spfd.SPFD_OK and info["rel_res_true"] <= 1e-13
        psi_p = np.asarray(psi_h)
        E_p = np.asarray(E_h)
        psi_d, E_d, info_d, st_d = _gpu_solve(torch, spfd, ph, a, tol=1e-13)
        np.testing.assert_array_equal(psi_p, psi_d)
        np.testing.assert_array_equal(E_p, E_d)
        assert info["iters"] == info_d["iters"]
        _compare(oracle_mod, ph, a, psi_p, E_p)


def test_sigma_at_an_8_byte_offset(torch_cuda, spfd):
    """A conductivity array that starts 8 bytes past a 16-byte boundary (a
    view into a larger tensor) gives the same operator, unknowns and Psi
    as an aligned copy: the classification falls back from paired loads."""
    torch = torch_cuda
    ph = body_phantom(32, 20, 112, h=16e-3)
    a = _dev(torch, loop_potential(ph.dims, ph.h, ph.origin))
    buf = torch.zeros(ph.sigma.size + 1, dtype=torch.float64, device="cuda")
    buf[1:] = torch.from_numpy(ph.sigma.reshape(-1)).cuda()
    sig_off = buf[1:].view(ph.sigma.shape)
    assert sig_off.data_ptr() % 16 == 8
    out = []
    for sig in (_dev(torch, ph.sigma), sig_off):
        with spfd.Solver(sig, ph.h) as S:
            psi, info, st = S.solve(a, 1e-10)
            assert st == spfd.SPFD_OK
            out.append((psi.clone(), info["n_dof"], info["iters"]))
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2]
    assert torch.equal(out[0][0], out[1][0])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_no_result_depends_on_unwritten_memory(torch_cuda, spfd, monkeypatch, precision):
    """Every device block the library hands out is first filled with NaN
    bytes (SPFD_POISON_ALLOC): build, solve to the rounding floor, |E| and the
    adjoint gradient on the 8 mm body give the same bits as with ordinary
    blocks, so nothing reads memory before writing it."""
    torch = torch_cuda
    ph = body_phantom(64, 40, 224, h=8e-3)
    a = _dev(torch, loop_potential(ph.dims, ph.h, ph.origin))
    sig = _dev(torch, ph.sigma)
    prec = spfd.SPFD_FP64 if precision == "fp64" else spfd.SPFD_MIXED
    out = []
    for poison in (False, True):
        if poison:
            monkeypatch.setenv("SPFD_POISON_ALLOC", "1")
        with spfd.Solver(sig, ph.h, precision=prec) as S:
            psi, info, st = S.solve(a, 1e-12)
            E = S.efield(a, psi, OMEGA)
            J, dJda, dJds, infoa, sta = S.energy_grad(a, psi, OMEGA, 1e-10)
            torch.cuda.synchronize()
            out.append((st, info["iters"], info["outer_iters"], psi.clone(), E.clone(), J,
                        dJds.clone()))
        monkeypatch.delenv("SPFD_POISON_ALLOC", raising=False)
    (s0, i0, o0, p0, e0, j0, d0), (s1, i1, o1, p1, e1, j1, d1) = out
    assert s0 == s1 == spfd.SPFD_OK and (i0, o0) == (i1, o1)
    assert torch.equal(p0, p1) and torch.equal(e0, e1) and j0 == j1
    assert torch.equal(d0, d1)


def test_cached_blocks_are_reused(torch_cuda, spfd):
    """A second build of the same model takes its device buffers from the
    library's cache: no net device memory is taken from the driver, and
    releasing the cache gives all of it back."""
    torch = torch_cuda
    ph = sphere_phantom()
    sig = _dev(torch, ph.sigma)
    torch.cuda.synchronize()
    spfd.spfd_release_cached_memory()
    with spfd.Solver(sig, ph.h) as S:
        held = S.info()["bytes_device"]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    with spfd.Solver(sig, ph.h) as S:
        assert S.info()["bytes_device"] == held
        free2, _ = torch.cuda.mem_get_info()
    assert free1 - free2 < (4 << 20)  # driver-internal allocations only
    assert spfd.spfd_release_cached_memory() >= held


def test_repeat_solves_are_deterministic(torch_cuda, spfd):
    torch = torch_cuda
    ph = body_phantom(32, 20, 112, h=16e-3)
    a = _dev(torch, loop_potential(ph.dims, ph.h, ph.origin))
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        p1, i1, _ = S.solve(a, 1e-10)
        p1 = p1.clone()
        p2, i2, _ = S.solve(a, 1e-10)
    assert i1["iters"] == i2["iters"]
    assert torch.equal(p1, p2)


@pytest.fixture(scope="module")
def body_2mm():
    """Full-size body phantom (256 x 160 x 896 voxels, h = 2 mm, 9,250,062
    unknowns) with the 0.3 m / 1000 A loop 0.4 m below it."""
    ph = body_phantom()
    a = loop_potential(ph.dims, ph.h, ph.origin)
    return ph, a


def test_body_full_size_properties(torch_cuda, spfd, oracle_mod, body_2mm):
    """At full size the oracle cannot solve in seconds, so the GPU result is
    checked through properties the oracle evaluates exactly: the true
    relative residual of Psi_gpu in the oracle's own assembled system, zero
    Psi off the unknowns, zero mean per component, and |E| against the
    oracle's Eq. 1 evaluation of the same Psi on every voxel."""
    torch = torch_cuda
    ph, a = body_2mm
    sig, ad = _dev(torch, ph.sigma), _dev(torch, a)
    with spfd.Solver(sig, ph.h) as S:
        psi_d, info, st = S.solve(ad, 1e-8)
        E = S.efield(ad, psi_d, OMEGA).cpu().numpy()
        psi = psi_d.cpu().numpy()
    assert st == spfd.SPFD_OK and info["n_dof"] == 9250062 and info["n_comp"] == 1
    sys = oracle_mod.assemble(ph.sigma, ph.h)
    assert sys.n == 9250062
    b = oracle_mod.project(sys, oracle_mod.rhs(sys, a))
    x = sys.gather(psi)
    r = b - oracle_mod.matvec(sys, x)
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert rel <= 1e-8
    assert abs(rel - info["rel_res_true"]) <= 1e-3 * rel + 1e-14
    assert abs(x.sum()) <= 1e-12 * np.abs(x).sum()
    full = psi.reshape(-1).copy()
    full[sys.nodes] = 0.0
    assert np.all(full == 0.0)
    E_r = oracle_mod.efield(ph.sigma, a, psi, ph.h, OMEGA)
    m = ph.sigma > 0
    floor = 1e-6 * max(E_r[m].max(), OMEGA / ph.h * np.abs(a).max())
    assert (np.abs(E - E_r)[m] / np.maximum(E_r[m], floor)).max() <= 1e-12
    assert np.all(E[~m] == 0.0)


def test_body_full_size_iteration_counts(torch_cuda, spfd, body_2mm):
    """Strength of the preconditioner at full size: the hierarchy takes the
    body to 1e-8 in 16 CG iterations in FP64 and in 17 inner iterations and
    2 refinement steps in the mixed form; the bounds leave two iterations of
    slack.  A weakened V-cycle (an inaccurate coarsest solve, a wrong
    transfer weight) shows here before it breaks convergence."""
    torch = torch_cuda
    ph, a = body_2mm
    sig, ad = _dev(torch, ph.sigma), _dev(torch, a)
    with spfd.Solver(sig, ph.h) as S:
        _, info, st = S.solve(ad, 1e-8)
    assert st == spfd.SPFD_OK and info["converged"] and info["rel_res_true"] <= 1e-8
    assert info["iters"] <= 18, info
    with spfd.Solver(sig, ph.h, precision=spfd.SPFD_MIXED) as S:
        _, info, st = S.solve(ad, 1e-8)
    assert st == spfd.SPFD_OK and info["converged"] and info["rel_res_true"] <= 1e-8
    assert info["iters"] <= 19 and info["outer_iters"] <= 3, info


def test_body_full_size_matches_oracle_samples(torch_cuda, spfd, body_2mm):
    """Full-size parity against the oracle's own solve of the same workload:
    tests/golden/body_2mm_oracle.json holds Psi (zero mean) of the oracle's
    Jacobi-PCG at its 1.4e-12 rounding floor at 4096 seeded unknowns, written
    by tests/golden/make_body_oracle_golden.py.  The GPU solve to 1e-12 must
    match those samples to 1e-9 relative (L2 over the samples)."""
    import json
    import os
    torch = torch_cuda
    ph, a = body_2mm
    with open(os.path.join(os.path.dirname(__file__), "golden", "body_2mm_oracle.json")) as f:
        gold = json.load(f)
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        psi, info, st = S.solve(_dev(torch, a), 1e-12)
    assert st == spfd.SPFD_OK and info["n_dof"] == gold["n_dof"]
    nodes = np.array(gold["psi_sample_nodes"], dtype=np.int64)
    want = np.array(gold["psi_sample_values"])
    got = psi.reshape(-1)[torch.from_numpy(nodes).cuda()].cpu().numpy()
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= 1e-9, f"sampled psi rel error {err:.3e}"


@pytest.mark.parametrize("precision,tol,psi_bar,E_bar", [
    ("fp64", 1e-12, 1e-9, 1e-7),
    ("mixed", 1e-12, 1e-9, 1e-7),
    ("fp64", 1e-8, 1e-5, 1e-5),
    ("mixed", 1e-8, 1e-5, 1e-5),
])
def test_body_full_size_error_against_oracle(torch_cuda, spfd, body_2mm, precision, tol,
                                             psi_bar, E_bar):
    """The error of each form against the oracle's floor solution of the full
    body (tests/golden/body_2mm_oracle.json): Psi at 4096 seeded unknowns
    (relative L2) and |E| at 8192 seeded conducting voxels (largest relative
    error, floor 1e-6 of the field scale, R9).  At the parity tolerance 1e-12
    both forms meet the 1e-9 / 1e-7 bars; at the timing tolerance 1e-8 a
    residual of 1e-8 bounds the error only through the conditioning of the
    operator, so the bound asserted is the stated one the benchmark reports
    against (1e-5)."""
    import json
    import os
    torch = torch_cuda
    ph, a = body_2mm
    with open(os.path.join(os.path.dirname(__file__), "golden", "body_2mm_oracle.json")) as f:
        gold = json.load(f)
    prec = spfd.SPFD_FP64 if precision == "fp64" else spfd.SPFD_MIXED
    ad = _dev(torch, a)
    with spfd.Solver(_dev(torch, ph.sigma), ph.h, precision=prec) as S:
        psi, info, st = S.solve(ad, tol)
        E = S.efield(ad, psi, OMEGA).reshape(-1)
    assert st == spfd.SPFD_OK and info["rel_res_true"] <= tol, (st, info)
    nodes = torch.tensor(gold["psi_sample_nodes"], dtype=torch.int64, device="cuda")
    vox = torch.tensor(gold["E_sample_voxels"], dtype=torch.int64, device="cuda")
    pw = np.array(gold["psi_sample_values"])
    ew = np.array(gold["E_sample_values"])
    pg = psi.reshape(-1)[nodes].cpu().numpy()
    eg = E[vox].cpu().numpy()
    err_psi = np.linalg.norm(pg - pw) / np.linalg.norm(pw)
    floor = 1e-6 * max(gold["E_max"], gold["E_floor_scale"])
    err_E = np.max(np.abs(eg - ew) / np.maximum(ew, floor))
    print(f"{precision} tol {tol:g}: psi {err_psi:.3e}, |E| {err_E:.3e}, "
          f"iters {info['iters']}/{info['outer_iters']}")
    assert err_psi <= psi_bar and err_E <= E_bar, (err_psi, err_E)


@pytest.mark.parametrize("dims", [(19, 10, 12), (150, 6, 5)])
def test_efield_complex_kernel_matches_oracle_on_given_psi(torch_cuda, spfd, oracle_mod, dims):
    """|E| of a complex source (reading R7) from given real and imaginary
    parts: the library's |E| of each part (bit-identical to the oracle's Eq. 1
    evaluation), squared, added and rooted with no contracted multiply-add,
    equals the oracle's definition bit for bit; a zero imaginary part gives
    the real |E|."""
    rng = np.random.default_rng(21)
    ph = random_phantom(*dims, rng, air_fraction=0.4)
    nx, ny, nz = ph.dims
    a_re = rng.normal(size=(3, nz + 1, ny + 1, nx + 1))
    a_im = rng.normal(size=(3, nz + 1, ny + 1, nx + 1))
    p_re = rng.normal(size=(nz + 1, ny + 1, nx + 1))
    p_im = rng.normal(size=(nz + 1, ny + 1, nx + 1))
    torch = torch_cuda
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        E = S.efield_complex(_dev(torch, a_re), _dev(torch, p_re), _dev(torch, a_im),
                             _dev(torch, p_im), OMEGA).cpu().numpy()
        z_a, z_p = torch.zeros_like(_dev(torch, a_im)), torch.zeros_like(_dev(torch, p_im))
        E0 = S.efield_complex(_dev(torch, a_re), _dev(torch, p_re), z_a, z_p, OMEGA).cpu().numpy()
        E_real = S.efield(_dev(torch, a_re), _dev(torch, p_re), OMEGA).cpu().numpy()
    E_r = oracle_mod.efield_complex(ph.sigma, a_re, p_re, a_im, p_im, ph.h, OMEGA)
    np.testing.assert_array_equal(E, E_r)
    np.testing.assert_array_equal(E0, E_real)


def test_complex_source_solved_as_a_batch_of_two(torch_cuda, spfd, oracle_mod):
    """A phasor source a = a_re + j a_im on the 8 mm body: its two parts
    solved as one batch of two right-hand sides to 1e-12, then |E| of the
    complex field, against the oracle's solves and its complex |E| at the
    parity bars (1e-9 in each Psi part, 1e-7 in |E|)."""
    torch = torch_cuda
    ph = body_phantom(64, 40, 224, h=8e-3)
    a_re = loop_potential(ph.dims, ph.h, ph.origin)
    a_im = loop_potential(ph.dims, ph.h, ph.origin, center=(0.1, -0.05, -0.5))
    A = torch.stack([_dev(torch, a_re), _dev(torch, a_im)])
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        psis, infos, st = S.solve_batch(A, 1e-12)
        assert st == spfd.SPFD_OK
        E = S.efield_complex(A[0], psis[0], A[1], psis[1], OMEGA).cpu().numpy()
        psis = psis.cpu().numpy()
    p_re, info_re, sys = oracle_mod.solve(ph.sigma, ph.h, a_re, tol=1e-13)
    p_im, info_im, _ = oracle_mod.solve(ph.sigma, ph.h, a_im, tol=1e-13, sys=sys)
    for g, r in ((psis[0], p_re), (psis[1], p_im)):
        gg, rr = oracle_mod.project(sys, sys.gather(g)), sys.gather(r)
        assert np.linalg.norm(gg - rr) <= 1e-9 * np.linalg.norm(rr)
    E_r = oracle_mod.efield_complex(ph.sigma, a_re, p_re, a_im, p_im, ph.h, OMEGA)
    m = ph.sigma > 0
    floor = 1e-6 * E_r[m].max()
    assert (np.abs(E - E_r)[m] / np.maximum(E_r[m], floor)).max() <= 1e-7
    assert np.all(E[~m] == 0)
