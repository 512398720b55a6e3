"""GPU parity of step 3 (Sec. II-A, Eq. 2): tree-cotree gauging of facet
fluxes into edge potentials, ``spfd_tree_cotree`` through the C ABI, against
the CPU oracle (``oracle.tree_cotree``, the definition solved by a sparse
least-squares solve on the same comb tree) and, at sizes the oracle cannot
solve, against properties that fix the result uniquely: a = 0 on the tree
edges, C a = b on every facet (the oracle's Eq. 2), and the same |E| as the
source potential through Eq. 3 and Eq. 1 (gauge invariance).

Tolerances: the kernel forms each potential as a running sum of up to n
facet fluxes (n <= 449 on the 2 mm grid), the oracle by a sparse solve whose
error grows with the condition number of the cotree normal equations; both
stay below 1e-11 of the largest |a| on the small grids.  C a = b then holds to
4 * n * eps * max|a| per facet.
"""

import ctypes
import json
import os

import numpy as np
import pytest

import oracle
from spfd_inputs import (body_phantom, loop_potential, random_phantom, sphere_phantom,
                         uniform_b_landau, uniform_b_symmetric)
from spfd_inputs.flux import loop_flux, uniform_flux

pytestmark = pytest.mark.gpu

OMEGA = 2 * np.pi * 85e3
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "body_2mm_oracle.json")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_12879_gb300 import build as b
    b.build()
    import paper_2010_12879_gb300 as spfd
    return torch, spfd


def _gpu_gauge(torch, spfd, b, j0, k0):
    """spfd_tree_cotree through the C ABI; returns a on the host."""
    _, nzp, nyp, nxp = b.shape
    bd = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    ad = torch.full_like(bd, float("nan"))  # every slot must be written
    st = spfd.lib().spfd_tree_cotree(ctypes.c_void_p(bd.data_ptr()), nxp - 1, nyp - 1,
                                     nzp - 1, j0, k0,
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                     ctypes.c_void_p(ad.data_ptr()))
    assert st == spfd.SPFD_OK, spfd.spfd_last_error()
    torch.cuda.synchronize()
    return ad.cpu().numpy()


def _edge_mask(dims):
    nx, ny, nz = dims
    m = np.zeros((3, nz + 1, ny + 1, nx + 1), dtype=bool)
    m[0, :, :, :nx] = True
    m[1, :, :ny, :] = True
    m[2, :nz, :, :] = True
    return m


@pytest.mark.parametrize("dims,root", [
    ((13, 9, 11), (4, 5)),     # interior root line
    ((13, 9, 11), (0, 0)),     # root line on the grid's corner edge
    ((13, 9, 11), (9, 11)),    # the opposite corner edge
    ((37, 21, 17), (10, 8)),   # several warps per plane, ragged last warp
    ((1, 1, 1), (1, 0)),       # one voxel
    ((40, 1, 3), (0, 2)),      # flat grids
    ((1, 30, 2), (30, 1)),
])
def test_tree_cotree_matches_oracle(env, dims, root):
    torch, spfd = env
    rng = np.random.default_rng(sum(dims) + 7 * root[0] + root[1])
    nx, ny, nz = dims
    a_src = rng.normal(size=(3, nz + 1, ny + 1, nx + 1)) * 1e-7 * _edge_mask(dims)
    b = oracle.curl(a_src)
    want = oracle.tree_cotree(b, oracle.comb_tree(dims, *root))
    got = _gpu_gauge(torch, spfd, b, *root)
    assert not np.any(np.isnan(got))
    scale = np.abs(want).max()
    assert np.max(np.abs(got - want)) <= 1e-11 * scale
    tree = oracle.comb_tree(dims, *root)
    assert np.all(got[tree] == 0.0) and np.all(got[~_edge_mask(dims)] == 0.0)


def test_uniform_field_gives_the_landau_gauge_and_the_same_field(env):
    """Sphere workload (32^3 voxels, h = 2 mm, B = 27 uT along z): the comb
    on the central root line turns the exact fluxes B h^2 into the Landau
    gauge a_x = -B y h, and the whole path (gauge, Eq. 3, Eq. 1) gives the
    oracle's |E| of the symmetric gauge."""
    torch, spfd = env
    ph = sphere_phantom()
    nx, ny, nz = ph.dims
    b = uniform_flux(ph.dims, ph.h, (0.0, 0.0, 27e-6))
    got = _gpu_gauge(torch, spfd, b, ny // 2, nz // 2)
    landau = uniform_b_landau(ph.dims, ph.h, ph.origin, 27e-6)
    assert np.max(np.abs(got - landau)) <= 1e-12 * np.abs(landau).max()
    a_sym = uniform_b_symmetric(ph.dims, ph.h, ph.origin, 27e-6)
    psi_r, _, _ = oracle.solve(ph.sigma, ph.h, a_sym, tol=1e-13)
    E_r = oracle.efield(ph.sigma, a_sym, psi_r, ph.h, OMEGA)
    sig = torch.from_numpy(ph.sigma).cuda()
    ad = torch.from_numpy(got).cuda()
    with spfd.Solver(sig, ph.h) as S:
        psi, info, st = S.solve(ad, 1e-13)
        E = S.efield(ad, psi, OMEGA).cpu().numpy()
    assert st == spfd.SPFD_OK
    m = ph.sigma > 0
    floor = 1e-6 * max(E_r.max(), OMEGA / ph.h * np.abs(a_sym).max())
    assert np.max(np.abs(E - E_r)[m] / np.maximum(E_r[m], floor)) <= 1e-7


def test_random_phantom_field_is_gauge_invariant(env):
    torch, spfd = env
    rng = np.random.default_rng(41)
    ph = random_phantom(21, 14, 17, rng, air_fraction=0.3)
    nx, ny, nz = ph.dims
    a = rng.normal(size=(3, nz + 1, ny + 1, nx + 1)) * 1e-8 * _edge_mask(ph.dims)
    ap = _gpu_gauge(torch, spfd, oracle.curl(a), 7, 8)
    psi_r, _, _ = oracle.solve(ph.sigma, ph.h, a, tol=1e-13)
    E_r = oracle.efield(ph.sigma, a, psi_r, ph.h, OMEGA)
    sig = torch.from_numpy(ph.sigma).cuda()
    ad = torch.from_numpy(ap).cuda()
    with spfd.Solver(sig, ph.h) as S:
        psi, info, st = S.solve(ad, 1e-13)
        E = S.efield(ad, psi, OMEGA).cpu().numpy()
    m = ph.sigma > 0
    floor = 1e-6 * max(E_r.max(), OMEGA / ph.h * np.abs(a).max())
    assert np.max(np.abs(E - E_r)[m] / np.maximum(E_r[m], floor)) <= 1e-7


def test_physical_loop_fluxes_give_the_midpoint_field_to_second_order(env):
    """Facet fluxes of the loop's closed-form B (the input generator's
    Gauss-Legendre rule) against the loop's midpoint-sampled potentials on
    the 16 mm body: the two discretisations of the same source agree to the
    midpoint rule's O(h^2), and the gauge reproduces C a = b."""
    torch, spfd = env
    ph = body_phantom(32, 20, 112, h=16e-3)
    nx, ny, nz = ph.dims
    b = loop_flux(ph.dims, ph.h, ph.origin)
    ap = _gpu_gauge(torch, spfd, b, ny // 2, nz // 2)
    assert np.max(np.abs(oracle.curl(ap) - b)) <= 1e-12 * np.abs(ap).max()
    a_mid = loop_potential(ph.dims, ph.h, ph.origin)
    sig = torch.from_numpy(ph.sigma).cuda()
    Es = []
    with spfd.Solver(sig, ph.h) as S:
        for a in (a_mid, ap):
            ad = torch.from_numpy(a).cuda()
            psi, info, st = S.solve(ad, 1e-12)
            assert st == spfd.SPFD_OK
            Es.append(S.efield(ad, psi, OMEGA).cpu().numpy())
    m = ph.sigma > 0
    rel = np.abs(Es[1] - Es[0])[m] / Es[0][m].max()
    assert rel.max() <= 1e-3


def test_full_size_body_properties(env):
    """The 2 mm body grid (256 x 160 x 896 voxels, 37.1 M nodes), the launch
    the benchmark times: b = C a of the loop's edge potentials (the oracle's
    Eq. 2); the gauged a vanishes on the tree, reproduces b on every facet,
    and through Eq. 3 (1e-12) and Eq. 1 gives the oracle's |E| at its seeded
    sample voxels."""
    torch, spfd = env
    with open(GOLDEN) as f:
        g = json.load(f)
    ph = body_phantom()
    nx, ny, nz = ph.dims
    a = loop_potential(ph.dims, ph.h, ph.origin)
    b = oracle.curl(a)
    j0, k0 = ny // 2, nz // 2
    ap = _gpu_gauge(torch, spfd, b, j0, k0)
    assert np.all(ap[2] == 0.0)
    assert np.all(ap[1, k0] == 0.0) and np.all(ap[0, k0, j0] == 0.0)
    # running sums of at most 449 terms, four of them per facet: 4 * 449 * eps
    # is about 4e-13 of max |a|
    assert np.max(np.abs(oracle.curl(ap) - b)) <= 1e-12 * np.abs(ap).max()
    if "E_sample_voxels" not in g:
        pytest.skip("golden file without |E| samples")
    sig = torch.from_numpy(ph.sigma).cuda()
    ad = torch.from_numpy(ap).cuda()
    del ap, b
    with spfd.Solver(sig, ph.h) as S:
        psi, info, st = S.solve(ad, 1e-12)
        assert st == spfd.SPFD_OK, spfd.spfd_last_error()
        E = S.efield(ad, psi, OMEGA).reshape(-1)
        vox = torch.tensor(g["E_sample_voxels"], dtype=torch.int64, device="cuda")
        Es = E[vox].cpu().numpy()
    ref = np.array(g["E_sample_values"])
    floor = 1e-6 * max(g["E_max"], g["E_floor_scale"])
    assert np.max(np.abs(Es - ref) / np.maximum(ref, floor)) <= 1e-7
