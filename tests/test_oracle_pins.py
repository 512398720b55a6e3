"""Pins for the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than its own formulas:
closed forms (graph-Laplacian spectra, linear fields), a hand-enumerated
fixture, brute-force dense solves on tiny grids, library routines for
sub-steps (connected-component labelling), and exact invariants of Eq. 1 /
Eq. 3 (gauge invariance, manufactured solutions, mirror symmetries).
"""

import os

import numpy as np
import pytest

from spfd_inputs import (random_phantom, sphere_phantom, uniform_b_landau,
                         uniform_b_symmetric)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
OMEGA = 2 * np.pi * 85e3
B0 = 27e-6


def _dense(sys):
    return sys.to_scipy().toarray()


def _node_xyz(dims, h, origin):
    nx, ny, nz = dims
    xs = np.arange(nx + 1) * h - origin[0]
    ys = np.arange(ny + 1) * h - origin[1]
    zs = np.arange(nz + 1) * h - origin[2]
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return X, Y, Z


def _grad(chi):
    """Edge differences of a node field (test-side, for manufactured inputs)."""
    nzp, nyp, nxp = chi.shape
    a = np.zeros((3, nzp, nyp, nxp))
    a[0, :, :, :-1] = chi[:, :, 1:] - chi[:, :, :-1]
    a[1, :, :-1, :] = chi[:, 1:, :] - chi[:, :-1, :]
    a[2, :-1, :, :] = chi[1:, :, :] - chi[:-1, :, :]
    return a


# ---------------------------------------------------------------- operator

def test_single_voxel_is_scaled_cube_laplacian(oracle_mod):
    """One conducting voxel: each of its 12 edges touches exactly one
    conducting voxel, so A = (h sigma / 4) * Laplacian of the cube graph,
    whose spectrum is {0, 2, 2, 2, 4, 4, 4, 6}."""
    h, s = 2e-3, 0.7
    sigma = np.zeros((3, 3, 3))
    sigma[1, 1, 1] = s
    sys = oracle_mod.assemble(sigma, h)
    assert sys.n == 8 and sys.ncomp == 1
    ev = np.linalg.eigvalsh(_dense(sys)) / (h * s / 4)
    np.testing.assert_allclose(ev, [0, 2, 2, 2, 4, 4, 4, 6], atol=1e-12)


def test_two_voxel_operator_matches_hand_enumeration(oracle_mod):
    """Against tests/golden/two_voxel_edges.txt (hand-derived conductances)."""
    h, s1, s2 = 2e-3, 0.3, 1.7
    sigma = np.array([[[s1, s2]]])  # [k][j][i], nx=2, ny=1, nz=1
    sys = oracle_mod.assemble(sigma, h)
    rows = np.loadtxt(os.path.join(GOLDEN, "two_voxel_edges.txt"), dtype=float)
    nx, ny, nz = 2, 1, 1
    nid = lambda i, j, k: (k * (ny + 1) + j) * (nx + 1) + i
    A = np.zeros((12, 12))
    for ax, i, j, k, c1, c2 in rows:
        i, j, k, ax = int(i), int(j), int(k), int(ax)
        ge = h / 4 * (c1 * s1 + c2 * s2)
        p = nid(i, j, k)
        q = nid(i + (ax == 0), j + (ax == 1), k + (ax == 2))
        A[p, p] += ge
        A[q, q] += ge
        A[p, q] -= ge
        A[q, p] -= ge
    assert sys.n == 12
    P = np.zeros((12, 12))
    P[np.arange(12), sys.nodes] = 1.0
    np.testing.assert_allclose(_dense(sys), P @ A @ P.T, rtol=0, atol=1e-15)
    # and the full edge array agrees slot by slot
    g = oracle_mod.conductances(sigma, h)
    expect = np.zeros_like(g)
    for ax, i, j, k, c1, c2 in rows:
        expect[int(ax), int(k), int(j), int(i)] = h / 4 * (c1 * s1 + c2 * s2)
    np.testing.assert_allclose(g, expect, rtol=0, atol=1e-16)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_operator_invariants(oracle_mod, seed):
    """Symmetric, zero row sums, positive semidefinite with exactly one zero
    eigenvalue per connected conducting component."""
    rng = np.random.default_rng(seed)
    ph = random_phantom(5, 4, 6, rng, air_fraction=0.55)
    sys = oracle_mod.assemble(ph.sigma, ph.h)
    A = _dense(sys)
    np.testing.assert_allclose(A, A.T, atol=0)
    np.testing.assert_allclose(A.sum(axis=1), 0, atol=1e-15)
    ev = np.linalg.eigvalsh(A)
    scale = ev.max()
    assert ev.min() > -1e-12 * scale
    assert int(np.sum(ev < 1e-10 * scale)) == sys.ncomp
    for c in range(sys.ncomp):
        one = (sys.comp == c).astype(float)
        assert np.abs(A @ one).max() < 1e-15 * scale


@pytest.mark.parametrize("seed", [3, 4])
def test_components_match_26_connectivity(oracle_mod, seed):
    """Components of the operator graph are the 26-connected clusters of
    conducting voxels (two voxels sharing only a corner share that node);
    checked with scipy.ndimage.label."""
    from scipy import ndimage
    rng = np.random.default_rng(seed)
    ph = random_phantom(7, 6, 5, rng, air_fraction=0.8)
    sys = oracle_mod.assemble(ph.sigma, ph.h)
    lab, nlab = ndimage.label(ph.sigma > 0, structure=np.ones((3, 3, 3)))
    assert sys.ncomp == nlab
    # every conducting voxel's 8 corners carry the component of its cluster
    nz, ny, nx = ph.sigma.shape
    comp_full = np.full(sys.dof.size, -1)
    comp_full[sys.nodes] = sys.comp
    comp_full = comp_full.reshape(nz + 1, ny + 1, nx + 1)
    mapping = {}
    for k, j, i in zip(*np.nonzero(lab)):
        corners = {comp_full[k + dk, j + dj, i + di]
                   for dk in (0, 1) for dj in (0, 1) for di in (0, 1)}
        assert len(corners) == 1 and -1 not in corners
        c = corners.pop()
        assert mapping.setdefault(lab[k, j, i], c) == c
    assert len(set(mapping.values())) == nlab


# ---------------------------------------------------------------- solver

@pytest.mark.parametrize("seed,dims", [(10, (4, 4, 4)), (11, (5, 3, 4)), (12, (6, 5, 4))])
def test_pcg_matches_dense_least_squares(oracle_mod, seed, dims):
    """Brute force: the minimum-norm least-squares solution of the assembled
    system equals the oracle's Psi.  The minimum-norm solution is orthogonal
    to the null space of A, which is spanned by the indicator vectors of the
    conducting components, so it already has zero unweighted mean on every
    component: it is compared as it comes, without re-projection, which pins
    the projection convention (R4) as well as the solve."""
    rng = np.random.default_rng(seed)
    ph = random_phantom(*dims, rng, air_fraction=0.35)
    nx, ny, nz = dims
    a = rng.normal(size=(3, nz + 1, ny + 1, nx + 1)) * 1e-6
    psi, info, sys = oracle_mod.solve(ph.sigma, ph.h, a, tol=1e-13)
    assert info["converged"] and info["rel_res"] <= 1e-13
    A = _dense(sys)
    b = oracle_mod.rhs(sys, a)
    x = np.linalg.lstsq(A, b, rcond=None)[0]
    got = sys.gather(psi)
    assert np.linalg.norm(got - x) <= 1e-11 * np.linalg.norm(x)
    # reported residual is the true one
    r = b - A @ sys.gather(psi)
    assert abs(np.linalg.norm(r) / np.linalg.norm(b) - info["rel_res"]) < 1e-13


def test_project_removes_the_unweighted_component_mean(oracle_mod):
    """R4: the projection subtracts each component's plain (unweighted) mean.
    A unit vector at one node of a component with m nodes becomes 1 - 1/m
    there and -1/m at the component's other nodes, and leaves every other
    component untouched; a per-component constant is removed entirely."""
    rng = np.random.default_rng(11)
    sigma = np.zeros((5, 6, 9))
    sigma[1:4, 1:5, 1:4] = rng.uniform(0.1, 1.0, size=(3, 4, 3))
    sigma[1:3, 2:4, 6:8] = rng.uniform(0.1, 1.0, size=(2, 2, 2))
    sys = oracle_mod.assemble(sigma, 2e-3)
    assert sys.ncomp == 2
    sizes = np.bincount(sys.comp, minlength=sys.ncomp)
    c = int(np.argmax(sizes))
    m = int(sizes[c])
    i = int(np.flatnonzero(sys.comp == c)[m // 2])
    x = np.zeros(sys.n)
    x[i] = 1.0
    y = oracle_mod.project(sys, x.copy())
    want = np.where(sys.comp == c, -1.0 / m, 0.0)
    want[i] += 1.0
    assert np.max(np.abs(y - want)) <= 1e-15
    k = rng.normal(size=sys.ncomp)
    assert np.max(np.abs(oracle_mod.project(sys, k[sys.comp].copy()))) <= 1e-15 * np.abs(k).max() * 4


def test_rhs_is_consistent(oracle_mod):
    """b = -G^T M a sums to zero over every component (it lies in the range
    of A), before any projection."""
    rng = np.random.default_rng(5)
    ph = random_phantom(6, 6, 6, rng, air_fraction=0.7)
    a = rng.normal(size=(3, 7, 7, 7))
    sys = oracle_mod.assemble(ph.sigma, ph.h)
    b = oracle_mod.rhs(sys, a)
    for c in range(sys.ncomp):
        m = sys.comp == c
        assert abs(b[m].sum()) <= 1e-13 * np.abs(b).sum()
    # and vanishes at removed nodes
    bf = oracle_mod.rhs_full(sys.g, a).reshape(-1)
    assert np.all(bf[sys.dof < 0] == 0)


def test_manufactured_solution(oracle_mod):
    """a = -G chi gives Psi = chi (per-component projected) and E = 0 exactly."""
    rng = np.random.default_rng(6)
    ph = random_phantom(6, 5, 7, rng, air_fraction=0.3)
    nx, ny, nz = ph.dims
    chi = rng.normal(size=(nz + 1, ny + 1, nx + 1))
    a = -_grad(chi)
    psi, info, sys = oracle_mod.solve(ph.sigma, ph.h, a, tol=1e-14)
    want = oracle_mod.project(sys, sys.gather(chi))
    got = sys.gather(psi)
    assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(want)
    E = oracle_mod.efield(ph.sigma, a, psi, ph.h, OMEGA)
    Escale = OMEGA / ph.h * np.abs(a).max()
    assert np.abs(E).max() <= 1e-10 * Escale


# ---------------------------------------------------------------- E field

def test_efield_of_linear_potential_is_exact(oracle_mod):
    """For a = 0 and Psi linear, Psi = c . r, every edge carries c_d h, so the
    voxel average is exact: |E| = omega |c| on conducting voxels, 0 in air."""
    rng = np.random.default_rng(7)
    ph = random_phantom(5, 4, 3, rng, air_fraction=0.4)
    X, Y, Z = _node_xyz(ph.dims, ph.h, ph.origin)
    c = np.array([3.0, -2.0, 0.5]) * 1e-6
    psi = c[0] * X + c[1] * Y + c[2] * Z
    a = np.zeros((3,) + psi.shape)
    E = oracle_mod.efield(ph.sigma, a, psi, ph.h, OMEGA)
    m = ph.sigma > 0
    np.testing.assert_allclose(E[m], OMEGA * np.linalg.norm(c), rtol=1e-12)
    assert np.all(E[~m] == 0)


def test_efield_of_uniform_edge_potential(oracle_mod):
    """Psi = 0 and a constant per axis: |E| = (omega/h) ||(ax, ay, az)||."""
    ph = random_phantom(3, 3, 3, np.random.default_rng(8), air_fraction=0.0)
    a = np.zeros((3, 4, 4, 4))
    a[0], a[1], a[2] = 1e-9, -2e-9, 2e-9
    E = oracle_mod.efield(ph.sigma, a, np.zeros((4, 4, 4)), ph.h, OMEGA)
    np.testing.assert_allclose(E, OMEGA / ph.h * 3e-9, rtol=1e-13)


def test_efield_complex_closed_forms(oracle_mod):
    """Complex source (R7): for Psi = 0 and a constant per axis with the
    phasor a = (1 + 2j) a0, the field is (1 + 2j) E0, whose magnitude is
    sqrt(5) (omega/h) ||a0||; a purely real source gives the real |E| bit for
    bit; and a quadrature pair of linear potentials, Psi = c.r + j (d.r),
    gives omega sqrt(|c|^2 + |d|^2) (the parts are not added before the
    magnitude)."""
    ph = random_phantom(3, 3, 3, np.random.default_rng(8), air_fraction=0.0)
    a0 = np.zeros((3, 4, 4, 4))
    a0[0], a0[1], a0[2] = 1e-9, -2e-9, 2e-9
    z = np.zeros((4, 4, 4))
    E = oracle_mod.efield_complex(ph.sigma, a0, z, 2 * a0, z, ph.h, OMEGA)
    np.testing.assert_allclose(E, np.sqrt(5.0) * OMEGA / ph.h * 3e-9, rtol=1e-13)
    E_re = oracle_mod.efield(ph.sigma, a0, z, ph.h, OMEGA)
    np.testing.assert_array_equal(
        oracle_mod.efield_complex(ph.sigma, a0, z, np.zeros_like(a0), z, ph.h, OMEGA), E_re)
    rng = np.random.default_rng(11)
    ph = random_phantom(5, 4, 3, rng, air_fraction=0.4)
    X, Y, Z = _node_xyz(ph.dims, ph.h, ph.origin)
    c = np.array([3.0, -2.0, 0.5]) * 1e-6
    d = np.array([-1.0, 0.5, 2.0]) * 1e-6
    zero_a = np.zeros((3,) + X.shape)
    E = oracle_mod.efield_complex(ph.sigma, zero_a, c[0] * X + c[1] * Y + c[2] * Z,
                                  zero_a, d[0] * X + d[1] * Y + d[2] * Z, ph.h, OMEGA)
    m = ph.sigma > 0
    np.testing.assert_allclose(E[m], OMEGA * np.sqrt(c @ c + d @ d), rtol=1e-12)
    assert np.all(E[~m] == 0)


# ---------------------------------------------------------------- sphere (32^3, R = 28 mm)

@pytest.fixture(scope="module")
def sphere_solutions(oracle_mod):
    ph = sphere_phantom()
    sys = oracle_mod.assemble(ph.sigma, ph.h)
    a_s = uniform_b_symmetric(ph.dims, ph.h, ph.origin, B0)
    a_l = uniform_b_landau(ph.dims, ph.h, ph.origin, B0)
    ps, info_s, _ = oracle_mod.solve(ph.sigma, ph.h, a_s, sys=sys)
    pl, info_l, _ = oracle_mod.solve(ph.sigma, ph.h, a_l, sys=sys)
    return ph, sys, a_s, a_l, ps, pl, info_s, info_l


def test_sphere_counts(sphere_solutions):
    ph, sys, *_ = sphere_solutions
    assert int((ph.sigma > 0).sum()) == 11536
    assert sys.n == 13469 and sys.ncomp == 1


def test_gauge_invariance(oracle_mod, sphere_solutions):
    """Landau gauge a_L = a_S + G chi with chi = -B x y / 2 at the nodes, so
    Psi_L = Psi_S - chi (mod constants) and E_L = E_S (Eq. 1)."""
    ph, sys, a_s, a_l, ps, pl, info_s, info_l = sphere_solutions
    assert info_s["converged"] and info_l["converged"]
    X, Y, _ = _node_xyz(ph.dims, ph.h, ph.origin)
    chi = -B0 * X * Y / 2
    np.testing.assert_allclose(a_l, a_s + _grad(chi), rtol=0, atol=1e-12 * np.abs(a_l).max())
    d = oracle_mod.project(sys, sys.gather(pl) - sys.gather(ps) + sys.gather(chi))
    assert np.abs(d).max() <= 1e-9 * np.abs(sys.gather(pl)).max()
    Es = oracle_mod.efield(ph.sigma, a_s, ps, ph.h, OMEGA)
    El = oracle_mod.efield(ph.sigma, a_l, pl, ph.h, OMEGA)
    m = ph.sigma > 0
    assert np.abs(Es - El)[m].max() <= 1e-9 * Es[m].max()


def test_sphere_symmetries(sphere_solutions):
    """Symmetric gauge on a grid-centred sphere: Psi_S is odd under x -> -x,
    y -> -y and x <-> y, even under z -> -z and invariant under a quarter turn
    about z; |E| shares all of these symmetries as an even function."""
    ph, sys, a_s, a_l, ps, pl, *_ = sphere_solutions
    scale = np.abs(ps).max()
    assert scale > 0
    tol = 1e-8 * scale
    assert np.abs(ps + ps[:, :, ::-1]).max() <= tol           # x -> -x
    assert np.abs(ps + ps[:, ::-1, :]).max() <= tol           # y -> -y
    assert np.abs(ps - ps[::-1, :, :]).max() <= tol           # z -> -z
    assert np.abs(ps + np.swapaxes(ps, 1, 2)).max() <= tol    # x <-> y
    rot = np.rot90(ps, k=1, axes=(1, 2))                      # quarter turn
    assert np.abs(ps - rot).max() <= tol
    E = __import__("oracle").efield(ph.sigma, a_s, ps, ph.h, OMEGA)
    Et = 1e-8 * E.max()
    assert np.abs(E - E[:, :, ::-1]).max() <= Et
    assert np.abs(E - E[::-1, :, :]).max() <= Et
    assert np.abs(E - np.swapaxes(E, 1, 2)).max() <= Et


def _sphere_interior_error(oracle_mod, n, h, limit):
    ph = sphere_phantom(n, h)
    a = uniform_b_symmetric(ph.dims, ph.h, ph.origin, B0)
    psi, info, _ = oracle_mod.solve(ph.sigma, ph.h, a)
    E = oracle_mod.efield(ph.sigma, a, psi, ph.h, OMEGA)
    c = (np.arange(n) + 0.5) * h - ph.origin[0]
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    rho = np.hypot(X, Y)
    Ea = OMEGA * B0 * rho / 2          # continuum: |E| = omega B rho / 2
    m = r <= limit
    return np.abs(E - Ea)[m].max() / Ea[m].max(), E, Ea, ph


def test_sphere_matches_analytic_field(oracle_mod):
    """Continuum answer for a = B x r / 2 in a homogeneous sphere: Psi = 0 and
    |E| = omega B rho / 2 (rho = distance to the field axis).  The staircase
    surface perturbs it; 8 mm inside the surface the 2 mm grid is within 1 %,
    4 mm inside within 2.5 %.  0.2019 V/m at rho = 28 mm."""
    assert abs(OMEGA * B0 * 0.028 / 2 - 0.2019) < 5e-5
    e8, *_ = _sphere_interior_error(oracle_mod, 32, 2e-3, 0.020)
    e4, *_ = _sphere_interior_error(oracle_mod, 32, 2e-3, 0.024)
    assert e8 < 0.01 and e4 < 0.025


def test_sphere_error_shrinks_under_refinement(oracle_mod):
    """Halving h (same sphere, same B) at least halves the interior error."""
    e2, *_ = _sphere_interior_error(oracle_mod, 32, 2e-3, 0.020)
    e1, *_ = _sphere_interior_error(oracle_mod, 64, 1e-3, 0.020)
    assert e1 < 0.5 * e2
