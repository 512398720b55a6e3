"""Pins of the oracle's Eq. 2 (b = C a, ``curl``) and of step 3 of the
pipeline, tree-cotree gauging (``comb_tree``, ``bfs_tree``, ``tree_cotree``),
against what the mathematics fixes without the oracle's own formulas:

* a hand-enumerated fixture: the unit potential on one edge appears with
  +1 / -1 in exactly the four facets that edge bounds (orientation, indices);
* C G = 0 exactly (curl of a gradient) and D C = 0 exactly (the net outward
  flux of every cell vanishes), on integer fields;
* Stokes for linear potentials: A = B x r / 2 sampled on the edges gives the
  flux B_d h^2 through every facet of normal d, for any constant B;
* the spanning trees are trees: nodes - 1 edges, one connected component;
* the gauged potentials solve the definition (C a' = b, a' = 0 on the tree)
  and differ from the source potential by an exact discrete gradient whose
  node values are recovered by walking the tree;
* closed form: for uniform B the comb tree on the root line (j0, k0) yields
  a'_x = h^2 (By (k - k0) - Bz (j - j0)), a'_y = -h^2 Bx (k - k0), a'_z = 0
  (for B along z and a central root this is the Landau gauge);
* gauge invariance through the whole pipeline: Eq. 3 + Eq. 1 give the same
  |E| from the source potential, the comb-gauged and the BFS-gauged one;
* the input generator's loop fluxes are divergence-free and equal C a of the
  loop's sampled edge potentials to the midpoint rule's O(h^2).
"""

import numpy as np
import pytest

import oracle
from spfd_inputs import body_phantom, loop_potential, random_phantom
from spfd_inputs.flux import loop_flux, uniform_flux

OMEGA = 2 * np.pi * 85e3


def _grad(chi):
    nzp, nyp, nxp = chi.shape
    a = np.zeros((3, nzp, nyp, nxp))
    a[0, :, :, :-1] = chi[:, :, 1:] - chi[:, :, :-1]
    a[1, :, :-1, :] = chi[:, 1:, :] - chi[:, :-1, :]
    a[2, :-1, :, :] = chi[1:, :, :] - chi[:-1, :, :]
    return a


def _div(b):
    """Net outward flux of every cell, from the facet fluxes (test-side)."""
    _, nzp, nyp, nxp = b.shape
    nz, ny, nx = nzp - 1, nyp - 1, nxp - 1
    return ((b[0, :nz, :ny, 1:] - b[0, :nz, :ny, :nx])
            + (b[1, :nz, 1:, :nx] - b[1, :nz, :ny, :nx])
            + (b[2, 1:, :ny, :nx] - b[2, :nz, :ny, :nx]))


def _edge_mask(dims):
    nx, ny, nz = dims
    m = np.zeros((3, nz + 1, ny + 1, nx + 1), dtype=bool)
    m[0, :, :, :nx] = True
    m[1, :, :ny, :] = True
    m[2, :nz, :, :] = True
    return m


def _facet_mask(dims):
    nx, ny, nz = dims
    m = np.zeros((3, nz + 1, ny + 1, nx + 1), dtype=bool)
    m[0, :nz, :ny, :] = True
    m[1, :nz, :, :nx] = True
    m[2, :, :ny, :nx] = True
    return m


def _linear_potential(dims, h, B, origin=(0.0, 0.0, 0.0)):
    """Edge integrals of A = B x r / 2 (exact at edge midpoints: A is linear)."""
    nx, ny, nz = dims
    Bx, By, Bz = B
    xs = np.arange(nx + 1) * h - origin[0]
    ys = np.arange(ny + 1) * h - origin[1]
    zs = np.arange(nz + 1) * h - origin[2]
    a = np.zeros((3, nz + 1, ny + 1, nx + 1))
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    # A = (By z - Bz y, Bz x - Bx z, Bx y - By x) / 2 at the edge midpoints
    a[0, :, :, :nx] = (0.5 * (By * Z - Bz * Y) * h)[:, :, :nx]
    a[1, :, :ny, :] = (0.5 * (Bz * X - Bx * Z) * h)[:, :ny, :]
    a[2, :nz, :, :] = (0.5 * (Bx * Y - By * X) * h)[:nz, :, :]
    return a


# ------------------------------------------------------------------ Eq. 2

def test_one_edge_bounds_four_facets():
    """Hand-enumerated: a = 1 on the x edge of node (1, 1, 1) of a 3x3x3
    voxel grid.  That edge is the first side of facet z at (1,1,1) (+1), the
    third side of facet z at (1,0,1) (-1), the last side of facet y at
    (1,1,1) (-1) and the second side of facet y at (1,1,0) (+1)."""
    a = np.zeros((3, 4, 4, 4))
    a[0, 1, 1, 1] = 1.0
    b = oracle.curl(a)
    want = np.zeros_like(b)
    want[2, 1, 1, 1] = 1.0
    want[2, 1, 0, 1] = -1.0
    want[1, 1, 1, 1] = -1.0
    want[1, 0, 1, 1] = 1.0
    np.testing.assert_array_equal(b, want)


def test_curl_of_gradient_and_divergence_of_curl_vanish():
    rng = np.random.default_rng(21)
    dims = (7, 5, 6)
    nx, ny, nz = dims
    chi = rng.integers(-1000, 1000, size=(nz + 1, ny + 1, nx + 1)).astype(float)
    assert np.all(oracle.curl(_grad(chi)) == 0.0)
    a = rng.integers(-1000, 1000, size=(3, nz + 1, ny + 1, nx + 1)).astype(float)
    b = oracle.curl(a)
    assert np.all(_div(b) == 0.0)
    assert np.all(b[~_facet_mask(dims)] == 0.0)
    assert np.any(b != 0.0)


@pytest.mark.parametrize("B", [(0.0, 0.0, 27e-6), (1.3e-5, -2.1e-5, 0.7e-5)])
def test_flux_of_uniform_field_is_exact(B):
    """Stokes for the linear potential B x r / 2: every facet of normal d
    carries B_d h^2 (the orientation of each facet is right-handed)."""
    dims, h = (6, 5, 4), 2e-3
    a = _linear_potential(dims, h, B, origin=(0.005, 0.004, 0.003))
    b = oracle.curl(a)
    want = uniform_flux(dims, h, B)
    assert np.max(np.abs(b - want)) <= 1e-12 * max(abs(v) for v in B) * h * h


# ------------------------------------------------------------- spanning trees

@pytest.mark.parametrize("kind", ["comb", "bfs"])
def test_trees_span_the_node_grid(kind):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    dims, root = (5, 4, 3), (2, 1, 2)
    nx, ny, nz = dims
    t = oracle.comb_tree(dims, root[1], root[2]) if kind == "comb" else oracle.bfs_tree(dims, root)
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    assert t.sum() == nn - 1
    assert not np.any(t & ~_edge_mask(dims))
    step = (1, nx + 1, (nx + 1) * (ny + 1))
    ids = np.arange(nn).reshape(nz + 1, ny + 1, nx + 1)
    r = np.concatenate([ids[t[d]] for d in range(3)])
    c = np.concatenate([ids[t[d]] + step[d] for d in range(3)])
    g = coo_matrix((np.ones(r.size), (r, c)), shape=(nn, nn))
    ncomp, _ = connected_components(g, directed=False)
    assert ncomp == 1


# ------------------------------------------------------- tree-cotree gauging

def _walk_potential(dims, tree, d_a, root):
    """chi with chi(root) = 0 and chi(head) - chi(tail) = d_a on every tree
    edge, found by walking the tree outward from the root (test-side)."""
    from collections import deque
    nx, ny, nz = dims
    shp = (nz + 1, ny + 1, nx + 1)
    step = (1, nx + 1, (nx + 1) * (ny + 1))
    nn = int(np.prod(shp))
    adj = [[] for _ in range(nn)]
    ids = np.arange(nn).reshape(shp)
    for d in range(3):
        for tail in ids[tree[d]]:
            head = tail + step[d]
            val = d_a.reshape(3, -1)[d, tail]
            adj[tail].append((head, val))
            adj[head].append((tail, -val))
    chi = np.full(nn, np.nan)
    r0 = int(ids[root[2], root[1], root[0]])
    chi[r0] = 0.0
    q = deque([r0])
    while q:
        u = q.popleft()
        for v, val in adj[u]:
            if np.isnan(chi[v]):
                chi[v] = chi[u] + val
                q.append(v)
    return chi.reshape(shp)


@pytest.mark.parametrize("kind", ["comb", "bfs"])
def test_gauged_potential_solves_the_definition(kind):
    rng = np.random.default_rng(22)
    dims, root = (6, 5, 7), (3, 2, 4)
    nx, ny, nz = dims
    a = rng.normal(size=(3, nz + 1, ny + 1, nx + 1)) * _edge_mask(dims)
    b = oracle.curl(a)
    t = oracle.comb_tree(dims, root[1], root[2]) if kind == "comb" else oracle.bfs_tree(dims, root)
    ap = oracle.tree_cotree(b, t)
    scale = np.abs(a).max()
    assert np.all(ap[t] == 0.0)
    assert np.all(ap[~_edge_mask(dims)] == 0.0)
    assert np.max(np.abs(oracle.curl(ap) - b)) <= 1e-12 * scale
    # a' - a is the gradient of the chi that the tree edges fix
    chi = _walk_potential(dims, t, ap - a, root)
    d = (ap - a) - _grad(chi)
    assert np.max(np.abs(d[_edge_mask(dims)])) <= 1e-11 * scale


@pytest.mark.parametrize("B", [(0.0, 0.0, 27e-6), (1.3e-5, -2.1e-5, 0.7e-5)])
def test_comb_gauge_of_uniform_field_closed_form(B):
    dims, h, (j0, k0) = (6, 5, 4), 2e-3, (3, 1)
    nx, ny, nz = dims
    b = uniform_flux(dims, h, B)
    ap = oracle.tree_cotree(b, oracle.comb_tree(dims, j0, k0))
    K, J, _ = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    want = np.zeros_like(ap)
    want[0] = h * h * (B[1] * (K - k0) - B[2] * (J - j0))
    want[1] = -h * h * B[0] * (K - k0)
    want *= _edge_mask(dims)
    assert np.max(np.abs(ap - want)) <= 1e-11 * max(abs(v) for v in B) * h * h


def test_gauged_potentials_give_the_same_field():
    """Eq. 3 then Eq. 1 on a random phantom: the source potential, its comb
    gauge and its BFS gauge produce the same voxel-averaged |E|."""
    rng = np.random.default_rng(23)
    ph = random_phantom(7, 6, 8, rng, air_fraction=0.3)
    nx, ny, nz = ph.dims
    a = rng.normal(size=(3, nz + 1, ny + 1, nx + 1)) * 1e-7 * _edge_mask(ph.dims)
    b = oracle.curl(a)
    Es = []
    for ap in (a, oracle.tree_cotree(b, oracle.comb_tree(ph.dims, 3, 4)),
               oracle.tree_cotree(b, oracle.bfs_tree(ph.dims, (0, 0, 0)))):
        psi, info, _ = oracle.solve(ph.sigma, ph.h, ap, tol=1e-13)
        Es.append(oracle.efield(ph.sigma, ap, psi, ph.h, OMEGA))
    floor = 1e-6 * Es[0].max()
    for E in Es[1:]:
        assert np.max(np.abs(E - Es[0]) / np.maximum(Es[0], floor)) <= 1e-7


# ------------------------------------------------------------ input fluxes

def test_loop_fluxes_are_divergence_free_and_match_the_potential():
    ph = body_phantom(32, 20, 112, h=16e-3)
    b = loop_flux(ph.dims, ph.h, ph.origin)
    assert np.max(np.abs(_div(b))) <= 1e-13 * np.abs(b).max()
    assert np.all(b[~_facet_mask(ph.dims)] == 0.0)
    bc = oracle.curl(loop_potential(ph.dims, ph.h, ph.origin))
    # the edge potentials are midpoint samples: O(h^2) apart from the fluxes
    assert np.max(np.abs(bc - b)) <= 2e-4 * np.abs(b).max()
