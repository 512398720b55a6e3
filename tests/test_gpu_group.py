"""Group solves: several bodies solved together by one launch of a captured
CUDA graph whose CG loop runs on the GPU (spfd_group_*).

The graph runs the kernels of the host-driven FP64 solve in the same order
and takes the same decisions on the same FP64 values, so each body's Psi must
be bit-identical to what spfd_solve returns for it alone, with the same
iteration count and true residual; one body is also held to the oracle at
the parity bar (1e-9 in Psi).
"""

import numpy as np
import pytest

from spfd_inputs import (body_phantom, loop_potential, random_phantom, scaled_body_phantom,
                         sphere_phantom, uniform_b_landau)

pytestmark = pytest.mark.gpu


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


def _bodies(rng):
    """Uneven bodies: a many-component random phantom, the sphere, two
    scaled ellipsoid bodies and the 8 mm body."""
    out = [random_phantom(13, 9, 11, rng, air_fraction=0.55), sphere_phantom(),
           scaled_body_phantom(32, 24, 112), scaled_body_phantom(48, 32, 160),
           body_phantom(64, 40, 224, h=8e-3)]
    srcs = []
    for ph in out:
        if ph.labels.max() > 0:
            srcs.append(loop_potential(ph.dims, ph.h, ph.origin))
        else:
            nx, ny, nz = ph.dims
            srcs.append(rng.normal(size=(3, nz + 1, ny + 1, nx + 1)))
    srcs[1] = uniform_b_landau(out[1].dims, out[1].h, out[1].origin, 27e-6)
    return out, srcs


def _assert_same_as_single(torch, S, a, psi_g, info_g, tol):
    psi_s, info_s, st_s = S.solve(a, tol)
    assert torch.equal(psi_g, psi_s)
    for k in ("iters", "outer_iters", "converged", "rel_res_true"):
        assert info_g[k] == info_s[k], (k, info_g[k], info_s[k])
    return st_s


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_group_equals_single_solves(torch_cuda, spfd, oracle_mod, precision):
    torch = torch_cuda
    rng = np.random.default_rng(44)
    phs, srcs = _bodies(rng)
    prec = spfd.SPFD_FP64 if precision == "fp64" else spfd.SPFD_MIXED
    solvers = [spfd.Solver(_dev(torch, ph.sigma), ph.h, precision=prec) for ph in phs]
    A = [_dev(torch, a) for a in srcs]
    try:
        with spfd.Group(solvers) as G:
            for tol in (1e-8, 1e-12):
                psis, infos, st = G.solve(A, tol)
                assert st == spfd.SPFD_OK
                for S, a, p, i in zip(solvers, A, psis, infos):
                    assert i["converged"] and i["iters"] > 0
                    if prec == spfd.SPFD_MIXED:
                        assert i["outer_iters"] >= 1
                    _assert_same_as_single(torch, S, a, p, i, tol)
            # new arrays (other pointers) for the same graph
            A2 = [(2.0 * a).contiguous() for a in A]
            psis2, infos2, st = G.solve(A2, 1e-10)
            for S, a, p, i in zip(solvers, A2, psis2, infos2):
                _assert_same_as_single(torch, S, a, p, i, 1e-10)
        # parity of one body against the oracle
        ph, a = phs[1], srcs[1]
        psi_r, info_r, sys = oracle_mod.solve(ph.sigma, ph.h, a, tol=1e-13)
        with spfd.Group([solvers[1]]) as G1:
            (psi,), (info,), st = G1.solve([A[1]], 1e-13)
        g = oracle_mod.project(sys, sys.gather(psi.cpu().numpy()))
        r = sys.gather(psi_r)
        assert np.linalg.norm(g - r) / np.linalg.norm(r) <= 1e-9
    finally:
        for S in solvers:
            S.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_group_edge_cases(torch_cuda, spfd, precision):
    torch = torch_cuda
    rng = np.random.default_rng(45)
    air = np.zeros((5, 6, 7))
    ph = random_phantom(9, 8, 10, rng, air_fraction=0.3)
    ph2 = random_phantom(11, 6, 9, rng, air_fraction=0.2)
    prec = spfd.SPFD_FP64 if precision == "fp64" else spfd.SPFD_MIXED
    S_air = spfd.Solver(_dev(torch, air), 2e-3, precision=prec)
    S1 = spfd.Solver(_dev(torch, ph.sigma), ph.h, precision=prec)
    S2 = spfd.Solver(_dev(torch, ph2.sigma), ph2.h, maxit=3, precision=prec)
    a_air = torch.ones((3, 6, 7, 8), dtype=torch.float64, device="cuda")
    a1 = torch.zeros((3,) + S1.node_shape, dtype=torch.float64, device="cuda")
    a2 = _dev(torch, rng.normal(size=(3,) + S2.node_shape))
    try:
        with spfd.Group([S_air, S1, S2]) as G:
            psis, infos, st = G.solve([a_air, a1, a2], 1e-12)
            assert st == spfd.SPFD_ENOTCONVERGED   # S2 stops at maxit = 3
            assert not torch.any(psis[0] != 0) and infos[0]["converged"]
            assert not torch.any(psis[1] != 0) and infos[1]["iters"] == 0
            assert infos[1]["converged"] and infos[1]["rel_res_true"] == 0.0
            assert infos[2]["iters"] <= 3 and not infos[2]["converged"]
            st2 = _assert_same_as_single(torch, S2, a2, psis[2], infos[2], 1e-12)
            assert st2 == spfd.SPFD_ENOTCONVERGED
            # a non-finite potential on a conducting edge
            bad = torch.full_like(a2, float("nan"))
            with pytest.raises(spfd.SpfdError) as ei:
                G.solve([a_air, a1, bad], 1e-12)
            assert ei.value.status == spfd.SPFD_EINVAL
            # the group keeps working afterwards
            psis, infos, st = G.solve([a_air, a1, a2], 1e-12)
            _assert_same_as_single(torch, S2, a2, psis[2], infos[2], 1e-12)
    finally:
        for S in (S_air, S1, S2):
            S.close()


def test_group_recaptures_after_batch(torch_cuda, spfd):
    """A batched solve reallocates the context's solve buffers; the next
    group solve must capture again rather than use stale pointers."""
    torch = torch_cuda
    rng = np.random.default_rng(46)
    ph = random_phantom(12, 10, 9, rng, air_fraction=0.25)
    S = spfd.Solver(_dev(torch, ph.sigma), ph.h)
    a = _dev(torch, rng.normal(size=(3,) + S.node_shape))
    try:
        with spfd.Group([S]) as G:
            (p0,), (i0,), _ = G.solve([a], 1e-11)
            S.solve_batch(torch.stack([a, 3 * a]).contiguous(), 1e-11)
            (p1,), (i1,), _ = G.solve([a], 1e-11)
            assert torch.equal(p0, p1) and i0["iters"] == i1["iters"]
            _assert_same_as_single(torch, S, a, p1, i1, 1e-11)
    finally:
        S.close()


def test_group_mixes_precisions_and_rejects_duplicates(torch_cuda, spfd):
    """A group may hold FP64 and mixed contexts side by side; a context may
    appear only once."""
    torch = torch_cuda
    rng = np.random.default_rng(47)
    ph = random_phantom(10, 9, 8, rng)
    S = spfd.Solver(_dev(torch, ph.sigma), ph.h)
    M = spfd.Solver(_dev(torch, ph.sigma), ph.h, precision=spfd.SPFD_MIXED)
    a = _dev(torch, rng.normal(size=(3,) + S.node_shape))
    try:
        with pytest.raises(spfd.SpfdError) as ei:
            spfd.Group([S, S])
        assert ei.value.status == spfd.SPFD_EINVAL
        with spfd.Group([S, M]) as G:
            psis, infos, st = G.solve([a, a], 1e-11)
            assert st == spfd.SPFD_OK
            _assert_same_as_single(torch, S, a, psis[0], infos[0], 1e-11)
            _assert_same_as_single(torch, M, a, psis[1], infos[1], 1e-11)
            assert infos[1]["outer_iters"] >= 2 and infos[0]["outer_iters"] == 0
    finally:
        S.close()
        M.close()
