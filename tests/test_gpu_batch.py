"""Batched solves: many source fields on one body in one spfd_solve_batch
call.  Each right-hand side keeps its own CG recurrence, scalars and stopping
decision inside the shared launches, so its Psi must be bit-identical to what
spfd_solve returns for that field alone, with the same iteration count; one
field per case is also held to the oracle at the parity bar (1e-9 in Psi).
"""

import numpy as np
import pytest

from spfd_inputs import (body_phantom, loop_potential, random_loops, random_phantom,
                         sphere_phantom)

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


def _singles(S, A, tol):
    out = []
    for j in range(A.shape[0]):
        psi, info, st = S.solve(A[j].contiguous(), tol)
        out.append((psi.clone(), info, st))
    return out


def _check_batch(torch, S, A, tol):
    psi_b, infos, st_b = S.solve_batch(A, tol)
    singles = _singles(S, A, tol)
    for j, (psi_s, info_s, st_s) in enumerate(singles):
        assert torch.equal(psi_b[j], psi_s), f"right-hand side {j} differs"
        assert infos[j]["iters"] == info_s["iters"]
        assert infos[j]["converged"] == info_s["converged"]
        assert infos[j]["rel_res_true"] == info_s["rel_res_true"]
    return psi_b, infos, st_b


def _oracle_psi_err(oracle, ph, a, psi_g):
    psi_r, info_r, sys = oracle.solve(ph.sigma, ph.h, a, tol=1e-13)
    assert info_r["converged"]
    g = oracle.project(sys, sys.gather(psi_g))
    r = sys.gather(psi_r)
    return np.linalg.norm(g - r) / np.linalg.norm(r)


@pytest.mark.parametrize("seed,dims,air", [(31, (13, 9, 11), 0.3), (32, (9, 17, 6), 0.55)])
def test_batch_equals_single_solves_random(torch_cuda, spfd, oracle_mod, seed, dims, air):
    """Random phantoms (ragged brick tails; many components at 55 % air) and
    five fields of very different scale, one of them zero."""
    torch = torch_cuda
    rng = np.random.default_rng(seed)
    ph = random_phantom(*dims, rng, air_fraction=air)
    nx, ny, nz = dims
    A = rng.normal(size=(5, 3, nz + 1, ny + 1, nx + 1))
    A[1] *= 1e3
    A[2] = 0.0
    A[3] *= 1e-12
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        psi_b, infos, st = _check_batch(torch, S, _dev(torch, A), 1e-13)
        assert st == spfd.SPFD_OK
        assert infos[2]["iters"] == 0 and not torch.any(psi_b[2] != 0)
        for j in (0, 3):
            assert _oracle_psi_err(oracle_mod, ph, A[j], psi_b[j].cpu().numpy()) <= 1e-9


def test_batch_sphere_loops(torch_cuda, spfd, oracle_mod):
    """The 32^3 sphere with six loop sources at seeded positions and
    orientations (the batched-source workload's placement rule)."""
    torch = torch_cuda
    ph = sphere_phantom(32)
    loops = random_loops(6, np.random.default_rng(40))
    A = np.stack([loop_potential(ph.dims, ph.h, ph.origin, center=c, normal=n)
                  for c, n in loops])
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        psi_b, infos, st = _check_batch(torch, S, _dev(torch, A), 1e-13)
        assert st == spfd.SPFD_OK and all(i["converged"] for i in infos)
        assert _oracle_psi_err(oracle_mod, ph, A[4], psi_b[4].cpu().numpy()) <= 1e-9


def test_batch_buffers_grow_and_are_reused(torch_cuda, spfd):
    """Batches of 2, 6 and 3 on one context, then single solves: every result
    stays equal to the single solve of its field."""
    torch = torch_cuda
    ph = body_phantom(32, 20, 112, h=16e-3)
    loops = random_loops(6, np.random.default_rng(41))
    A = _dev(torch, np.stack([loop_potential(ph.dims, ph.h, ph.origin, center=c, normal=n)
                              for c, n in loops]))
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        for k in (2, 6, 3):
            _, infos, st = _check_batch(torch, S, A[:k].contiguous(), 1e-10)
            assert st == spfd.SPFD_OK


def test_batch_mixed_precision_equals_single(torch_cuda, spfd):
    """With SPFD_MIXED the batch shares the FP32 inner CG's launches while
    each right-hand side keeps its own refinement state: the same results as
    single mixed solves, bit for bit."""
    torch = torch_cuda
    ph = body_phantom(64, 40, 224, h=8e-3)
    loops = random_loops(3, np.random.default_rng(42))
    A = _dev(torch, np.stack([loop_potential(ph.dims, ph.h, ph.origin, center=c, normal=n)
                              for c, n in loops]))
    with spfd.Solver(_dev(torch, ph.sigma), ph.h, precision=spfd.SPFD_MIXED) as S:
        _, infos, st = _check_batch(torch, S, A, 1e-10)
        assert st == spfd.SPFD_OK and all(i["outer_iters"] >= 1 for i in infos)


@pytest.mark.parametrize("seed,air", [(48, 0.55), (49, 0.2)])
def test_batch_mixed_random_and_zero(torch_cuda, spfd, oracle_mod, seed, air):
    """Mixed batches on random phantoms (many components at 55 % air), with a
    zero field and fields of very different scale; one, solved to 1e-11, is
    held to the oracle to 1e-7."""
    torch = torch_cuda
    rng = np.random.default_rng(seed)
    ph = random_phantom(15, 11, 13, rng, air_fraction=air)
    nx, ny, nz = ph.dims
    A = rng.normal(size=(4, 3, nz + 1, ny + 1, nx + 1))
    A[1] = 0.0
    A[2] *= 1e4
    with spfd.Solver(_dev(torch, ph.sigma), ph.h, precision=spfd.SPFD_MIXED) as S:
        psi_b, infos, st = _check_batch(torch, S, _dev(torch, A), 1e-11)
        assert st == spfd.SPFD_OK
        assert infos[1]["iters"] == 0 and not torch.any(psi_b[1] != 0)
        assert _oracle_psi_err(oracle_mod, ph, A[3], psi_b[3].cpu().numpy()) <= 1e-7


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("force", [None, 1, 2])
def test_batch_autotuned_orders_keep_results(torch_cuda, spfd, precision, force, monkeypatch):
    """Every block order runs the same arithmetic per right-hand side: the
    batch solved with the autotuner's orders (or with order 1 or the
    right-hand-side tile forced wherever it exists) equals, bit for bit, the
    same batch in the fixed order 0; the autotuner records one decision per
    tuned family and level, for this batch size only.  Six right-hand sides
    leave a ragged second tile of two."""
    torch = torch_cuda
    if force is not None:
        monkeypatch.setenv("SPFD_TUNE_FORCE", str(force))
    ph = body_phantom(64, 40, 224, h=8e-3)
    loops = random_loops(6, np.random.default_rng(50))
    A = _dev(torch, np.stack([loop_potential(ph.dims, ph.h, ph.origin, center=c, normal=n)
                              for c, n in loops]))
    prec = spfd.SPFD_FP64 if precision == "fp64" else spfd.SPFD_MIXED
    sig = _dev(torch, ph.sigma)
    with spfd.Solver(sig, ph.h, precision=prec) as S1, \
            spfd.Solver(sig, ph.h, precision=prec, autotune=0) as S0:
        p1, i1, st1 = S1.solve_batch(A, 1e-10)
        p0, i0, st0 = S0.solve_batch(A, 1e-10)
        assert st1 == st0 == spfd.SPFD_OK
        assert torch.equal(p1, p0)
        assert [i["iters"] for i in i1] == [i["iters"] for i in i0]
        rep = S1.autotune_report()
        nl = S1.info()["n_levels"]
        # per non-coarsest level: first sweep, smooth, residual, restrict,
        # prolong; apply_dot on level 0
        assert len(rep) == 5 * (nl - 1) + 1
        assert all(r["order"] in (0, 1, 2) and r["nrhs"] == 6 for r in rep)
        assert all(r["ms_order0"] > 0 and r["ms_order1"] > 0 for r in rep)
        # the tile exists for the 27-point smoother and residual (levels >= 1)
        # and for both transfers
        for r in rep:
            tile = r["family"] in ("restrict", "prolong") or (
                r["family"] in ("smooth", "residual") and r["level"] >= 1)
            assert (r["ms_order2"] > 0) if tile else (r["ms_order2"] == -1), r
            if force is not None and (force == 1 or tile):
                assert r["order"] == force, r
        assert S0.autotune_report() == []
        # a second batch of the same size reuses the decisions
        S1.solve_batch(A, 1e-10)
        assert len(S1.autotune_report()) == len(rep)


def test_batch_argument_errors(torch_cuda, spfd):
    torch = torch_cuda
    rng = np.random.default_rng(43)
    ph = random_phantom(6, 5, 4, rng, air_fraction=0.0)
    A = rng.normal(size=(3, 3, 5, 6, 7))
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        Ad = _dev(torch, A)
        psi = torch.empty((3, 5, 6, 7), dtype=torch.float64, device="cuda")
        with pytest.raises(spfd.SpfdError) as e:
            spfd.spfd_solve_batch(S.ctx, 0, Ad.data_ptr(), 1e-10, psi.data_ptr())
        assert e.value.status == spfd.SPFD_EINVAL
        A[2, 0, 1, 1, 1] = np.nan  # an x edge inside the all-conducting grid
        with pytest.raises(spfd.SpfdError) as e:
            S.solve_batch(_dev(torch, A), 1e-10)
        assert e.value.status == spfd.SPFD_EINVAL
        # the context stays usable
        A[2, 0, 1, 1, 1] = 0.0
        _check_batch(torch, S, _dev(torch, A), 1e-12)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_full_size_body_loops(torch_cuda, spfd, precision):
    """The 256 x 160 x 896 body (h = 2 mm, 9.25 M unknowns) with four of the
    batched-source loops at 1e-8, in both precisions: each Psi bit-identical
    to its single solve, all converged."""
    torch = torch_cuda
    from spfd_inputs.sources_torch import loop_potential_t
    ph = body_phantom()
    loops = random_loops(4, np.random.default_rng(44))
    A = torch.empty((4, 3) + tuple(d + 1 for d in ph.dims[::-1]), dtype=torch.float64,
                    device="cuda")
    for j, (c, n) in enumerate(loops):
        loop_potential_t(ph.dims, ph.h, ph.origin, center=c, normal=n, device="cuda", out=A[j])
    prec = spfd.SPFD_FP64 if precision == "fp64" else spfd.SPFD_MIXED
    with spfd.Solver(_dev(torch, ph.sigma), ph.h, precision=prec) as S:
        _, infos, st = _check_batch(torch, S, A, 1e-8)
        assert st == spfd.SPFD_OK and all(i["converged"] for i in infos)
        assert all(i["rel_res_true"] <= 1e-8 for i in infos)


def test_repeated_solves_bit_identical_many_components(torch_cuda, spfd):
    """Per-component sums are exact in fixed point, so two solves of the same
    field on a phantom with many components agree bit for bit."""
    torch = torch_cuda
    rng = np.random.default_rng(45)
    ph = random_phantom(20, 16, 18, rng, air_fraction=0.55)
    a = _dev(torch, rng.normal(size=(3, 19, 17, 21)))
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        p1, i1, _ = S.solve(a, 1e-12)
        p1 = p1.clone()
        p2, i2, _ = S.solve(a, 1e-12)
        assert torch.equal(p1, p2) and i1["iters"] == i2["iters"]
