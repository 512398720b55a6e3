"""Step 6 on the GPU: the nearest-rank 99th percentile of |E| per tissue and
over the whole body (Sec. II-A step 6, Sec. III-E), through spfd_percentile.

The selection returns one of its inputs, so the GPU must equal the oracle bit
for bit on the same |E| and labels.  Inputs are seeded: tie-heavy values on
random phantoms with ragged tails, the oracle's own |E| of the sphere, and
seeded log-normal fields on the full-size 2 mm body (8.95 M conducting
voxels, 40 tissues), plus the edge cases (p = 1, tiny p, no labels, empty
tissues, stray labels, an all-air grid, invalid |E|).
"""

import math

import numpy as np
import pytest

from spfd_inputs import (body_phantom, random_phantom, sphere_phantom,
                         uniform_b_landau)

pytestmark = pytest.mark.gpu
OMEGA = 2 * np.pi * 85e3


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


def _same(got, want):
    """Bit-exact equality, NaN for NaN."""
    got, want = np.asarray(got), np.asarray(want)
    assert got.shape == want.shape
    for g, w in zip(got, want):
        if math.isnan(w):
            assert math.isnan(g)
        else:
            assert g == w and np.float64(g).tobytes() == np.float64(w).tobytes()


def _compare(torch, spfd, oracle, S, sigma, E, lab, nlab, p):
    vals, cnts = S.percentile(_dev(torch, E), _dev(torch, lab.astype(np.int32)), nlab, p)
    want, wcnt = oracle.percentile(sigma, E, lab, nlab, p)
    assert list(cnts) == list(wcnt)
    _same(vals, want)
    return vals, cnts


@pytest.mark.parametrize("seed,dims,nlab", [(5, (13, 9, 11), 6), (6, (37, 21, 19), 40),
                                             (7, (8, 8, 8), 1)])
def test_percentile_random_ties(torch_cuda, spfd, oracle_mod, seed, dims, nlab):
    torch = torch_cuda
    rng = np.random.default_rng(seed)
    ph = random_phantom(*dims, rng, air_fraction=0.3)
    nx, ny, nz = dims
    # few distinct values (ties across digit boundaries), zeros, one huge value
    E = rng.integers(0, 9, (nz, ny, nx)) * rng.choice([1e-3, 2.5e-7, 3.0], (nz, ny, nx))
    E.reshape(-1)[0] = 1e300
    lab = rng.integers(-2, nlab + 2, (nz, ny, nx)).astype(np.int32)
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        for p in (0.99, 0.5, 1.0, 1e-9, 0.73):
            _compare(torch, spfd, oracle_mod, S, ph.sigma, E, lab, nlab, p)


def test_percentile_no_labels_and_empty(torch_cuda, spfd, oracle_mod):
    torch = torch_cuda
    rng = np.random.default_rng(8)
    ph = random_phantom(10, 7, 9, rng, air_fraction=0.4)
    E = rng.lognormal(-2.0, 1.5, ph.sigma.shape)
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        vals, cnts = S.percentile(_dev(torch, E), None, 0, 0.99)
        want, wcnt = oracle_mod.percentile(ph.sigma, E, np.zeros(E.shape, np.int32), 0, 0.99)
        _same(vals, want)
        assert cnts == list(wcnt) and cnts[0] == int((ph.sigma > 0).sum())
        # labels 0..2 used, 3..4 empty
        lab = rng.integers(0, 3, E.shape).astype(np.int32)
        vals, cnts = _compare(torch, spfd, oracle_mod, S, ph.sigma, E, lab, 5, 0.99)
        assert math.isnan(vals[3]) and cnts[3] == 0


def test_percentile_of_oracle_field(torch_cuda, spfd, oracle_mod):
    """The oracle's |E| of the sphere in the Landau-gauge field: GPU and
    oracle select the same voxel; the GPU's own |E| gives the same 99th
    percentile to the |E| parity bar."""
    torch = torch_cuda
    ph = sphere_phantom()
    a = uniform_b_landau(ph.dims, ph.h, ph.origin, 27e-6)
    psi_r, _, _ = oracle_mod.solve(ph.sigma, ph.h, a, tol=1e-13)
    E_r = oracle_mod.efield(ph.sigma, a, psi_r, ph.h, OMEGA)
    lab = np.where(ph.sigma > 0, (np.arange(E_r.size).reshape(E_r.shape) % 3), -1).astype(np.int32)
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        want, _ = _compare(torch, spfd, oracle_mod, S, ph.sigma, E_r, lab, 3, 0.99)
        ad = _dev(torch, a)
        psi, info, st = S.solve(ad, 1e-13)
        E = S.efield(ad, psi, OMEGA)
        got, _ = S.percentile(E, _dev(torch, lab), 3, 0.99)
    assert np.max(np.abs(np.array(got) - want) / np.array(want)) <= 1e-7


def test_percentile_body_full_size(torch_cuda, spfd, oracle_mod):
    """The 2 mm body (256 x 160 x 896 voxels, 40 tissues): seeded log-normal
    |E| with a share of exact ties, every tissue and the body bit-exact."""
    torch = torch_cuda
    ph = body_phantom()
    rng = np.random.default_rng(12879)
    E = rng.lognormal(-4.0, 1.2, ph.sigma.shape)
    tie = rng.random(ph.sigma.shape) < 0.05
    E[tie] = np.round(E[tie], 3)
    E[ph.sigma == 0] = 0.0
    lab = ph.labels.astype(np.int32)
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        vals, cnts = _compare(torch, spfd, oracle_mod, S, ph.sigma, E, lab, 40, 0.99)
        assert cnts[40] == 8_954_036
        # a second call on the same context reuses its scratch
        _compare(torch, spfd, oracle_mod, S, ph.sigma, E, lab, 40, 0.5)


def test_percentile_errors_and_air(torch_cuda, spfd):
    torch = torch_cuda
    sig = np.zeros((4, 4, 4))
    with spfd.Solver(_dev(torch, sig), 2e-3) as S:
        vals, cnts = S.percentile(_dev(torch, np.ones((4, 4, 4))), None, 0, 0.99)
        assert math.isnan(vals[0]) and cnts == [0]
    rng = np.random.default_rng(9)
    ph = random_phantom(6, 6, 6, rng, air_fraction=0.0)
    E = np.ones((6, 6, 6))
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        for bad in (-1.0, np.nan, np.inf):
            Eb = E.copy()
            Eb[2, 3, 1] = bad
            with pytest.raises(spfd.SpfdError) as ei:
                S.percentile(_dev(torch, Eb), None, 0, 0.99)
            assert ei.value.status == spfd.SPFD_EINVAL
        for p in (0.0, 1.5, np.nan):
            with pytest.raises(spfd.SpfdError):
                S.percentile(_dev(torch, E), None, 0, p)
        vals, _ = S.percentile(_dev(torch, E), None, 0, 0.99)
        assert vals == [1.0]
