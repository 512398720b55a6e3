"""GPU adjoint gradient of J = mean over conducting voxels of |E|^2 against
the oracle's (tests/test_oracle_adjoint.py pins the oracle against finite
differences).  Bars: J to 1e-9 relative, per-tissue dJ/dsigma and dJ/da to
1e-6 relative (the spec bar for the gradient), with both GPU solves at
1e-12 and the oracle's at 1e-13.  Edge and voxel arrays are compared in the
relative L2 norm; per-tissue sums one by one.
"""

import numpy as np
import pytest

from spfd_inputs import loop_potential, random_phantom, scaled_body_phantom

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


def _rel(x, y):
    return np.linalg.norm(x - y) / np.linalg.norm(y)


def _gpu_grad(torch, spfd, sigma, h, a, tol=1e-12, **opts):
    with spfd.Solver(_dev(torch, sigma), h, **opts) as S:
        ad = _dev(torch, a)
        psi, _, st = S.solve(ad, tol)
        assert st == spfd.SPFD_OK
        J, dJda, dJds, info, st = S.energy_grad(ad, psi, OMEGA, tol)
        assert st == spfd.SPFD_OK and info["converged"]
        return J, dJda.cpu().numpy(), dJds.cpu().numpy(), info


def _check(oracle, ph, a, J, dJda, dJds, tol_grad=1e-6):
    ref = oracle.energy_gradient(ph.sigma, ph.h, a, OMEGA, tol=1e-13)
    assert ref["info"]["converged"] and ref["info_adj"]["converged"]
    assert J == pytest.approx(ref["J"], rel=1e-9)
    assert _rel(dJda, ref["dJda"]) <= tol_grad
    assert _rel(dJds, ref["dJdsigma"]) <= tol_grad
    assert np.all(dJds[ph.sigma == 0] == 0.0)
    return ref


def test_energy_grad_scaled_body(torch_cuda, spfd, oracle_mod):
    """The body's ellipsoids scaled to a 32 x 24 x 112 voxel box, 40
    tissues, loop source; per-tissue gradients."""
    ph = scaled_body_phantom(32, 24, 112)
    a = loop_potential(ph.dims, ph.h, ph.origin)
    J, dJda, dJds, info = _gpu_grad(torch_cuda, spfd, ph.sigma, ph.h, a)
    ref = _check(oracle_mod, ph, a, J, dJda, dJds)
    for t in np.unique(ph.labels[ph.labels >= 0]):
        m = ph.labels == t
        want = ref["dJdsigma"][m].sum()
        assert dJds[m].sum() == pytest.approx(want, rel=1e-6, abs=1e-9 * np.abs(ref["dJdsigma"]).sum())


@pytest.mark.parametrize("seed,dims,air", [(21, (13, 9, 11), 0.3), (22, (9, 17, 6), 0.55)])
def test_energy_grad_random_phantoms(torch_cuda, spfd, oracle_mod, seed, dims, air):
    """Random conductivities, random a, ragged brick tails; many components
    at 55 % air."""
    rng = np.random.default_rng(seed)
    ph = random_phantom(*dims, rng, air_fraction=air)
    nx, ny, nz = dims
    a = rng.normal(size=(3, nz + 1, ny + 1, nx + 1)) * 1e-9
    J, dJda, dJds, _ = _gpu_grad(torch_cuda, spfd, ph.sigma, ph.h, a)
    _check(oracle_mod, ph, a, J, dJda, dJds)


def test_energy_grad_mixed_precision(torch_cuda, spfd, oracle_mod):
    """The mixed-precision solver reaches the same gradient: both solves go
    to 1e-12 by FP64 refinement around the FP32 V-cycle."""
    ph = scaled_body_phantom(32, 24, 112)
    a = loop_potential(ph.dims, ph.h, ph.origin)
    J, dJda, dJds, _ = _gpu_grad(torch_cuda, spfd, ph.sigma, ph.h, a,
                                 precision=spfd.SPFD_MIXED)
    _check(oracle_mod, ph, a, J, dJda, dJds)


def test_field_energy_autograd_per_tissue(torch_cuda, spfd, oracle_mod):
    """torch.autograd through sigma = table[labels]: the tissue gradient is
    the per-label sum of dJ/dsigma, and dJ/da along a direction matches the
    exact central difference of the GPU objective (J is quadratic in a)."""
    torch = torch_cuda
    from paper_2010_12879_gb300.autograd import field_energy
    ph = scaled_body_phantom(32, 24, 112)
    a_np = loop_potential(ph.dims, ph.h, ph.origin)
    lab = torch.from_numpy(ph.labels.astype(np.int64)).cuda()
    table = torch.tensor(ph.tissue_sigma, dtype=torch.float64, device="cuda", requires_grad=True)
    a = _dev(torch, a_np).requires_grad_(True)

    def sigma_of(tab):
        s = torch.zeros(lab.shape, dtype=torch.float64, device="cuda")
        m = lab >= 0
        s[m] = tab[lab[m]]
        return s

    J = field_energy(sigma_of(table), a, ph.h, OMEGA, tol=1e-12)
    J.backward()
    ref = oracle_mod.energy_gradient(ph.sigma, ph.h, a_np, OMEGA, tol=1e-13)
    want = np.array([ref["dJdsigma"][ph.labels == t].sum() for t in range(len(ph.tissue_sigma))])
    got = table.grad.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max()
    w = torch.from_numpy(np.random.default_rng(7).normal(size=a_np.shape)).cuda()
    eps = 1e-3 * float(a.detach().abs().max()) / float(w.abs().max())
    with torch.no_grad():
        s0 = sigma_of(table)
        Jp = field_energy(s0, a + eps * w, ph.h, OMEGA, tol=1e-12)
        Jm = field_energy(s0, a - eps * w, ph.h, OMEGA, tol=1e-12)
    fd = float((Jp - Jm) / (2 * eps))
    an = float((a.grad * w).sum())
    assert fd == pytest.approx(an, rel=1e-6)


def test_energy_grad_scaled_body_128_properties(torch_cuda, spfd, oracle_mod):
    """The scaled body at full size (128 x 96 x 448 voxels, h = 2 mm): the
    oracle cannot solve it in seconds, so the GPU gradient is checked
    through what holds at any size.  J and dJ/du follow from the GPU's Psi
    by the oracle's own evaluation, and G^T dJ/da = G^T dJ/du - A lambda is
    the adjoint solve's residual, at most its tolerance times ||G^T dJ/du||
    (gauge invariance makes it 0 at the exact solution)."""
    torch = torch_cuda
    ph = scaled_body_phantom(128, 96, 448)
    a = loop_potential(ph.dims, ph.h, ph.origin)
    with spfd.Solver(_dev(torch, ph.sigma), ph.h) as S:
        ad = _dev(torch, a)
        psi, _, st = S.solve(ad, 1e-10)
        assert st == spfd.SPFD_OK
        J, dJda, dJds, info, st = S.energy_grad(ad, psi, OMEGA, 1e-10)
        assert st == spfd.SPFD_OK and info["converged"]
        psi = psi.cpu().numpy()
        dJda = dJda.cpu().numpy()
    J_ref, gJ = oracle_mod.energy(ph.sigma, a, psi, ph.h, OMEGA)
    assert J == pytest.approx(J_ref, rel=1e-12)
    b = oracle_mod.div(gJ)
    assert np.linalg.norm(oracle_mod.div(dJda)) <= 2e-10 * np.linalg.norm(b)


def test_energy_grad_scaled_body_128_finite_differences(torch_cuda, spfd):
    """The adjoint gradient at the full size of the adjoint workload (the
    body scaled to 128 x 96 x 448 voxels, 40 tissues, loop source) against
    central differences of the GPU's own objective:
    * dJ/dsigma summed per tissue, for a seeded subset of 8 tissues, against
      (J(t_i (1 + d)) - J(t_i (1 - d))) / (2 d t_i) at relative step d = 1e-6
      of the tissue's table entry, every solve to 1e-12;
    * dJ/da along 3 seeded random directions w against the central
      difference of J(a +- eps w): J is quadratic in a, so the difference is
      exact up to rounding at any step.
    Bar: 1e-6 relative, normwise over the 8 tissues (the largest error
    against the largest gradient), per direction for dJ/da."""
    torch = torch_cuda
    ph = scaled_body_phantom(128, 96, 448)
    a = _dev(torch, loop_potential(ph.dims, ph.h, ph.origin))
    lab = ph.labels.astype(np.int64)
    air = lab < 0
    tol = 1e-12

    def sigma_of(table):
        s = np.asarray(table)[np.where(air, 0, lab)]
        s[air] = 0.0
        return s

    def run(table, av, grads=False):
        with spfd.Solver(_dev(torch, sigma_of(table)), ph.h) as S:
            psi, _, st = S.solve(av, tol)
            assert st == spfd.SPFD_OK
            J, dJda, dJds, info, st = S.energy_grad(av, psi, OMEGA, tol)
            assert st == spfd.SPFD_OK and info["converged"]
            return (J, dJda, dJds) if grads else J

    table = np.array(ph.tissue_sigma, dtype=np.float64)
    J0, dJda, dJds = run(table, a, grads=True)
    dJds = dJds.cpu().numpy()
    rng = np.random.default_rng(128)
    present = np.unique(lab[~air])
    pick = np.sort(rng.choice(present, size=8, replace=False))
    adj = np.array([dJds[lab == t].sum() for t in pick])
    fd = []
    d = 1e-6
    for t in pick:
        tp, tm = table.copy(), table.copy()
        tp[t] *= 1 + d
        tm[t] *= 1 - d
        fd.append((run(tp, a) - run(tm, a)) / (2 * d * table[t]))
    fd = np.array(fd)
    err_sigma = np.abs(fd - adj).max() / np.abs(adj).max()
    errs_a = []
    for _ in range(3):
        w = torch.from_numpy(rng.normal(size=tuple(a.shape))).cuda()
        eps = 1e-3 * float(a.abs().max()) / float(w.abs().max())
        Jp, Jm = run(table, a + eps * w), run(table, a - eps * w)
        fd_a = (Jp - Jm) / (2 * eps)
        an = float((dJda * w).sum())
        errs_a.append(abs(fd_a - an) / abs(an))
    print(f"128x96x448 adjoint vs central differences: dJ/dsigma {err_sigma:.2e}, "
          f"dJ/da {max(errs_a):.2e}")
    assert err_sigma <= 1e-6, (fd, adj)
    assert max(errs_a) <= 1e-6, errs_a
