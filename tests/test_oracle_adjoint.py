"""Pins of the oracle's adjoint gradient of J = mean over conducting voxels of
|E|^2 (Eq. 1, reading R6), against what the mathematics fixes without the
oracle's own gradient formulas:

* J is the mean square of the oracle's own |E| (Eq. 1 evaluation);
* G^T (``div``) is the transpose of G (head minus tail) under the dot product;
* gJ = dJ/du: J is a quadratic form in u, so central differences in one edge
  value of a (Psi held) are exact up to rounding;
* dJ/da: for fixed sigma the whole map a -> Psi(a) -> J is quadratic, so a
  central difference along any direction is exact up to rounding;
* dJ/dsigma summed per tissue label against central differences at relative
  step 1e-6 (solves to 1e-13, so the solver error is ~1e-7 of the step);
* gauge invariance (a -> a + G chi leaves J unchanged) forces G^T dJ/da = 0.
"""

import numpy as np
import pytest

import oracle

H = 2e-3
OMEGA = 2 * np.pi * 85e3


@pytest.fixture(scope="module")
def case():
    rng = np.random.default_rng(3)
    labels = rng.integers(0, 3, size=(4, 5, 6))
    air = rng.random((4, 5, 6)) < 0.2
    table = np.array([0.2, 0.7, 1.5])
    a = rng.normal(size=(3, 5, 6, 7)) * 1e-6

    def sigma(t):
        s = t[labels]
        s[air] = 0.0
        return s

    res = oracle.energy_gradient(sigma(table), H, a, OMEGA)
    return dict(rng=rng, labels=labels, air=air, table=table, a=a, sigma=sigma, res=res)


def test_energy_is_mean_square_of_efield(case):
    s = case["sigma"](case["table"])
    res = case["res"]
    E = oracle.efield(s, case["a"], res["psi"], H, OMEGA)
    m = s > 0
    assert res["J"] == pytest.approx((E[m] ** 2).mean(), rel=1e-13)


def test_div_is_transpose_of_gradient():
    rng = np.random.default_rng(11)
    nx, ny, nz = 5, 4, 3
    v = rng.normal(size=(3, nz + 1, ny + 1, nx + 1))
    x = rng.normal(size=(nz + 1, ny + 1, nx + 1))
    gx = np.zeros_like(v)      # (G x)_e = x_head - x_tail, edges leaving each node in +d
    gx[0, :, :, :-1] = x[:, :, 1:] - x[:, :, :-1]
    gx[1, :, :-1, :] = x[:, 1:, :] - x[:, :-1, :]
    gx[2, :-1, :, :] = x[1:, :, :] - x[:-1, :, :]
    v[0, :, :, -1] = 0.0       # no edges leave the grid
    v[1, :, -1, :] = 0.0
    v[2, -1, :, :] = 0.0
    assert (oracle.div(v) * x).sum() == pytest.approx((v * gx).sum(), rel=1e-12)


def test_gJ_is_derivative_of_J_in_u(case):
    s = case["sigma"](case["table"])
    a, psi = case["a"], case["res"]["psi"]
    J0, gJ = oracle.energy(s, a, psi, H, OMEGA)
    rng = np.random.default_rng(5)
    edges = np.argwhere(np.abs(gJ) > 0)
    for e in edges[rng.choice(len(edges), 6, replace=False)]:
        da = np.zeros_like(a)
        eps = 1e-7
        da[tuple(e)] = eps
        fd = (oracle.energy(s, a + da, psi, H, OMEGA)[0] -
              oracle.energy(s, a - da, psi, H, OMEGA)[0]) / (2 * eps)
        assert fd == pytest.approx(gJ[tuple(e)], rel=1e-7)


def test_dJda_along_random_directions(case):
    s = case["sigma"](case["table"])
    a, res = case["a"], case["res"]
    rng = np.random.default_rng(6)
    for _ in range(3):
        w = rng.normal(size=a.shape)
        eps = 1e-6
        fd = (oracle.energy_gradient(s, H, a + eps * w, OMEGA)["J"] -
              oracle.energy_gradient(s, H, a - eps * w, OMEGA)["J"]) / (2 * eps)
        assert fd == pytest.approx((res["dJda"] * w).sum(), rel=1e-9)


def test_dJdsigma_per_tissue_against_central_differences(case):
    table, labels, air, res = case["table"], case["labels"], case["air"], case["res"]
    for t in range(len(table)):
        d = 1e-6 * table[t]
        tp, tm = table.copy(), table.copy()
        tp[t] += d
        tm[t] -= d
        fd = (oracle.energy_gradient(case["sigma"](tp), H, case["a"], OMEGA)["J"] -
              oracle.energy_gradient(case["sigma"](tm), H, case["a"], OMEGA)["J"]) / (2 * d)
        adj = res["dJdsigma"][(labels == t) & ~air].sum()
        assert fd == pytest.approx(adj, rel=1e-6)


def test_gauge_invariance_of_dJda(case):
    res = case["res"]
    scale = np.abs(res["dJda"]).max()
    assert np.abs(oracle.div(res["dJda"])).max() <= 1e-10 * scale
    assert np.all(res["dJdsigma"][case["air"]] == 0.0)
