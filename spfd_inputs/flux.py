"""Facet fluxes of analytic magneto-quasistatic sources.

Step 2 of the paper's pipeline delivers the magnetic flux through every facet
of the fine grid (the vector ``b`` of Eq. 2); here it is computed from the
closed-form flux density of the sources instead of from measurements:

    b_f = integral over facet f of B . n_f dS

by a tensor Gauss-Legendre rule on the square facet.  Facet ``d`` at node
``(i, j, k)`` is the square spanned by the edges that leave that node along
the two other axes; its normal is ``+d``.  Output layout: float64
``[3][nz+1][ny+1][nx+1]`` (the edge layout); slots of facets that would leave
the grid are zero.

Only input generation lives here: the flux density is evaluated from its
textbook closed form and integrated over each facet; no discrete operator of
the method is applied.
"""

from __future__ import annotations

import os

import numpy as np

from .sources import MU0


def gauss_legendre01(order: int):
    """Nodes and weights of the Gauss-Legendre rule on [0, 1] (weights sum
    to 1)."""
    x, w = np.polynomial.legendre.leggauss(order)
    return 0.5 * (x + 1.0), 0.5 * w


def loop_flux_density(x, y, z, center, normal, radius: float, current: float,
                      max_iter: int = 40):
    """Flux density (T) of a thin circular current loop (one turn).

    In the loop's cylinder coordinates (rho, z') the field is (Simpson et al.,
    "Simple analytic expressions for the magnetic field of a circular current
    loop", NASA 2001; Smythe, Static and Dynamic Electricity, Sec. 7.10)

        B_z'  = C / (2 alpha^2 beta) [(R^2 - r^2) E(k) + alpha^2 K(k)]
        B_rho = C z' / (2 alpha^2 beta rho) [(R^2 + r^2) E(k) - alpha^2 K(k)]

    with C = mu0 I / pi, r^2 = rho^2 + z'^2, alpha^2 = (R - rho)^2 + z'^2,
    beta^2 = (R + rho)^2 + z'^2, k^2 = 4 R rho / beta^2.  K and E come from
    the arithmetic-geometric mean (a_0 = 1, b_0 = sqrt(1 - k^2), c_0 = k):
    K = pi / (2 a_N), E = K (1 - k^2/2 - S) with S = sum_{n>=1} 2^(n-1) c_n^2.
    Writing S = rho^2 T (T finite on the axis, gamma_n = c_n / rho) turns the
    bracket of B_rho, which vanishes like rho^2, into
    K rho^2 (4 R^2 / beta^2 - (R^2 + r^2) T), so B_rho / rho is evaluated
    without cancellation and B = B_z' n + (B_rho / rho) p, p the part of
    r - centre normal to n.  The current circulates right-handed about
    ``normal``.
    """
    n = np.asarray(normal, dtype=np.float64)
    n = n / np.linalg.norm(n)
    rx = np.asarray(x, dtype=np.float64) - center[0]
    ry = np.asarray(y, dtype=np.float64) - center[1]
    rz = np.asarray(z, dtype=np.float64) - center[2]
    rx, ry, rz = np.broadcast_arrays(rx, ry, rz)
    zp = rx * n[0] + ry * n[1] + rz * n[2]
    px, py, pz = rx - zp * n[0], ry - zp * n[1], rz - zp * n[2]
    rho = np.sqrt(px * px + py * py + pz * pz)
    R = float(radius)
    r2 = rho * rho + zp * zp
    beta2 = (R + rho) ** 2 + zp * zp
    beta = np.sqrt(beta2)
    alpha2 = (R - rho) ** 2 + zp * zp
    m = 4.0 * R * rho / beta2
    a_n = np.ones_like(m)
    b_n = np.sqrt(np.maximum(1.0 - m, 0.0))
    g = 2.0 * R / (beta2 * (1.0 + b_n))  # gamma_1 = c_1 / rho
    T = g * g
    w = 1.0
    a_n, b_n = 0.5 * (a_n + b_n), np.sqrt(a_n * b_n)
    for _ in range(max_iter):
        a_next = 0.5 * (a_n + b_n)
        b_next = np.sqrt(a_n * b_n)
        g = g * g * rho / (4.0 * a_next)
        w *= 2.0
        term = w * g * g
        T = T + term
        a_n, b_n = a_next, b_next
        if not np.any(term > 1e-18 * T):
            break
    K = np.pi / (2.0 * a_n)
    C = MU0 * current / np.pi
    E_over_K = 1.0 - 0.5 * m - rho * rho * T
    bz = C * K / (2.0 * alpha2 * beta) * ((R * R - r2) * E_over_K + alpha2)
    brho_over_rho = C * zp * K / (2.0 * alpha2 * beta) * (4.0 * R * R / beta2 - (R * R + r2) * T)
    return (bz * n[0] + brho_over_rho * px, bz * n[1] + brho_over_rho * py,
            bz * n[2] + brho_over_rho * pz)


def facet_flux(field, dims, h: float, origin, order: int = 4, chunk_nodes: int = 1 << 18):
    """Integrate a flux density ``field(x, y, z) -> (Bx, By, Bz)`` over every
    facet of a voxel grid with an ``order`` x ``order`` Gauss-Legendre rule.
    Work is chunked over z-planes of nodes."""
    nx, ny, nz = dims
    ox, oy, oz = origin
    b = np.zeros((3, nz + 1, ny + 1, nx + 1), dtype=np.float64)
    xs = np.arange(nx + 1, dtype=np.float64) * h - ox
    ys = np.arange(ny + 1, dtype=np.float64) * h - oy
    zs = np.arange(nz + 1, dtype=np.float64) * h - oz
    t, wt = gauss_legendre01(order)
    plane = (ny + 1) * (nx + 1)
    step = max(1, chunk_nodes // plane)
    hh = h * h

    def work(k0):
        k1 = min(nz + 1, k0 + step)
        z = zs[k0:k1][:, None, None]
        kz1 = min(k1, nz)
        for p in range(order):
            for q in range(order):
                wpq = wt[p] * wt[q] * hh
                # facet x at (i, j, k): spans y in [y_j, y_j+h], z in [z_k, z_k+h]
                if kz1 > k0:
                    zz = (zs[k0:kz1] + t[q] * h)[:, None, None]
                    b[0, k0:kz1, :ny, :] += wpq * field(
                        xs[None, None, :], (ys[:-1] + t[p] * h)[None, :, None], zz)[0]
                    # facet y: spans z in [z_k, z_k+h], x in [x_i, x_i+h]
                    b[1, k0:kz1, :, :nx] += wpq * field(
                        (xs[:-1] + t[q] * h)[None, None, :], ys[None, :, None],
                        (zs[k0:kz1] + t[p] * h)[:, None, None])[1]
                # facet z: spans x in [x_i, x_i+h], y in [y_j, y_j+h]
                b[2, k0:k1, :ny, :nx] += wpq * field(
                    (xs[:-1] + t[p] * h)[None, None, :], (ys[:-1] + t[q] * h)[None, :, None],
                    z)[2]

    starts = list(range(0, nz + 1, step))
    if len(starts) > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=min(len(starts), os.cpu_count() or 1)) as ex:
            list(ex.map(work, starts))
    else:
        work(0)
    return b


def uniform_flux(dims, h: float, B=(0.0, 0.0, 27e-6)):
    """Facet fluxes of a uniform flux density B = (Bx, By, Bz): B_d h^2 on
    every facet with normal d."""
    nx, ny, nz = dims
    b = np.zeros((3, nz + 1, ny + 1, nx + 1), dtype=np.float64)
    b[0, :nz, :ny, :] = B[0] * h * h
    b[1, :nz, :, :nx] = B[1] * h * h
    b[2, :, :ny, :nx] = B[2] * h * h
    return b


def loop_flux(dims, h: float, origin, center=(0.0, 0.0, -0.4), normal=(0.0, 0.0, 1.0),
              radius: float = 0.3, current: float = 1000.0, order: int = 4):
    """Facet fluxes of the circular loop of ``sources.loop_potential``
    (radius 0.3 m, 1000 A-turns, 0.4 m below the grid's bottom face by
    default)."""

    def f(x, y, z):
        return loop_flux_density(x, y, z, center, normal, radius, current)

    return facet_flux(f, dims, h, origin, order)
