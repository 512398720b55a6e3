"""Edge vector potentials of analytic magneto-quasistatic sources.

The SPFD right-hand side needs the discrete magnetic vector potential on the
grid edges (the vector ``a`` of Eq. 1 and Eq. 3).  The paper obtains it from
measured or simulated flux densities by tree-cotree gauging (Eq. 2); here it
is sampled from closed-form potentials instead:

    a_e = A(midpoint of e) . t_e * h

with ``t_e`` the unit vector of the edge's axis.  The samples are exact line
integrals for the linear potentials of a uniform field and a midpoint rule for
the current loop.  Output layout: float64 ``[3][nz+1][ny+1][nx+1]``; the slot
of a d-edge past the last node along d is zero.
"""

from __future__ import annotations

import os

import numpy as np

MU0 = 4.0e-7 * np.pi  # vacuum permeability, H/m


def _node_coords(n: int, h: float, o: float) -> np.ndarray:
    return np.arange(n + 1, dtype=np.float64) * h - o


def edge_potential(field, dims, h: float, origin, chunk_nodes: int = 1 << 20):
    """Sample a vector potential ``field(x, y, z) -> (Ax, Ay, Az)`` at the edge
    midpoints of a voxel grid and return the edge line integrals.

    ``field`` receives broadcastable float64 arrays in metres and returns the
    three components in T*m.  Work is chunked over z-planes of nodes.
    """
    nx, ny, nz = dims
    ox, oy, oz = origin
    a = np.zeros((3, nz + 1, ny + 1, nx + 1), dtype=np.float64)
    xs, ys, zs = (_node_coords(nx, h, ox), _node_coords(ny, h, oy),
                  _node_coords(nz, h, oz))
    xm, ym, zm = xs[:-1] + 0.5 * h, ys[:-1] + 0.5 * h, zs[:-1] + 0.5 * h
    plane = (ny + 1) * (nx + 1)
    step = max(1, chunk_nodes // plane)

    def work(k0):
        k1 = min(nz + 1, k0 + step)
        z = zs[k0:k1][:, None, None]
        # x edges: midpoints (xm, y_j, z_k)
        a[0, k0:k1, :, :nx] = field(xm[None, None, :], ys[None, :, None], z)[0] * h
        # y edges: midpoints (x_i, ym, z_k)
        a[1, k0:k1, :ny, :] = field(xs[None, None, :], ym[None, :, None], z)[1] * h
        # z edges: midpoints (x_i, y_j, zm), only for k < nz
        kz1 = min(k1, nz)
        if kz1 > k0:
            zz = zm[k0:kz1][:, None, None]
            a[2, k0:kz1, :, :] = field(xs[None, None, :], ys[None, :, None], zz)[2] * h

    starts = list(range(0, nz + 1, step))
    if len(starts) > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=min(len(starts), os.cpu_count() or 1)) as ex:
            list(ex.map(work, starts))
    else:
        work(0)
    return a


def uniform_b_symmetric(dims, h: float, origin, B: float = 27e-6):
    """Uniform flux density B along +z in the symmetric gauge A = B x r / 2."""

    def f(x, y, z):
        zero = np.zeros(np.broadcast_shapes(np.shape(x), np.shape(y), np.shape(z)))
        return (-0.5 * B * y + zero, 0.5 * B * x + zero, zero)

    return edge_potential(f, dims, h, origin)


def uniform_b_landau(dims, h: float, origin, B: float = 27e-6):
    """Uniform flux density B along +z in the Landau gauge A = (-B y, 0, 0)."""

    def f(x, y, z):
        zero = np.zeros(np.broadcast_shapes(np.shape(x), np.shape(y), np.shape(z)))
        return (-B * y + zero, zero, zero)

    return edge_potential(f, dims, h, origin)


def loop_vector_potential(x, y, z, center, normal, radius: float,
                          current: float, max_iter: int = 40):
    """Vector potential of a thin circular current loop (one turn).

    In the loop's own cylinder coordinates (rho, z') the potential is
    azimuthal with (Jackson, Classical Electrodynamics, Sec. 5.5)

        A_phi = mu0 I / (pi k) sqrt(R/rho) [(1 - k^2/2) K(k) - E(k)],
        k^2 = 4 R rho / ((R + rho)^2 + z'^2).

    The bracket equals ``K * sum_{n>=1} 2^(n-1) c_n^2`` in the arithmetic-
    geometric-mean recursion (a_0 = 1, b_0 = sqrt(1-k^2), c_0 = k), which has
    no cancellation for small k.  Dividing out rho analytically gives

        A(r) = mu0 I / (2 pi) * D * K * T * (n x r),
        D = sqrt((R + rho)^2 + z'^2),   T = sum_n 2^(n-1) (c_n / rho)^2,

    finite on the axis.  ``r`` is relative to the loop centre; the current
    circulates right-handed about ``normal``.
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
    D2 = (R + rho) ** 2 + zp * zp
    D = np.sqrt(D2)
    m = 4.0 * R * rho / D2
    a_n = np.ones_like(m)
    b_n = np.sqrt(np.maximum(1.0 - m, 0.0))
    # gamma_1 = c_1 / rho = m / (2 (1 + b_0) rho) = 2 R / (D^2 (1 + b_0))
    g = 2.0 * R / (D2 * (1.0 + b_n))
    T = g * g
    w = 1.0
    a_next = 0.5 * (a_n + b_n)
    b_next = np.sqrt(a_n * b_n)
    a_n, b_n = a_next, b_next
    for _ in range(max_iter):
        # c_{n+1} = c_n^2 / (4 a_{n+1})  ->  gamma_{n+1} = gamma_n^2 rho / (4 a_{n+1})
        a_next = 0.5 * (a_n + b_n)
        b_next = np.sqrt(a_n * b_n)
        g = g * g * rho / (4.0 * a_next)
        w *= 2.0
        term = w * g * g
        T = T + term
        a_n, b_n = a_next, b_next
        # quadratic convergence: stop once the last term no longer changes T
        if not np.any(term > 1e-18 * T):
            break
    K = np.pi / (2.0 * a_n)
    f = MU0 * current / (2.0 * np.pi) * D * K * T
    # n x r
    cx = n[1] * rz - n[2] * ry
    cy = n[2] * rx - n[0] * rz
    cz = n[0] * ry - n[1] * rx
    return f * cx, f * cy, f * cz


def loop_potential(dims, h: float, origin, center=(0.0, 0.0, -0.4),
                   normal=(0.0, 0.0, 1.0), radius: float = 0.3,
                   current: float = 1000.0):
    """Edge potentials of a circular loop (radius 0.3 m, 1000 A-turns, 0.4 m
    below the grid's bottom face by default)."""

    def f(x, y, z):
        return loop_vector_potential(x, y, z, center, normal, radius, current)

    return edge_potential(f, dims, h, origin)


def random_loops(n: int, rng: np.random.Generator):
    """Loop placements for a batch of sources: centre x, y ~ U(-0.5, 0.5) m,
    z ~ U(-0.6, -0.3) m, unit normal uniform on the sphere."""
    cx = rng.uniform(-0.5, 0.5, size=n)
    cy = rng.uniform(-0.5, 0.5, size=n)
    cz = rng.uniform(-0.6, -0.3, size=n)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return [((cx[i], cy[i], cz[i]), tuple(v[i])) for i in range(n)]
