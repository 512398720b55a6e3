"""The current-loop edge potentials of ``sources.py`` evaluated with torch ops,
so that large batches of source fields can be generated where they are used
(e.g. on a GPU) instead of on the host.

Same sampling (edge midpoints, ``a_e = A(midpoint) . t_e * h``), same closed
form and the same arithmetic-geometric-mean series as
``sources.loop_vector_potential``; the two agree to rounding.  Input
generation only: nothing of the SPFD method is computed here.
"""

from __future__ import annotations

import math

import torch

from .sources import MU0


def loop_vector_potential_t(x, y, z, center, normal, radius: float, current: float,
                            max_iter: int = 40):
    """torch version of ``sources.loop_vector_potential`` (float64 tensors,
    broadcastable)."""
    nrm = math.sqrt(sum(float(v) * float(v) for v in normal))
    n = [float(v) / nrm for v in normal]
    rx, ry, rz = torch.broadcast_tensors(x - center[0], y - center[1], z - center[2])
    zp = rx * n[0] + ry * n[1] + rz * n[2]
    px, py, pz = rx - zp * n[0], ry - zp * n[1], rz - zp * n[2]
    rho = torch.sqrt(px * px + py * py + pz * pz)
    R = float(radius)
    D2 = (R + rho) ** 2 + zp * zp
    D = torch.sqrt(D2)
    m = 4.0 * R * rho / D2
    a_n = torch.ones_like(m)
    b_n = torch.sqrt(torch.clamp(1.0 - m, min=0.0))
    g = 2.0 * R / (D2 * (1.0 + b_n))
    T = g * g
    w = 1.0
    a_n, b_n = 0.5 * (a_n + b_n), torch.sqrt(a_n * b_n)
    for _ in range(max_iter):
        a_next = 0.5 * (a_n + b_n)
        b_next = torch.sqrt(a_n * b_n)
        g = g * g * rho / (4.0 * a_next)
        w *= 2.0
        term = w * g * g
        T = T + term
        a_n, b_n = a_next, b_next
        if not bool(torch.any(term > 1e-18 * T)):
            break
    K = math.pi / (2.0 * a_n)
    f = MU0 * current / (2.0 * math.pi) * D * K * T
    return (f * (n[1] * rz - n[2] * ry), f * (n[2] * rx - n[0] * rz),
            f * (n[0] * ry - n[1] * rx))


def loop_potential_t(dims, h: float, origin, center=(0.0, 0.0, -0.4),
                     normal=(0.0, 0.0, 1.0), radius: float = 0.3, current: float = 1000.0,
                     device="cpu", out=None):
    """Edge potentials ``[3][nz+1][ny+1][nx+1]`` (float64 on ``device``, or
    written into ``out``) of the loop of ``sources.loop_potential``."""
    nx, ny, nz = dims
    ox, oy, oz = origin
    kw = dict(dtype=torch.float64, device=device)
    xs = torch.arange(nx + 1, **kw) * h - ox
    ys = torch.arange(ny + 1, **kw) * h - oy
    zs = torch.arange(nz + 1, **kw) * h - oz
    a = out if out is not None else torch.empty((3, nz + 1, ny + 1, nx + 1), **kw)
    a.zero_()

    def f(x, y, z):
        return loop_vector_potential_t(x, y, z, center, normal, radius, current)

    # z-planes in chunks bound the temporaries
    step = max(1, (1 << 22) // ((ny + 1) * (nx + 1)))
    X, Y = xs[None, None, :], ys[None, :, None]
    Xm, Ym = (xs[:-1] + 0.5 * h)[None, None, :], (ys[:-1] + 0.5 * h)[None, :, None]
    for k0 in range(0, nz + 1, step):
        k1 = min(nz + 1, k0 + step)
        z = zs[k0:k1][:, None, None]
        a[0, k0:k1, :, :nx] = f(Xm, Y, z)[0] * h
        a[1, k0:k1, :ny, :] = f(X, Ym, z)[1] * h
        kz1 = min(k1, nz)
        if kz1 > k0:
            zz = (zs[k0:kz1] + 0.5 * h)[:, None, None]
            a[2, k0:kz1, :, :] = f(X, Y, zz)[2] * h
    return a


def loop_flux_density_t(x, y, z, center, normal, radius: float, current: float,
                        max_iter: int = 40):
    """torch version of ``flux.loop_flux_density`` (float64 tensors,
    broadcastable): the same closed form and arithmetic-geometric-mean
    series."""
    nrm = math.sqrt(sum(float(v) * float(v) for v in normal))
    n = [float(v) / nrm for v in normal]
    rx, ry, rz = torch.broadcast_tensors(x - center[0], y - center[1], z - center[2])
    zp = rx * n[0] + ry * n[1] + rz * n[2]
    px, py, pz = rx - zp * n[0], ry - zp * n[1], rz - zp * n[2]
    rho = torch.sqrt(px * px + py * py + pz * pz)
    R = float(radius)
    r2 = rho * rho + zp * zp
    beta2 = (R + rho) ** 2 + zp * zp
    beta = torch.sqrt(beta2)
    alpha2 = (R - rho) ** 2 + zp * zp
    m = 4.0 * R * rho / beta2
    a_n = torch.ones_like(m)
    b_n = torch.sqrt(torch.clamp(1.0 - m, min=0.0))
    g = 2.0 * R / (beta2 * (1.0 + b_n))
    T = g * g
    w = 1.0
    a_n, b_n = 0.5 * (a_n + b_n), torch.sqrt(a_n * b_n)
    for _ in range(max_iter):
        a_next = 0.5 * (a_n + b_n)
        b_next = torch.sqrt(a_n * b_n)
        g = g * g * rho / (4.0 * a_next)
        w *= 2.0
        term = w * g * g
        T = T + term
        a_n, b_n = a_next, b_next
        if not bool(torch.any(term > 1e-18 * T)):
            break
    K = math.pi / (2.0 * a_n)
    C = MU0 * current / math.pi
    E_over_K = 1.0 - 0.5 * m - rho * rho * T
    bz = C * K / (2.0 * alpha2 * beta) * ((R * R - r2) * E_over_K + alpha2)
    bro = C * zp * K / (2.0 * alpha2 * beta) * (4.0 * R * R / beta2 - (R * R + r2) * T)
    return (bz * n[0] + bro * px, bz * n[1] + bro * py, bz * n[2] + bro * pz)


def loop_flux_t(dims, h: float, origin, center=(0.0, 0.0, -0.4), normal=(0.0, 0.0, 1.0),
                radius: float = 0.3, current: float = 1000.0, order: int = 4,
                device="cpu", out=None):
    """Facet fluxes ``[3][nz+1][ny+1][nx+1]`` (float64 on ``device``, or
    written into ``out``) of the loop of ``flux.loop_flux``: the same
    Gauss-Legendre rule on every facet."""
    import numpy as np
    nx, ny, nz = dims
    ox, oy, oz = origin
    kw = dict(dtype=torch.float64, device=device)
    xs = torch.arange(nx + 1, **kw) * h - ox
    ys = torch.arange(ny + 1, **kw) * h - oy
    zs = torch.arange(nz + 1, **kw) * h - oz
    xg, wg = np.polynomial.legendre.leggauss(order)
    t = [float(v) for v in 0.5 * (xg + 1.0)]
    wt = [float(v) for v in 0.5 * wg]
    b = out if out is not None else torch.empty((3, nz + 1, ny + 1, nx + 1), **kw)
    b.zero_()

    def f(x, y, z):
        return loop_flux_density_t(x, y, z, center, normal, radius, current)

    step = max(1, (1 << 21) // ((ny + 1) * (nx + 1)))
    X, Y = xs[None, None, :], ys[None, :, None]
    hh = h * h
    for k0 in range(0, nz + 1, step):
        k1 = min(nz + 1, k0 + step)
        kz1 = min(k1, nz)
        for p in range(order):
            for q in range(order):
                wpq = wt[p] * wt[q] * hh
                if kz1 > k0:
                    b[0, k0:kz1, :ny, :] += wpq * f(
                        X, (ys[:-1] + t[p] * h)[None, :, None],
                        (zs[k0:kz1] + t[q] * h)[:, None, None])[0]
                    b[1, k0:kz1, :, :nx] += wpq * f(
                        (xs[:-1] + t[q] * h)[None, None, :], Y,
                        (zs[k0:kz1] + t[p] * h)[:, None, None])[1]
                b[2, k0:k1, :ny, :nx] += wpq * f(
                    (xs[:-1] + t[p] * h)[None, None, :], (ys[:-1] + t[q] * h)[None, :, None],
                    zs[k0:k1][:, None, None])[2]
    return b
