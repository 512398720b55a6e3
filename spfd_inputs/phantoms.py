"""Seeded voxel conductivity phantoms.

The paper's workload is the 2 mm "Duke" voxel model (about 8.9 M node
unknowns, Section III-A).  That model is licensed and absent here, so a
synthetic body stands in for it: a union of ellipsoids (torso, head, neck,
arms, legs) with piecewise-constant tissue conductivities on seeded Voronoi
blobs, air (sigma = 0) elsewhere.  At 256 x 160 x 896 voxels, h = 2 mm it
has 8,954,036 conducting voxels and 9,250,062 conducting nodes, one
26-connected body.

All phantoms return float64 arrays indexed ``[k][j][i]`` (z, y, x).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# (centre x, y, z; semi-axes a, b, c) in metres, in the frame with x, y
# centred on the grid and z = 0 at the grid's bottom face.
BODY_ELLIPSOIDS = (
    (0.0, 0.0, 1.10, 0.175, 0.125, 0.35),   # torso
    (0.0, 0.0, 1.62, 0.085, 0.100, 0.12),   # head
    (0.0, 0.0, 1.46, 0.065, 0.065, 0.10),   # neck
    (0.205, 0.0, 1.08, 0.045, 0.050, 0.34),  # right arm
    (-0.205, 0.0, 1.08, 0.045, 0.050, 0.34),  # left arm
    (0.09, 0.0, 0.47, 0.085, 0.090, 0.46),  # right leg
    (-0.09, 0.0, 0.47, 0.085, 0.090, 0.46),  # left leg
)


@dataclass
class Phantom:
    """A voxel model: conductivities, tissue labels and the grid frame."""

    sigma: np.ndarray          # float64 [nz][ny][nx], S/m, 0 = air
    labels: np.ndarray         # int16 [nz][ny][nx], -1 = air, else tissue id
    h: float                   # voxel edge length, m
    origin: tuple              # (ox, oy, oz): node (i,j,k) sits at (i*h-ox, j*h-oy, k*h-oz)
    tissue_sigma: np.ndarray   # float64 [n_labels], sigma of each tissue label

    @property
    def dims(self):
        nz, ny, nx = self.sigma.shape
        return nx, ny, nz


def _centres(n: int, h: float, o: float) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) * h - o


def sphere_phantom(n: int = 32, h: float = 2e-3, radius: float = 0.028,
                   sigma: float = 0.2) -> Phantom:
    """Homogeneous sphere centred on an n^3 grid, origin at the grid centre.

    A voxel conducts iff its centre lies inside the sphere.  With the defaults
    (32^3, h = 2 mm, R = 28 mm) that is 11,536 voxels.
    """
    o = n * h / 2.0
    c = _centres(n, h, o)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    inside = x * x + y * y + z * z <= radius * radius
    s = np.where(inside, sigma, 0.0).astype(np.float64)
    lab = np.where(inside, 0, -1).astype(np.int16)
    return Phantom(s, lab, h, (o, o, o), np.array([sigma]))


def body_mask(nx: int, ny: int, nz: int, h: float,
              scale=(1.0, 1.0, 1.0)) -> np.ndarray:
    """Union of the body ellipsoids, each scaled by ``scale`` in (x, y, z)."""
    ox, oy = nx * h / 2.0, ny * h / 2.0
    xs, ys, zs = _centres(nx, h, ox), _centres(ny, h, oy), _centres(nz, h, 0.0)
    sx, sy, sz = scale
    m = np.zeros((nz, ny, nx), dtype=bool)
    for cx, cy, cz, a, b, c in BODY_ELLIPSOIDS:
        cx, a = cx * sx, a * sx
        cy, b = cy * sy, b * sy
        cz, c = cz * sz, c * sz
        # separable evaluation, then one broadcast sum per ellipsoid
        tx = ((xs - cx) / a) ** 2
        ty = ((ys - cy) / b) ** 2
        tz = ((zs - cz) / c) ** 2
        m |= (tz[:, None, None] + ty[None, :, None] + tx[None, None, :]) <= 1.0
    return m


def body_phantom(nx: int = 256, ny: int = 160, nz: int = 896, h: float = 2e-3,
                 scale=(1.0, 1.0, 1.0), n_seeds: int = 200, n_labels: int = 40,
                 seed_geometry: int = 2010, seed_sigma: int = 12879,
                 sigma_range=(0.02, 2.0)) -> Phantom:
    """Synthetic ellipsoid body with seeded Voronoi tissue blobs.

    ``n_seeds`` seeds are drawn without replacement among the body's voxels
    (``default_rng(seed_geometry)``), each jittered uniformly inside its voxel
    and given a label uniform in ``0..n_labels-1``; each body voxel takes the
    label of the nearest seed.  Tissue conductivities are log-uniform in
    ``sigma_range`` (``default_rng(seed_sigma)``).
    """
    from scipy.spatial import cKDTree

    m = body_mask(nx, ny, nz, h, scale)
    ox, oy = nx * h / 2.0, ny * h / 2.0
    idx = np.flatnonzero(m)
    rng = np.random.default_rng(seed_geometry)
    n_seeds = min(n_seeds, idx.size)
    pick = rng.choice(idx.size, size=n_seeds, replace=False)
    seed_flat = idx[np.sort(pick)]
    sk, sj, si = np.unravel_index(seed_flat, m.shape)
    jitter = rng.uniform(-0.5, 0.5, size=(n_seeds, 3))
    seed_pos = np.stack([(si + 0.5 + jitter[:, 0]) * h - ox,
                         (sj + 0.5 + jitter[:, 1]) * h - oy,
                         (sk + 0.5 + jitter[:, 2]) * h], axis=1)
    seed_label = rng.integers(0, n_labels, size=n_seeds)

    rs = np.random.default_rng(seed_sigma)
    lo, hi = np.log(sigma_range[0]), np.log(sigma_range[1])
    tissue_sigma = np.exp(rs.uniform(lo, hi, size=n_labels))

    labels = np.full(m.shape, -1, dtype=np.int16)
    if idx.size:
        tree = cKDTree(seed_pos)
        vk, vj, vi = np.unravel_index(idx, m.shape)
        pts = np.stack([(vi + 0.5) * h - ox, (vj + 0.5) * h - oy,
                        (vk + 0.5) * h], axis=1)
        _, near = tree.query(pts, k=1, workers=-1)
        labels.reshape(-1)[idx] = seed_label[near].astype(np.int16)
    sigma = np.where(labels >= 0, tissue_sigma[np.maximum(labels, 0)], 0.0)
    return Phantom(sigma.astype(np.float64), labels, h, (ox, oy, 0.0),
                   tissue_sigma)


def scaled_body_phantom(nx: int, ny: int, nz: int, h: float = 2e-3,
                        **kw) -> Phantom:
    """Body phantom whose ellipsoids are scaled to fill an (nx, ny, nz) box
    the way the 256 x 160 x 896 body fills its own box."""
    return body_phantom(nx, ny, nz, h,
                        scale=(nx / 256.0, ny / 160.0, nz / 896.0), **kw)


def random_phantom(nx: int, ny: int, nz: int, rng: np.random.Generator,
                   h: float = 2e-3, air_fraction: float = 0.3,
                   sigma_range=(0.02, 2.0)) -> Phantom:
    """I.i.d. random voxels: air with probability ``air_fraction``, else a
    log-uniform conductivity.  Used for small brute-force and parity cases."""
    air = rng.random((nz, ny, nx)) < air_fraction
    lo, hi = np.log(sigma_range[0]), np.log(sigma_range[1])
    s = np.exp(rng.uniform(lo, hi, size=(nz, ny, nx)))
    s[air] = 0.0
    lab = np.where(air, -1, 0).astype(np.int16)
    return Phantom(s, lab, h, (nx * h / 2.0, ny * h / 2.0, nz * h / 2.0),
                   np.array([]))
