"""The torch evaluation of the current-loop edge potentials (used to make
large batches of source fields where they are consumed) agrees with the numpy
one to rounding, for random loop placements and orientations."""

import numpy as np
import torch

from spfd_inputs import loop_potential, random_loops, sphere_phantom
from spfd_inputs.sources_torch import loop_potential_t


def test_loop_potential_torch_matches_numpy():
    ph = sphere_phantom(12)
    for c, n in random_loops(4, np.random.default_rng(5)) + [((0.0, 0.0, -0.4), (0, 0, 1))]:
        a_np = loop_potential(ph.dims, ph.h, ph.origin, center=c, normal=n)
        a_t = loop_potential_t(ph.dims, ph.h, ph.origin, center=c, normal=n).numpy()
        assert a_t.shape == a_np.shape
        assert np.abs(a_t - a_np).max() <= 1e-13 * np.abs(a_np).max()
        # slots past the last node along each edge's axis stay zero
        assert np.all(a_t[0, :, :, -1] == 0) and np.all(a_t[1, :, -1, :] == 0)
        assert np.all(a_t[2, -1] == 0)


def test_loop_potential_torch_into_preallocated():
    ph = sphere_phantom(6)
    out = torch.full((3, 7, 7, 7), 5.0, dtype=torch.float64)
    a = loop_potential_t(ph.dims, ph.h, ph.origin, out=out)
    assert a.data_ptr() == out.data_ptr()
    assert np.abs(a.numpy() - loop_potential(ph.dims, ph.h, ph.origin)).max() <= \
        1e-13 * np.abs(a.numpy()).max()
