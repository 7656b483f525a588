"""The seeded input generators (vrc_workloads) are the one module the oracle
and the CUDA path share: the same seed must give the same arrays, a
different seed different ones, and the ray records must have the layout and
value ranges both sides assume (float32 SoA, positions inside the box,
non-zero directions, energies inside the table range, positive weights)."""
from __future__ import annotations

import numpy as np
import pytest

import vrc_workloads as W

SMALL = {
    "slab": lambda seed: W.slab_room(seed=seed, n=24, n_rays=4096, n_points=300, n_resonances=6,
                                     n_groups=3),
    "lattice": lambda seed: W.pin_lattice(seed=seed, pins=2, cells_per_pin=8, nz=3, n_rays=4096,
                                          n_points=300, n_resonances=6),
    "graded": lambda seed: W.graded_assembly(seed=seed, pins=2, cells_per_pin=5, reflector=4.0,
                                             n_rays=4096, n_points=300, n_resonances=6),
}


def _arrays(p):
    out = [np.asarray(p.rays[k]) for k in W.RAY_FIELDS]
    out.append(np.asarray(p.mesh.material))
    for t in p.tables:
        if t is not None:
            out += [np.asarray(t[0]), np.asarray(t[1])]
    return out


@pytest.mark.parametrize("name", sorted(SMALL))
def test_same_seed_same_inputs(name):
    a, b = SMALL[name](7), SMALL[name](7)
    for x, y in zip(_arrays(a), _arrays(b)):
        assert x.dtype == y.dtype and np.array_equal(x, y)
    c = SMALL[name](8)
    assert not np.array_equal(a.rays["x"], c.rays["x"])


@pytest.mark.parametrize("name", sorted(SMALL))
def test_ray_records(name):
    p = SMALL[name](3)
    lo, hi = np.array(p.mesh.lo), np.array(p.mesh.hi)
    for k in W.RAY_FIELDS:
        assert p.rays[k].dtype == np.float32 and p.rays[k].shape == (p.n_rays,)
        assert np.isfinite(p.rays[k]).all()
    pos = np.stack([p.rays[k] for k in ("x", "y", "z")], 1).astype(np.float64)
    assert (pos >= lo).all() and (pos < hi).all()
    d = np.stack([p.rays[k] for k in ("u", "v", "w")], 1).astype(np.float64)
    assert (np.linalg.norm(d, axis=1) > 0.5).all()
    assert (p.rays["E"] >= W.E_MIN_EV * (1 - 1e-6)).all() and (p.rays["E"] <= W.E_MAX_EV * (1 + 1e-6)).all()
    assert (p.rays["wt"] > 0).all()
