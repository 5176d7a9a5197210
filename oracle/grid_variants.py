"""Oracle of the estimator-update variants (TEST INFRASTRUCTURE ONLY).

* Dynamic scenes (Sec. 4.3 "Dynamic NeRFs"): one occupancy grid for all frames
  marks the maximum occupancy over the timestamps -- the EMA update of
  ``oracle.update_grid`` fed with the per-cell maximum over the frames.
* Gradient-descent update (the Plenoxels variant named in Sec. 3.1 "Spatial
  Skipping"): the grid holds a density per cell; a sample reads the density
  of the cell of its midpoint (the lattice march's FP32 definition of level
  and cell); the adjoint adds each sample's dL/dsigma into its cell; an SGD
  step clamps at 0 and re-binarises at a threshold.

numpy only; shares no code with the CUDA library.  Pins in
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import numpy as np


def sample_cells(rays_o, rays_d, ray_indices, t0, t1, geom, res) -> np.ndarray:
    """Flat cell index of each sample's midpoint (-1 outside every level).
    ``geom`` = ``oracle.level_geometry(...)``: [L][lmin, lmax, scale, width][3]
    float32.  Every operation is an individually rounded float32 operation:
    tm = (t0 + t1) * 0.5, x = o + d * tm, level = the finest whose closed box
    holds x, cell = clamp(floor((x - lmin) * scale), 0, res - 1)."""
    f = np.float32
    o = np.asarray(rays_o, f)[ray_indices]
    d = np.asarray(rays_d, f)[ray_indices]
    tm = ((np.asarray(t0, f) + np.asarray(t1, f)).astype(f) * f(0.5)).astype(f)
    x = (o + (d * tm[:, None]).astype(f)).astype(f)
    L = geom.shape[0]
    level = np.full(len(tm), -1, np.int64)
    for l in range(L - 1, -1, -1):  # the finest level wins: visit it last
        inside = np.all((x >= geom[l, 0]) & (x <= geom[l, 1]), axis=1)
        level[inside] = l
    cells = np.full(len(tm), -1, np.int64)
    ok = level >= 0
    lm, sc = geom[level[ok], 0], geom[level[ok], 2]
    u = ((x[ok] - lm).astype(f) * sc).astype(f)
    ic = np.clip(np.floor(u).astype(np.int64), 0, res - 1)
    cells[ok] = level[ok] * res ** 3 + (ic[:, 0] * res + ic[:, 1]) * res + ic[:, 2]
    return cells


def density_lookup(density, cells) -> np.ndarray:
    d = np.asarray(density, np.float32)
    out = np.zeros(len(cells), np.float32)
    ok = cells >= 0
    out[ok] = d[cells[ok]]
    return out


def density_backward(g_sigma, cells, n_cells) -> np.ndarray:
    g = np.zeros(n_cells, np.float64)
    ok = cells >= 0
    np.add.at(g, cells[ok], np.asarray(g_sigma, np.float64)[ok])
    return g


def sgd_step(density, g_density, lr, thresh):
    """density <- max(density - lr g, 0) (float32, rounded in this order);
    returns (density, occupancy bits as booleans)."""
    f = np.float32
    d = np.maximum((np.asarray(density, f) - (f(lr) * np.asarray(g_density, f)).astype(f)).astype(f), f(0))
    return d, d > f(thresh)


def frames_max(densities) -> np.ndarray:
    return np.max(np.asarray(densities, np.float32), axis=0)
