"""The seeded synthetic workloads match the stated recipe of the five
evaluation configurations (ray counts, camera geometry, field statistics, grid
and lattice settings) and are deterministic.  CPU only."""
import math

import numpy as np

import workloads


def _unit(d):
    return np.allclose(np.linalg.norm(d.astype(np.float64), axis=1), 1.0, atol=1e-5)


def test_sphere_rays_and_blob_field_of_the_forward_config():
    w = workloads.c1_forward()
    assert w.n_rays == 4096 and _unit(w.rays_d)
    assert np.allclose(np.linalg.norm(w.rays_o.astype(np.float64), axis=1), 4.0, atol=1e-5)
    # every ray is aimed at a point of the box, so it enters it
    o, d = w.rays_o.astype(np.float64), w.rays_d.astype(np.float64)
    with np.errstate(divide="ignore"):
        ta, tb = (-1.5 - o) / d, (1.5 - o) / d
    assert (np.minimum(ta, tb).max(1) < np.maximum(ta, tb).min(1)).all()
    b = w.blobs
    assert b.n == 8 and (np.abs(b.mu) <= 1.0).all() and (b.peak == 50.0).all()
    assert (b.std >= 0.1).all() and (b.std <= 0.3).all() and (b.rgb >= 0).all() and (b.rgb <= 1).all()
    assert (w.grid.res, w.grid.n_levels) == (128, 1)
    assert abs(w.march.step - math.sqrt(3) * 3 / 1024) < 1e-12  # 1024 steps span the box diagonal
    assert w.march.max_steps == 1024 and w.march.early_stop_eps == 1e-4 and w.bg == (1.0, 1.0, 1.0)


def test_image_config_is_one_pinhole_camera():
    w = workloads.c2_image()
    assert w.n_rays == 640_000 and _unit(w.rays_d)
    assert (w.rays_o == w.rays_o[0]).all()
    assert abs(np.linalg.norm(w.rays_o[0].astype(np.float64)) - 4.0) < 1e-5
    assert (w.grid.res, w.grid.n_levels) == (128, 4) and w.march.max_steps == 1024
    assert w.target.shape == (640_000, 3) and (w.target >= 0).all() and (w.target < 1).all()
    # the central pixel looks at the origin
    c = w.rays_d[400 * 800 + 400].astype(np.float64)
    assert np.dot(c, -w.rays_o[0] / np.linalg.norm(w.rays_o[0])) > 0.999


def test_training_batch_comes_from_a_hundred_cameras():
    w = workloads.c3_training()
    assert w.n_rays == 262_144 and _unit(w.rays_d)
    cams = np.unique(w.rays_o, axis=0)
    assert 1 < len(cams) <= 100
    assert np.allclose(np.linalg.norm(cams.astype(np.float64), axis=1), 4.0, atol=1e-5)
    assert w.blobs.n == 64 and (w.grid.res, w.grid.n_levels) == (128, 4)


def test_unbounded_config_ring_of_sixteen_cameras():
    w = workloads.c5_unbounded()
    assert w.n_rays == 16 * 1024 * 256 == 4_194_304 and _unit(w.rays_d)
    cams = np.unique(w.rays_o, axis=0).astype(np.float64)
    assert len(cams) == 16
    assert np.allclose(np.hypot(cams[:, 0], cams[:, 2]), 4.0, atol=1e-5) and np.allclose(cams[:, 1], 0.5)
    b = w.blobs
    assert b.n == 256 and np.linalg.norm(b.mu.astype(np.float64), axis=1).max() <= 20.0 + 1e-4
    assert (w.grid.res, w.grid.n_levels) == (256, 4)
    # the outermost level covers the contracted cube [-2, 2]^3
    half = (w.grid.aabb_max[0] - w.grid.aabb_min[0]) / 2 * 2 ** (w.grid.n_levels - 1)
    assert abs(half - 2.0) < 1e-12


def test_generators_are_deterministic():
    a, b = workloads.c1_forward(256), workloads.c1_forward(256)
    assert np.array_equal(a.rays_o, b.rays_o) and np.array_equal(a.rays_d, b.rays_d)
    assert np.array_equal(a.blobs.mu, b.blobs.mu)
    p, q = workloads.random_packed(100, 9), workloads.random_packed(100, 9)
    assert all(np.array_equal(p[k], q[k]) for k in p)
