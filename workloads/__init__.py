"""Seeded synthetic inputs for the occupancy-grid sampling and compositing path.

This module only *generates data*: analytic Gaussian-blob scene parameters,
camera rays, target images, random occupancy bitfields and random packed
sample sets.  It holds none of the method's arithmetic (no marching, no
transmittance, no compositing, no grid update, no inverse-CDF sampling), so
both the CPU oracle and the CUDA path may consume it.

Every generator is deterministic given its arguments (numpy PCG64 seeded from
``SEED_BASE + config_id`` plus a stream number).  Arrays are C-contiguous
float32 / int64 / uint32 in the layouts the C ABI uses:
rays ``[n][3]``, blob centres ``[B][3]``, blob colours ``[B][3]``, packed
samples as CSR ``offsets[n+1]`` plus flat per-sample arrays.

The recipes stand in for the paper's datasets (NeRF-Synthetic style bounded
scenes with much empty space, Sec. 4.3 / Fig. 5 discussion): isotropic
Gaussian density blobs with peak density 50 inside the scene box, viewed from
cameras on a sphere of radius 4.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 0x5EED

# Lattice step used by every bounded config: 1024 steps span the diagonal of
# the 3-unit scene box (the marching step size is a hyper-parameter of the
# occupancy-grid estimator, Appendix B "Hyper-parameter Space").
STEP_BOUNDED = math.sqrt(3.0) * 3.0 / 1024.0


def rng(config_id: int, stream: int = 0) -> np.random.Generator:
    """PCG64 generator for ``config_id`` / ``stream``."""
    return np.random.Generator(np.random.PCG64([SEED_BASE + int(config_id), int(stream)]))


@dataclasses.dataclass
class Blobs:
    """Analytic density field: ``sigma(x) = sum_b peak_b exp(-|x-mu_b|^2 / (2 std_b^2))``."""

    mu: np.ndarray    # [B][3] float32
    std: np.ndarray   # [B] float32
    peak: np.ndarray  # [B] float32
    rgb: np.ndarray   # [B][3] float32

    @property
    def n(self) -> int:
        return int(self.std.shape[0])


def blob_field(n_blobs: int, config_id: int, centre_half: float = 1.0,
               std_lo: float = 0.1, std_hi: float = 0.3, peak: float = 50.0) -> Blobs:
    """``n_blobs`` isotropic Gaussian blobs: centres uniform in ``[-centre_half, centre_half]^3``,
    std uniform in ``[std_lo, std_hi]``, constant peak density, colours uniform in ``[0,1]^3``."""
    g = rng(config_id, 1)
    mu = g.uniform(-centre_half, centre_half, size=(n_blobs, 3))
    std = g.uniform(std_lo, std_hi, size=(n_blobs,))
    rgb = g.uniform(0.0, 1.0, size=(n_blobs, 3))
    return Blobs(mu=mu.astype(np.float32), std=std.astype(np.float32),
                 peak=np.full((n_blobs,), peak, np.float32), rgb=rgb.astype(np.float32))


def _normalise(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def sphere_rays(n_rays: int, config_id: int, radius: float = 4.0, box_half: float = 1.5):
    """Origins uniform on a sphere of ``radius``; each direction points at a
    uniform random point of the box ``[-box_half, box_half]^3``.  Directions are
    unit length in float64 before the cast to float32."""
    g = rng(config_id, 2)
    o = _normalise(g.standard_normal((n_rays, 3))) * radius
    p = g.uniform(-box_half, box_half, size=(n_rays, 3))
    d = _normalise(p - o)
    return o.astype(np.float32), d.astype(np.float32)


def look_at(cam_pos: np.ndarray, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Camera-to-world rotation (columns right, up, backward) for a camera looking at ``target``."""
    f = _normalise(np.asarray(target, np.float64) - cam_pos)
    upv = np.asarray(up, np.float64)
    if abs(float(np.dot(f, upv))) > 0.999:
        upv = np.array([0.0, 1.0, 0.0])
    r = _normalise(np.cross(f, upv))
    u = np.cross(r, f)
    return np.stack([r, u, -f], axis=1)


def pinhole_rays(cam_pos: np.ndarray, width: int, height: int, focal: float,
                 pix_i: np.ndarray | None = None, pix_j: np.ndarray | None = None):
    """Rays through pixel centres of a pinhole camera at ``cam_pos`` looking at the
    origin.  With ``pix_i``/``pix_j`` given, only those pixels (rows/cols)."""
    cam_pos = np.asarray(cam_pos, np.float64)
    if pix_i is None:
        jj, ii = np.meshgrid(np.arange(width), np.arange(height))
        pix_i, pix_j = ii.reshape(-1), jj.reshape(-1)
    x = (pix_j + 0.5 - width * 0.5) / focal
    y = -(pix_i + 0.5 - height * 0.5) / focal
    dirs_cam = np.stack([x, y, -np.ones_like(x)], axis=-1)
    R = look_at(cam_pos)
    d = _normalise(dirs_cam @ R.T)
    o = np.broadcast_to(cam_pos, d.shape)
    return np.ascontiguousarray(o, dtype=np.float32), np.ascontiguousarray(d, dtype=np.float32)


def camera_position(config_id: int, radius: float = 4.0) -> np.ndarray:
    """One seeded camera position on the sphere of ``radius``."""
    g = rng(config_id, 3)
    v = _normalise(g.standard_normal(3))
    return v * radius


def fibonacci_cameras(n: int, radius: float = 4.0) -> np.ndarray:
    """``n`` camera centres on a Fibonacci lattice over the sphere of ``radius``."""
    k = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * k / n
    phi = math.pi * (1.0 + math.sqrt(5.0)) * k
    rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], axis=-1) * radius


def multi_camera_rays(n_rays: int, config_id: int, n_cams: int = 100, width: int = 800,
                      height: int = 800, focal: float = 1111.0, radius: float = 4.0):
    """``n_rays`` rays drawn uniformly at random over (camera, pixel) pairs of
    ``n_cams`` Fibonacci-lattice cameras that look at the origin."""
    g = rng(config_id, 4)
    cams = fibonacci_cameras(n_cams, radius)
    cam = g.integers(0, n_cams, size=n_rays)
    pi = g.integers(0, height, size=n_rays)
    pj = g.integers(0, width, size=n_rays)
    o = np.empty((n_rays, 3), np.float32)
    d = np.empty((n_rays, 3), np.float32)
    for c in range(n_cams):
        m = cam == c
        if not m.any():
            continue
        oc, dc = pinhole_rays(cams[c], width, height, focal, pi[m], pj[m])
        o[m], d[m] = oc, dc
    return o, d


def target_image(n_rays: int, config_id: int) -> np.ndarray:
    """Seeded uniform-noise target colours ``[n][3]`` in [0, 1)."""
    return rng(config_id, 5).uniform(0.0, 1.0, size=(n_rays, 3)).astype(np.float32)


def random_bitfield(n_levels: int, res: int, config_id: int, p_block: float = 0.3,
                    block: int = 8, p_cell: float = 0.7, stream: int = 6) -> np.ndarray:
    """Random occupancy bitfield with spatial structure: a coarse ``res/block``
    mask (probability ``p_block``) refined by per-cell probability ``p_cell``, so
    that empty runs of many cells exist for skipping.  Layout: cell index
    ``level*res^3 + (x*res + y)*res + z``, bit ``idx & 31`` of word ``idx >> 5``."""
    g = rng(config_id, stream)
    nb = max(1, res // block)
    coarse = g.random((n_levels, nb, nb, nb)) < p_block
    fine = np.repeat(np.repeat(np.repeat(coarse, block, 1), block, 2), block, 3)[:, :res, :res, :res]
    if fine.shape[1] < res:
        pad = res - fine.shape[1]
        fine = np.pad(fine, ((0, 0), (0, pad), (0, pad), (0, pad)))
    occ = fine & (g.random((n_levels, res, res, res)) < p_cell)
    return pack_bits(occ.reshape(-1))


def pack_bits(occ: np.ndarray) -> np.ndarray:
    """Pack a flat boolean array (length multiple of 32) into uint32 words, bit i of word w = element 32*w+i."""
    occ = np.asarray(occ, bool).reshape(-1, 32)
    weights = (np.uint64(1) << np.arange(32, dtype=np.uint64))
    return (occ.astype(np.uint64) * weights).sum(axis=1).astype(np.uint32)


def unpack_bits(words: np.ndarray) -> np.ndarray:
    """Inverse of :func:`pack_bits`."""
    w = np.asarray(words, np.uint32).astype(np.uint64)[:, None]
    return ((w >> np.arange(32, dtype=np.uint64)) & np.uint64(1)).astype(bool).reshape(-1)


def random_packed(n_rays: int, config_id: int, max_len: int = 64, p_empty: float = 0.2,
                  sigma_hi: float = 60.0, step: float = STEP_BOUNDED, stream: int = 7,
                  lengths: np.ndarray | None = None):
    """Random packed sample set for compositing tests: per-ray counts (some 0),
    contiguous lattice intervals starting at a random near distance, densities
    in [0, sigma_hi) with many zeros, colours in [0,1)."""
    g = rng(config_id, stream)
    if lengths is None:
        lengths = g.integers(1, max_len + 1, size=n_rays)
        lengths[g.random(n_rays) < p_empty] = 0
    lengths = np.asarray(lengths, np.int64)
    offsets = np.zeros(n_rays + 1, np.int64)
    np.cumsum(lengths, out=offsets[1:])
    S = int(offsets[-1])
    t_near = np.repeat(g.uniform(2.0, 3.0, size=n_rays), lengths)
    k = np.arange(S, dtype=np.int64) - np.repeat(offsets[:-1], lengths)
    t0 = (t_near + k * step).astype(np.float32)
    t1 = (t0.astype(np.float64) + step).astype(np.float32)
    sig = g.uniform(0.0, sigma_hi, size=S)
    sig[g.random(S) < 0.3] = 0.0
    rgb = g.uniform(0.0, 1.0, size=(S, 3))
    ray_ids = np.repeat(np.arange(n_rays, dtype=np.int32), lengths)
    return dict(offsets=offsets, t_starts=t0, t_ends=t1, sigmas=sig.astype(np.float32),
                rgbs=rgb.astype(np.float32), ray_indices=ray_ids)


# --------------------------------------------------------------------------
# Named workloads (sizes of the five evaluation configurations)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class GridSpec:
    aabb_min: tuple
    aabb_max: tuple
    res: int
    n_levels: int

    @property
    def n_cells(self) -> int:
        return self.n_levels * self.res ** 3


@dataclasses.dataclass
class MarchSpec:
    step: float
    max_steps: int
    t_min: float
    t_max: float
    early_stop_eps: float


@dataclasses.dataclass
class Workload:
    name: str
    rays_o: np.ndarray
    rays_d: np.ndarray
    blobs: Blobs
    grid: GridSpec
    march: MarchSpec
    bg: tuple = (1.0, 1.0, 1.0)
    target: np.ndarray | None = None

    @property
    def n_rays(self) -> int:
        return int(self.rays_o.shape[0])


def c1_forward(n_rays: int = 4096) -> Workload:
    """4096 rays from a radius-4 sphere aimed into the box [-1.5,1.5]^3; 8 blobs;
    one 128^3 level; early stop at T < 1e-4; white background."""
    o, d = sphere_rays(n_rays, 1)
    return Workload("sphere4096_grid1x128", o, d, blob_field(8, 1),
                    GridSpec((-1.5, -1.5, -1.5), (1.5, 1.5, 1.5), 128, 1),
                    MarchSpec(STEP_BOUNDED, 1024, 0.0, 1e10, 1e-4))


def c2_image(width: int = 800, height: int = 800, focal: float = 1111.0, view: int = 0) -> Workload:
    """Full 800x800 pinhole image (640,000 rays) of the C1 blob field, camera at
    radius 4 looking at the origin, near plane 2; 4-level cascaded 128^3 grid;
    up to 1024 lattice steps; seeded uniform-noise target for an L2 loss.
    ``view`` > 0 picks another seeded camera on the same sphere (one image per
    GPU when several GPUs each render their own view)."""
    cam = camera_position(2) if view == 0 else camera_position(1000 + view)
    o, d = pinhole_rays(cam, width, height, focal)
    n = o.shape[0]
    return Workload(f"image{width}x{height}_grid4x128", o, d, blob_field(8, 1),
                    GridSpec((-1.5, -1.5, -1.5), (1.5, 1.5, 1.5), 128, 4),
                    MarchSpec(STEP_BOUNDED, 1024, 2.0, 1e10, 1e-4),
                    target=target_image(n, 2 if view == 0 else 1000 + view))


def c3_training(n_rays: int = 262144) -> Workload:
    """262,144 rays drawn at random from 100 cameras on the radius-4 sphere around
    a 64-blob field; 4-level cascaded 128^3 grid; uniform-noise target."""
    o, d = multi_camera_rays(n_rays, 3)
    return Workload(f"batch{n_rays}_blobs64_grid4x128", o, d, blob_field(64, 3),
                    GridSpec((-1.5, -1.5, -1.5), (1.5, 1.5, 1.5), 128, 4),
                    MarchSpec(STEP_BOUNDED, 1024, 2.0, 1e10, 1e-4),
                    target=target_image(n_rays, 3))


def ball_blob_field(n_blobs: int, config_id: int, radius: float = 20.0, std_lo: float = 0.1, std_hi: float = 0.3,
                    peak: float = 50.0) -> Blobs:
    """Blobs for an unbounded scene: centres uniform in a ball of ``radius``
    (r = radius * U^(1/3), uniform direction), std U[std_lo, std_hi] scaled by
    (1 + r/4) so that far blobs stay a few pixels wide, constant peak, colours
    uniform in [0,1]^3."""
    g = rng(config_id, 1)
    r = radius * g.random(n_blobs) ** (1.0 / 3.0)
    mu = _normalise(g.standard_normal((n_blobs, 3))) * r[:, None]
    std = g.uniform(std_lo, std_hi, size=n_blobs) * (1.0 + r / 4.0)
    rgb = g.uniform(0.0, 1.0, size=(n_blobs, 3))
    return Blobs(mu=mu.astype(np.float32), std=std.astype(np.float32), peak=np.full(n_blobs, peak, np.float32),
                 rgb=rgb.astype(np.float32))


def ring_cameras(n_cams: int, radius: float = 4.0, height: float = 0.5) -> np.ndarray:
    """Camera centres evenly spaced on a horizontal circle, all looking at the origin."""
    a = 2.0 * math.pi * np.arange(n_cams) / n_cams
    return np.stack([radius * np.cos(a), np.full(n_cams, height), radius * np.sin(a)], axis=-1)


# Unbounded scenes: lattice of 1024 steps in s in [0, 1], mapped to t in
# [T_NEAR_UNBOUNDED, T_FAR_UNBOUNDED]; the grid covers the contracted cube
# [-2, 2]^3 as 4 cascaded levels around [-0.25, 0.25]^3.
T_NEAR_UNBOUNDED = 0.2
T_FAR_UNBOUNDED = 1000.0


def c5_unbounded(n_cams: int = 16, width: int = 1024, height: int = 256, res: int = 256) -> Workload:
    """16 inward-facing 1024x256 cameras (90 degree horizontal field of view) on
    a radius-4 ring over a 256-blob field spread across radius 20; 4-level
    cascaded res^3 grid over the contracted space; 4,194,304 rays."""
    focal = width / 2.0  # tan(45 deg) = 1
    os_, ds_ = [], []
    for c in ring_cameras(n_cams):
        o, d = pinhole_rays(c, width, height, focal)
        os_.append(o)
        ds_.append(d)
    o, d = np.concatenate(os_), np.concatenate(ds_)
    return Workload(f"unbounded{n_cams}x{width}x{height}_blobs256_grid4x{res}", o, d, ball_blob_field(256, 5),
                    GridSpec((-0.25, -0.25, -0.25), (0.25, 0.25, 0.25), res, 4),
                    MarchSpec(0.0, 1024, T_NEAR_UNBOUNDED, T_FAR_UNBOUNDED, 1e-4),
                    target=target_image(o.shape[0], 5))


def subsample(w: Workload, every: int, offset: int = 0) -> Workload:
    """Every ``every``-th ray of a workload (a bounded sample for CPU timing)."""
    sl = slice(offset, None, every)
    return dataclasses.replace(
        w, name=f"{w.name}_every{every}", rays_o=np.ascontiguousarray(w.rays_o[sl]),
        rays_d=np.ascontiguousarray(w.rays_d[sl]),
        target=None if w.target is None else np.ascontiguousarray(w.target[sl]))
