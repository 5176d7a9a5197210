"""CPU oracle for the occupancy-grid sampling and compositing path (NerfAcc, arXiv 2305.04966).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import this package.  It
wraps the plain C reference in ``oracle.c`` (built with gcc, loaded with
ctypes) behind numpy functions.  It shares no code with the CUDA library and
never imports it.

Precision: the lattice march is FP32 with every operation rounded (the
definition of the packed sample set); compositing and its gradient are FP64;
inverse-CDF sampling is FP32 (bin choices are float decisions taken in the
kernel's precision); the EMA update is FP32 with an FP64 mean.

Pins (``tests/test_oracle_pins.py``): closed-form uniform marching (Sec. 3.1
"Uniform"), geometric single-cell marching, homogeneous-slab transmittance,
Eq. 3 (sum of weights = 1 - T_N), the erf line integral of a Gaussian blob,
finite differences for the gradient, published SplitMix64 outputs, analytic
inversion of piecewise-constant CDFs, the float64 slab clip.  Parity
unpinned: none.  ``tests/test_oracle_mutants.py`` plants one-line mistakes in
copies of this oracle and checks that the pins catch every one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (OpenMP if available)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    for extra in (["-fopenmp"], []):
        cmd = base + extra + [_SRC, "-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, _LIB_PATH)
            return _LIB_PATH
    raise RuntimeError(f"oracle build failed:\n{r.stderr}")


def _P(t):
    return ctypes.POINTER(t)


def load(path: str):
    """ctypes handle on a compiled copy of ``oracle.c`` at ``path``, with the
    signatures of its entry points declared (``lib()`` loads the in-tree
    build; the planted-mistake tests load mutated copies)."""
    L = ctypes.CDLL(path)
    i64, i32, f32, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_uint64
    vp = ctypes.c_void_p
    L.orc_splitmix64_at.restype = u64
    L.orc_splitmix64_at.argtypes = [u64, u64]
    L.orc_march.restype = i32
    L.orc_march.argtypes = [i64, vp, vp, vp, vp, i32, i32, vp, f32, i32, f32, f32, i32, vp, vp,
                            vp, f32, vp, vp, vp, vp, vp, i32]
    L.orc_ray_clip.restype = None
    L.orc_ray_clip.argtypes = [i64, vp, vp, vp, vp, i32, i32, f32, f32, vp, vp, vp]
    L.orc_level_geometry.restype = None
    L.orc_level_geometry.argtypes = [vp, vp, i32, i32, vp]
    L.orc_field_samples.restype = None
    L.orc_field_samples.argtypes = [i64, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp, i32]
    L.orc_field_points.restype = None
    L.orc_field_points.argtypes = [i64, vp, i32, vp, vp, vp, vp, vp, i32]
    L.orc_render_fwd.restype = None
    L.orc_render_fwd.argtypes = [i64, vp, vp, vp, vp, vp, vp, f32, vp, vp, vp, vp, vp, i32]
    L.orc_render_bwd.restype = None
    L.orc_render_bwd.argtypes = [i64, vp, vp, vp, vp, vp, vp, f32, vp, vp, vp, vp, vp, i32]
    L.orc_grid_points.restype = None
    L.orc_grid_points.argtypes = [vp, vp, i32, i32, u64, i64, i32, vp, i32]
    L.orc_update_grid.restype = None
    L.orc_update_grid.argtypes = [i64, vp, vp, f32, f32, f32, vp, vp]
    L.orc_sample_pdf.restype = None
    L.orc_sample_pdf.argtypes = [i64, i32, vp, vp, i32, i32, u64, vp, i32]
    L.orc_march_unbounded.restype = i32
    L.orc_march_unbounded.argtypes = [i64, vp, vp, vp, vp, i32, i32, vp, i32, f32, f32, i32, vp, vp, vp, f32,
                                      vp, vp, vp, vp, vp, i32]
    L.orc_s_to_t.restype = f32
    L.orc_s_to_t.argtypes = [f32, f32, f32]
    L.orc_contract_points.restype = None
    L.orc_contract_points.argtypes = [i64, vp, vp]
    L.orc_uncontract_points.restype = None
    L.orc_uncontract_points.argtypes = [i64, vp, vp]
    L.orc_max_threads.restype = i32
    L.orc_max_threads.argtypes = []
    L.orc_exp_steps_array.restype = None
    L.orc_exp_steps_array.argtypes = [i64, vp, vp]
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = load(_LIB_PATH)
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def max_threads() -> int:
    return int(lib().orc_max_threads())


def _threads(n):
    return max_threads() if n is None else int(n)


def exp_steps(a):
    """The early-stop density's exponential, defined by its steps (Cody-Waite
    reduction, degree-7 Taylor polynomial, FP32; 0 below -86): float32 in,
    float32 out."""
    a = _c(a, np.float32)
    out = np.empty_like(a)
    lib().orc_exp_steps_array(a.size, _ptr(a), _ptr(out))
    return out


def splitmix64_at(seed: int, counter: int) -> int:
    return int(lib().orc_splitmix64_at(seed & (2**64 - 1), counter & (2**64 - 1)))


def level_geometry(aabb_min, aabb_max, res, n_levels):
    """[L][4][3] float32: lmin, lmax, scale, width per level."""
    out = np.zeros((n_levels, 4, 3), np.float32)
    lib().orc_level_geometry(_ptr(_c(aabb_min, np.float32)), _ptr(_c(aabb_max, np.float32)),
                             res, n_levels, _ptr(out))
    return out


def ray_clip(rays_o, rays_d, aabb_min, aabb_max, res, n_levels, t_min, t_max):
    o, d = _c(rays_o, np.float32), _c(rays_d, np.float32)
    n = o.shape[0]
    tn, tf, hit = np.zeros(n, np.float32), np.zeros(n, np.float32), np.zeros(n, np.int32)
    lib().orc_ray_clip(n, _ptr(o), _ptr(d), _ptr(_c(aabb_min, np.float32)),
                       _ptr(_c(aabb_max, np.float32)), res, n_levels, t_min, t_max,
                       _ptr(tn), _ptr(tf), _ptr(hit))
    return tn, tf, hit.astype(bool)


def march(rays_o, rays_d, aabb_min, aabb_max, res, n_levels, bits, step, max_steps, t_min,
          t_max, blobs=None, eps=1e-4, n_threads=None):
    """Dense lattice march.  Returns dict(offsets int64[n+1], ray_indices int32[S],
    t_starts float32[S], t_ends float32[S]).  ``blobs`` (a workloads.Blobs) enables
    early termination at T < eps with the FP32 field."""
    o, d = _c(rays_o, np.float32), _c(rays_d, np.float32)
    n = o.shape[0]
    bits = _c(bits, np.uint32)
    amin, amax = _c(aabb_min, np.float32), _c(aabb_max, np.float32)
    if blobs is not None:
        nb, mu, sd, pk = blobs.n, _c(blobs.mu, np.float32), _c(blobs.std, np.float32), _c(blobs.peak, np.float32)
    else:
        nb, mu, sd, pk = 0, None, None, None
    counts = np.zeros(n, np.int64)
    nt = _threads(n_threads)
    L = lib()
    args = (n, _ptr(o), _ptr(d), _ptr(amin), _ptr(amax), res, n_levels, _ptr(bits), step, max_steps,
            t_min, t_max, nb, _ptr(mu), _ptr(sd), _ptr(pk), eps)
    if L.orc_march(*args, _ptr(counts), None, None, None, None, nt) != 0:
        raise ValueError("orc_march: invalid arguments")
    offsets = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=offsets[1:])
    S = int(offsets[-1])
    ri, t0, t1 = np.zeros(S, np.int32), np.zeros(S, np.float32), np.zeros(S, np.float32)
    counts2 = np.zeros(n, np.int64)
    L.orc_march(*args, _ptr(counts2), _ptr(offsets), _ptr(ri), _ptr(t0), _ptr(t1), nt)
    assert np.array_equal(counts, counts2)
    return dict(offsets=offsets, ray_indices=ri, t_starts=t0, t_ends=t1)


def s_to_t(s, t_near, t_far):
    """Disparity-linear s -> t (FP32 definition of the unbounded lattice)."""
    L = lib()
    return np.array([L.orc_s_to_t(float(v), float(t_near), float(t_far)) for v in np.ravel(s)], np.float32)


def contract(xyz):
    """L-infinity contraction of points [n][3] into [-2, 2]^3 (FP32 definition)."""
    x = _c(xyz, np.float32).reshape(-1, 3)
    out = np.zeros_like(x)
    lib().orc_contract_points(x.shape[0], _ptr(x), _ptr(out))
    return out


def march_unbounded(rays_o, rays_d, aabb_min, aabb_max, res, n_levels, bits, K, t_near, t_far, blobs=None,
                    eps=1e-4, n_threads=None):
    """Unbounded-scene march: K uniform steps in s mapped to t by the
    disparity-linear bijection, occupancy of the contracted midpoint.  Same
    return value as :func:`march`."""
    o, d = _c(rays_o, np.float32), _c(rays_d, np.float32)
    n = o.shape[0]
    bits = _c(bits, np.uint32)
    amin, amax = _c(aabb_min, np.float32), _c(aabb_max, np.float32)
    if blobs is not None:
        nb, mu, sd, pk = blobs.n, _c(blobs.mu, np.float32), _c(blobs.std, np.float32), _c(blobs.peak, np.float32)
    else:
        nb, mu, sd, pk = 0, None, None, None
    counts = np.zeros(n, np.int64)
    nt = _threads(n_threads)
    L = lib()
    args = (n, _ptr(o), _ptr(d), _ptr(amin), _ptr(amax), res, n_levels, _ptr(bits), K, t_near, t_far, nb, _ptr(mu),
            _ptr(sd), _ptr(pk), eps)
    if L.orc_march_unbounded(*args, _ptr(counts), None, None, None, None, nt) != 0:
        raise ValueError("orc_march_unbounded: invalid arguments")
    offsets = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=offsets[1:])
    S = int(offsets[-1])
    ri, t0, t1 = np.zeros(S, np.int32), np.zeros(S, np.float32), np.zeros(S, np.float32)
    counts2 = np.zeros(n, np.int64)
    L.orc_march_unbounded(*args, _ptr(counts2), _ptr(offsets), _ptr(ri), _ptr(t0), _ptr(t1), nt)
    assert np.array_equal(counts, counts2)
    return dict(offsets=offsets, ray_indices=ri, t_starts=t0, t_ends=t1)


def uncontract(c):
    """Inverse of :func:`contract` in FP64: y with m' = max|y_a| > 1 maps back to
    y * (m / m') with m = 1 / (2 - m') (m' < 2)."""
    y = np.asarray(c, np.float64).reshape(-1, 3)
    mp = np.abs(y).max(1)
    out = y.copy()
    far = mp > 1.0
    m = 1.0 / np.maximum(2.0 - mp[far], 1e-300)
    out[far] = y[far] * (m / mp[far])[:, None]
    return out


def uncontract32(c):
    """Inverse contraction in FP32 (the definition the grid update uses):
    x = c * (inv / m'), inv = 1 / (2 - min(m', 2 - 2^-23)) for m' = max|c_a| > 1."""
    y = _c(c, np.float32).reshape(-1, 3)
    out = np.zeros_like(y)
    lib().orc_uncontract_points(y.shape[0], _ptr(y), _ptr(out))
    return out


def density_grid_contracted(grid_spec, blobs, thresh=0.01, n_threads=None):
    """Occupancy bits of a grid over the contracted space: cell centres (in
    contracted coordinates) mapped back to the scene (FP32), FP64 field > thresh."""
    pts = grid_points(grid_spec.aabb_min, grid_spec.aabb_max, grid_spec.res, grid_spec.n_levels, jitter=False,
                      n_threads=n_threads)
    sig = field_points(uncontract32(pts), blobs, n_threads)
    occ = sig > thresh
    w = occ.reshape(-1, 32).astype(np.uint64) * (np.uint64(1) << np.arange(32, dtype=np.uint64))
    return w.sum(1).astype(np.uint32), sig


def field_samples(rays_o, rays_d, ray_indices, t_starts, t_ends, blobs, n_threads=None):
    """FP64 density [S] and colour [S][3] of the blob field at interval midpoints."""
    ri = _c(ray_indices, np.int32)
    S = ri.shape[0]
    sig, rgb = np.zeros(S, np.float64), np.zeros((S, 3), np.float64)
    lib().orc_field_samples(S, _ptr(_c(rays_o, np.float32)), _ptr(_c(rays_d, np.float32)), _ptr(ri),
                            _ptr(_c(t_starts, np.float32)), _ptr(_c(t_ends, np.float32)), blobs.n,
                            _ptr(_c(blobs.mu, np.float32)), _ptr(_c(blobs.std, np.float32)),
                            _ptr(_c(blobs.peak, np.float32)), _ptr(_c(blobs.rgb, np.float32)),
                            _ptr(sig), _ptr(rgb), _threads(n_threads))
    return sig, rgb


def field_points(xyz, blobs, n_threads=None):
    """FP64 density of the blob field at points [n][3]."""
    xyz = _c(xyz, np.float32).reshape(-1, 3)
    out = np.zeros(xyz.shape[0], np.float64)
    lib().orc_field_points(xyz.shape[0], _ptr(xyz), blobs.n, _ptr(_c(blobs.mu, np.float32)),
                           _ptr(_c(blobs.std, np.float32)), _ptr(_c(blobs.peak, np.float32)),
                           _ptr(_c(blobs.rgb, np.float32)), _ptr(out), _threads(n_threads))
    return out


def render_fwd(offsets, t_starts, t_ends, sigmas, rgbs, bg=(1.0, 1.0, 1.0), eps=0.0, n_threads=None):
    """FP64 compositing.  Returns dict(rgb [n][3], opacity [n], depth [n], trans [n], weights [S])."""
    off = _c(offsets, np.int64)
    n = off.shape[0] - 1
    S = int(off[-1])
    rgb, op, dep, tr = np.zeros((n, 3)), np.zeros(n), np.zeros(n), np.zeros(n)
    w = np.zeros(S)
    lib().orc_render_fwd(n, _ptr(off), _ptr(_c(t_starts, np.float32)), _ptr(_c(t_ends, np.float32)),
                         _ptr(_c(sigmas, np.float64)), _ptr(_c(rgbs, np.float64)),
                         _ptr(_c(bg, np.float64)), eps, _ptr(rgb), _ptr(op), _ptr(dep), _ptr(tr),
                         _ptr(w), _threads(n_threads))
    return dict(rgb=rgb, opacity=op, depth=dep, trans=tr, weights=w)


def render_bwd(offsets, t_starts, t_ends, sigmas, rgbs, g_rgb, g_opacity, g_depth,
               bg=(1.0, 1.0, 1.0), eps=0.0, n_threads=None):
    """FP64 gradient of :func:`render_fwd`.  Returns (g_sigmas [S], g_rgbs [S][3])."""
    off = _c(offsets, np.int64)
    n = off.shape[0] - 1
    S = int(off[-1])
    gs, gr = np.zeros(S), np.zeros((S, 3))
    lib().orc_render_bwd(n, _ptr(off), _ptr(_c(t_starts, np.float32)), _ptr(_c(t_ends, np.float32)),
                         _ptr(_c(sigmas, np.float64)), _ptr(_c(rgbs, np.float64)),
                         _ptr(_c(bg, np.float64)), eps, _ptr(_c(g_rgb, np.float64)),
                         _ptr(_c(g_opacity, np.float64)), _ptr(_c(g_depth, np.float64)),
                         _ptr(gs), _ptr(gr), _threads(n_threads))
    return gs, gr


def grid_points(aabb_min, aabb_max, res, n_levels, seed=0, step=0, jitter=True, n_threads=None):
    """Cell sample points [n_levels*res^3][3] float32 (centres if not jitter)."""
    n = n_levels * res ** 3
    out = np.zeros((n, 3), np.float32)
    lib().orc_grid_points(_ptr(_c(aabb_min, np.float32)), _ptr(_c(aabb_max, np.float32)), res,
                          n_levels, seed & (2**64 - 1), step, int(bool(jitter)), _ptr(out),
                          _threads(n_threads))
    return out


def update_grid(ema, density, decay, thresh_frac, thresh_abs=0.0):
    """EMA update + threshold.  Returns (new ema float32, bits uint32, mean float64); input not modified."""
    e = np.array(ema, dtype=np.float32, copy=True)
    den = _c(density, np.float32)
    n = e.shape[0]
    bits = np.zeros((n + 31) // 32, np.uint32)
    mean = ctypes.c_double(0.0)
    lib().orc_update_grid(n, _ptr(e), _ptr(den), decay, thresh_frac, thresh_abs, _ptr(bits),
                          ctypes.cast(ctypes.pointer(mean), ctypes.c_void_p))
    return e, bits, mean.value


def sample_pdf(edges, weights, n_out, stratified=False, seed=0, n_threads=None):
    """Inverse-CDF resampling.  edges [n][nb+1], weights [n][nb] -> [n][n_out+1] float32."""
    e, w = _c(edges, np.float32), _c(weights, np.float32)
    n, nb = w.shape
    out = np.zeros((n, n_out + 1), np.float32)
    lib().orc_sample_pdf(n, nb, _ptr(e), _ptr(w), n_out, int(bool(stratified)), seed & (2**64 - 1),
                         _ptr(out), _threads(n_threads))
    return out


def density_grid(grid_spec, blobs, thresh=0.01, n_threads=None):
    """Occupancy bits of ``grid_spec`` where the FP64 field at the cell centre exceeds ``thresh``,
    plus the FP32 centre densities (the initial EMA state)."""
    pts = grid_points(grid_spec.aabb_min, grid_spec.aabb_max, grid_spec.res, grid_spec.n_levels,
                      jitter=False, n_threads=n_threads)
    sig = field_points(pts, blobs, n_threads=n_threads)
    occ = sig > thresh
    words = occ.reshape(-1, 32).astype(np.uint64) << np.arange(32, dtype=np.uint64)
    return words.sum(axis=1).astype(np.uint32), sig.astype(np.float32)


from . import proposal  # noqa: E402  (density-proposal network oracle)
from . import grid_variants  # noqa: E402  (estimator-update variants)
