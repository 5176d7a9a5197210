"""PyTorch-facing binding of the C ABI (argument marshalling only).

Every function here checks tensor placement / dtype / shape, allocates the
output tensors, and calls the corresponding ``nacc_*`` entry point on the
current CUDA stream.  All arithmetic of the path runs in the CUDA library;
there is no CPU fallback.  Names follow Algorithm 1 of NerfAcc
(arXiv 2305.04966): ``march_grid`` is its ``sampling`` with an occupancy-grid
estimator, ``render`` its differentiable ``rendering``, ``update_grid`` its
``estimator.update_every_n_steps``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math

import torch

from . import _abi

_F32, _I32, _I64 = torch.float32, torch.int32, torch.int64


def _stream(dev: torch.device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


_EMPTY = {}


def _ptr(t):
    """Device pointer of ``t``; a zero-element tensor maps to a small valid
    buffer so that the ABI's non-NULL checks hold (nothing is read from it)."""
    if t is None:
        return None
    if t.numel() == 0:
        key = t.device
        if key not in _EMPTY:
            _EMPTY[key] = torch.zeros(16, dtype=torch.float32, device=t.device)
        return ctypes.c_void_p(_EMPTY[key].data_ptr())
    return ctypes.c_void_p(t.data_ptr())


def _check(t, name, dtype, dev=None, shape=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (no CPU path exists)")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dev is not None and t.device != dev:
        raise ValueError(f"{name} is on {t.device}, expected {dev}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


def _scratch(nbytes: int, dev) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)


# ---------------------------------------------------------------------------
# occupancy grid
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class OccupancyGrid:
    """Cascaded occupancy grid: ``n_levels`` levels of ``res^3`` cells; level l
    covers the level-0 box scaled by 2^l about its centre.  ``bits`` packs one
    occupancy bit per cell (int32 words, bit c%32 of word c//32); ``ema`` is the
    running density estimate the update refreshes (Eq. 4)."""

    aabb_min: tuple
    aabb_max: tuple
    res: int
    n_levels: int
    bits: torch.Tensor  # int32 [n_cells/32]
    ema: torch.Tensor | None = None  # float32 [n_cells]

    @property
    def n_cells(self) -> int:
        return self.n_levels * self.res ** 3

    @classmethod
    def empty(cls, aabb_min, aabb_max, res, n_levels, device="cuda"):
        n = n_levels * res ** 3
        return cls(tuple(map(float, aabb_min)), tuple(map(float, aabb_max)), int(res), int(n_levels),
                   torch.zeros(n // 32, dtype=_I32, device=device),
                   torch.zeros(n, dtype=_F32, device=device))

    def state_dict(self) -> dict:
        """The estimator's state for a training checkpoint (the update runs every
        few steps and carries the EMA across them): geometry, bits, EMA; copies."""
        return {"aabb_min": [float(v) for v in self.aabb_min], "aabb_max": [float(v) for v in self.aabb_max],
                "res": int(self.res), "n_levels": int(self.n_levels), "bits": self.bits.detach().clone(),
                "ema": None if self.ema is None else self.ema.detach().clone()}

    @classmethod
    def from_state_dict(cls, state: dict, device=None) -> "OccupancyGrid":
        """Rebuild a grid saved by :meth:`state_dict` (on ``device``, default the
        device the tensors were saved on); checks the sizes against the geometry."""
        res, levels = int(state["res"]), int(state["n_levels"])
        n = levels * res ** 3
        bits, ema = state["bits"], state.get("ema")
        if res < 1 or levels < 1 or n % 32:
            raise ValueError(f"grid of {levels} levels of {res}^3 cells cannot be bit-packed")
        if bits.dtype != _I32 or tuple(bits.shape) != (n // 32,):
            raise ValueError(f"bits must be int32 [{n // 32}], got {bits.dtype} {tuple(bits.shape)}")
        if ema is not None and (ema.dtype != _F32 or tuple(ema.shape) != (n,)):
            raise ValueError(f"ema must be float32 [{n}], got {ema.dtype} {tuple(ema.shape)}")
        dev = bits.device if device is None else torch.device(device)
        return cls(tuple(float(v) for v in state["aabb_min"]), tuple(float(v) for v in state["aabb_max"]), res,
                   levels, bits.to(dev).contiguous().clone(),
                   None if ema is None else ema.to(dev).contiguous().clone())

    def c_struct(self) -> _abi.Grid:
        g = _abi.Grid()
        g.aabb_min[:] = [float(v) for v in self.aabb_min]
        g.aabb_max[:] = [float(v) for v in self.aabb_max]
        g.res = int(self.res)
        g.n_levels = int(self.n_levels)
        g.bits = _ptr(self.bits)
        return g


@dataclasses.dataclass
class BlobField:
    """Analytic density field sum_b peak_b exp(-|x-mu_b|^2/(2 std_b^2)) (harness stand-in
    for the radiance field); tensors on the device."""

    mu: torch.Tensor    # [B][3]
    std: torch.Tensor   # [B]
    peak: torch.Tensor  # [B]
    rgb: torch.Tensor   # [B][3]

    @classmethod
    def from_numpy(cls, blobs, device="cuda"):
        t = lambda a: torch.as_tensor(a, dtype=_F32).contiguous().to(device)
        return cls(t(blobs.mu), t(blobs.std), t(blobs.peak), t(blobs.rgb))

    @property
    def n(self) -> int:
        return int(self.std.shape[0])

    def c_struct(self) -> _abi.BlobField:
        f = _abi.BlobField()
        f.n_blobs = self.n
        f.mu, f.std, f.peak, f.rgb = _ptr(self.mu), _ptr(self.std), _ptr(self.peak), _ptr(self.rgb)
        return f


# ---------------------------------------------------------------------------
# sampling (Algorithm 1 "sampling"; Sec. 4.2 packed intervals)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class PackedSamples:
    """Packed intervals: sample s = [t_starts[s], t_ends[s]] on ray ray_indices[s];
    ray r owns samples offsets[r]:offsets[r+1].  Sample arrays have ``capacity``
    entries; the first ``n_samples`` are valid."""

    offsets: torch.Tensor      # int64 [n_rays+1]
    ray_indices: torch.Tensor | None  # int32 [capacity]
    t_starts: torch.Tensor     # float32 [capacity]
    t_ends: torch.Tensor       # float32 [capacity]
    n_samples_dev: torch.Tensor  # int64 [1] on the device

    @property
    def capacity(self) -> int:
        return int(self.t_starts.shape[0])

    def n_samples(self) -> int:
        """Total sample count (synchronises)."""
        return int(self.n_samples_dev.item())

    def trimmed(self) -> "PackedSamples":
        n = self.n_samples()
        return PackedSamples(self.offsets, None if self.ray_indices is None else self.ray_indices[:n],
                             self.t_starts[:n], self.t_ends[:n], self.n_samples_dev)


class MarchBuffers:
    """Reusable device buffers for :func:`march_grid` (no allocation per call,
    capture-safe when ``capacity >= n_rays*max_steps``)."""

    def __init__(self, n_rays: int, capacity: int, device="cuda", with_ray_indices: bool = True):
        dev = torch.device(device)
        self.n_rays = int(n_rays)
        self.packed = PackedSamples(
            torch.empty(n_rays + 1, dtype=_I64, device=dev),
            torch.empty(capacity, dtype=_I32, device=dev) if with_ray_indices else None,
            torch.empty(capacity, dtype=_F32, device=dev),
            torch.empty(capacity, dtype=_F32, device=dev),
            torch.zeros(1, dtype=_I64, device=dev))
        self.scratch = _scratch(_abi.load().nacc_march_scratch_bytes(n_rays), dev)


def march_grid(grid: OccupancyGrid, rays_o: torch.Tensor, rays_d: torch.Tensor, step: float,
               max_steps: int = 1024, t_min: float = 0.0, t_max: float = 1e10,
               early_stop_eps: float = 1e-4, field: BlobField | None = None,
               capacity: int | None = None, buffers: MarchBuffers | None = None,
               with_ray_indices: bool = True, exact_stops: bool = False) -> PackedSamples:
    """Occupancy-grid lattice march into packed samples (``nacc_march_grid``).

    With ``field`` given, samples are filtered at T < early_stop_eps while
    marching (Sec. 4.2 "No Gradient Filtering"); ``exact_stops`` takes every
    such decision in the exact arithmetic (same result, slower: validation).
    Without ``buffers``, a capacity is chosen (worst case when it is small,
    else a guess that is grown on NACC_ERR_CAPACITY)."""
    dev = rays_o.device
    _check(rays_o, "rays_o", _F32, dev)
    n = int(rays_o.shape[0])
    _check(rays_d, "rays_d", _F32, dev, (n, 3))
    if rays_o.dim() != 2 or rays_o.shape[1] != 3:
        raise ValueError("rays_o must be [n][3]")
    _check(grid.bits, "grid.bits", _I32, dev, (grid.n_cells // 32,))
    params = _abi.MarchParams(float(step), int(max_steps), float(t_min), float(t_max),
                              float(early_stop_eps), int(bool(exact_stops)))
    fs = field.c_struct() if field is not None else None
    worst = n * int(max_steps)
    while True:
        if buffers is None:
            cap = capacity if capacity is not None else (worst if worst * 12 <= (1 << 31) else max(n * 64, 1 << 20))
            buf = MarchBuffers(n, cap, dev, with_ray_indices)
        else:
            buf = buffers
            if buf.n_rays != n:
                raise ValueError("buffers were made for a different ray count")
        pk = buf.packed
        out = _abi.Packed(_ptr(pk.offsets), _ptr(pk.ray_indices), _ptr(pk.t_starts), _ptr(pk.t_ends),
                          pk.capacity, _ptr(pk.n_samples_dev))
        rc = _abi.call("nacc_march_grid", ctypes.byref(grid.c_struct()), _ptr(rays_o), _ptr(rays_d), n,
                       ctypes.byref(params), ctypes.byref(fs) if fs is not None else None,
                       ctypes.byref(out), _ptr(buf.scratch), buf.scratch.numel(), _stream(dev))
        if rc == _abi.NACC_OK:
            return pk
        if buffers is not None or capacity is not None:
            raise _abi.NaccError("nacc_march_grid", rc, "capacity too small")
        capacity = int(pk.n_samples_dev.item())


# ---------------------------------------------------------------------------
# rendering (Algorithm 1 "rendering"; Eq. 2)
# ---------------------------------------------------------------------------

def march_unbounded(grid: OccupancyGrid, rays_o: torch.Tensor, rays_d: torch.Tensor, max_steps: int = 1024,
                    t_near: float = 0.2, t_far: float = 1000.0, early_stop_eps: float = 1e-4,
                    field: BlobField | None = None, capacity: int | None = None,
                    buffers: MarchBuffers | None = None, with_ray_indices: bool = True,
                    exact_stops: bool = False) -> PackedSamples:
    """Unbounded-scene march (``nacc_march_unbounded``): max_steps uniform
    steps in s mapped to [t_near, t_far] by the disparity-linear bijection,
    occupancy of the contracted midpoint; ``exact_stops`` as in
    ``march_grid``."""
    dev = rays_o.device
    n = int(rays_o.shape[0])
    _check(rays_o, "rays_o", _F32, dev, (n, 3))
    _check(rays_d, "rays_d", _F32, dev, (n, 3))
    _check(grid.bits, "grid.bits", _I32, dev, (grid.n_cells // 32,))
    params = _abi.MarchParams(0.0, int(max_steps), float(t_near), float(t_far), float(early_stop_eps),
                              int(bool(exact_stops)))
    fs = field.c_struct() if field is not None else None
    worst = n * int(max_steps)
    scratch = _scratch(_abi.load().nacc_march_unbounded_scratch_bytes(n, int(max_steps)), dev)
    while True:
        if buffers is None:
            cap = capacity if capacity is not None else (worst if worst * 12 <= (1 << 31) else max(n * 64, 1 << 20))
            buf = MarchBuffers(n, cap, dev, with_ray_indices)
        else:
            buf = buffers
        pk = buf.packed
        out = _abi.Packed(_ptr(pk.offsets), _ptr(pk.ray_indices), _ptr(pk.t_starts), _ptr(pk.t_ends),
                          pk.capacity, _ptr(pk.n_samples_dev))
        rc = _abi.call("nacc_march_unbounded", ctypes.byref(grid.c_struct()), _ptr(rays_o), _ptr(rays_d), n,
                       ctypes.byref(params), ctypes.byref(fs) if fs is not None else None, ctypes.byref(out),
                       _ptr(scratch), scratch.numel(), _stream(dev))
        if rc == _abi.NACC_OK:
            return pk
        if buffers is not None or capacity is not None:
            raise _abi.NaccError("nacc_march_unbounded", rc, "capacity too small")
        capacity = int(pk.n_samples_dev.item())


def uncontract_points(c: torch.Tensor, out=None) -> torch.Tensor:
    """Scene points of contracted points [n][3] (``nacc_uncontract_points``)."""
    dev = c.device
    n = int(c.shape[0])
    _check(c, "c", _F32, dev, (n, 3))
    x = out if out is not None else torch.empty_like(c)
    _check(x, "out", _F32, dev, (n, 3))
    _abi.call("nacc_uncontract_points", n, _ptr(c), _ptr(x), _stream(dev))
    return x


def density_grid_unbounded(grid: OccupancyGrid, field: BlobField, thresh: float = 0.01):
    """Initialise a grid over the contracted space from the field at the scene
    points of the cell centres (bits = sigma > thresh)."""
    pts = uncontract_points(grid_points(grid, jitter=False))
    dens = field_points(field, pts)
    update_grid(grid, dens, decay=0.0, thresh_frac=0.0, thresh_abs=thresh)
    return grid


def _bg(bg):
    return (ctypes.c_float * 3)(*[float(v) for v in bg])


def render_ckpt_buffer(n_rays: int, device) -> torch.Tensor:
    """Device buffer for the per-ray checkpoint records of :func:`render_fwd` /
    :func:`render_bwd` (16 words per ray)."""
    words = int(_abi.load().nacc_render_ckpt_bytes(int(n_rays))) // 4
    return torch.empty(words, dtype=_F32, device=device)


def render_fwd(offsets, t_starts, t_ends, sigmas, rgbs, bg=(1.0, 1.0, 1.0), early_stop_eps=0.0,
               want_weights=False, ckpt=None):
    """Composite packed samples.  Returns (rgb [n][3], opacity [n], depth [n], trans [n],
    weights [S] or None).  With ``ckpt`` (from :func:`render_ckpt_buffer`) the pass
    also writes the per-ray records that let :func:`render_bwd` skip its first sweep."""
    dev = offsets.device
    _check(offsets, "offsets", _I64, dev)
    n = int(offsets.shape[0]) - 1
    cap = int(t_starts.shape[0])
    _check(t_starts, "t_starts", _F32, dev)
    _check(t_ends, "t_ends", _F32, dev, (cap,))
    _check(sigmas, "sigmas", _F32, dev)
    _check(rgbs, "rgbs", _F32, dev)
    if sigmas.shape[0] > cap or rgbs.shape[0] != sigmas.shape[0] or rgbs.dim() != 2 or rgbs.shape[1] != 3:
        raise ValueError("sigmas [S] / rgbs [S][3] must match the sample arrays")
    rgb = torch.empty((n, 3), dtype=_F32, device=dev)
    op = torch.empty(n, dtype=_F32, device=dev)
    dep = torch.empty(n, dtype=_F32, device=dev)
    tr = torch.empty(n, dtype=_F32, device=dev)
    w = torch.empty(sigmas.shape[0], dtype=_F32, device=dev) if want_weights else None
    if ckpt is None:
        _abi.call("nacc_render_fwd", n, _ptr(offsets), _ptr(t_starts), _ptr(t_ends), _ptr(sigmas), _ptr(rgbs),
                  _bg(bg), float(early_stop_eps), _ptr(rgb), _ptr(op), _ptr(dep), _ptr(tr), _ptr(w), _stream(dev))
    else:
        _check(ckpt, "ckpt", _F32, dev, (16 * n,))
        _abi.call("nacc_render_fwd_ckpt", n, _ptr(offsets), _ptr(t_starts), _ptr(t_ends), _ptr(sigmas),
                  _ptr(rgbs), _bg(bg), float(early_stop_eps), _ptr(rgb), _ptr(op), _ptr(dep), _ptr(tr), _ptr(w),
                  _ptr(ckpt), _stream(dev))
    return rgb, op, dep, tr, w


def render_bwd(offsets, t_starts, t_ends, sigmas, rgbs, g_rgb, g_opacity, g_depth, bg=(1.0, 1.0, 1.0),
               early_stop_eps=0.0, out=None, ckpt=None):
    """Adjoint of :func:`render_fwd`.  Returns (g_sigmas [S], g_rgbs [S][3]).  ``ckpt``:
    the records a :func:`render_fwd` call on the same samples and eps wrote."""
    dev = offsets.device
    n = int(offsets.shape[0]) - 1
    for t, nm, shp in ((g_rgb, "g_rgb", (n, 3)), (g_opacity, "g_opacity", (n,)), (g_depth, "g_depth", (n,))):
        if t is not None:
            _check(t, nm, _F32, dev, shp)
    if out is None:
        gs = torch.empty_like(sigmas)
        gc = torch.empty_like(rgbs)
    else:
        gs, gc = out
    if ckpt is None:
        _abi.call("nacc_render_bwd", n, _ptr(offsets), _ptr(t_starts), _ptr(t_ends), _ptr(sigmas), _ptr(rgbs),
                  _bg(bg), float(early_stop_eps), _ptr(g_rgb), _ptr(g_opacity), _ptr(g_depth), _ptr(gs),
                  _ptr(gc), _stream(dev))
    else:
        _check(ckpt, "ckpt", _F32, dev, (16 * n,))
        _abi.call("nacc_render_bwd_ckpt", n, _ptr(offsets), _ptr(t_starts), _ptr(t_ends), _ptr(sigmas),
                  _ptr(rgbs), _bg(bg), float(early_stop_eps), _ptr(g_rgb), _ptr(g_opacity), _ptr(g_depth),
                  _ptr(ckpt), _ptr(gs), _ptr(gc), _stream(dev))
    return gs, gc


class RenderFn(torch.autograd.Function):
    """Differentiable compositing: (sigmas, rgbs) -> (rgb, opacity, depth).  The
    backward recomputes per-sample transmittance from the samples; the forward
    saves only a 64-byte record per ray (chunk carries, mask cut, kept depth)."""

    @staticmethod
    def forward(ctx, sigmas, rgbs, offsets, t_starts, t_ends, bg=(1.0, 1.0, 1.0), early_stop_eps=0.0):
        ckpt = render_ckpt_buffer(offsets.shape[0] - 1, offsets.device)
        rgb, op, dep, _, _ = render_fwd(offsets, t_starts, t_ends, sigmas, rgbs, bg, early_stop_eps, ckpt=ckpt)
        ctx.save_for_backward(sigmas, rgbs, offsets, t_starts, t_ends, ckpt)
        ctx.bg, ctx.eps = bg, early_stop_eps
        return rgb, op, dep

    @staticmethod
    def backward(ctx, g_rgb, g_op, g_dep):
        sigmas, rgbs, offsets, t_starts, t_ends, ckpt = ctx.saved_tensors
        c = lambda t: None if t is None else t.contiguous()
        gs, gc = render_bwd(offsets, t_starts, t_ends, sigmas, rgbs, c(g_rgb), c(g_op), c(g_dep),
                            ctx.bg, ctx.eps, ckpt=ckpt)
        return gs, gc, None, None, None, None, None


def render(sigmas, rgbs, packed: PackedSamples, bg=(1.0, 1.0, 1.0), early_stop_eps=0.0):
    """Algorithm 1 ``rendering``: differentiable colour, opacity, depth per ray."""
    return RenderFn.apply(sigmas, rgbs, packed.offsets, packed.t_starts, packed.t_ends, tuple(bg),
                          float(early_stop_eps))


# ---------------------------------------------------------------------------
# estimator update (Eq. 4) and resampling (Eq. 1 / Eq. 3)
# ---------------------------------------------------------------------------

def grid_points(grid: OccupancyGrid, seed: int = 0, step: int = 0, jitter: bool = True, out=None):
    """Sample point of every cell (jittered or centre), [n_cells][3]."""
    dev = grid.bits.device
    xyz = out if out is not None else torch.empty((grid.n_cells, 3), dtype=_F32, device=dev)
    _check(xyz, "xyz", _F32, dev, (grid.n_cells, 3))
    _abi.call("nacc_grid_points", ctypes.byref(grid.c_struct()), int(seed) & (2**64 - 1), int(step),
              int(bool(jitter)), _ptr(xyz), _stream(dev))
    return xyz


class UpdateBuffers:
    def __init__(self, n_cells: int, device="cuda"):
        self.scratch = _scratch(_abi.load().nacc_update_grid_scratch_bytes(n_cells), torch.device(device))


def update_grid(grid: OccupancyGrid, density: torch.Tensor, decay: float = 0.95,
                thresh_frac: float = 0.01, thresh_abs: float = 0.0, buffers: UpdateBuffers | None = None):
    """EMA update of ``grid.ema`` with ``density`` at the cell points, then
    ``grid.bits`` = ema > max(thresh_abs, thresh_frac * mean(ema))."""
    dev = grid.bits.device
    _check(grid.ema, "grid.ema", _F32, dev, (grid.n_cells,))
    _check(density, "density", _F32, dev, (grid.n_cells,))
    buf = buffers if buffers is not None else UpdateBuffers(grid.n_cells, dev)
    _abi.call("nacc_update_grid", ctypes.byref(grid.c_struct()), _ptr(grid.ema), _ptr(density),
              float(decay), float(thresh_frac), float(thresh_abs), _ptr(grid.bits), _ptr(buf.scratch),
              buf.scratch.numel(), _stream(dev))
    return grid


def update_grid_frames(grid: OccupancyGrid, densities: torch.Tensor, decay: float = 0.95,
                       thresh_frac: float = 0.01, thresh_abs: float = 0.0, buffers: UpdateBuffers | None = None):
    """Dynamic scenes: the EMA update with the per-cell maximum over frames of
    ``densities`` [n_frames][n_cells] (one grid for all timestamps)."""
    dev = grid.bits.device
    nf = int(densities.shape[0])
    _check(densities, "densities", _F32, dev, (nf, grid.n_cells))
    buf = buffers if buffers is not None else UpdateBuffers(grid.n_cells, dev)
    _abi.call("nacc_update_grid_frames", ctypes.byref(grid.c_struct()), _ptr(grid.ema), _ptr(densities), nf,
              float(decay), float(thresh_frac), float(thresh_abs), _ptr(grid.bits), _ptr(buf.scratch),
              buf.scratch.numel(), _stream(dev))
    return grid


def grid_density_lookup(grid: OccupancyGrid, density: torch.Tensor, rays_o, rays_d, packed: PackedSamples,
                        out=None) -> torch.Tensor:
    """SGD-updated grid: density of each sample's cell -> [capacity]."""
    dev = density.device
    sig = out if out is not None else torch.empty(packed.capacity, dtype=_F32, device=dev)
    _abi.call("nacc_grid_density_lookup", ctypes.byref(grid.c_struct()), _ptr(density), _ptr(rays_o),
              _ptr(rays_d), _ptr(packed.ray_indices), _ptr(packed.t_starts), _ptr(packed.t_ends),
              _ptr(packed.n_samples_dev), _ptr(sig), _stream(dev))
    return sig


def grid_density_backward(grid: OccupancyGrid, rays_o, rays_d, packed: PackedSamples, g_sigma: torch.Tensor,
                          g_density: torch.Tensor) -> torch.Tensor:
    """Adds each sample's dL/dsigma into its cell's entry of ``g_density``."""
    _abi.call("nacc_grid_density_backward", ctypes.byref(grid.c_struct()), _ptr(rays_o), _ptr(rays_d),
              _ptr(packed.ray_indices), _ptr(packed.t_starts), _ptr(packed.t_ends), _ptr(packed.n_samples_dev),
              _ptr(g_sigma), _ptr(g_density), _stream(g_density.device))
    return g_density


def update_grid_sgd(grid: OccupancyGrid, density: torch.Tensor, g_density: torch.Tensor, lr: float,
                    thresh: float = 0.01) -> OccupancyGrid:
    """density = max(density - lr g, 0), g = 0, bits = density > thresh."""
    _abi.call("nacc_update_grid_sgd", ctypes.byref(grid.c_struct()), _ptr(density), _ptr(g_density), float(lr),
              float(thresh), _ptr(grid.bits), _stream(density.device))
    return grid


def sample_pdf(edges: torch.Tensor, weights: torch.Tensor, n_out: int, stratified: bool = False,
               seed: int = 0, out=None):
    """Inverse-CDF resampling: edges [n][nb+1], weights [n][nb] -> [n][n_out+1]."""
    dev = edges.device
    _check(weights, "weights", _F32, dev)
    n, nb = int(weights.shape[0]), int(weights.shape[1])
    _check(edges, "edges", _F32, dev, (n, nb + 1))
    res = out if out is not None else torch.empty((n, n_out + 1), dtype=_F32, device=dev)
    _check(res, "out", _F32, dev, (n, n_out + 1))
    _abi.call("nacc_sample_pdf", n, nb, _ptr(edges), _ptr(weights), int(n_out), int(bool(stratified)),
              int(seed) & (2**64 - 1), _ptr(res), _stream(dev))
    return res


# ---------------------------------------------------------------------------
# harness (not the method): analytic field and loss
# ---------------------------------------------------------------------------

def field_eval(field: BlobField, rays_o, rays_d, packed: PackedSamples, out=None, per_sample=False):
    """Blob field at interval midpoints: (sigmas [cap], rgbs [cap][3]).

    By default one warp per ray through the CSR offsets
    (``nacc_harness_field_rays``, up to 256 blobs); ``per_sample`` (or more
    blobs) uses one thread per sample through ``ray_indices``."""
    dev = rays_o.device
    cap = packed.capacity
    if out is None:
        sig = torch.empty(cap, dtype=_F32, device=dev)
        rgb = torch.empty((cap, 3), dtype=_F32, device=dev)
    else:
        sig, rgb = out
    if not per_sample and field.n <= 256:
        n = int(rays_o.shape[0])
        _abi.call("nacc_harness_field_rays", _ptr(rays_o), _ptr(rays_d), n, _ptr(packed.offsets),
                  _ptr(packed.t_starts), _ptr(packed.t_ends), ctypes.byref(field.c_struct()), _ptr(sig),
                  _ptr(rgb), _stream(dev))
        return sig, rgb
    if packed.ray_indices is None:
        raise ValueError("field_eval per sample needs ray_indices")
    _abi.call("nacc_harness_field", _ptr(rays_o), _ptr(rays_d), _ptr(packed.ray_indices),
              _ptr(packed.t_starts), _ptr(packed.t_ends), _ptr(packed.n_samples_dev),
              ctypes.byref(field.c_struct()), _ptr(sig), _ptr(rgb), _stream(dev))
    return sig, rgb


def field_points(field: BlobField, xyz: torch.Tensor, out=None):
    dev = xyz.device
    _check(xyz, "xyz", _F32, dev)
    n = int(xyz.shape[0])
    sig = out if out is not None else torch.empty(n, dtype=_F32, device=dev)
    _abi.call("nacc_harness_field_points", n, _ptr(xyz), ctypes.byref(field.c_struct()), _ptr(sig),
              _stream(dev))
    return sig


def l2_loss(rgb: torch.Tensor, target: torch.Tensor, out=None):
    """(loss [1], g_rgb [n][3]) for the mean squared error."""
    dev = rgb.device
    n = int(rgb.shape[0])
    _check(rgb, "rgb", _F32, dev, (n, 3))
    _check(target, "target", _F32, dev, (n, 3))
    if out is None:
        g = torch.empty_like(rgb)
        loss = torch.empty(1, dtype=_F32, device=dev)
    else:
        g, loss = out
    _abi.call("nacc_harness_l2_loss", n, _ptr(rgb), _ptr(target), _ptr(g), _ptr(loss), _stream(dev))
    return loss, g


def density_grid(grid: OccupancyGrid, field: BlobField, thresh: float = 0.01, seed: int = 0):
    """Initialise ``grid`` from the field at cell centres: ema = sigma(centre),
    bits = sigma(centre) > thresh (update with decay 0 and an absolute threshold)."""
    pts = grid_points(grid, jitter=False)
    dens = field_points(field, pts)
    update_grid(grid, dens, decay=0.0, thresh_frac=0.0, thresh_abs=thresh)
    return grid


# ---------------------------------------------------------------------------
# learned density proposal (Table 1 "PDF Approaches"; nacc_proposal.h)
# ---------------------------------------------------------------------------

class ProposalMLP:
    """The proposal network: FP32 master parameters (layout of
    ``nacc_proposal.h``), their BF16 weight copy used by the tensor-core
    kernels, Adam moments and a gradient accumulator, all on one device."""

    def __init__(self, params: torch.Tensor):
        dev = params.device
        _check(params, "params", _F32, dev, (_abi.MLP_PARAMS,))
        self.params = params.contiguous()
        self.weights = torch.empty(_abi.MLP_WEIGHTS, dtype=torch.int16, device=dev)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grads = torch.zeros_like(self.params)
        self.loss_sum = torch.zeros(1, dtype=_F32, device=dev)
        self.step = 0
        self.sync()

    @classmethod
    def init(cls, seed: int = 7, device="cuda"):
        """Uniform(+-1/sqrt(fan_in)) weights (fan-in 51 for the encoding, the
        padding columns of W1 zero), zero biases."""
        g = torch.Generator().manual_seed(seed)
        p = torch.zeros(_abi.MLP_PARAMS, dtype=_F32)
        W1 = (torch.rand((64, 64), generator=g, dtype=torch.float64) * 2 - 1) / math.sqrt(51)
        W1[:, 51:] = 0
        p[0:4096] = W1.reshape(-1).float()
        p[4160:8256] = ((torch.rand(4096, generator=g, dtype=torch.float64) * 2 - 1) / 8.0).float()
        p[8320:8384] = ((torch.rand(64, generator=g, dtype=torch.float64) * 2 - 1) / 8.0).float()
        return cls(p.to(device))

    def sync(self):
        _abi.call("nacc_mlp_sync", _ptr(self.params), _ptr(self.weights), _stream(self.params.device))

    def forward(self, xyz: torch.Tensor, out=None) -> torch.Tensor:
        dev = xyz.device
        n = int(xyz.shape[0])
        _check(xyz, "xyz", _F32, dev, (n, 3))
        sig = out if out is not None else torch.empty(n, dtype=_F32, device=dev)
        _abi.call("nacc_mlp_forward", n, _ptr(xyz), _ptr(self.params), _ptr(self.weights), _ptr(sig),
                  _stream(dev))
        return sig

    def forward_rays(self, rays_o, rays_d, edges: torch.Tensor, out=None, contracted: bool = False) -> torch.Tensor:
        """Density at the bin midpoints of rays: edges [n][nb+1] -> [n][nb]
        (``contracted``: at the contracted midpoints, for unbounded scenes)."""
        dev = edges.device
        n, nb = int(edges.shape[0]), int(edges.shape[1]) - 1
        _check(edges, "edges", _F32, dev, (n, nb + 1))
        _check(rays_o, "rays_o", _F32, dev, (n, 3))
        _check(rays_d, "rays_d", _F32, dev, (n, 3))
        sig = out if out is not None else torch.empty((n, nb), dtype=_F32, device=dev)
        _check(sig, "out", _F32, dev, (n, nb))
        fn = "nacc_mlp_forward_rays_contracted" if contracted else "nacc_mlp_forward_rays"
        _abi.call(fn, n, nb, _ptr(rays_o), _ptr(rays_d), _ptr(edges), _ptr(self.params), _ptr(self.weights),
                  _ptr(sig), _stream(dev))
        return sig

    def forward_encoded(self, enc: torch.Tensor, out=None) -> torch.Tensor:
        """The network on rows that are already its layer-1 input: enc [n][64]
        int16 holding BF16 bit patterns (``nacc_mlp_forward_encoded``)."""
        dev = enc.device
        n = int(enc.shape[0])
        _check(enc, "enc", torch.int16, dev, (n, 64))
        sig = out if out is not None else torch.empty(n, dtype=_F32, device=dev)
        _abi.call("nacc_mlp_forward_encoded", n, _ptr(enc), _ptr(self.params), _ptr(self.weights), _ptr(sig),
                  _stream(dev))
        return sig

    def accumulate_grads_encoded(self, enc: torch.Tensor, target: torch.Tensor):
        """As :meth:`accumulate_grads` on encoded rows (``nacc_mlp_train_grads_encoded``)."""
        dev = enc.device
        n = int(enc.shape[0])
        _check(enc, "enc", torch.int16, dev, (n, 64))
        _check(target, "target", _F32, dev, (n,))
        _abi.call("nacc_mlp_train_grads_encoded", n, _ptr(enc), _ptr(target), _ptr(self.params),
                  _ptr(self.weights), _ptr(self.grads), _ptr(self.loss_sum), _stream(dev))

    def accumulate_grads(self, xyz: torch.Tensor, target: torch.Tensor):
        """Adds dL/dparams of L = mean (density - target)^2 into ``grads``
        and sum (density - target)^2 into ``loss_sum``."""
        dev = xyz.device
        n = int(xyz.shape[0])
        _check(xyz, "xyz", _F32, dev, (n, 3))
        _check(target, "target", _F32, dev, (n,))
        _abi.call("nacc_mlp_train_grads", n, _ptr(xyz), _ptr(target), _ptr(self.params), _ptr(self.weights),
                  _ptr(self.grads), _ptr(self.loss_sum), _stream(dev))

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step += 1
        _abi.call("nacc_mlp_adam", _ptr(self.params), _ptr(self.grads), _ptr(self.m), _ptr(self.v), self.step,
                  float(lr), float(beta1), float(beta2), float(eps), _ptr(self.weights),
                  _stream(self.params.device))

    def train_step(self, xyz, target, lr=1e-3) -> torch.Tensor:
        """One fused forward/adjoint pass and an Adam step; returns the batch's
        mean squared error (a device tensor, read before the step)."""
        self.loss_sum.zero_()
        self.accumulate_grads(xyz, target)
        loss = self.loss_sum / xyz.shape[0]
        self.adam(lr)
        return loss


def contract_points(x: torch.Tensor, out=None) -> torch.Tensor:
    """The L-infinity contraction of points [n][3] into [-2, 2]^3 (``nacc_contract_points``)."""
    dev = x.device
    n = int(x.shape[0])
    _check(x, "x", _F32, dev, (n, 3))
    c = out if out is not None else torch.empty_like(x)
    _check(c, "out", _F32, dev, (n, 3))
    _abi.call("nacc_contract_points", n, _ptr(x), _ptr(c), _stream(dev))
    return c


def phi_edges(n_rays: int, n_bins: int, t_near: float, t_far: float, device="cuda", out=None) -> torch.Tensor:
    """Bins uniform in s mapped to t by the disparity-linear Phi -> edges [n_rays][n_bins+1]."""
    e = out if out is not None else torch.empty((n_rays, n_bins + 1), dtype=_F32, device=device)
    dev = e.device
    _check(e, "edges", _F32, dev, (n_rays, n_bins + 1))
    _abi.call("nacc_phi_edges", int(n_rays), int(n_bins), float(t_near), float(t_far), _ptr(e), _stream(dev))
    return e


def uniform_edges(grid: OccupancyGrid, rays_o, rays_d, n_bins: int, t_min: float = 0.0, t_max: float = 1e10,
                  out=None) -> torch.Tensor:
    """Initial bins of the proposal estimator: n_bins equal bins of each ray's
    clip against the box of the grid's level 0 -> edges [n][n_bins+1]."""
    dev = rays_o.device
    n = int(rays_o.shape[0])
    _check(rays_o, "rays_o", _F32, dev, (n, 3))
    _check(rays_d, "rays_d", _F32, dev, (n, 3))
    e = out if out is not None else torch.empty((n, n_bins + 1), dtype=_F32, device=dev)
    _check(e, "edges", _F32, dev, (n, n_bins + 1))
    _abi.call("nacc_uniform_edges", ctypes.byref(grid.c_struct()), _ptr(rays_o), _ptr(rays_d), n, float(t_min),
              float(t_max), int(n_bins), _ptr(e), _stream(dev))
    return e


def dense_weights(edges: torch.Tensor, sigmas: torch.Tensor, out=None, trans=None) -> torch.Tensor:
    """w_j = T_j (1 - exp(-sigma_j dt_j)) on a dense [n][n_bins] layout (Eq. 2)."""
    dev = edges.device
    n, nb = int(sigmas.shape[0]), int(sigmas.shape[1])
    _check(edges, "edges", _F32, dev, (n, nb + 1))
    _check(sigmas, "sigmas", _F32, dev, (n, nb))
    w = out if out is not None else torch.empty((n, nb), dtype=_F32, device=dev)
    _abi.call("nacc_dense_weights", n, nb, _ptr(edges), _ptr(sigmas), _ptr(w), _ptr(trans) if trans is not None
              else None, _stream(dev))
    return w


def edges_to_packed(edges: torch.Tensor, out: PackedSamples | None = None) -> PackedSamples:
    """Bins [n][nb+1] -> packed samples (nb per ray, no ray_indices)."""
    dev = edges.device
    n, nb = int(edges.shape[0]), int(edges.shape[1]) - 1
    if out is None:
        out = PackedSamples(torch.empty(n + 1, dtype=torch.int64, device=dev), None,
                            torch.empty(n * nb, dtype=_F32, device=dev), torch.empty(n * nb, dtype=_F32, device=dev),
                            torch.empty(1, dtype=torch.int64, device=dev))
    _abi.call("nacc_edges_to_packed", n, nb, _ptr(edges), _ptr(out.offsets), _ptr(out.t_starts), _ptr(out.t_ends),
              _ptr(out.n_samples_dev), _stream(dev))
    return out


class ProposalSampler:
    """The learned-proposal estimator (Table 1 "PDF Approaches"): n0 uniform
    bins per ray; for each round, the proposal density at the bin midpoints,
    its transmittance weights (Eq. 2) and inverse transform sampling (Eq. 1)
    to the next round's bins; the last round's bins become the packed samples
    the radiance field and the renderer consume.  Rounds (64, 32) then 32
    final samples by default."""

    def __init__(self, mlp: ProposalMLP, grid: OccupancyGrid, n_rays: int, rounds=(64, 32), n_final: int = 32,
                 device="cuda"):
        self.mlp, self.grid, self.rounds, self.n_final = mlp, grid, tuple(rounds), int(n_final)
        dev = torch.device(device)
        self.n_rays = int(n_rays)
        sizes = list(self.rounds) + [self.n_final]
        self.edges = [torch.empty((n_rays, nb + 1), dtype=_F32, device=dev) for nb in sizes]
        self.sig = [torch.empty((n_rays, nb), dtype=_F32, device=dev) for nb in self.rounds]
        self.w = [torch.empty((n_rays, nb), dtype=_F32, device=dev) for nb in self.rounds]
        self.packed = edges_to_packed(self.edges[-1])
        self.contracted = False

    def sample(self, rays_o, rays_d, t_min: float = 0.0, t_max: float = 1e10, stratified: bool = False,
               seed: int = 0) -> PackedSamples:
        e = uniform_edges(self.grid, rays_o, rays_d, self.rounds[0], t_min, t_max, out=self.edges[0])
        return self.resample(rays_o, rays_d, e, stratified, seed)

    def resample(self, rays_o, rays_d, e: torch.Tensor, stratified: bool = False, seed: int = 0) -> PackedSamples:
        """The proposal rounds from given initial bins e [n][rounds[0]+1]."""
        for i, nb in enumerate(self.rounds):
            s = self.mlp.forward_rays(rays_o, rays_d, e, out=self.sig[i], contracted=self.contracted)
            w = dense_weights(e, s, out=self.w[i])
            n_next = self.rounds[i + 1] if i + 1 < len(self.rounds) else self.n_final
            e = sample_pdf(e, w, n_next, stratified, seed + i, out=self.edges[i + 1])
        return edges_to_packed(e, out=self.packed)


class UnboundedProposalSampler(ProposalSampler):
    """The proposal estimator for unbounded scenes (Sec. 3.2): initial bins
    uniform in s over [t_near, t_far] (disparity-linear Phi), the network
    evaluated at the contracted bin midpoints; the rounds and the inverse
    transform sampling act on the bins in t."""

    def __init__(self, mlp: ProposalMLP, n_rays: int, t_near: float, t_far: float, rounds=(64, 32),
                 n_final: int = 32, device="cuda"):
        super().__init__(mlp, None, n_rays, rounds, n_final, device)
        self.t_near, self.t_far = float(t_near), float(t_far)
        self.contracted = True

    def sample(self, rays_o, rays_d, t_min: float | None = None, t_max: float | None = None,
               stratified: bool = False, seed: int = 0) -> PackedSamples:
        """Same call as :meth:`ProposalSampler.sample`; ``t_min`` / ``t_max``, if
        given, replace the sampler's t_near / t_far for this call."""
        tn = self.t_near if t_min is None else float(t_min)
        tf = self.t_far if t_max is None else float(t_max)
        e = phi_edges(self.n_rays, self.rounds[0], tn, tf, out=self.edges[0])
        return self.resample(rays_o, rays_d, e, stratified, seed)


def occupied_range(grid: OccupancyGrid, rays_o, rays_d, step: float, max_steps: int = 1024, t_min: float = 0.0,
                   t_max: float = 1e10, out=None, scratch=None):
    """t0 of the first and t1 of the last occupied lattice point of each ray
    (``nacc_occupied_range``): (t_lo [n], t_hi [n])."""
    dev = rays_o.device
    n = int(rays_o.shape[0])
    _check(rays_o, "rays_o", _F32, dev, (n, 3))
    _check(rays_d, "rays_d", _F32, dev, (n, 3))
    lo, hi = out if out is not None else (torch.empty(n, dtype=_F32, device=dev), torch.empty(n, dtype=_F32, device=dev))
    if scratch is None:
        scratch = _scratch(_abi.load().nacc_occupied_range_scratch_bytes(), dev)
    params = _abi.MarchParams(float(step), int(max_steps), float(t_min), float(t_max), 0.0)
    _abi.call("nacc_occupied_range", ctypes.byref(grid.c_struct()), _ptr(rays_o), _ptr(rays_d), n,
              ctypes.byref(params), _ptr(lo), _ptr(hi), _ptr(scratch), scratch.numel(), _stream(dev))
    return lo, hi


def range_edges(t_lo: torch.Tensor, t_hi: torch.Tensor, n_bins: int, out=None) -> torch.Tensor:
    """n_bins equal bins of [t_lo, t_hi] per ray -> edges [n][n_bins+1]."""
    dev = t_lo.device
    n = int(t_lo.shape[0])
    e = out if out is not None else torch.empty((n, n_bins + 1), dtype=_F32, device=dev)
    _abi.call("nacc_range_edges", n, _ptr(t_lo), _ptr(t_hi), int(n_bins), _ptr(e), _stream(dev))
    return e


class CombinedSampler(ProposalSampler):
    """Occupancy grid stacked on the proposal network: the grid gives each
    ray's occupied range (first to last occupied lattice point), the proposal
    rounds resample inside it."""

    def __init__(self, mlp: ProposalMLP, grid: OccupancyGrid, n_rays: int, step: float, max_steps: int = 1024,
                 rounds=(64, 32), n_final: int = 32, device="cuda"):
        super().__init__(mlp, grid, n_rays, rounds, n_final, device)
        self.step, self.max_steps = float(step), int(max_steps)
        dev = torch.device(device)
        self.lo = torch.empty(n_rays, dtype=_F32, device=dev)
        self.hi = torch.empty(n_rays, dtype=_F32, device=dev)
        self.scratch = _scratch(_abi.load().nacc_occupied_range_scratch_bytes(), dev)

    def sample(self, rays_o, rays_d, t_min: float = 0.0, t_max: float = 1e10, stratified: bool = False,
               seed: int = 0) -> PackedSamples:
        occupied_range(self.grid, rays_o, rays_d, self.step, self.max_steps, t_min, t_max, out=(self.lo, self.hi),
                       scratch=self.scratch)
        e = range_edges(self.lo, self.hi, self.rounds[0], out=self.edges[0])
        return self.resample(rays_o, rays_d, e, stratified, seed)


def mlp_encode(xyz: torch.Tensor) -> torch.Tensor:
    """Diagnostics: the FP32 frequency encoding [n][64] of points [n][3]."""
    dev = xyz.device
    n = int(xyz.shape[0])
    enc = torch.empty((n, 64), dtype=_F32, device=dev)
    _abi.call("nacc_mlp_encode", n, _ptr(xyz), _ptr(enc), _stream(dev))
    return enc
