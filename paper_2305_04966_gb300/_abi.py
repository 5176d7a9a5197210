"""ctypes declarations of the C ABI in ``include/nacc.h``, ``include/nacc_harness.h``
and ``include/nacc_proposal.h``.

Loads the in-tree ``libnacc.so``.  There is no fallback: if the library is
missing or fails to load, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_i32, c_i64, c_u64, c_f32, c_sz, c_vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                         ctypes.c_float, ctypes.c_size_t, ctypes.c_void_p)

NACC_OK = 0
NACC_ERR_INVALID_ARG = -1
NACC_ERR_CAPACITY = -2
NACC_ERR_CUDA = -3
NACC_ERR_TIMEOUT = -4
NACC_ERR_UNSUPPORTED = -5
MAX_LEVELS = 8


class Grid(ctypes.Structure):
    _fields_ = [("aabb_min", c_f32 * 3), ("aabb_max", c_f32 * 3), ("res", c_i32),
                ("n_levels", c_i32), ("bits", c_vp)]


class MarchParams(ctypes.Structure):
    _fields_ = [("step", c_f32), ("max_steps", c_i32), ("t_min", c_f32), ("t_max", c_f32),
                ("early_stop_eps", c_f32), ("exact_stops", c_i32)]


class BlobField(ctypes.Structure):
    _fields_ = [("n_blobs", c_i32), ("mu", c_vp), ("std", c_vp), ("peak", c_vp), ("rgb", c_vp)]


class Packed(ctypes.Structure):
    _fields_ = [("offsets", c_vp), ("ray_indices", c_vp), ("t_starts", c_vp), ("t_ends", c_vp),
                ("capacity", c_i64), ("n_samples", c_vp)]


P = ctypes.POINTER

# name -> (restype, argtypes)
SIGNATURES = {
    "nacc_last_error": (ctypes.c_char_p, []),
    "nacc_version": (c_i32, []),
    "nacc_march_scratch_bytes": (c_sz, [c_i64]),
    "nacc_march_grid": (c_i32, [P(Grid), c_vp, c_vp, c_i64, P(MarchParams), P(BlobField), P(Packed),
                                c_vp, c_sz, c_vp]),
    "nacc_grid_points": (c_i32, [P(Grid), c_u64, c_i64, c_i32, c_vp, c_vp]),
    "nacc_march_unbounded_scratch_bytes": (c_sz, [c_i64, c_i32]),
    "nacc_march_unbounded": (c_i32, [P(Grid), c_vp, c_vp, c_i64, P(MarchParams), P(BlobField), P(Packed),
                                     c_vp, c_sz, c_vp]),
    "nacc_uncontract_points": (c_i32, [c_i64, c_vp, c_vp, c_vp]),
    "nacc_update_grid_scratch_bytes": (c_sz, [c_i64]),
    "nacc_update_grid": (c_i32, [P(Grid), c_vp, c_vp, c_f32, c_f32, c_f32, c_vp, c_vp, c_sz, c_vp]),
    "nacc_update_grid_noalloc": (c_i32, [P(Grid), c_vp, c_vp, c_f32, c_f32, c_f32, c_vp, c_vp]),
    "nacc_update_grid_frames": (c_i32, [P(Grid), c_vp, c_vp, c_i32, c_f32, c_f32, c_f32, c_vp, c_vp, c_sz, c_vp]),
    "nacc_grid_density_lookup": (c_i32, [P(Grid), c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "nacc_grid_density_backward": (c_i32, [P(Grid), c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "nacc_update_grid_sgd": (c_i32, [P(Grid), c_vp, c_vp, c_f32, c_f32, c_vp, c_vp]),
    "nacc_sample_pdf": (c_i32, [c_i64, c_i32, c_vp, c_vp, c_i32, c_i32, c_u64, c_vp, c_vp]),
    "nacc_render_fwd": (c_i32, [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, P(c_f32), c_f32, c_vp, c_vp,
                                c_vp, c_vp, c_vp, c_vp]),
    "nacc_render_bwd": (c_i32, [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, P(c_f32), c_f32, c_vp, c_vp,
                                c_vp, c_vp, c_vp, c_vp]),
    "nacc_render_ckpt_bytes": (c_sz, [c_i64]),
    "nacc_render_fwd_ckpt": (c_i32, [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, P(c_f32), c_f32, c_vp, c_vp,
                                     c_vp, c_vp, c_vp, c_vp, c_vp]),
    "nacc_render_bwd_ckpt": (c_i32, [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, P(c_f32), c_f32, c_vp, c_vp,
                                     c_vp, c_vp, c_vp, c_vp, c_vp]),
    "nacc_harness_field": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, P(BlobField), c_vp, c_vp, c_vp]),
    "nacc_harness_field_points": (c_i32, [c_i64, c_vp, P(BlobField), c_vp, c_vp]),
    "nacc_harness_field_rays": (c_i32, [c_vp, c_vp, c_i64, c_vp, c_vp, c_vp, P(BlobField), c_vp, c_vp, c_vp]),
    "nacc_harness_l2_loss": (c_i32, [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "nacc_device_status": (c_i32, [c_vp, P(c_i32)]),
    "nacc_selftest_wait_timeout": (c_i32, [c_i64, c_vp]),
    "nacc_set_march_count_events": (c_i32, [c_vp, c_vp]),
    "nacc_mlp_sync": (c_i32, [c_vp, c_vp, c_vp]),
    "nacc_mlp_forward": (c_i32, [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "nacc_mlp_train_grads": (c_i32, [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "nacc_mlp_forward_encoded": (c_i32, [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "nacc_mlp_train_grads_encoded": (c_i32, [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "nacc_mlp_adam": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i64, c_f32, c_f32, c_f32, c_f32, c_vp, c_vp]),
    "nacc_mlp_encode": (c_i32, [c_i64, c_vp, c_vp, c_vp]),
    "nacc_mlp_forward_rays": (c_i32, [c_i64, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "nacc_mlp_forward_rays_contracted": (c_i32, [c_i64, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "nacc_contract_points": (c_i32, [c_i64, c_vp, c_vp, c_vp]),
    "nacc_phi_edges": (c_i32, [c_i64, c_i32, c_f32, c_f32, c_vp, c_vp]),
    "nacc_uniform_edges": (c_i32, [P(Grid), c_vp, c_vp, c_i64, c_f32, c_f32, c_i32, c_vp, c_vp]),
    "nacc_dense_weights": (c_i32, [c_i64, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "nacc_edges_to_packed": (c_i32, [c_i64, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "nacc_occupied_range_scratch_bytes": (c_sz, []),
    "nacc_occupied_range": (c_i32, [P(Grid), c_vp, c_vp, c_i64, P(MarchParams), c_vp, c_vp, c_vp, c_sz, c_vp]),
    "nacc_range_edges": (c_i32, [c_i64, c_vp, c_vp, c_i32, c_vp, c_vp]),
}

MLP_PARAMS = 8385
MLP_WEIGHTS = 8256

_lib = None


class NaccError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} failed with status {code}: {msg}")
        self.code = code


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load ``libnacc.so`` (raises if absent, unless ``build_if_missing``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build() "
                               f"(or python -m paper_2305_04966_gb300.build)")
        _build.build()
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def call(name: str, *args) -> int:
    """Call an entry point; raise NaccError on a non-OK status (except CAPACITY, returned)."""
    L = load()
    rc = getattr(L, name)(*args)
    if rc != NACC_OK and rc != NACC_ERR_CAPACITY:
        raise NaccError(name, rc, L.nacc_last_error().decode(errors="replace"))
    return rc
