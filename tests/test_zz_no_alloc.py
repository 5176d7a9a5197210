"""nacc_update_grid_noalloc: the grid update for callers that cannot allocate
device memory on the path that refreshes the grid (for example code hosted in
an application that owns the whole device memory budget, or a latency-critical
thread that must not pay for an allocation's synchronisation).  It must give
exactly the EMA and occupancy bits of nacc_update_grid, call after call, while
using the library's own scratch array instead of a caller buffer.

Collected last on purpose, so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_update_matches_update_grid_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_04966_gb300 as nacc
    from paper_2305_04966_gb300 import _abi

    lib = nacc.load_library()
    res, L = 96, 3
    n = L * res ** 3
    g = workloads.rng(500)
    ema0 = torch.as_tensor(g.exponential(1.0, n).astype(np.float32)).cuda()
    ref = nacc.OccupancyGrid.empty((-1.5,) * 3, (1.5,) * 3, res, L)
    alt = nacc.OccupancyGrid.empty((-1.5,) * 3, (1.5,) * 3, res, L)
    ref.ema.copy_(ema0)
    alt.ema.copy_(ema0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        dens = torch.as_tensor((g.exponential(0.5, n) * (g.random(n) < 0.4)).astype(np.float32)).cuda()
        nacc.update_grid(ref, dens, decay=0.95, thresh_frac=0.01)
        rc = lib.nacc_update_grid_noalloc(ctypes.byref(alt.c_struct()), _ptr(alt.ema), _ptr(dens),
                                          0.95, 0.01, 0.0, _ptr(alt.bits), stream)
        assert rc == _abi.NACC_OK, lib.nacc_last_error()
        torch.cuda.synchronize()
        assert torch.equal(alt.ema, ref.ema), f"EMA differs on call {call}"
        assert torch.equal(alt.bits, ref.bits), f"occupancy bits differ on call {call}"
        assert 0 < int(workloads.unpack_bits(alt.bits.cpu().numpy().view(np.uint32)).sum()) < n


def test_noalloc_update_at_its_limit():
    """Exactly 2^27 cells (8 levels of 256^3): the 65,536 partial sums fill the
    whole array and the (mean, threshold) words sit right after them.  EMA
    and bits equal nacc_update_grid's on two consecutive calls."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_04966_gb300 as nacc
    from paper_2305_04966_gb300 import _abi

    lib = nacc.load_library()
    res, L = 256, 8
    n = L * res ** 3
    assert n == 1 << 27
    gen = torch.Generator(device="cuda")
    gen.manual_seed(501)
    ref = nacc.OccupancyGrid.empty((-1.5,) * 3, (1.5,) * 3, res, L)
    alt = nacc.OccupancyGrid.empty((-1.5,) * 3, (1.5,) * 3, res, L)
    ref.ema.copy_(-torch.log1p(-torch.rand(n, generator=gen, device="cuda") * 0.999))
    alt.ema.copy_(ref.ema)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        dens = torch.rand(n, generator=gen, device="cuda") * (torch.rand(n, generator=gen, device="cuda") < 0.3)
        nacc.update_grid(ref, dens, decay=0.95, thresh_frac=0.01)
        rc = lib.nacc_update_grid_noalloc(ctypes.byref(alt.c_struct()), _ptr(alt.ema), _ptr(dens),
                                          0.95, 0.01, 0.0, _ptr(alt.bits), stream)
        assert rc == _abi.NACC_OK, lib.nacc_last_error()
        torch.cuda.synchronize()
        assert torch.equal(alt.ema, ref.ema), f"EMA differs on call {call}"
        assert torch.equal(alt.bits, ref.bits), f"occupancy bits differ on call {call}"
        del dens
    words = alt.bits.view(torch.int32)
    assert bool((words != 0).any()) and bool((words != -1).any())  # some cells occupied, some not
    del ref, alt
    torch.cuda.empty_cache()


def test_noalloc_update_rejects_grids_beyond_its_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_04966_gb300 as nacc
    from paper_2305_04966_gb300 import _abi

    lib = nacc.load_library()
    g = _abi.Grid()
    g.aabb_min[:] = [-1.0, -1.0, -1.0]
    g.aabb_max[:] = [1.0, 1.0, 1.0]
    g.res, g.n_levels, g.bits = 512, 2, None  # 2^28 cells > 2^27
    dummy = torch.zeros(8, device="cuda")
    rc = lib.nacc_update_grid_noalloc(ctypes.byref(g), _ptr(dummy), _ptr(dummy), 0.95, 0.01, 0.0,
                                      _ptr(dummy), None)
    assert rc == _abi.NACC_ERR_INVALID_ARG
    assert b"134217728" in lib.nacc_last_error()
