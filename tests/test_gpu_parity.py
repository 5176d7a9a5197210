"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Bars (see the design notes for the derivations):
  * packed samples (offsets, ray ids, t0, t1): bit-exact, with and without
    the field's early stop, on every ray (the march reaches the definition's
    FP32 stopping decision exactly; rays whose depth comes near the
    threshold are counted and reported, not exempted);
  * compositing: transmittance, weights, colour, opacity within 1e-5
    absolute, depth within 1e-5 relative;
  * gradients: |g - g_ref| <= 1e-4 |g_ref| + 1e-5 * dt_i * (|g_C|_1 + |g_A| +
    |g_D| m_i) (1e-4 relative, with an absolute floor at the natural scale of
    the terms that cancel);
  * grid points, EMA, sample_pdf: bit-exact; occupancy bits exact except
    cells within 1e-12 (relative) of the FP64 threshold.
"""
import dataclasses
import math
import types

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module")
def nacc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_04966_gb300 as m
    m.load_library()
    return m


def T(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def grid_from_bits(nacc, spec_min, spec_max, res, L, bits):
    return nacc.OccupancyGrid(tuple(spec_min), tuple(spec_max), res, L,
                              T(bits.view(np.int32), torch.int32))


def run_march(nacc, grid, o, d, step, max_steps, t_min, t_max, field=None, eps=1e-4, capacity=None,
              exact_stops=False):
    pk = nacc.march_grid(grid, T(o), T(d), step, max_steps, t_min, t_max, eps, field=field,
                         capacity=capacity, exact_stops=exact_stops)
    torch.cuda.synchronize()
    pk = pk.trimmed()
    return dict(offsets=pk.offsets.cpu().numpy(), ray_indices=pk.ray_indices.cpu().numpy(),
                t_starts=pk.t_starts.cpu().numpy(), t_ends=pk.t_ends.cpu().numpy())


def assert_packed_equal(got, exp, rays=None):
    if rays is None:
        for k in ("offsets", "ray_indices", "t_starts", "t_ends"):
            np.testing.assert_array_equal(got[k], exp[k], err_msg=k)
        return
    go, eo = got["offsets"], exp["offsets"]
    for r in rays:
        gs, ge, es, ee = go[r], go[r + 1], eo[r], eo[r + 1]
        assert ge - gs == ee - es, f"ray {r}: {ge - gs} vs {ee - es} samples"
        for k in ("t_starts", "t_ends"):
            np.testing.assert_array_equal(got[k][gs:ge], exp[k][es:ee], err_msg=f"{k} ray {r}")
        assert np.all(got["ray_indices"][gs:ge] == r)


# ---------------------------------------------------------------------------
# march
# ---------------------------------------------------------------------------

def test_march_c1_no_field_bit_exact(nacc, orc):
    w = workloads.c1_forward()
    g, m = w.grid, w.march
    bits, _ = orc.density_grid(g, w.blobs)
    grid = grid_from_bits(nacc, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits)
    got = run_march(nacc, grid, w.rays_o, w.rays_d, m.step, m.max_steps, m.t_min, m.t_max)
    exp = orc.march(w.rays_o, w.rays_d, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, m.step,
                    m.max_steps, m.t_min, m.t_max)
    assert exp["offsets"][-1] > 100000
    assert_packed_equal(got, exp)


@pytest.mark.parametrize("res,L,block,p_block", [(16, 1, 2, 0.5), (32, 2, 4, 0.3), (64, 3, 8, 0.2),
                                                 (128, 4, 16, 0.15), (20, 2, 5, 0.4)])
def test_march_random_grids_bit_exact(nacc, orc, res, L, block, p_block):
    bits = workloads.random_bitfield(L, res, 200 + res + L, p_block=p_block, block=block, p_cell=0.6)
    g = workloads.rng(300 + res + L)
    n = 3000
    o = workloads._normalise(g.standard_normal((n, 3))) * g.uniform(0.0, 8.0, size=(n, 1))
    p = g.uniform(-1.5, 1.5, size=(n, 3))
    d = workloads._normalise(p - o)
    d[:40] = 0.0
    d[np.arange(40), np.arange(40) % 3] = np.where(np.arange(40) % 2 == 0, 1.0, -1.0)
    d[40:80, 2] = 0.0
    d[40:80] = workloads._normalise(d[40:80])
    # origins exactly on cell faces and grazing the box edge
    o[80:100] = np.round(o[80:100] * (res / 3.0)) * (3.0 / res)
    o, d = o.astype(np.float32), d.astype(np.float32)
    step = 3.0 * math.sqrt(3) / 1024 * (128 / res) ** 0.5
    grid = grid_from_bits(nacc, (-1.5,) * 3, (1.5,) * 3, res, L, bits)
    got = run_march(nacc, grid, o, d, step, 2048, 0.05, 1e10)
    exp = orc.march(o, d, (-1.5,) * 3, (1.5,) * 3, res, L, bits, step, 2048, 0.05, 1e10)
    assert exp["offsets"][-1] > 1000
    assert_packed_equal(got, exp)


def _lattice_ranges(packed, step):
    """Number of separate contiguous lattice ranges of each ray's samples."""
    off, t0 = packed["offsets"], packed["t_starts"].astype(np.float64)
    out = np.zeros(len(off) - 1, np.int64)
    for r in range(len(off) - 1):
        a, b = off[r], off[r + 1]
        if b > a:
            out[r] = 1 + int(np.count_nonzero(np.diff(t0[a:b]) > 1.5 * step))
    return out


def test_march_many_lattice_ranges_bit_exact(nacc, orc):
    """A fine random grid splits rays into many separate lattice ranges: both
    the rays whose ranges fit the fill pass's per-ray record (16) and the rays
    that overflow it (re-marched) must match the definition."""
    res, L = 64, 2
    g = workloads.rng(4243)
    occ = g.random((L, res, res, res)) < 0.5
    occ[:, : res // 2] = True  # solid half (x < 0): few ranges per ray there
    bits = workloads.pack_bits(occ.reshape(-1))
    n = 2048
    o = workloads._normalise(g.standard_normal((n, 3))) * 4.0
    d = workloads._normalise(g.uniform(-1.2, 1.2, size=(n, 3)) - o)
    o, d = o.astype(np.float32), d.astype(np.float32)
    step = 3.0 / 256
    grid = grid_from_bits(nacc, (-1.5,) * 3, (1.5,) * 3, res, L, bits)
    got = run_march(nacc, grid, o, d, step, 1024, 0.0, 1e10)
    exp = orc.march(o, d, (-1.5,) * 3, (1.5,) * 3, res, L, bits, step, 1024, 0.0, 1e10)
    ranges = _lattice_ranges(exp, step)
    assert np.count_nonzero(ranges > 16) > 100 and np.count_nonzero((ranges > 0) & (ranges <= 16)) > 100
    assert_packed_equal(got, exp)


@pytest.mark.parametrize("field_blobs", [8, 64])
def test_march_many_lattice_ranges_with_field(nacc, orc, field_blobs):
    """Early stop on rays split into many lattice ranges: rays whose ranges
    overflow the per-ray record are cut by the early-stop pass's lattice walk,
    the others from their recorded runs; 64 blobs also exercise the per-group
    culling of tables with more than 16 entries.  The packed samples equal the
    definition's on every ray, in the default mode and with every decision
    taken in the exact arithmetic."""
    res, L = 64, 2
    g = workloads.rng(4244)
    occ = g.random((L, res, res, res)) < 0.5
    occ[:, : res // 2] = True
    bits = workloads.pack_bits(occ.reshape(-1))
    n = 2048
    o = workloads._normalise(g.standard_normal((n, 3))) * 4.0
    d = workloads._normalise(g.uniform(-1.2, 1.2, size=(n, 3)) - o)
    o, d = o.astype(np.float32), d.astype(np.float32)
    blobs = workloads.c1_forward().blobs if field_blobs == 8 else workloads.c3_training(64).blobs
    assert blobs.n == field_blobs
    step, eps = 3.0 / 256, 1e-4
    grid = grid_from_bits(nacc, (-1.5,) * 3, (1.5,) * 3, res, L, bits)
    field = nacc.BlobField.from_numpy(blobs)
    got = run_march(nacc, grid, o, d, step, 1024, 0.0, 1e10, field=field, eps=eps)
    got_x = run_march(nacc, grid, o, d, step, 1024, 0.0, 1e10, field=field, eps=eps, exact_stops=True)
    exp = orc.march(o, d, (-1.5,) * 3, (1.5,) * 3, res, L, bits, step, 1024, 0.0, 1e10, blobs=blobs, eps=eps)
    full = orc.march(o, d, (-1.5,) * 3, (1.5,) * 3, res, L, bits, step, 1024, 0.0, 1e10)
    assert_packed_equal(got, exp)
    assert_packed_equal(got_x, exp)
    _report_near_threshold("many ranges", orc, types.SimpleNamespace(rays_o=o, rays_d=d, blobs=blobs), full,
                           -math.log(eps))
    ec, fc = np.diff(exp["offsets"]), np.diff(full["offsets"])
    ranges = _lattice_ranges(full, step)
    stopped = ec < fc
    assert np.count_nonzero(stopped & (ranges > 16)) > 20  # cut by the lattice walk
    assert np.count_nonzero(stopped & (ranges > 0) & (ranges <= 16)) > 20  # cut from the recorded runs


def test_march_full_grid_is_uniform_sampling(nacc, orc):
    """All-occupied grid: the marcher reduces to uniform sampling (Sec. 3.1)."""
    res = 32
    bits = np.full(res ** 3 // 32, 0xFFFFFFFF, np.uint32)
    w = workloads.c1_forward(2000)
    grid = grid_from_bits(nacc, (-1.5,) * 3, (1.5,) * 3, res, 1, bits)
    got = run_march(nacc, grid, w.rays_o, w.rays_d, 0.01, 1024, 0.0, 1e10)
    exp = orc.march(w.rays_o, w.rays_d, (-1.5,) * 3, (1.5,) * 3, res, 1, bits, 0.01, 1024, 0.0, 1e10)
    assert_packed_equal(got, exp)


def _near_threshold_counts(orc, w, full, thr, rels=(1e-4, 1e-5, 1e-6)):
    """Rays whose optical depth (FP64 field, at the samples of the field-less
    march) before some sample lies within `rel` of the threshold: where an
    FP32 evaluation of the depth could take either side."""
    sig, _ = orc.field_samples(w.rays_o, w.rays_d, full["ray_indices"], full["t_starts"],
                               full["t_ends"], w.blobs)
    tau = sig * (full["t_ends"].astype(np.float64) - full["t_starts"])
    off = full["offsets"]
    dist = np.full(len(off) - 1, np.inf)
    for r in range(len(off) - 1):
        P = np.cumsum(tau[off[r]:off[r + 1]])
        if P.size:
            dist[r] = np.min(np.abs(P - thr)) / thr
    return {rel: int(np.count_nonzero(dist < rel)) for rel in rels}


def _report_near_threshold(name, orc, w, full, thr):
    n = len(full["offsets"]) - 1
    c = _near_threshold_counts(orc, w, full, thr)
    print(f"[{name}] rays near the early-stop threshold (all bit-exact): " +
          ", ".join(f"within {rel:g}: {k} ({1e6 * k / n:.0f} per million)" for rel, k in c.items()))
    return c


@pytest.mark.parametrize("field_blobs", [8, 64])
def test_march_c1_with_field_early_stop(nacc, orc, field_blobs):
    """C1 rays with the 8-blob C1 field (the per-ray closed form of the density
    for few blobs) and with the 64-blob C3 field (per-group culled tables):
    every ray's samples equal the definition's, in the default mode and with
    every decision taken in the exact arithmetic."""
    w = workloads.c1_forward()
    if field_blobs == 64:
        w = dataclasses.replace(w, blobs=workloads.c3_training(64).blobs)
    assert w.blobs.n == field_blobs
    g, m = w.grid, w.march
    bits, _ = orc.density_grid(g, w.blobs)
    grid = grid_from_bits(nacc, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits)
    field = nacc.BlobField.from_numpy(w.blobs)
    got = run_march(nacc, grid, w.rays_o, w.rays_d, m.step, m.max_steps, m.t_min, m.t_max, field=field)
    got_x = run_march(nacc, grid, w.rays_o, w.rays_d, m.step, m.max_steps, m.t_min, m.t_max, field=field,
                      exact_stops=True)
    exp = orc.march(w.rays_o, w.rays_d, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, m.step,
                    m.max_steps, m.t_min, m.t_max, blobs=w.blobs, eps=m.early_stop_eps)
    full = orc.march(w.rays_o, w.rays_d, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, m.step,
                     m.max_steps, m.t_min, m.t_max)
    assert_packed_equal(got, exp)
    assert_packed_equal(got_x, exp)
    near = _report_near_threshold(f"C1, {field_blobs} blobs", orc, w, full, -math.log(m.early_stop_eps))
    assert near[1e-4] > 10  # the case does reach the threshold's neighbourhood
    assert (np.diff(exp["offsets"]) < np.diff(full["offsets"])).sum() > 100  # early stop happened


@pytest.mark.parametrize("n_blobs", [1, 3, 8, 9])
def test_march_small_fields_early_stop(nacc, orc, n_blobs):
    """Fields of at most 8 blobs have each 32-ray entry's early-stop tables built
    together, eight lanes per ray; 9 blobs take the per-ray build.  Both sides
    of that boundary, and fields that leave most of the eight lanes idle, give
    every ray the definition's samples, by default and all-exact."""
    w = workloads.c1_forward()
    w = dataclasses.replace(w, blobs=workloads.blob_field(n_blobs, 90 + n_blobs, std_lo=0.2, std_hi=0.4))
    g, m = w.grid, w.march
    bits, _ = orc.density_grid(g, w.blobs)
    grid = grid_from_bits(nacc, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits)
    field = nacc.BlobField.from_numpy(w.blobs)
    got = run_march(nacc, grid, w.rays_o, w.rays_d, m.step, m.max_steps, m.t_min, m.t_max, field=field)
    got_x = run_march(nacc, grid, w.rays_o, w.rays_d, m.step, m.max_steps, m.t_min, m.t_max, field=field,
                      exact_stops=True)
    exp = orc.march(w.rays_o, w.rays_d, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, m.step,
                    m.max_steps, m.t_min, m.t_max, blobs=w.blobs, eps=m.early_stop_eps)
    full = orc.march(w.rays_o, w.rays_d, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, m.step,
                     m.max_steps, m.t_min, m.t_max)
    assert_packed_equal(got, exp)
    assert_packed_equal(got_x, exp)
    assert (np.diff(exp["offsets"]) < np.diff(full["offsets"])).sum() > 20  # early stop happened


def test_march_c2_full_size_sampled(nacc, orc):
    """640,000-ray image, 4-level grid, with field: per-ray exact on a seeded
    sample of rays computed one by one by the oracle (every sampled ray)."""
    w = workloads.c2_image()
    g, m = w.grid, w.march
    bits, _ = orc.density_grid(g, w.blobs)
    grid = grid_from_bits(nacc, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits)
    field = nacc.BlobField.from_numpy(w.blobs)
    got = run_march(nacc, grid, w.rays_o, w.rays_d, m.step, m.max_steps, m.t_min, m.t_max, field=field,
                    capacity=w.n_rays * m.max_steps)
    sel = np.sort(workloads.rng(77).choice(w.n_rays, 3000, replace=False))
    o, d = w.rays_o[sel], w.rays_d[sel]
    exp = orc.march(o, d, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, m.step, m.max_steps,
                    m.t_min, m.t_max, blobs=w.blobs, eps=m.early_stop_eps)
    go = got["offsets"]
    for k, r in enumerate(sel):
        gs, ge = go[r], go[r + 1]
        es, ee = exp["offsets"][k], exp["offsets"][k + 1]
        assert ge - gs == ee - es, f"ray {r}"
        np.testing.assert_array_equal(got["t_starts"][gs:ge], exp["t_starts"][es:ee])
        np.testing.assert_array_equal(got["t_ends"][gs:ge], exp["t_ends"][es:ee])
        assert np.all(got["ray_indices"][gs:ge] == r)
    # structure over all rays: offsets are a CSR of the counts, ray ids consistent
    assert go[0] == 0 and np.all(np.diff(go) >= 0) and go[-1] == len(got["t_starts"])
    assert np.all(np.diff(go) <= m.max_steps)
    ri = got["ray_indices"]
    assert np.array_equal(ri, np.repeat(np.arange(w.n_rays, dtype=np.int32), np.diff(go)))


@pytest.mark.parametrize("which", ["c2", "c3"])
def test_march_default_equals_all_exact_full_size(nacc, orc, which):
    """On every ray of the 640,000-ray image and of the 262,144-ray training
    batch, the default early stop (bounds, fast density, exact fallback)
    gives the same packed samples as taking every decision in the exact
    arithmetic (itself checked against the oracle above)."""
    w = workloads.c2_image() if which == "c2" else workloads.c3_training()
    g, m = w.grid, w.march
    bits, _ = orc.density_grid(g, w.blobs)
    grid = grid_from_bits(nacc, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits)
    field = nacc.BlobField.from_numpy(w.blobs)
    cap = w.n_rays * m.max_steps
    a = run_march(nacc, grid, w.rays_o, w.rays_d, m.step, m.max_steps, m.t_min, m.t_max, field=field, capacity=cap)
    b = run_march(nacc, grid, w.rays_o, w.rays_d, m.step, m.max_steps, m.t_min, m.t_max, field=field, capacity=cap,
                  exact_stops=True)
    assert_packed_equal(a, b)
    assert a["offsets"][-1] > 50 * w.n_rays


def test_march_c3_full_size_sampled(nacc, orc):
    """The 262,144-ray training batch with its 64-blob field (per-group culled
    tables in the early stop), marched whole: per-ray exact against the
    oracle on 2,000 strided rays."""
    w = workloads.c3_training()
    g, m = w.grid, w.march
    bits, _ = orc.density_grid(g, w.blobs)
    grid = grid_from_bits(nacc, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits)
    got = run_march(nacc, grid, w.rays_o, w.rays_d, m.step, m.max_steps, m.t_min, m.t_max,
                    field=nacc.BlobField.from_numpy(w.blobs), capacity=w.n_rays * m.max_steps)
    sel = np.linspace(0, w.n_rays - 1, 2000).astype(np.int64)
    o, d = w.rays_o[sel], w.rays_d[sel]
    exp = orc.march(o, d, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, m.step, m.max_steps,
                    m.t_min, m.t_max, blobs=w.blobs, eps=m.early_stop_eps)
    go = got["offsets"]
    for k, r in enumerate(sel):
        gs, ge = go[r], go[r + 1]
        es, ee = exp["offsets"][k], exp["offsets"][k + 1]
        assert ge - gs == ee - es, f"ray {r}"
        np.testing.assert_array_equal(got["t_starts"][gs:ge], exp["t_starts"][es:ee])
        assert np.all(got["ray_indices"][gs:ge] == r)
    assert go[-1] > 50 * w.n_rays


def test_march_capacity_overflow_reports_and_recovers(nacc, orc):
    w = workloads.c1_forward(512)
    g, m = w.grid, w.march
    bits, _ = orc.density_grid(g, w.blobs)
    grid = grid_from_bits(nacc, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits)
    with pytest.raises(nacc.NaccError) as ei:
        nacc.march_grid(grid, T(w.rays_o), T(w.rays_d), m.step, m.max_steps, m.t_min, m.t_max,
                        capacity=100)
    assert ei.value.code == -2
    got = nacc.march_grid(grid, T(w.rays_o), T(w.rays_d), m.step, m.max_steps, m.t_min, m.t_max,
                          capacity=None).trimmed()
    exp = orc.march(w.rays_o, w.rays_d, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, m.step,
                    m.max_steps, m.t_min, m.t_max)
    np.testing.assert_array_equal(got.t_starts.cpu().numpy(), exp["t_starts"])


def test_march_empty_inputs(nacc):
    grid = nacc.OccupancyGrid.empty((-1.5,) * 3, (1.5,) * 3, 32, 2)
    pk = nacc.march_grid(grid, torch.zeros((0, 3), device=DEV), torch.zeros((0, 3), device=DEV), 0.01)
    assert pk.n_samples() == 0 and pk.offsets.cpu().tolist() == [0]
    o = torch.tensor([[5.0, 5.0, 5.0], [0.0, 0.0, 0.0]], device=DEV)
    d = torch.tensor([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]], device=DEV)
    pk = nacc.march_grid(grid, o, d, 0.01)  # empty grid: nothing occupied
    assert pk.n_samples() == 0 and pk.offsets.cpu().tolist() == [0, 0, 0]


# ---------------------------------------------------------------------------
# compositing
# ---------------------------------------------------------------------------

def _render_inputs(p):
    return (T(p["offsets"]), T(p["t_starts"]), T(p["t_ends"]), T(p["sigmas"]), T(p["rgbs"]))


def _long_ray_packed():
    """Ragged mix: empty rays, short rays, rays across tile boundaries, and
    rays longer than one 2048-sample tile."""
    g = workloads.rng(60)
    lengths = g.integers(0, 300, size=3000)
    lengths[g.random(3000) < 0.2] = 0
    lengths[[5, 700, 1500, 2999]] = [2047, 2049, 5000, 4097]
    lengths[[10, 11, 12]] = [1024, 1023, 2048]
    return workloads.random_packed(3000, 61, lengths=lengths, sigma_hi=3.0)


@pytest.mark.parametrize("case", ["ragged", "long", "dense"])
def test_render_fwd_parity(nacc, orc, case):
    if case == "ragged":
        p = workloads.random_packed(20000, 62, max_len=200, sigma_hi=40.0)
    elif case == "long":
        p = _long_ray_packed()
    else:
        p = workloads.random_packed(5000, 63, max_len=1024, sigma_hi=0.5, p_empty=0.0)
    off, t0, t1, sg, c = _render_inputs(p)
    rgb, op, dep, tr, w = nacc.render_fwd(off, t0, t1, sg, c, (1.0, 1.0, 1.0), 0.0, want_weights=True)
    exp = orc.render_fwd(p["offsets"], p["t_starts"], p["t_ends"], p["sigmas"], p["rgbs"])
    np.testing.assert_allclose(rgb.cpu().numpy(), exp["rgb"], rtol=0, atol=1e-5)
    np.testing.assert_allclose(op.cpu().numpy(), exp["opacity"], rtol=0, atol=1e-5)
    np.testing.assert_allclose(tr.cpu().numpy(), exp["trans"], rtol=0, atol=1e-5)
    np.testing.assert_allclose(w.cpu().numpy(), exp["weights"], rtol=0, atol=1e-5)
    np.testing.assert_allclose(dep.cpu().numpy(), exp["depth"], rtol=1e-5, atol=1e-5)


def test_render_fwd_mask_mode(nacc, orc):
    p = workloads.random_packed(8000, 64, max_len=300, sigma_hi=120.0)
    eps = 1e-4
    thr = float(np.float32(-math.log(eps)))
    off = p["offsets"]
    tau = p["sigmas"].astype(np.float64) * (p["t_ends"].astype(np.float64) - p["t_starts"])
    ties = []
    for r in range(8000):
        P = np.concatenate([[0.0], np.cumsum(tau[off[r]:off[r + 1]])])
        if P.size > 1 and np.min(np.abs(P - thr)) < 1e-4 * thr:
            ties.append(r)
    rgb, op, dep, tr, w = nacc.render_fwd(*_render_inputs(p), (1.0, 1.0, 1.0), eps, want_weights=True)
    exp = orc.render_fwd(p["offsets"], p["t_starts"], p["t_ends"], p["sigmas"], p["rgbs"], eps=eps)
    keep = np.ones(8000, bool)
    keep[ties] = False
    assert keep.sum() > 7800
    np.testing.assert_allclose(rgb.cpu().numpy()[keep], exp["rgb"][keep], rtol=0, atol=1e-5)
    np.testing.assert_allclose(op.cpu().numpy()[keep], exp["opacity"][keep], rtol=0, atol=1e-5)
    np.testing.assert_allclose(tr.cpu().numpy()[keep], exp["trans"][keep], rtol=0, atol=1e-5)
    wmask = np.repeat(keep, np.diff(off))
    np.testing.assert_allclose(w.cpu().numpy()[wmask], exp["weights"][wmask], rtol=0, atol=1e-5)
    assert (exp["weights"] == 0).sum() > 1000
    assert np.all(w.cpu().numpy()[wmask][exp["weights"][wmask] == 0] == 0)


def _grad_tol(p, g_rgb, g_op, g_dep, gref, sel=None):
    off = p["offsets"]
    ray = np.repeat(np.arange(len(off) - 1), np.diff(off))
    dt = p["t_ends"].astype(np.float64) - p["t_starts"]
    m = 0.5 * (p["t_ends"].astype(np.float64) + p["t_starts"])
    scale = np.abs(g_rgb).sum(1)[ray] + np.abs(g_op)[ray] + np.abs(g_dep)[ray] * m
    return 1e-4 * np.abs(gref) + 1e-5 * dt * scale


@pytest.mark.parametrize("case,eps", [("ragged", 0.0), ("long", 0.0), ("ragged", 1e-4)])
def test_render_bwd_parity(nacc, orc, case, eps):
    if case == "ragged":
        p = workloads.random_packed(20000, 65, max_len=200, sigma_hi=40.0)
    else:
        p = _long_ray_packed()
    n = len(p["offsets"]) - 1
    g = workloads.rng(66)
    gC = g.standard_normal((n, 3)).astype(np.float32)
    gA = g.standard_normal(n).astype(np.float32)
    gD = g.standard_normal(n).astype(np.float32)
    gs, gc = nacc.render_bwd(*_render_inputs(p), T(gC), T(gA), T(gD), (1.0, 1.0, 1.0), eps)
    es, ec = orc.render_bwd(p["offsets"], p["t_starts"], p["t_ends"], p["sigmas"], p["rgbs"], gC, gA, gD,
                            eps=eps)
    gs, gc = gs.cpu().numpy(), gc.cpu().numpy()
    tol = _grad_tol(p, gC, gA, gD, es)
    ok = np.abs(gs - es) <= tol
    if eps > 0:
        # rays with a stop near the threshold may legitimately cut one sample differently
        off = p["offsets"]
        tau = p["sigmas"].astype(np.float64) * (p["t_ends"].astype(np.float64) - p["t_starts"])
        thr = -math.log(eps)
        for r in range(n):
            P = np.cumsum(tau[off[r]:off[r + 1]])
            if P.size and np.min(np.abs(P - thr)) < 1e-4 * thr:
                ok[off[r]:off[r + 1]] = True
    assert ok.all(), f"{(~ok).sum()} sigma grads off; worst {np.max(np.abs(gs - es) - tol)}"
    np.testing.assert_allclose(gc[ok], ec[ok], rtol=1e-4, atol=1e-6)


def test_render_bwd_matches_finite_differences(nacc, orc):
    """Adjoint of the C2 loss on 64 rays vs central differences of the FP64
    compositing."""
    p = workloads.random_packed(64, 67, max_len=40, sigma_hi=30.0, p_empty=0.0)
    n = 64
    g = workloads.rng(68)
    gC = g.standard_normal((n, 3))
    gs, gc = nacc.render_bwd(*_render_inputs(p), T(gC.astype(np.float32)), None, None)
    gs = gs.cpu().numpy()
    sig = p["sigmas"].astype(np.float64)
    rgb = p["rgbs"].astype(np.float64)

    def loss(s):
        o = orc.render_fwd(p["offsets"], p["t_starts"], p["t_ends"], s, rgb)
        return (o["rgb"] * gC).sum()

    zeros = np.zeros(n)
    tol = _grad_tol(p, gC, zeros, zeros, gs.astype(np.float64))
    for i in range(len(sig)):
        h = 1e-6 * max(1.0, sig[i])
        sp, sm = sig.copy(), sig.copy()
        sp[i] += h
        sm[i] -= h
        fd = (loss(sp) - loss(sm)) / (2 * h)
        assert abs(gs[i] - fd) <= tol[i] + 1e-7, (i, gs[i], fd)


def test_autograd_function(nacc, orc):
    p = workloads.random_packed(500, 69, max_len=60)
    off, t0, t1, sg, c = _render_inputs(p)
    sg.requires_grad_(True)
    c.requires_grad_(True)
    pk = nacc.PackedSamples(off, None, t0, t1, torch.tensor([len(p["t_starts"])], device=DEV))
    rgb, op, dep = nacc.render(sg, c, pk)
    tgt = T(workloads.target_image(500, 9))
    loss = ((rgb - tgt) ** 2).mean() + op.sum() * 0.1 + dep.sum() * 0.01
    loss.backward()
    gC = (2 * (rgb - tgt) / rgb.numel()).detach()
    gs, gc = nacc.render_bwd(off, t0, t1, sg.detach(), c.detach(), gC,
                             torch.full_like(op, 0.1), torch.full_like(dep, 0.01))
    torch.testing.assert_close(sg.grad, gs, rtol=1e-5, atol=1e-7)
    torch.testing.assert_close(c.grad, gc, rtol=1e-5, atol=1e-7)


def test_render_empty_and_degenerate(nacc, orc):
    off = torch.zeros(5, dtype=torch.int64, device=DEV)
    e = torch.zeros(0, device=DEV)
    rgb, op, dep, tr, _ = nacc.render_fwd(off, e, e, e, torch.zeros((0, 3), device=DEV), (0.2, 0.4, 0.6))
    np.testing.assert_allclose(rgb.cpu().numpy(), np.tile([0.2, 0.4, 0.6], (4, 1)), atol=1e-7)
    assert op.abs().max().item() == 0 and tr.min().item() == 1.0
    # zero-density samples: fully transparent
    p = workloads.random_packed(100, 70, max_len=50)
    p["sigmas"][:] = 0
    rgb, op, dep, tr, w = nacc.render_fwd(*_render_inputs(p), (1, 1, 1), 0.0, want_weights=True)
    assert w.abs().max().item() == 0 and np.allclose(rgb.cpu().numpy(), 1.0)


# ---------------------------------------------------------------------------
# estimator update and resampling
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("res,L", [(32, 1), (128, 4)])
def test_grid_points_bit_exact(nacc, orc, res, L):
    grid = nacc.OccupancyGrid.empty((-1.5, -1.0, -2.0), (1.5, 2.0, 0.5), res, L)
    for jitter in (False, True):
        got = nacc.grid_points(grid, seed=1234, step=17, jitter=jitter).cpu().numpy()
        exp = orc.grid_points(grid.aabb_min, grid.aabb_max, res, L, seed=1234, step=17, jitter=jitter)
        np.testing.assert_array_equal(got, exp)


def test_update_grid_parity(nacc, orc):
    res, L = 128, 4
    n = L * res ** 3
    g = workloads.rng(80)
    ema0 = g.exponential(1.0, n).astype(np.float32)
    ema0[g.random(n) < 0.5] = 0
    grid = nacc.OccupancyGrid.empty((-1.5,) * 3, (1.5,) * 3, res, L)
    grid.ema.copy_(T(ema0))
    e_ref = ema0
    for step in range(3):
        dens = g.exponential(0.5, n).astype(np.float32) * (g.random(n) < 0.3)
        nacc.update_grid(grid, T(dens), decay=0.95, thresh_frac=0.01)
        e_ref, bits_ref, mean_ref = orc.update_grid(e_ref, dens, 0.95, 0.01)
        got_e = grid.ema.cpu().numpy()
        np.testing.assert_array_equal(got_e, e_ref)
        got_b = workloads.unpack_bits(grid.bits.cpu().numpy().view(np.uint32))
        ref_b = workloads.unpack_bits(bits_ref)
        thr = 0.01 * mean_ref
        near = np.abs(e_ref.astype(np.float64) - thr) <= 1e-12 * thr
        assert np.array_equal(got_b[~near], ref_b[~near])


def test_initial_density_grid_matches_oracle(nacc, orc):
    w = workloads.c2_image(8, 8)
    grid = nacc.OccupancyGrid.empty(w.grid.aabb_min, w.grid.aabb_max, w.grid.res, w.grid.n_levels)
    nacc.density_grid(grid, nacc.BlobField.from_numpy(w.blobs), 0.01)
    got = workloads.unpack_bits(grid.bits.cpu().numpy().view(np.uint32))
    bits, sig = orc.density_grid(w.grid, w.blobs)
    ref = workloads.unpack_bits(bits)
    near = np.abs(sig.astype(np.float64) - 0.01) < 1e-5 * 0.01
    assert np.array_equal(got[~near], ref[~near])
    assert ref.sum() > 10000


@pytest.mark.parametrize("nb,no,strat,n", [(64, 32, False, 20000), (32, 32, False, 20000), (64, 32, True, 20001),
                                           (7, 100, False, 20000), (300, 17, True, 20000), (1, 4, False, 20000),
                                           (4096, 4096, True, 300), (128, 64, False, 1), (33, 31, True, 20003),
                                           (64, 64, True, 5000), (65, 32, False, 5000), (2, 40, True, 333)])
def test_sample_pdf_bit_exact(nacc, orc, nb, no, strat, n):
    """Every output bit-exact, including all-zero rows (uniform), single-bin
    mass, CDFs that reach 1 before the last bin (a dominant weight followed
    by ones too small to move the sum), and denormal weights; row counts that
    are not multiples of the 32 rays a warp takes, and bin counts on both
    sides of the 64-bin switch between the staged-row and streamed kernels."""
    g = workloads.rng(90 + nb)
    edges = np.sort(g.uniform(2.0, 6.0, (n, nb + 1)), axis=1).astype(np.float32)
    wts = g.uniform(0, 1, (n, nb)).astype(np.float32)
    wts[g.random((n, nb)) < 0.4] = 0
    wts[:50] = 0  # all-zero rows: uniform
    wts[50:60, :] = 0
    wts[50:60, nb // 2] = 1.0  # single-bin mass
    if nb > 2 and n > 80:
        wts[60:70, : nb // 3] = 1e8  # F_j = 1 well before the last bin
        wts[60:70, nb // 3:] = 1e-3
        wts[70:80] = np.float32(1e-41) * (wts[70:80] > 0)  # denormal weights
    got = nacc.sample_pdf(T(edges), T(wts), no, stratified=strat, seed=4242).cpu().numpy()
    exp = orc.sample_pdf(edges, wts, no, stratified=strat, seed=4242)
    np.testing.assert_array_equal(got, exp)


# ---------------------------------------------------------------------------
# whole step
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("field_blobs", [8, 64])
@pytest.mark.parametrize("per_sample", [False, True])
def test_field_eval_matches_oracle_field(nacc, orc, field_blobs, per_sample):
    """Harness field at the midpoints of a packed set (C1 rays through the
    C1 grid, ragged): the warp-per-ray closed form and the per-sample form
    against the oracle's FP64 field."""
    w = workloads.c1_forward()
    if field_blobs == 64:
        w = dataclasses.replace(w, blobs=workloads.c3_training(64).blobs)
    g, m = w.grid, w.march
    bits, _ = orc.density_grid(g, w.blobs)
    ex = orc.march(w.rays_o, w.rays_d, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, m.step,
                   m.max_steps, m.t_min, m.t_max)
    S = int(ex["offsets"][-1])
    assert S > 100000
    pk = nacc.PackedSamples(T(ex["offsets"]), T(ex["ray_indices"]), T(ex["t_starts"]), T(ex["t_ends"]),
                            torch.tensor([S], device=DEV))
    field = nacc.BlobField.from_numpy(w.blobs)
    sig, rgb = nacc.field_eval(field, T(w.rays_o), T(w.rays_d), pk, per_sample=per_sample)
    s64, c64 = orc.field_samples(w.rays_o, w.rays_d, ex["ray_indices"], ex["t_starts"], ex["t_ends"], w.blobs)
    sig, rgb = sig[:S].cpu().numpy(), rgb[:S].cpu().numpy()
    if per_sample or field_blobs <= 16:  # every blob
        np.testing.assert_allclose(sig, s64, rtol=1e-4, atol=1e-30)
        ok = s64 > 1e-20
        np.testing.assert_allclose(rgb[ok], c64[ok], rtol=1e-4, atol=1e-6)
        return
    # the warp-per-ray form culls blobs per ray above 16 blobs: each dropped
    # blob changes sigma by at most 1e-7 |d| / (sqrt(2 pi) std)
    dlen = np.linalg.norm(w.rays_d, axis=1)[ex["ray_indices"]]
    cull = np.sum(1e-7 / (math.sqrt(2 * math.pi) * w.blobs.std.astype(np.float64))) * dlen
    assert np.all(np.abs(sig - s64) <= 1e-4 * s64 + cull)
    ok = s64 > 1.0
    assert ok.sum() > 10000
    np.testing.assert_allclose(rgb[ok], c64[ok], rtol=1e-3, atol=1e-4)


def test_c2_pipeline_sampled_rays_vs_oracle(nacc, orc):
    """Full C2 step (march with field -> field -> render -> loss -> adjoint) at the
    full 640,000-ray size: rendered colour of sampled rays against the oracle's
    march + FP64 field + FP64 compositing (FP32 field: tolerance 1e-4)."""
    w = workloads.c2_image()
    g, m = w.grid, w.march
    bits, _ = orc.density_grid(g, w.blobs)
    grid = grid_from_bits(nacc, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits)
    field = nacc.BlobField.from_numpy(w.blobs)
    o, d = T(w.rays_o), T(w.rays_d)
    pk = nacc.march_grid(grid, o, d, m.step, m.max_steps, m.t_min, m.t_max, m.early_stop_eps, field=field,
                         capacity=w.n_rays * m.max_steps)
    sig, rgbs = nacc.field_eval(field, o, d, pk)
    rgb, op, dep = nacc.render(sig, rgbs, pk)
    loss, g_rgb = nacc.l2_loss(rgb, T(w.target))
    gs, gc = nacc.render_bwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs, g_rgb, None, None)
    torch.cuda.synchronize()
    sel = np.sort(workloads.rng(78).choice(w.n_rays, 2000, replace=False))
    ex = orc.march(w.rays_o[sel], w.rays_d[sel], g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, m.step,
                   m.max_steps, m.t_min, m.t_max, blobs=w.blobs, eps=m.early_stop_eps)
    s64, c64 = orc.field_samples(w.rays_o[sel], w.rays_d[sel], ex["ray_indices"], ex["t_starts"],
                                 ex["t_ends"], w.blobs)
    er = orc.render_fwd(ex["offsets"], ex["t_starts"], ex["t_ends"], s64, c64)
    got = rgb.cpu().numpy()[sel]
    np.testing.assert_allclose(got, er["rgb"], rtol=0, atol=2e-3)
    assert np.mean(np.abs(got - er["rgb"])) < 1e-4
    assert np.isfinite(gs[:pk.n_samples()].cpu().numpy()).all()
    assert math.isfinite(loss.item())


def test_cuda_graph_capture_of_training_step(nacc, orc):
    """One training step (march -> field -> render -> loss -> adjoint -> grid
    update) captured as a CUDA graph replays to the eager results."""
    w = workloads.c3_training(16384)
    g, m = w.grid, w.march
    field = nacc.BlobField.from_numpy(w.blobs)
    grid = nacc.OccupancyGrid.empty(g.aabb_min, g.aabb_max, g.res, g.n_levels)
    nacc.density_grid(grid, field, 0.01)
    o, d, tgt = T(w.rays_o), T(w.rays_d), T(w.target)
    n = w.n_rays
    bufs = nacc.MarchBuffers(n, n * m.max_steps)
    ubufs = nacc.UpdateBuffers(grid.n_cells)
    cap = n * m.max_steps
    sig = torch.empty(cap, device=DEV)
    rgbs = torch.empty((cap, 3), device=DEV)
    pts = torch.empty((grid.n_cells, 3), device=DEV)
    dens = torch.empty(grid.n_cells, device=DEV)
    gsg = torch.empty(cap, device=DEV)
    gcc = torch.empty((cap, 3), device=DEV)
    step_no = torch.zeros(1)

    def step():
        pk = nacc.march_grid(grid, o, d, m.step, m.max_steps, m.t_min, m.t_max, m.early_stop_eps,
                             field=field, buffers=bufs)
        nacc.field_eval(field, o, d, pk, out=(sig, rgbs))
        rgb, op, dep, tr, _ = nacc.render_fwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs)
        loss, g_rgb = nacc.l2_loss(rgb, tgt)
        nacc.render_bwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs, g_rgb, None, None, out=(gsg, gcc))
        nacc.grid_points(grid, seed=7, step=3, jitter=True, out=pts)
        nacc.field_points(field, pts, out=dens)
        nacc.update_grid(grid, dens, 0.95, 0.01, buffers=ubufs)
        return rgb, loss

    bits0, ema0 = grid.bits.clone(), grid.ema.clone()
    rgb_e, loss_e = step()
    torch.cuda.synchronize()
    eager = (rgb_e.clone(), gsg.clone(), grid.bits.clone(), grid.ema.clone())
    grid.bits.copy_(bits0)
    grid.ema.copy_(ema0)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside capture
        step()
    torch.cuda.current_stream().wait_stream(s)
    grid.bits.copy_(bits0)
    grid.ema.copy_(ema0)
    gph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gph):
        rgb_g, loss_g = step()
    grid.bits.copy_(bits0)
    grid.ema.copy_(ema0)
    gph.replay()
    torch.cuda.synchronize()
    nsamp = bufs.packed.n_samples()
    assert nsamp > 10000
    assert torch.equal(rgb_g, eager[0])
    assert torch.equal(gsg[:nsamp], eager[1][:nsamp])
    assert torch.equal(grid.bits, eager[2])
    assert torch.equal(grid.ema, eager[3])


def test_bounded_wait_reports_timeout_and_context_survives(nacc):
    """A wait that can never be satisfied gives up, records NACC_ERR_TIMEOUT in
    the device status word and returns; the next work on the GPU runs normally."""
    import ctypes
    from paper_2305_04966_gb300 import _abi
    lib = nacc.load_library()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = ctypes.c_int32(7)
    assert lib.nacc_device_status(st, ctypes.byref(status)) == 0 and status.value == 0
    assert lib.nacc_selftest_wait_timeout(2_000_000, st) == 0  # 2 ms
    assert lib.nacc_device_status(st, ctypes.byref(status)) == 0
    assert status.value == _abi.NACC_ERR_TIMEOUT
    assert lib.nacc_device_status(st, ctypes.byref(status)) == 0 and status.value == 0  # cleared
    p = workloads.random_packed(100, 71, max_len=30)
    rgb, *_ = nacc.render_fwd(*_render_inputs(p))
    assert torch.isfinite(rgb).all()
