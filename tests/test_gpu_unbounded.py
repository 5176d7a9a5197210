"""GPU parity of the unbounded-scene march (Sec. 3.2): s-lattice uniform in
[0, 1], disparity-linear map to [t_near, t_far], occupancy of the contracted
midpoint.

Bars: the packed samples are bit-exact against the oracle on every ray,
with and without the field's early stop (the march reaches the
definition's FP32 stopping decision exactly; rays whose depth comes near the
threshold are counted and reported, not exempted).
"""
import math

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


def _T(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).to(DEV)


def _grid(nacc, g, bits):
    return nacc.OccupancyGrid(tuple(g.aabb_min), tuple(g.aabb_max), g.res, g.n_levels,
                              _T(bits.view(np.int32), torch.int32))


def _run(nacc, grid, w, K, field=None, capacity=None, with_ray_indices=True, exact_stops=False):
    pk = nacc.march_unbounded(grid, _T(w.rays_o), _T(w.rays_d), K, w.march.t_min, w.march.t_max,
                              w.march.early_stop_eps, field=field, capacity=capacity,
                              with_ray_indices=with_ray_indices, exact_stops=exact_stops)
    torch.cuda.synchronize()
    pk = pk.trimmed()
    return dict(offsets=pk.offsets.cpu().numpy(),
                ray_indices=None if pk.ray_indices is None else pk.ray_indices.cpu().numpy(),
                t_starts=pk.t_starts.cpu().numpy(), t_ends=pk.t_ends.cpu().numpy())


def _oracle(orc, w, bits, K, blobs=None):
    g, m = w.grid, w.march
    return orc.march_unbounded(w.rays_o, w.rays_d, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, K,
                               m.t_min, m.t_max, blobs=blobs, eps=m.early_stop_eps)


def _equal(got, exp, rays=None):
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


@pytest.fixture(scope="module")
def small_c5(orc):
    """Two 64x16 cameras of the 16-camera ring, grid 4 x 32^3 over the contracted cube."""
    w = workloads.c5_unbounded(n_cams=2, width=64, height=16, res=32)
    bits, _ = orc.density_grid_contracted(w.grid, w.blobs)
    return w, bits


@pytest.mark.parametrize("K", [1024, 333])
def test_unbounded_no_field_bit_exact(nacc, orc, small_c5, K):
    w, bits = small_c5
    got = _run(nacc, _grid(nacc, w.grid, bits), w, K, field=None)
    exp = _oracle(orc, w, bits, K)
    assert exp["offsets"][-1] > 10 * w.n_rays
    _equal(got, exp)


@pytest.mark.parametrize("res,L,seed", [(16, 4, 1), (20, 3, 2), (32, 1, 3)])
def test_unbounded_random_grids_bit_exact(nacc, orc, res, L, seed):
    """Random block-structured occupancy over the contracted cube; rays from
    inside and outside the unit cube, axis-aligned and zero directions."""
    bits = workloads.random_bitfield(L, res, 500 + seed, p_block=0.3, block=4 if res % 4 == 0 else 5, p_cell=0.6)
    g = workloads.rng(600 + seed)
    n = 3000
    o = workloads._normalise(g.standard_normal((n, 3))) * g.uniform(0.0, 30.0, size=(n, 1))
    d = workloads._normalise(g.standard_normal((n, 3)))
    d[:30] = 0.0
    d[np.arange(30), np.arange(30) % 3] = np.where(np.arange(30) % 2 == 0, 1.0, -1.0)
    d[30:40] = 0.0  # degenerate direction: every sample at the origin
    w = workloads.Workload("random", o.astype(np.float32), d.astype(np.float32), None,
                           workloads.GridSpec((-0.5,) * 3, (0.5,) * 3, res, L),
                           workloads.MarchSpec(0.0, 512, 0.05, 500.0, 1e-4))
    got = _run(nacc, _grid(nacc, w.grid, bits), w, 512)
    exp = _oracle(orc, w, bits, 512)
    assert exp["offsets"][-1] > 1000
    _equal(got, exp)


def _runs(packed, t_lattice):
    """Number of runs of consecutive lattice points of each ray's samples."""
    k = np.searchsorted(t_lattice, packed["t_starts"])
    off = packed["offsets"]
    return np.array([1 + int(np.count_nonzero(np.diff(k[off[r]:off[r + 1]]) != 1)) if off[r + 1] > off[r] else 0
                     for r in range(len(off) - 1)])


def test_unbounded_many_runs_bit_exact(nacc, orc):
    """A fine random grid breaks rays into many runs: rays whose runs fit the
    count pass's record (16) and rays that overflow it (re-walked) both match."""
    res, L = 64, 3
    g = workloads.rng(4343)
    occ = g.random((L, res, res, res)) < 0.5
    occ[:, : res // 2] = True
    bits = workloads.pack_bits(occ.reshape(-1))
    n = 2048
    o = workloads._normalise(g.standard_normal((n, 3))) * g.uniform(0.0, 3.0, size=(n, 1))
    d = workloads._normalise(g.standard_normal((n, 3)))
    K = 768
    w = workloads.Workload("runs", o.astype(np.float32), d.astype(np.float32), None,
                           workloads.GridSpec((-0.5,) * 3, (0.5,) * 3, res, L),
                           workloads.MarchSpec(0.0, K, 0.05, 100.0, 1e-4))
    got = _run(nacc, _grid(nacc, w.grid, bits), w, K)
    exp = _oracle(orc, w, bits, K)
    s = (np.arange(K + 1, dtype=np.float32) / np.float32(K)).astype(np.float32)
    runs = _runs(exp, orc.s_to_t(s, 0.05, 100.0))
    assert np.count_nonzero(runs > 16) > 100 and np.count_nonzero((runs > 0) & (runs <= 16)) > 100
    _equal(got, exp)


def test_unbounded_full_grid_is_the_s_lattice(nacc, orc, small_c5):
    """All-occupied grid: every ray gets all K samples, t_k = Phi(k / K)."""
    w, bits = small_c5
    K = 256
    full = np.full_like(bits, 0xFFFFFFFF)
    got = _run(nacc, _grid(nacc, w.grid, full), w, K)
    assert np.array_equal(np.diff(got["offsets"]), np.full(w.n_rays, K))
    s = (np.arange(K + 1, dtype=np.float32) / np.float32(K)).astype(np.float32)
    t = orc.s_to_t(s, w.march.t_min, w.march.t_max)
    np.testing.assert_array_equal(got["t_starts"].reshape(w.n_rays, K), np.broadcast_to(t[:-1], (w.n_rays, K)))
    np.testing.assert_array_equal(got["t_ends"].reshape(w.n_rays, K), np.broadcast_to(t[1:], (w.n_rays, K)))


def _near_threshold(orc, w, full, thr, rels=(1e-4, 1e-5, 1e-6)):
    """Rays whose optical depth (FP64 field) before some sample lies within
    `rel` of the threshold, where an FP32 evaluation could take either side:
    counted and printed (they are bit-exact like the rest)."""
    sig, _ = orc.field_samples(w.rays_o, w.rays_d, full["ray_indices"], full["t_starts"], full["t_ends"], w.blobs)
    tau = sig * (full["t_ends"].astype(np.float64) - full["t_starts"])
    off = full["offsets"]
    dist = np.full(len(off) - 1, np.inf)
    for r in range(len(off) - 1):
        P = np.cumsum(tau[off[r]:off[r + 1]])
        if P.size:
            dist[r] = np.min(np.abs(P - thr)) / thr
    n = len(off) - 1
    c = {rel: int(np.count_nonzero(dist < rel)) for rel in rels}
    print("rays near the early-stop threshold (all bit-exact): " +
          ", ".join(f"within {rel:g}: {k} ({1e6 * k / n:.0f} per million)" for rel, k in c.items()))
    return c


def _check_early_stop(nacc, orc, w, bits, K):
    grid = _grid(nacc, w.grid, bits)
    field = nacc.BlobField.from_numpy(w.blobs)
    got = _run(nacc, grid, w, K, field=field)
    got_x = _run(nacc, grid, w, K, field=field, exact_stops=True)
    exp = _oracle(orc, w, bits, K, blobs=w.blobs)
    full = _oracle(orc, w, bits, K)
    _equal(got, exp)
    _equal(got_x, exp)
    _near_threshold(orc, w, full, -math.log(w.march.early_stop_eps))
    ec = np.diff(exp["offsets"])
    stopped = int((ec < np.diff(full["offsets"])).sum())
    assert stopped > 0.2 * w.n_rays
    return stopped


def test_unbounded_early_stop_culled_table(nacc, orc, small_c5):
    """The ring workload's 256-blob field: each ray keeps 16-42 blobs in its table."""
    w, bits = small_c5
    _check_early_stop(nacc, orc, w, bits, 1024)


def test_unbounded_early_stop_dense_field_direct_sum(nacc, orc):
    """256 blobs packed within radius 2.5: most rays keep more than the table
    holds and sum every blob per sample."""
    w = workloads.c5_unbounded(n_cams=2, width=32, height=16, res=32)
    blobs = workloads.ball_blob_field(256, 7, radius=2.5, std_lo=0.15, std_hi=0.3, peak=20.0)
    w = workloads.dataclasses.replace(w, blobs=blobs)
    # same culling bound as the kernel, in FP64: rays with more than 48 blobs
    o, d = w.rays_o.astype(np.float64), w.rays_d.astype(np.float64)
    mu, sd, pk = blobs.mu.astype(np.float64), blobs.std.astype(np.float64), blobs.peak.astype(np.float64)
    rel = mu[None] - o[:, None]
    pp = (np.cross(rel, np.broadcast_to(d[:, None], rel.shape)) ** 2).sum(-1) / (d * d).sum(1)[:, None]
    bound = pk[None] * np.exp(-pp / (2 * sd[None] ** 2)) * math.sqrt(2 * math.pi) * sd[None]
    assert (bound > 1e-7).sum(1).max() > 60
    bits, _ = orc.density_grid_contracted(w.grid, blobs)
    _check_early_stop(nacc, orc, w, bits, 512)


def test_unbounded_capacity_and_empty(nacc, orc, small_c5):
    w, bits = small_c5
    grid = _grid(nacc, w.grid, bits)
    exp = _oracle(orc, w, bits, 1024)
    S = int(exp["offsets"][-1])
    with pytest.raises(nacc.NaccError):
        _run(nacc, grid, w, 1024, capacity=S - 1)
    got = _run(nacc, grid, w, 1024, capacity=S)
    _equal(got, exp)
    got = _run(nacc, grid, w, 1024, with_ray_indices=False)
    np.testing.assert_array_equal(got["t_starts"], exp["t_starts"])
    empty = workloads.dataclasses.replace(w, rays_o=w.rays_o[:0], rays_d=w.rays_d[:0])
    got = _run(nacc, grid, empty, 1024)
    assert got["offsets"].tolist() == [0] and got["t_starts"].size == 0


def test_uncontract_points_bit_exact(nacc, orc):
    g0 = np.random.default_rng(11)
    c = g0.uniform(-2.05, 2.05, (100003, 3)).astype(np.float32)
    c[:5] = [[2.0, 0.0, 0.0], [0.3, -2.0, 1.0], [1.0, 1.0, 1.0], [0.0, 0.0, 0.0], [-1.0000001, 0.2, 0.1]]
    got = nacc.uncontract_points(_T(c)).cpu().numpy()
    np.testing.assert_array_equal(got, orc.uncontract32(c))
    assert nacc.uncontract_points(_T(c[:0])).shape == (0, 3)


def test_density_grid_unbounded_matches_oracle(nacc, orc, small_c5):
    """Grid over the contracted space from the field at the scene points of
    the cell centres: bits exact except cells whose density is within 1e-5
    (relative) of the threshold (FP32 field on the device, FP64 in the oracle)."""
    w, bits = small_c5
    _, sig = orc.density_grid_contracted(w.grid, w.blobs)
    grid = nacc.OccupancyGrid.empty(w.grid.aabb_min, w.grid.aabb_max, w.grid.res, w.grid.n_levels)
    nacc.density_grid_unbounded(grid, nacc.BlobField.from_numpy(w.blobs), 0.01)
    got = workloads.unpack_bits(grid.bits.cpu().numpy().view(np.uint32))
    ref = workloads.unpack_bits(bits)
    near = np.abs(sig - 0.01) < 1e-5 * 0.01
    assert np.array_equal(got[~near], ref[~near])
    assert 0.02 < ref.mean() < 0.5


# ---------------------------------------------------------------------------
# learned proposal for unbounded scenes
# ---------------------------------------------------------------------------

def test_contract_points_bit_exact(nacc, orc):
    g0 = np.random.default_rng(12)
    x = (g0.standard_normal((50001, 3)) * g0.lognormal(0.0, 2.0, (50001, 1))).astype(np.float32)
    x[:4] = [[1.0, -1.0, 0.5], [0.0, 0.0, 0.0], [1.0000001, 0.0, 0.0], [-3e7, 1.0, 2.0]]
    got = nacc.contract_points(_T(x)).cpu().numpy()
    np.testing.assert_array_equal(got, orc.contract(x))


@pytest.mark.parametrize("nb", [1, 64, 1000])
def test_phi_edges_bit_exact(nacc, orc, nb):
    e = nacc.phi_edges(37, nb, 0.2, 1000.0).cpu().numpy()
    s = (np.arange(nb + 1, dtype=np.float32) / np.float32(nb)).astype(np.float32)
    row = orc.s_to_t(s, 0.2, 1000.0)
    np.testing.assert_array_equal(e, np.broadcast_to(row, (37, nb + 1)))


def _proposal_params(seed):
    from oracle import proposal as P
    p = P.init_params(seed)
    g = np.random.default_rng(seed + 1)
    p["b1"] = g.uniform(-0.3, 0.3, 64).astype(np.float32)
    p["b2"] = g.uniform(-0.3, 0.3, 64).astype(np.float32)
    p["b3"] = np.array([0.2], np.float32)
    flat = np.concatenate([p["W1"].reshape(-1), p["b1"], p["W2"].reshape(-1), p["b2"], p["w3"], p["b3"]])
    return p, flat.astype(np.float32)


def _contracted_midpoints(orc, o, d, e):
    """FP32 midpoints o + d t (t = (e_j + e_j+1) / 2, one FMA per axis as the
    kernel's point source) then the oracle's FP32 contraction."""
    t = (0.5 * (e[:, :-1].astype(np.float64) + e[:, 1:])).astype(np.float32)
    x = (o[:, None, :].astype(np.float64) + d[:, None, :].astype(np.float64) * t[:, :, None]).astype(np.float32)
    return orc.contract(x.reshape(-1, 3))


def test_forward_rays_contracted_matches_oracle(nacc, orc, small_c5):
    from oracle import proposal as P
    w, _ = small_c5
    o, d = w.rays_o[:1024], w.rays_d[:1024]
    p, flat = _proposal_params(120)
    mlp = nacc.ProposalMLP(_T(flat))
    e = nacc.phi_edges(o.shape[0], 64, w.march.t_min, w.march.t_max).cpu().numpy()
    got = mlp.forward_rays(_T(o), _T(d), _T(e), contracted=True).cpu().numpy().reshape(-1)
    c = _contracted_midpoints(orc, o, d, e)
    assert np.abs(c).max() < 2.0 and np.abs(c).max() > 1.9
    exp = P.forward(p, c)["sigma"]
    rel = np.abs(got - exp) / np.maximum(np.abs(exp), 1e-3)
    assert np.median(rel) < 1e-4 and np.mean(rel) < 3e-3 and rel.max() < 5e-2, (np.median(rel), rel.mean(), rel.max())


def test_unbounded_sampler_matches_oracle_composition(nacc, orc, small_c5):
    """Phi bins (64) -> contracted proposal density -> weights -> inverse CDF
    (32) -> again -> 32 final bins, against the same chain of oracle functions."""
    from oracle import proposal as P
    w, _ = small_c5
    o, d = w.rays_o[:1536], w.rays_d[:1536]
    n = o.shape[0]
    p, flat = _proposal_params(121)
    p["b3"] = np.array([-1.0], np.float32)
    flat[-1] = -1.0
    mlp = nacc.ProposalMLP(_T(flat))
    sampler = nacc.UnboundedProposalSampler(mlp, n, w.march.t_min, w.march.t_max, rounds=(64, 32), n_final=32,
                                            device=DEV)
    pk = sampler.sample(_T(o), _T(d))
    got = np.stack([pk.t_starts.cpu().numpy().reshape(n, 32), pk.t_ends.cpu().numpy().reshape(n, 32)])
    s = (np.arange(65, dtype=np.float32) / np.float32(64)).astype(np.float32)
    e = np.broadcast_to(orc.s_to_t(s, w.march.t_min, w.march.t_max), (n, 65)).astype(np.float32)
    for nb, n_next in ((64, 32), (32, 32)):
        sg = P.forward(p, _contracted_midpoints(orc, o, d, e))["sigma"]
        off = np.arange(n + 1, dtype=np.int64) * nb
        wts = orc.render_fwd(off, e[:, :-1].reshape(-1), e[:, 1:].reshape(-1), sg, np.zeros((n * nb, 3)))["weights"]
        e = orc.sample_pdf(e, wts.reshape(n, nb).astype(np.float32), n_next)
    exp = np.stack([e[:, :-1], e[:, 1:]])

    def s_of(t):  # inverse of Phi, in FP64: the bins' positions in s
        a, b = 1.0 / w.march.t_min, 1.0 / w.march.t_max
        return (1.0 / t.astype(np.float64) - a) / (b - a)

    err = np.abs(s_of(got) - s_of(exp))
    assert np.quantile(err, 0.99) < 2e-3 and err.mean() < 2e-4, (np.quantile(err, 0.99), err.mean(), err.max())


def test_field_eval_culled_256_blobs(nacc, orc, small_c5):
    """The harness field with the unbounded scene's 256 blobs (per-ray culling
    above 64 blobs) against the oracle's FP64 field on the oracle's samples:
    sigma within 1e-4 relative plus the culling bound (1e-7 |d| / (sqrt(2 pi)
    std) per dropped blob, summed over all blobs), colour where sigma > 1."""
    w, bits = small_c5
    ex = _oracle(orc, w, bits, 1024)
    S = int(ex["offsets"][-1])
    pk = nacc.PackedSamples(_T(ex["offsets"]), _T(ex["ray_indices"]), _T(ex["t_starts"]), _T(ex["t_ends"]),
                            torch.tensor([S], device=DEV))
    sig, rgb = nacc.field_eval(nacc.BlobField.from_numpy(w.blobs), _T(w.rays_o), _T(w.rays_d), pk)
    s64, c64 = orc.field_samples(w.rays_o, w.rays_d, ex["ray_indices"], ex["t_starts"], ex["t_ends"], w.blobs)
    sig, rgb = sig[:S].cpu().numpy(), rgb[:S].cpu().numpy()
    dlen = np.linalg.norm(w.rays_d, axis=1)[ex["ray_indices"]]
    cull = np.sum(1e-7 / (math.sqrt(2 * math.pi) * w.blobs.std.astype(np.float64))) * dlen
    assert np.all(np.abs(sig - s64) <= 1e-4 * s64 + cull), np.max(np.abs(sig - s64) - 1e-4 * s64 - cull)
    ok = s64 > 1.0
    assert ok.sum() > 1000
    np.testing.assert_allclose(rgb[ok], c64[ok], rtol=1e-3, atol=1e-4)


def _gather_rays(pk, rays):
    """Samples of the given rays of a device-resident packed set, copied out
    ray by ray (the full set is too large to copy)."""
    off = pk.offsets.cpu().numpy()
    idx = np.concatenate([np.arange(off[r], off[r + 1]) for r in rays]).astype(np.int64)
    it = torch.as_tensor(idx, device=DEV)
    cnt = np.array([off[r + 1] - off[r] for r in rays], np.int64)
    return dict(offsets=np.concatenate([[0], np.cumsum(cnt)]), t_starts=pk.t_starts[it].cpu().numpy(),
                t_ends=pk.t_ends[it].cpu().numpy(), ray_indices=pk.ray_indices[it].cpu().numpy())


def test_unbounded_full_size_sampled(nacc, orc):
    """The 4,194,304-ray workload on a full 4 x 256^3 grid over the contracted
    space (seeded block-structured bits: building the field's grid on the CPU
    would take minutes), marched whole on the GPU as the bench launches it;
    3,000 strided rays compared with the oracle, bit-exact with and without
    the 256-blob field; with the field, the default early stop also equals
    the all-exact one on every ray."""
    w = workloads.c5_unbounded()
    g, m = w.grid, w.march
    bits = workloads.random_bitfield(g.n_levels, g.res, 505, p_block=0.15, block=8, p_cell=0.7)
    grid = _grid(nacc, g, bits)
    o, d = _T(w.rays_o), _T(w.rays_d)
    sel = np.linspace(0, w.n_rays - 1, 3000).astype(np.int64)
    sub = workloads.dataclasses.replace(w, rays_o=np.ascontiguousarray(w.rays_o[sel]),
                                        rays_d=np.ascontiguousarray(w.rays_d[sel]),
                                        target=None)
    full = _oracle(orc, sub, bits, m.max_steps)
    for field in (None, nacc.BlobField.from_numpy(w.blobs)):
        pk = nacc.march_unbounded(grid, o, d, m.max_steps, m.t_min, m.t_max, m.early_stop_eps, field=field)
        torch.cuda.synchronize()
        got = _gather_rays(pk, sel)
        got["ray_indices"] = np.repeat(np.arange(len(sel), dtype=np.int32), np.diff(got["offsets"]))
        if field is None:
            assert pk.n_samples() > 50 * w.n_rays
            _equal(got, full)
            continue
        exp = _oracle(orc, sub, bits, m.max_steps, blobs=w.blobs)
        _equal(got, exp)
        _near_threshold(orc, sub, full, -math.log(m.early_stop_eps))
        off_a = pk.offsets.cpu().numpy()
        t0_a = pk.t_starts[: int(off_a[-1])].cpu().numpy()
        del pk
        torch.cuda.empty_cache()
        pk = nacc.march_unbounded(grid, o, d, m.max_steps, m.t_min, m.t_max, m.early_stop_eps, field=field,
                                  exact_stops=True)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(pk.offsets.cpu().numpy(), off_a)
        np.testing.assert_array_equal(pk.t_starts[: int(off_a[-1])].cpu().numpy(), t0_a)
        del pk
        torch.cuda.empty_cache()


def test_unbounded_early_stop_table_overflow_direct_sum(nacc, orc):
    """320 wide blobs within radius 2: more than half the rays keep more than
    the 256 table entries of the early-stop pass and sum every blob per point."""
    w = workloads.c5_unbounded(n_cams=1, width=32, height=16, res=32)
    blobs = workloads.ball_blob_field(320, 9, radius=2.0, std_lo=0.3, std_hi=0.5, peak=2.0)
    w = workloads.dataclasses.replace(w, blobs=blobs)
    o, d = w.rays_o.astype(np.float64), w.rays_d.astype(np.float64)
    mu, sd, pk = blobs.mu.astype(np.float64), blobs.std.astype(np.float64), blobs.peak.astype(np.float64)
    rel = mu[None] - o[:, None]
    pp = (np.cross(rel, np.broadcast_to(d[:, None], rel.shape)) ** 2).sum(-1) / (d * d).sum(1)[:, None]
    bound = pk[None] * np.exp(-pp / (2 * sd[None] ** 2)) * math.sqrt(2 * math.pi) * sd[None]
    assert ((bound > 1e-7).sum(1) > 256).mean() > 0.3
    bits, _ = orc.density_grid_contracted(w.grid, blobs)
    _check_early_stop(nacc, orc, w, bits, 256)
