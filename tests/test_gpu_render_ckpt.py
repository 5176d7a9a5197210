"""The checkpointed render pair (nacc_render_fwd_ckpt / nacc_render_bwd_ckpt)
against the plain pair, through the C ABI.

The forward pass's per-ray record (chunk carries, mask cut, kept optical
depth) replaces the adjoint's own first sweep; both compute the carries with
the same FP32 operations, so every output must be bit-identical to the plain
pair's, which the parity tests hold against the oracle.  Covered: empty rays,
short rays, rays across the record's 14-chunk limit (where the adjoint falls
back to its own sweep), rays far beyond it, masked and unmasked rendering,
the full 800x800 image step that the benchmark times, the proposal paths'
short rays, and the unbounded scene's long rays.
"""
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


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV)


def _ragged():
    g = workloads.rng(66)
    n = 2500
    lengths = g.integers(0, 700, size=n)
    lengths[g.random(n) < 0.15] = 0
    lengths[:40] = np.arange(1770, 1810)  # the 14-chunk limit at every alignment of the start
    lengths[40:44] = [1, 2, 3, 4]
    lengths[44:47] = [4096, 5000, 8191]
    return workloads.random_packed(n, 67, lengths=lengths, sigma_hi=0.4)


def _both(nacc, p, eps, grads, bg=(1.0, 0.5, 0.25)):
    off, t0, t1, sg, c = (x if torch.is_tensor(x) else T(x)
                          for x in (p[k] for k in ("offsets", "t_starts", "t_ends", "sigmas", "rgbs")))
    n = off.shape[0] - 1
    ck = nacc.render_ckpt_buffer(n, off.device)
    plain = nacc.render_fwd(off, t0, t1, sg, c, bg, eps, want_weights=True)
    chk = nacc.render_fwd(off, t0, t1, sg, c, bg, eps, want_weights=True, ckpt=ck)
    gC, gA, gD = grads
    gp = nacc.render_bwd(off, t0, t1, sg, c, gC, gA, gD, bg, eps)
    gk = nacc.render_bwd(off, t0, t1, sg, c, gC, gA, gD, bg, eps, ckpt=ck)
    torch.cuda.synchronize()
    return plain, chk, gp, gk, ck


@pytest.mark.parametrize("eps", [0.0, 1e-4])
@pytest.mark.parametrize("dense", [False, True])
def test_ckpt_pair_is_bit_identical_to_plain_pair(nacc, eps, dense):
    p = _ragged()
    if dense:  # opaque media: most rays are cut by the mask well inside their samples
        p["sigmas"] = (p["sigmas"] * 300.0).astype(np.float32)
    n = len(p["offsets"]) - 1
    g = workloads.rng(68)
    grads = (T(g.standard_normal((n, 3)).astype(np.float32)), T(g.standard_normal(n).astype(np.float32)),
             T(g.standard_normal(n).astype(np.float32)))
    plain, chk, gp, gk, ck = _both(nacc, p, eps, grads)
    for a, b, name in zip(plain, chk, ("rgb", "opacity", "depth", "trans", "weights")):
        assert torch.equal(a, b), f"forward {name} differs with the checkpoint"
    assert torch.equal(gp[0], gk[0]), "g_sigmas differ with the checkpoint"
    assert torch.equal(gp[1], gk[1]), "g_rgbs differ with the checkpoint"
    # the records: chunk counts, cut positions; absent beyond 14 chunks
    rec = ck.view(torch.int32).view(n, 16).cpu().numpy()
    off = p["offsets"]
    s, e = off[:-1], off[1:]
    nch = np.where(e > s, (e - (s & ~3) + 127) // 128, 0)
    assert (rec[nch > 14, 0] == -1).all() and (nch > 14).sum() >= 10
    ok = nch <= 14
    assert (rec[ok, 0] >= 0).all() and (rec[ok, 0] <= nch[ok]).all()
    assert (rec[ok, 1] >= 0).all() and (rec[ok, 1] <= (e - s)[ok]).all()
    if eps == 0.0:  # no mask: every chunk is kept and the cut is the ray's end
        assert (rec[ok, 0] == nch[ok]).all() and (rec[ok, 1] == (e - s)[ok]).all()
    elif dense:
        assert (rec[ok, 0] < nch[ok]).sum() > 100


def test_ckpt_pair_on_the_full_image_step(nacc):
    """The 800x800 image step as the benchmark runs it (march with early stop,
    field, render, L2 loss, adjoint): the checkpointed pair equals the plain
    pair bit for bit on all 640,000 rays."""
    w = workloads.c2_image()
    g, m = w.grid, w.march
    field = nacc.BlobField.from_numpy(w.blobs)
    grid = nacc.OccupancyGrid.empty(g.aabb_min, g.aabb_max, g.res, g.n_levels)
    nacc.density_grid(grid, field, 0.01)
    o, d = T(w.rays_o), T(w.rays_d)
    pk = nacc.march_grid(grid, o, d, m.step, m.max_steps, m.t_min, m.t_max, m.early_stop_eps, field=field,
                         capacity=w.n_rays * m.max_steps)
    pk = pk.trimmed()
    sig, rgbs = nacc.field_eval(field, o, d, pk)
    ck = nacc.render_ckpt_buffer(w.n_rays, o.device)
    rgb_p, op_p, dep_p, tr_p, _ = nacc.render_fwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs, w.bg, 0.0)
    rgb_k, op_k, dep_k, tr_k, _ = nacc.render_fwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs, w.bg, 0.0,
                                                  ckpt=ck)
    _, g_rgb = nacc.l2_loss(rgb_k, T(w.target))
    gp = nacc.render_bwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs, g_rgb, None, None, w.bg, 0.0)
    gk = nacc.render_bwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs, g_rgb, None, None, w.bg, 0.0, ckpt=ck)
    torch.cuda.synchronize()
    for a, b in ((rgb_p, rgb_k), (op_p, op_k), (dep_p, dep_k), (tr_p, tr_k), (gp[0], gk[0]), (gp[1], gk[1])):
        assert torch.equal(a, b)
    assert pk.n_samples() > 100_000_000


def _subset(p, rows):
    """Packed samples of the rays `rows` (in that order), renumbered."""
    off = p["offsets"]
    lens = off[rows + 1] - off[rows]
    idx = np.concatenate([np.arange(off[r], off[r + 1]) for r in rows]) if lens.sum() else np.zeros(0, np.int64)
    return np.concatenate([[0], np.cumsum(lens)]).astype(np.int64), idx


def test_ckpt_pair_full_image_against_oracle(nacc, orc):
    """All 640,000 rays of the 800x800 image as the benchmark renders them
    (checkpointed pair, white background, no mask): the oracle's own packed
    samples (its march with the early stop) and its FP64 field rounded to FP32
    are the inputs on both sides.  On 4,000 seeded rays, rgb, opacity and
    T_N match the oracle's FP64 compositing within 1e-5 absolute and depth
    within 1e-5 relative; their sigma gradients within 1e-4 relative (with the
    absolute floor of the parity tests at the natural scale of the terms that
    cancel) and colour gradients within 1e-4 relative, for seeded upstream
    gradients of colour, opacity and depth."""
    w = workloads.c2_image()
    g, m = w.grid, w.march
    bits, _ = orc.density_grid(g, w.blobs)
    pk = orc.march(w.rays_o, w.rays_d, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, m.step, m.max_steps,
                   m.t_min, m.t_max, blobs=w.blobs, eps=m.early_stop_eps)
    S = int(pk["offsets"][-1])
    assert S > 100_000_000
    sig64, rgb64 = orc.field_samples(w.rays_o, w.rays_d, pk["ray_indices"], pk["t_starts"], pk["t_ends"], w.blobs)
    p = dict(offsets=pk["offsets"], t_starts=pk["t_starts"], t_ends=pk["t_ends"],
             sigmas=sig64.astype(np.float32), rgbs=rgb64.astype(np.float32))
    del sig64, rgb64, pk
    n = w.n_rays
    gen = workloads.rng(90)
    gC = gen.standard_normal((n, 3)).astype(np.float32)
    gA = gen.standard_normal(n).astype(np.float32)
    gD = gen.standard_normal(n).astype(np.float32)
    off, t0, t1, sg, c = (T(p[k]) for k in ("offsets", "t_starts", "t_ends", "sigmas", "rgbs"))
    ck = nacc.render_ckpt_buffer(n, off.device)
    rgb, op, dep, tr, _ = nacc.render_fwd(off, t0, t1, sg, c, w.bg, 0.0, ckpt=ck)
    gs, gc = nacc.render_bwd(off, t0, t1, sg, c, T(gC), T(gA), T(gD), w.bg, 0.0, ckpt=ck)
    torch.cuda.synchronize()
    rgb, op, dep, tr = (x.cpu().numpy() for x in (rgb, op, dep, tr))
    rows = np.sort(workloads.rng(91).choice(n, 4000, replace=False))
    soff, idx = _subset(p, rows)
    gs, gc = gs[T(idx)].cpu().numpy(), gc[T(idx)].cpu().numpy()
    del off, t0, t1, sg, c, ck
    torch.cuda.empty_cache()
    sub = dict(offsets=soff, t_starts=p["t_starts"][idx], t_ends=p["t_ends"][idx], sigmas=p["sigmas"][idx],
               rgbs=p["rgbs"][idx])
    assert (np.diff(soff) > 0).sum() > 1000  # many of the sampled rays hit the blobs
    exp = orc.render_fwd(sub["offsets"], sub["t_starts"], sub["t_ends"], sub["sigmas"], sub["rgbs"], w.bg)
    np.testing.assert_allclose(rgb[rows], exp["rgb"], rtol=0, atol=1e-5)
    np.testing.assert_allclose(op[rows], exp["opacity"], rtol=0, atol=1e-5)
    np.testing.assert_allclose(tr[rows], exp["trans"], rtol=0, atol=1e-5)
    np.testing.assert_allclose(dep[rows], exp["depth"], rtol=1e-5, atol=1e-5)
    es, ec = orc.render_bwd(sub["offsets"], sub["t_starts"], sub["t_ends"], sub["sigmas"], sub["rgbs"], gC[rows],
                            gA[rows], gD[rows], w.bg)
    ray = np.repeat(np.arange(len(rows)), np.diff(soff))
    dt = sub["t_ends"].astype(np.float64) - sub["t_starts"]
    mid = 0.5 * (sub["t_ends"].astype(np.float64) + sub["t_starts"])
    scale = np.abs(gC[rows]).sum(1)[ray] + np.abs(gA[rows])[ray] + np.abs(gD[rows])[ray] * mid
    tol = 1e-4 * np.abs(es) + 1e-5 * dt * scale
    bad = np.abs(gs - es) > tol
    assert not bad.any(), f"{bad.sum()} sigma gradients off; worst excess {np.max(np.abs(gs - es) - tol)}"
    np.testing.assert_allclose(gc, ec, rtol=1e-4, atol=1e-6)


def _assert_pair_identical(nacc, o, d, field, pk, bg, eps, seed):
    """Field at the samples, then the plain and the checkpointed pair on them
    with seeded upstream gradients of colour, opacity and depth: every output
    bit-identical.  Returns the per-ray sample counts."""
    pk = pk.trimmed()
    sig, rgbs = nacc.field_eval(field, o, d, pk)
    n = pk.offsets.shape[0] - 1
    g = workloads.rng(seed)
    grads = (T(g.standard_normal((n, 3)).astype(np.float32)), T(g.standard_normal(n).astype(np.float32)),
             T(g.standard_normal(n).astype(np.float32)))
    plain, chk, gp, gk, _ = _both(nacc, dict(offsets=pk.offsets, t_starts=pk.t_starts, t_ends=pk.t_ends,
                                             sigmas=sig, rgbs=rgbs), eps, grads, bg=bg)
    for a, b, name in zip(plain, chk, ("rgb", "opacity", "depth", "trans", "weights")):
        assert torch.equal(a, b), f"forward {name} differs with the checkpoint"
    assert torch.equal(gp[0], gk[0]) and torch.equal(gp[1], gk[1])
    return np.diff(pk.offsets.cpu().numpy())


@pytest.mark.parametrize("eps", [0.0, 1e-4])
def test_ckpt_pair_on_proposal_rays(nacc, eps):
    """Short rays of the learned-proposal paths (32 and 128 final samples per
    ray, scene-box bins and the grid's occupied range) on 32,768 rays of the
    training batch with its 64-blob field."""
    w = workloads.c3_training(32768)
    g, m = w.grid, w.march
    field = nacc.BlobField.from_numpy(w.blobs)
    grid = nacc.OccupancyGrid.empty(g.aabb_min, g.aabb_max, g.res, g.n_levels)
    nacc.density_grid(grid, field, 0.01)
    box = nacc.OccupancyGrid.empty(g.aabb_min, g.aabb_max, 32, 1)
    mlp = nacc.ProposalMLP.init(seed=11)
    o, d = T(w.rays_o), T(w.rays_d)
    n = w.n_rays
    for rounds, nf in (((64, 32), 32), ((256, 128), 128)):
        smp = nacc.ProposalSampler(mlp, box, n, rounds=rounds, n_final=nf)
        lens = _assert_pair_identical(nacc, o, d, field, smp.sample(o, d, m.t_min, m.t_max), w.bg, eps, 92)
        assert (lens == nf).all()
    comb = nacc.CombinedSampler(mlp, grid, n, m.step, m.max_steps, rounds=(64, 32), n_final=32)
    lens = _assert_pair_identical(nacc, o, d, field, comb.sample(o, d, m.t_min, m.t_max), w.bg, eps, 93)
    assert set(np.unique(lens)) <= {0, 32}


def test_ckpt_pair_on_unbounded_long_rays(nacc):
    """One 1024x256 camera of the unbounded scene (256 blobs over radius 20,
    4x256^3 grid over the contracted space): the s-lattice march at K = 2048
    with the early stop on the grid from the field, and on a fully occupied
    grid without it, whose 2048-sample rays run past the record's 14-chunk
    limit (the adjoint's own sweep); and the unbounded proposal sampler's
    128-sample rays."""
    w = workloads.c5_unbounded(n_cams=1)
    g, m = w.grid, w.march
    field = nacc.BlobField.from_numpy(w.blobs)
    grid = nacc.OccupancyGrid.empty(g.aabb_min, g.aabb_max, g.res, g.n_levels)
    nacc.density_grid_unbounded(grid, field, 0.01)
    o, d = T(w.rays_o), T(w.rays_d)
    # the grid from the field, with the early stop, at K = 2048
    pk = nacc.march_unbounded(grid, o, d, 2048, m.t_min, m.t_max, m.early_stop_eps, field=field)
    lens = _assert_pair_identical(nacc, o, d, field, pk, w.bg, 0.0, 94)
    assert (lens > 128).sum() > 1000  # several chunks
    del pk
    # every cell occupied, no early stop: all 2048 lattice points of every
    # ray, 16 chunks, past the record's 14-chunk limit
    full = nacc.OccupancyGrid.empty(g.aabb_min, g.aabb_max, g.res, g.n_levels)
    full.bits.fill_(-1)
    pk = nacc.march_unbounded(full, o, d, 2048, m.t_min, m.t_max, m.early_stop_eps)
    lens = _assert_pair_identical(nacc, o, d, field, pk, w.bg, 1e-4, 96)
    assert (lens == 2048).all()
    del pk, full
    mlp = nacc.ProposalMLP.init(seed=12)
    smp = nacc.UnboundedProposalSampler(mlp, w.n_rays, m.t_min, m.t_max, rounds=(256, 128), n_final=128)
    lens = _assert_pair_identical(nacc, o, d, field, smp.sample(o, d), w.bg, 1e-4, 95)
    assert (lens == 128).all()
