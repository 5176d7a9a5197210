"""The checkpointed render pair (nacc_render_fwd_ckpt / nacc_render_bwd_ckpt)
against the plain pair, through the C ABI.

The forward pass's per-ray record (chunk carries, mask cut, kept optical
depth) replaces the adjoint's own first sweep; both compute the carries with
the same FP32 operations, so every output must be bit-identical to the plain
pair's, which the parity tests hold against the oracle.  Covered: empty rays,
short rays, rays across the record's 14-chunk limit (where the adjoint falls
back to its own sweep), rays far beyond it, masked and unmasked rendering,
and the full 800x800 image step that the benchmark times.
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


def _both(nacc, p, eps, grads):
    off, t0, t1, sg, c = (T(p[k]) for k in ("offsets", "t_starts", "t_ends", "sigmas", "rgbs"))
    n = off.shape[0] - 1
    ck = nacc.render_ckpt_buffer(n, off.device)
    plain = nacc.render_fwd(off, t0, t1, sg, c, (1.0, 0.5, 0.25), eps, want_weights=True)
    chk = nacc.render_fwd(off, t0, t1, sg, c, (1.0, 0.5, 0.25), eps, want_weights=True, ckpt=ck)
    gC, gA, gD = grads
    gp = nacc.render_bwd(off, t0, t1, sg, c, gC, gA, gD, (1.0, 0.5, 0.25), eps)
    gk = nacc.render_bwd(off, t0, t1, sg, c, gC, gA, gD, (1.0, 0.5, 0.25), eps, ckpt=ck)
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
