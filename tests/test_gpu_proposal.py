"""Proposal network on the GPU (tcgen05 kernels) against the oracle
(oracle/proposal.py): encoding, forward, fused adjoint, Adam, training."""
import math

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def nacc():
    import paper_2305_04966_gb300 as m
    from paper_2305_04966_gb300 import build
    build.build()
    return m


@pytest.fixture(scope="module")
def P():
    from oracle import proposal
    return proposal


def _flat(p):
    """oracle parameter dict -> the library's FP32 layout"""
    return np.concatenate([p["W1"].reshape(-1), p["b1"], p["W2"].reshape(-1), p["b2"], p["w3"], p["b3"]]).astype(np.float32)


def _unflat(a):
    a = np.asarray(a, np.float64)
    return {"W1": a[0:4096].reshape(64, 64), "b1": a[4096:4160], "W2": a[4160:8256].reshape(64, 64),
            "b2": a[8256:8320], "w3": a[8320:8384], "b3": a[8384:8385]}


def _params(P, seed):
    p = P.init_params(seed)
    g = np.random.default_rng(seed + 1)
    p["b1"] = g.uniform(-0.3, 0.3, 64).astype(np.float32)
    p["b2"] = g.uniform(-0.3, 0.3, 64).astype(np.float32)
    p["b3"] = np.array([0.2], np.float32)
    return p


def _points(n, seed):
    return workloads.rng(seed).uniform(-1.5, 1.5, (n, 3)).astype(np.float32)


def test_encoding_matches_oracle(nacc, P):
    x = _points(20000, 90)
    got = nacc.mlp_encode(torch.as_tensor(x, device=DEV)).cpu().numpy()
    exp = P.encode(x)
    np.testing.assert_allclose(got, exp, rtol=0, atol=2e-6)


@pytest.mark.parametrize("n", [1, 127, 128, 129, 20000])
def test_forward_matches_oracle(nacc, P, n):
    p = _params(P, 91)
    x = _points(n, 92)
    mlp = nacc.ProposalMLP(torch.as_tensor(_flat(p), device=DEV))
    got = mlp.forward(torch.as_tensor(x, device=DEV)).cpu().numpy()
    exp = P.forward(p, x)["sigma"]
    rel = np.abs(got - exp) / np.maximum(np.abs(exp), 1e-3)
    # BF16 operands: the GPU's FP32 encoding and sums may round an operand one
    # BF16 step apart from the oracle's (a few points in 1e3)
    assert np.median(rel) < 1e-4 and np.mean(rel) < 2e-3 and rel.max() < 3e-2, (np.median(rel), rel.mean(), rel.max())


U32 = 2.0 ** -24  # FP32 unit roundoff


def _bf16_bits(a):
    """float64 values that are BF16 numbers -> their 16-bit patterns (int16)."""
    f = np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))
    return (f.view(np.uint32) >> 16).astype(np.uint16).view(np.int16)


def _exact_case(P, n, seed):
    """Encoded rows and parameters on dyadic grids that make layers 1 and 2
    exact in FP32 whatever the order of the sums (every partial sum is a
    multiple of 2^-16 or 2^-20 below 2^8 or 2^4: at most 24 bits), so the GPU
    and the oracle take every BF16 rounding and ReLU decision of the hidden
    layers on the same values: rows k/256 in [-1, 1] (columns 51..63 zero,
    the encoding's padding), W1 in multiples of 2^-8 within 1/32, b1 in
    multiples of 2^-16 within 1/2 (hi + lo BF16 is then b1 itself), W2 in
    {-1/16, 0, 1/16}, b2 in multiples of 2^-20 within 1/2; w3, b3 and the
    targets unconstrained (no rounding decision follows them)."""
    g = workloads.rng(seed)
    enc = np.zeros((n, 64))
    enc[:, :51] = g.integers(-256, 257, (n, 51)) / 256.0
    p = {"W1": np.zeros((64, 64), np.float32)}
    p["W1"][:, :51] = g.integers(-8, 9, (64, 51)) / 256.0
    p["b1"] = (g.integers(-2 ** 15, 2 ** 15, 64) / 2.0 ** 16).astype(np.float32)
    p["W2"] = (g.integers(-1, 2, (64, 64)) / 16.0).astype(np.float32)
    p["b2"] = (g.integers(-2 ** 19, 2 ** 19, 64) / 2.0 ** 20).astype(np.float32)
    p["w3"] = P.bf16(g.standard_normal(64) * 0.3).astype(np.float32)
    p["b3"] = np.array([0.3], np.float32)
    t = g.uniform(0.0, 3.0, n).astype(np.float32)
    f = P.forward(p, None, enc=enc)
    for z in (f["z1"], f["z2"]):  # the sums are FP32 numbers: exact in FP32
        assert np.array_equal(z.astype(np.float32).astype(np.float64), z)
    assert 0.2 < (f["z1"] > 0).mean() < 0.8 and 0.2 < (f["z2"] > 0).mean() < 0.8  # the ReLUs bind both ways
    return p, enc, t, f


def test_forward_encoded_elementwise(nacc, P):
    """The forward on identical BF16 layer-1 inputs whose hidden layers are
    exact (_exact_case): every density within the FP32 error of the last
    layer's sum (64 products and b3, at most 2u per addition) through
    softplus, and 16 ulp of softplus itself."""
    p, enc, _, f = _exact_case(P, 3000, 101)
    mlp = nacc.ProposalMLP(torch.as_tensor(_flat(p), device=DEV))
    got = mlp.forward_encoded(torch.as_tensor(_bf16_bits(enc), device=DEV)).cpu().numpy().astype(np.float64)
    w3 = P.bf16(p["w3"])
    d3 = 160 * U32 * (np.abs(f["h2"]) @ np.abs(w3) + abs(float(p["b3"][0])))
    sig = 1.0 / (1.0 + np.exp(-f["z3"]))
    tol = sig * d3 * 1.1 + 16 * U32 * np.abs(f["sigma"]) + 1e-30
    err = np.abs(got - f["sigma"])
    assert np.all(err <= tol), (int((err > tol).sum()), float(np.max(err / tol)))
    assert np.median(err) < 1e-6 * np.median(f["sigma"])


def test_train_gradients_match_oracle(nacc, P):
    """The fused adjoint on identical BF16 layer-1 inputs whose hidden layers
    are exact (_exact_case): the loss and all 8,385 gradient entries element
    by element.  Each entry's
    bound is the FP32 error of its computation on the GPU: the FP32 output
    error d3 of every point (its sum of 64 products, softplus and logistic)
    carried through the adjoint by absolute values, the error terms' split
    into two BF16 parts (2^-18 relative), and 2 (n + 32) u times the sum of
    the absolute terms of every accumulation over the batch (2u per
    addition: tensor-core accumulation need not round to nearest)."""
    n = 1024
    p, enc, t, f = _exact_case(P, n, 93)
    mlp = nacc.ProposalMLP(torch.as_tensor(_flat(p), device=DEV))
    mlp.accumulate_grads_encoded(torch.as_tensor(_bf16_bits(enc), device=DEV), torch.as_tensor(t, device=DEV))
    got = _unflat(mlp.grads.cpu().numpy())
    loss = mlp.loss_sum.item()
    L, exp = P.loss_and_grads(p, None, t, enc=enc)
    W2, w3 = P.bf16(p["W2"]), P.bf16(p["w3"])
    t64 = t.astype(np.float64)
    z3, sp = f["z3"], f["sigma"]
    sig = 1.0 / (1.0 + np.exp(-z3))
    dz3 = 160 * U32 * (np.abs(f["h2"]) @ np.abs(w3) + abs(float(p["b3"][0])))
    d3 = (2.0 / n) * (sp - t64) * sig
    # FP32 error of d3 per point: z3's sum through softplus and the logistic, their own rounding
    e_sp = sig * dz3 + 16 * U32 * (np.abs(sp) + np.abs(t64))
    e_sig = sig * (1 - sig) * dz3 + 16 * U32 * sig
    e_d3 = (2.0 / n) * (e_sp * sig + np.abs(sp - t64) * e_sig) + 8 * U32 * np.abs(d3)
    m2 = (f["z2"] > 0).astype(np.float64)
    m1 = (f["z1"] > 0).astype(np.float64)
    D2 = d3[:, None] * w3[None, :] * m2
    e_D2 = (e_d3[:, None] * np.abs(w3)[None, :] + (2.0 ** -18 + 2 * U32) * np.abs(D2)) * m2
    D1 = (D2 @ W2) * m1
    e_D1 = (e_D2 @ np.abs(W2) + 160 * U32 * (np.abs(D2) @ np.abs(W2))) * m1 + 2.0 ** -18 * np.abs(D1)
    acc = 2 * (n + 32) * U32  # accumulations: at most 2u per addition (the tensor cores may truncate)
    tol = {
        "b3": np.array([e_d3.sum() + acc * np.abs(d3).sum()]),
        "w3": e_d3 @ np.abs(f["h2"]) + acc * (np.abs(d3) @ np.abs(f["h2"])),
        "b2": e_D2.sum(0) + acc * np.abs(D2).sum(0),
        "W2": e_D2.T @ np.abs(f["h1"]) + acc * (np.abs(D2).T @ np.abs(f["h1"])),
        "b1": e_D1.sum(0) + acc * np.abs(D1).sum(0),
        "W1": e_D1.T @ np.abs(enc) + acc * (np.abs(D1).T @ np.abs(enc)),
    }
    n_checked = 0
    for k in exp:
        e, g, tk = (np.asarray(a, np.float64).reshape(-1) for a in (exp[k], got[k], tol[k]))
        bad = np.abs(g - e) > tk * 1.05 + 1e-30
        assert not bad.any(), (k, int(bad.sum()), float(np.max(np.abs(g - e) / (tk + 1e-30))))
        n_checked += e.size
    assert n_checked == 8385
    # the loss: n squared differences, FP32
    e_loss = np.sum(2 * np.abs(sp - t64) * e_sp) + acc * np.sum((sp - t64) ** 2)
    assert abs(loss - L * n) <= e_loss * 1.05, (loss, L * n, e_loss)
    # the comparison is not vacuous: gradients well above their bounds
    assert np.median(np.abs(np.asarray(exp["W2"])).reshape(-1) / (tol["W2"].reshape(-1) + 1e-30)) > 10


def test_adam_matches_oracle(nacc, P):
    p = _params(P, 96)
    g = np.random.default_rng(97)
    grads = {k: g.standard_normal(v.shape) * 0.1 for k, v in p.items()}
    grads["W1"][:, 51:] = 0.0
    mlp = nacc.ProposalMLP(torch.as_tensor(_flat(p), device=DEV))
    st = {}
    for step in range(3):
        mlp.grads.copy_(torch.as_tensor(_flat({k: v.astype(np.float32) for k, v in grads.items()}), device=DEV))
        mlp.adam(lr=1e-2)
        P.adam_step(p, grads, st, lr=1e-2)
    got = mlp.params.cpu().numpy()
    np.testing.assert_allclose(got, _flat(p), rtol=1e-5, atol=1e-7)
    assert float(mlp.grads.abs().max()) == 0.0  # zeroed by the step
    # the BF16 weight copy follows the master parameters
    w = mlp.weights.cpu().numpy().view(np.uint16)
    np.testing.assert_array_equal(w[0:4096], (P.bf16(got[0:4096]).astype(np.float32).view(np.uint32) >> 16))


def test_training_fits_the_blob_field(nacc, P):
    """Densities of the 8-blob field along C1 rays: 300 Adam steps of 16384
    points cut the mean squared error by 10x or more."""
    w = workloads.c1_forward(4096)
    field = nacc.BlobField.from_numpy(w.blobs)
    g = torch.Generator(device=DEV).manual_seed(5)
    mlp = nacc.ProposalMLP.init(seed=3, device=DEV)
    o = torch.as_tensor(w.rays_o, device=DEV)
    d = torch.as_tensor(w.rays_d, device=DEV)
    losses = []
    for it in range(300):
        r = torch.randint(0, w.n_rays, (16384,), generator=g, device=DEV)
        tt = 2.5 + 3.0 * torch.rand(16384, generator=g, device=DEV)
        xyz = (o[r] + d[r] * tt[:, None]).contiguous()
        sig = nacc.field_points(field, xyz)
        losses.append(mlp.train_step(xyz, sig, lr=3e-3))
    first = float(losses[0].item())
    last = float(torch.stack(losses[-20:]).mean().item())
    assert math.isfinite(last) and last < first / 10.0, (first, last)


# ---------------------------------------------------------------------------
# proposal sampling pipeline
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _c1_rays_with_misses(n=4096):
    w = workloads.c1_forward(n)
    o, d = w.rays_o.copy(), w.rays_d.copy()
    d[:64] = -d[:64]  # pointing away from the box: misses
    return o, d


def _edges_oracle(orc, o, d, nb, t_min=0.0, t_max=1e10):
    tn, tf, hit = orc.ray_clip(o, d, (-1.5,) * 3, (1.5,) * 3, 32, 1, t_min, t_max)
    tn = np.where(hit, tn, np.float32(max(t_min, 0.0))).astype(np.float32)
    tf = np.where(hit, tf, tn).astype(np.float32)
    span = (tf - tn).astype(np.float32)
    frac = (np.arange(nb, dtype=np.float32) / np.float32(nb)).astype(np.float32)
    e = (tn[:, None] + (span[:, None] * frac[None, :]).astype(np.float32)).astype(np.float32)
    return np.concatenate([e, tf[:, None]], 1)


def test_uniform_edges_bit_exact(nacc, orc):
    o, d = _c1_rays_with_misses()
    grid = nacc.OccupancyGrid.empty((-1.5,) * 3, (1.5,) * 3, 32, 1, DEV)
    got = nacc.uniform_edges(grid, torch.as_tensor(o, device=DEV), torch.as_tensor(d, device=DEV), 64).cpu().numpy()
    np.testing.assert_array_equal(got, _edges_oracle(orc, o, d, 64))


def test_dense_weights_match_oracle(nacc, orc):
    g = workloads.rng(98)
    n, nb = 3000, 64
    e = np.sort(g.uniform(1.0, 6.0, (n, nb + 1)), axis=1).astype(np.float32)
    s = (g.exponential(3.0, (n, nb)) * (g.random((n, nb)) < 0.4)).astype(np.float32)
    tr = torch.empty(n, device=DEV)
    got = nacc.dense_weights(torch.as_tensor(e, device=DEV), torch.as_tensor(s, device=DEV), trans=tr).cpu().numpy()
    off = np.arange(n + 1, dtype=np.int64) * nb
    exp = orc.render_fwd(off, e[:, :-1].reshape(-1), e[:, 1:].reshape(-1), s.reshape(-1), np.zeros((n * nb, 3)))
    np.testing.assert_allclose(got.reshape(-1), exp["weights"], rtol=0, atol=1e-5)
    np.testing.assert_allclose(tr.cpu().numpy(), exp["trans"], rtol=0, atol=1e-5)


def test_edges_to_packed_exact(nacc):
    g = workloads.rng(99)
    e = np.sort(g.uniform(0.0, 5.0, (777, 33)), axis=1).astype(np.float32)
    pk = nacc.edges_to_packed(torch.as_tensor(e, device=DEV))
    assert pk.n_samples() == 777 * 32
    np.testing.assert_array_equal(pk.offsets.cpu().numpy(), np.arange(778) * 32)
    np.testing.assert_array_equal(pk.t_starts.cpu().numpy(), e[:, :-1].reshape(-1))
    np.testing.assert_array_equal(pk.t_ends.cpu().numpy(), e[:, 1:].reshape(-1))


def _midpoints(o, d, e):
    t = (0.5 * (e[:, :-1].astype(np.float64) + e[:, 1:])).astype(np.float32)
    return (o[:, None, :] + d[:, None, :] * t[:, :, None]).reshape(-1, 3)


def test_forward_rays_matches_oracle(nacc, P, orc):
    o, d = _c1_rays_with_misses(2048)
    p = _params(P, 100)
    mlp = nacc.ProposalMLP(torch.as_tensor(_flat(p), device=DEV))
    e = _edges_oracle(orc, o, d, 64)
    got = mlp.forward_rays(torch.as_tensor(o, device=DEV), torch.as_tensor(d, device=DEV),
                           torch.as_tensor(e, device=DEV)).cpu().numpy().reshape(-1)
    exp = P.forward(p, _midpoints(o, d, e))["sigma"]
    rel = np.abs(got - exp) / np.maximum(np.abs(exp), 1e-3)
    assert np.median(rel) < 1e-4 and np.mean(rel) < 3e-3 and rel.max() < 5e-2, (np.median(rel), rel.mean(), rel.max())


def test_sampler_matches_oracle_composition(nacc, P, orc):
    """Two rounds (64 -> 32 -> 32 bins) of proposal density, weights and
    inverse-CDF resampling against the same chain of oracle functions."""
    o, d = _c1_rays_with_misses(2048)
    n = o.shape[0]
    p = _params(P, 101)
    p["b3"] = np.array([1.0], np.float32)  # some opacity for untrained weights
    mlp = nacc.ProposalMLP(torch.as_tensor(_flat(p), device=DEV))
    grid = nacc.OccupancyGrid.empty((-1.5,) * 3, (1.5,) * 3, 32, 1, DEV)
    sampler = nacc.ProposalSampler(mlp, grid, n, rounds=(64, 32), n_final=32, device=DEV)
    pk = sampler.sample(torch.as_tensor(o, device=DEV), torch.as_tensor(d, device=DEV))
    got = np.stack([pk.t_starts.cpu().numpy().reshape(n, 32), pk.t_ends.cpu().numpy().reshape(n, 32)])
    e = _edges_oracle(orc, o, d, 64)
    for nb, n_next in ((64, 32), (32, 32)):
        s = P.forward(p, _midpoints(o, d, e))["sigma"]
        off = np.arange(n + 1, dtype=np.int64) * nb
        w = orc.render_fwd(off, e[:, :-1].reshape(-1), e[:, 1:].reshape(-1), s, np.zeros((n * nb, 3)))["weights"]
        e = orc.sample_pdf(e, w.reshape(n, nb).astype(np.float32), n_next)
    exp = np.stack([e[:, :-1], e[:, 1:]])
    span = np.maximum(e[:, -1] - e[:, 0], 1e-6)[None, :, None]
    err = np.abs(got - exp) / span
    assert np.quantile(err, 0.99) < 2e-3 and err.mean() < 2e-4, (np.quantile(err, 0.99), err.mean(), err.max())
    np.testing.assert_array_equal(got[:, :64], exp[:, :64])  # misses: empty bins, identical


# ---------------------------------------------------------------------------
# combined estimator: occupancy grid + proposal network
# ---------------------------------------------------------------------------

def _grid(nacc, bits, res, L):
    return nacc.OccupancyGrid((-1.5,) * 3, (1.5,) * 3, res, L, torch.as_tensor(bits.view(np.int32)).to(DEV))


@pytest.mark.parametrize("case", ["c1", "cascade"])
def test_occupied_range_bit_exact(nacc, orc, case):
    o, d = _c1_rays_with_misses(3000)
    if case == "c1":
        w = workloads.c1_forward()
        res, L = w.grid.res, w.grid.n_levels
        bits, _ = orc.density_grid(w.grid, w.blobs)
        step, tmin = w.march.step, 0.0
    else:
        res, L = 64, 4
        bits = workloads.random_bitfield(L, res, 555, p_block=0.3, block=4, p_cell=0.6)
        step, tmin = 3.0 * math.sqrt(3) / 512, 0.5
        o = o * 2.0  # origins out to radius 8: through the outer levels
        o[:64] *= 4.0  # the 64 rays pointing away start at radius 32: they miss the +-12 outer box
    got_lo, got_hi = nacc.occupied_range(_grid(nacc, bits, res, L), torch.as_tensor(o, device=DEV),
                                         torch.as_tensor(d, device=DEV), step, 1024, tmin, 1e10)
    ex = orc.march(o, d, (-1.5,) * 3, (1.5,) * 3, res, L, bits, step, 1024, tmin, 1e10)
    tn, tf, hit = orc.ray_clip(o, d, (-1.5,) * 3, (1.5,) * 3, res, L, tmin, 1e10)
    off = ex["offsets"]
    cnt = np.diff(off)
    lo = np.where(hit, tn, np.float32(max(tmin, 0.0))).astype(np.float32)
    hi = lo.copy()
    has = cnt > 0
    lo[has] = ex["t_starts"][off[:-1][has]]
    hi[has] = ex["t_ends"][off[1:][has] - 1]
    assert has.sum() > 500 and (~has).sum() > 50
    np.testing.assert_array_equal(got_lo.cpu().numpy(), lo)
    np.testing.assert_array_equal(got_hi.cpu().numpy(), hi)


def test_range_edges_exact(nacc):
    g = workloads.rng(102)
    lo = g.uniform(0.0, 3.0, 1000).astype(np.float32)
    hi = (lo + g.uniform(0.0, 2.0, 1000) * (g.random(1000) < 0.9)).astype(np.float32)
    got = nacc.range_edges(torch.as_tensor(lo, device=DEV), torch.as_tensor(hi, device=DEV), 64).cpu().numpy()
    span = (hi - lo).astype(np.float32)
    frac = (np.arange(64, dtype=np.float32) / np.float32(64)).astype(np.float32)
    exp = np.concatenate([(lo[:, None] + (span[:, None] * frac).astype(np.float32)).astype(np.float32), hi[:, None]], 1)
    np.testing.assert_array_equal(got, exp)


def test_combined_sampler_matches_oracle_composition(nacc, P, orc):
    w = workloads.c1_forward(2048)
    o, d = w.rays_o, w.rays_d
    n = o.shape[0]
    bits, _ = orc.density_grid(w.grid, w.blobs)
    p = _params(P, 103)
    p["b3"] = np.array([1.0], np.float32)
    mlp = nacc.ProposalMLP(torch.as_tensor(_flat(p), device=DEV))
    grid = _grid(nacc, bits, w.grid.res, w.grid.n_levels)
    cs = nacc.CombinedSampler(mlp, grid, n, w.march.step, 1024, rounds=(64, 32), n_final=32, device=DEV)
    pk = cs.sample(torch.as_tensor(o, device=DEV), torch.as_tensor(d, device=DEV))
    got = np.stack([pk.t_starts.cpu().numpy().reshape(n, 32), pk.t_ends.cpu().numpy().reshape(n, 32)])
    ex = orc.march(o, d, (-1.5,) * 3, (1.5,) * 3, w.grid.res, 1, bits, w.march.step, 1024, 0.0, 1e10)
    tn, tf, hit = orc.ray_clip(o, d, (-1.5,) * 3, (1.5,) * 3, w.grid.res, 1, 0.0, 1e10)
    off, cnt = ex["offsets"], np.diff(ex["offsets"])
    lo = np.where(hit, tn, np.float32(0.0)).astype(np.float32)
    hi = lo.copy()
    lo[cnt > 0] = ex["t_starts"][off[:-1][cnt > 0]]
    hi[cnt > 0] = ex["t_ends"][off[1:][cnt > 0] - 1]
    span0 = (hi - lo).astype(np.float32)
    frac = (np.arange(64, dtype=np.float32) / np.float32(64)).astype(np.float32)
    e = np.concatenate([(lo[:, None] + (span0[:, None] * frac).astype(np.float32)).astype(np.float32), hi[:, None]], 1)
    for nb, n_next in ((64, 32), (32, 32)):
        s = P.forward(p, _midpoints(o, d, e))["sigma"]
        off2 = np.arange(n + 1, dtype=np.int64) * nb
        wts = orc.render_fwd(off2, e[:, :-1].reshape(-1), e[:, 1:].reshape(-1), s, np.zeros((n * nb, 3)))["weights"]
        e = orc.sample_pdf(e, wts.reshape(n, nb).astype(np.float32), n_next)
    exp = np.stack([e[:, :-1], e[:, 1:]])
    span = np.maximum(e[:, -1] - e[:, 0], 1e-6)[None, :, None]
    err = np.abs(got - exp) / span
    assert np.quantile(err, 0.99) < 2e-3 and err.mean() < 2e-4, (np.quantile(err, 0.99), err.mean(), err.max())


def test_sampler_full_batch_sampled_rays(nacc, P, orc):
    """The whole 262,144-ray training batch through the proposal rounds
    (64 -> 32 -> 32) as the bench runs them; 1,000 strided rays against the
    oracle chain (same tolerance as the small composition test)."""
    w = workloads.c3_training()
    n = w.n_rays
    p = _params(P, 102)
    p["b3"] = np.array([1.0], np.float32)
    mlp = nacc.ProposalMLP(torch.as_tensor(_flat(p), device=DEV))
    grid = nacc.OccupancyGrid.empty((-1.5,) * 3, (1.5,) * 3, 32, 1, DEV)
    sampler = nacc.ProposalSampler(mlp, grid, n, rounds=(64, 32), n_final=32, device=DEV)
    pk = sampler.sample(torch.as_tensor(w.rays_o, device=DEV), torch.as_tensor(w.rays_d, device=DEV))
    sel = np.linspace(0, n - 1, 1000).astype(np.int64)
    got = np.stack([pk.t_starts.reshape(n, 32)[sel].cpu().numpy(), pk.t_ends.reshape(n, 32)[sel].cpu().numpy()])
    o, d = w.rays_o[sel], w.rays_d[sel]
    e = _edges_oracle(orc, o, d, 64)
    for nb, n_next in ((64, 32), (32, 32)):
        s = P.forward(p, _midpoints(o, d, e))["sigma"]
        off = np.arange(len(sel) + 1, dtype=np.int64) * nb
        wts = orc.render_fwd(off, e[:, :-1].reshape(-1), e[:, 1:].reshape(-1), s, np.zeros((len(sel) * nb, 3)))
        e = orc.sample_pdf(e, wts["weights"].reshape(len(sel), nb).astype(np.float32), n_next)
    exp = np.stack([e[:, :-1], e[:, 1:]])
    span = np.maximum(e[:, -1] - e[:, 0], 1e-6)[None, :, None]
    err = np.abs(got - exp) / span
    assert np.quantile(err, 0.99) < 2e-3 and err.mean() < 2e-4, (np.quantile(err, 0.99), err.mean(), err.max())
