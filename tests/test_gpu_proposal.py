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


def test_train_gradients_match_oracle(nacc, P):
    p = _params(P, 93)
    n = 5000
    x = _points(n, 94)
    t = workloads.rng(95).uniform(0.0, 3.0, n).astype(np.float32)
    mlp = nacc.ProposalMLP(torch.as_tensor(_flat(p), device=DEV))
    mlp.accumulate_grads(torch.as_tensor(x, device=DEV), torch.as_tensor(t, device=DEV))
    got = _unflat(mlp.grads.cpu().numpy())
    loss = mlp.loss_sum.item() / n
    L, exp = P.loss_and_grads(p, x, t)
    assert loss == pytest.approx(L, rel=2e-3)
    for k in exp:
        e, g = np.asarray(exp[k]).reshape(-1), got[k].reshape(-1)
        scale = np.abs(e).max()
        cos = float(e @ g / (np.linalg.norm(e) * np.linalg.norm(g) + 1e-30))
        assert cos > 0.999 and np.abs(g - e).max() < 3e-2 * scale, (k, cos, np.abs(g - e).max(), scale)


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
