"""Estimator-update variants on the GPU against oracle/grid_variants.py:
the dynamic-scene grid (maximum over frames) and the gradient-descent grid
(density lookup, its adjoint, the SGD step, and a small fit)."""
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
def orc():
    import oracle
    oracle.build()
    return oracle


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV)


def test_update_grid_frames_parity(nacc, orc):
    from oracle import grid_variants as G
    res, L, nf = 64, 2, 3
    n = L * res ** 3
    g = workloads.rng(120)
    ema0 = (g.exponential(1.0, n) * (g.random(n) < 0.5)).astype(np.float32)
    dens = (g.exponential(0.5, (nf, n)) * (g.random((nf, n)) < 0.3)).astype(np.float32)
    grid = nacc.OccupancyGrid.empty((-1.5,) * 3, (1.5,) * 3, res, L, DEV)
    grid.ema.copy_(T(ema0))
    nacc.update_grid_frames(grid, T(dens), decay=0.95, thresh_frac=0.01)
    e_ref, bits_ref, mean_ref = orc.update_grid(ema0, G.frames_max(dens), 0.95, 0.01)
    np.testing.assert_array_equal(grid.ema.cpu().numpy(), e_ref)
    thr = 0.01 * mean_ref
    near = np.abs(e_ref.astype(np.float64) - thr) <= 1e-12 * thr
    got_b = workloads.unpack_bits(grid.bits.cpu().numpy().view(np.uint32))
    assert np.array_equal(got_b[~near], workloads.unpack_bits(bits_ref)[~near])


def _packed(nacc, orc, res=32, L=3):
    w = workloads.c1_forward(3000)
    bits = workloads.random_bitfield(L, res, 121, p_block=0.5, block=4, p_cell=0.6)
    ex = orc.march(w.rays_o, w.rays_d, (-1.5,) * 3, (1.5,) * 3, res, L, bits, 0.01, 1024, 0.0, 1e10)
    S = int(ex["offsets"][-1])
    pk = nacc.PackedSamples(T(ex["offsets"]), T(ex["ray_indices"]), T(ex["t_starts"]), T(ex["t_ends"]),
                            torch.tensor([S], device=DEV))
    grid = nacc.OccupancyGrid((-1.5,) * 3, (1.5,) * 3, res, L, T(bits.view(np.int32)))
    return w, ex, pk, grid, S


def test_density_lookup_bit_exact_and_backward(nacc, orc):
    from oracle import grid_variants as G
    w, ex, pk, grid, S = _packed(nacc, orc)
    n = grid.n_cells
    g = workloads.rng(122)
    dens = g.uniform(0.0, 5.0, n).astype(np.float32)
    got = nacc.grid_density_lookup(grid, T(dens), T(w.rays_o), T(w.rays_d), pk).cpu().numpy()
    cells = G.sample_cells(w.rays_o, w.rays_d, ex["ray_indices"], ex["t_starts"], ex["t_ends"],
                           orc.level_geometry((-1.5,) * 3, (1.5,) * 3, grid.res, grid.n_levels), grid.res)
    np.testing.assert_array_equal(got, G.density_lookup(dens, cells))
    gs = g.standard_normal(S).astype(np.float32)
    gd = torch.zeros(n, device=DEV)
    nacc.grid_density_backward(grid, T(w.rays_o), T(w.rays_d), pk, T(gs), gd)
    np.testing.assert_allclose(gd.cpu().numpy(), G.density_backward(gs, cells, n), rtol=1e-5, atol=1e-5)


def test_sgd_step_exact(nacc, orc):
    from oracle import grid_variants as G
    grid = nacc.OccupancyGrid.empty((-1.5,) * 3, (1.5,) * 3, 32, 2, DEV)
    g = workloads.rng(123)
    d0 = g.uniform(0.0, 1.0, grid.n_cells).astype(np.float32)
    g0 = g.standard_normal(grid.n_cells).astype(np.float32)
    dens, grad = T(d0), T(g0)
    nacc.update_grid_sgd(grid, dens, grad, 0.3, 0.25)
    ed, eb = G.sgd_step(d0, g0, 0.3, 0.25)
    np.testing.assert_array_equal(dens.cpu().numpy(), ed)
    np.testing.assert_array_equal(workloads.unpack_bits(grid.bits.cpu().numpy().view(np.uint32)), eb)
    assert float(grad.abs().max()) == 0.0


def test_sgd_grid_fits_a_target_opacity(nacc, orc):
    """Render the grid's densities (lookup -> render_fwd), L2 loss against the
    opacity of a fixed density field, adjoint (render_bwd -> backward), SGD:
    the loss falls by 5x in 60 steps (the oracle's FP64 run of the same loop
    falls by 25x)."""
    w, ex, pk, grid, S = _packed(nacc, orc)
    n = grid.n_cells
    g = workloads.rng(124)
    target_d = T(g.uniform(0.0, 8.0, n).astype(np.float32))
    o, d = T(w.rays_o), T(w.rays_d)
    tgt = nacc.render_fwd(pk.offsets, pk.t_starts, pk.t_ends, nacc.grid_density_lookup(grid, target_d, o, d, pk),
                          torch.zeros((S, 3), device=DEV))[1]
    dens = torch.full((n,), 1.0, device=DEV)
    gd = torch.zeros(n, device=DEV)
    zc = torch.zeros((S, 3), device=DEV)
    losses = []
    for it in range(60):
        sig = nacc.grid_density_lookup(grid, dens, o, d, pk)
        rgb, op, dep, tr, _ = nacc.render_fwd(pk.offsets, pk.t_starts, pk.t_ends, sig, zc)
        losses.append(float(((op - tgt) ** 2).mean()))
        g_op = (2.0 * (op - tgt) / op.numel()).contiguous()
        gs, _ = nacc.render_bwd(pk.offsets, pk.t_starts, pk.t_ends, sig, zc, None, g_op, None)
        nacc.grid_density_backward(grid, o, d, pk, gs, gd)
        nacc.update_grid_sgd(grid, dens, gd, 2e4, -1.0)  # threshold below 0: keep every cell occupied
    assert losses[-1] < losses[0] / 5.0, (losses[0], losses[-1])
