"""GB300 (sm_103a) occupancy-grid sampling and differentiable volume rendering.

The hot path of NerfAcc (arXiv 2305.04966), Algorithm 1: ``march_grid``
(transmittance-estimator sampling with an occupancy grid, Table 1 "Spatial
Skipping", Sec. 4.2), ``render`` / ``render_fwd`` / ``render_bwd`` (Eq. 2
and its adjoint), ``update_grid`` (Eq. 4, EMA), ``sample_pdf`` (Eq. 1 with
F = 1 - T, Eq. 3).  The kernels live in ``libnacc.so`` behind the C ABI of
``include/nacc.h``; this package only marshals torch tensors.
"""
from ._abi import NaccError, load as load_library
from .api import (BlobField, CombinedSampler, MarchBuffers, OccupancyGrid, PackedSamples, ProposalMLP,
                  ProposalSampler, RenderFn, occupied_range, range_edges,
                  UpdateBuffers, dense_weights, density_grid, edges_to_packed, field_eval, field_points,
                  grid_points, l2_loss, march_grid, mlp_encode, render, render_bwd, render_ckpt_buffer, render_fwd,
                  sample_pdf,
                  uniform_edges, update_grid, update_grid_frames, grid_density_lookup, grid_density_backward,
                  update_grid_sgd, march_unbounded, uncontract_points, density_grid_unbounded,
                  contract_points, phi_edges, UnboundedProposalSampler)

__all__ = [
    "NaccError", "load_library", "BlobField", "MarchBuffers", "OccupancyGrid", "PackedSamples",
    "RenderFn", "UpdateBuffers", "density_grid", "field_eval", "field_points", "grid_points",
    "l2_loss", "march_grid", "render", "render_bwd", "render_ckpt_buffer", "render_fwd", "sample_pdf",
    "update_grid",
    "ProposalMLP", "ProposalSampler", "mlp_encode", "uniform_edges", "dense_weights", "edges_to_packed",
    "CombinedSampler", "occupied_range", "range_edges", "update_grid_frames", "grid_density_lookup",
    "grid_density_backward", "update_grid_sgd", "march_unbounded", "uncontract_points",
    "density_grid_unbounded", "contract_points", "phi_edges", "UnboundedProposalSampler",
]
