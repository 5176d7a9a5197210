"""Checkpoint and resume of the occupancy-grid estimator (host only).

The grid's update runs every few training steps and carries its EMA from one
update to the next (Eq. 4, Sec. 3.1), so a training checkpoint has to hold
the bits and the EMA.  These tests round-trip that state through torch's
serialisation on the CPU and check that malformed states are refused.
"""
import io

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")


def _grid(nacc):
    g = nacc.OccupancyGrid.empty((-1.5, -1.0, -0.5), (1.5, 1.0, 0.5), 16, 3, device="cpu")
    r = workloads.rng(501)
    g.ema.copy_(torch.as_tensor(r.exponential(1.0, g.n_cells).astype(np.float32)))
    occ = r.random(g.n_cells) < 0.3
    g.bits.copy_(torch.as_tensor(workloads.pack_bits(occ).view(np.int32)))
    return g


def test_grid_state_round_trip_through_torch_save():
    import paper_2305_04966_gb300 as nacc
    g = _grid(nacc)
    buf = io.BytesIO()
    torch.save(g.state_dict(), buf)
    buf.seek(0)
    h = nacc.OccupancyGrid.from_state_dict(torch.load(buf))
    assert (h.aabb_min, h.aabb_max, h.res, h.n_levels) == (g.aabb_min, g.aabb_max, g.res, g.n_levels)
    assert torch.equal(h.bits, g.bits) and torch.equal(h.ema, g.ema)
    # the state is a copy: later updates of the live grid do not change it
    st = g.state_dict()
    g.ema.mul_(0.5)
    assert not torch.equal(st["ema"], g.ema)
    # the C view of the restored grid carries the same geometry
    c = h.c_struct()
    assert list(c.aabb_min) == [-1.5, -1.0, -0.5] and (c.res, c.n_levels) == (16, 3)


def test_grid_state_without_ema_and_on_another_device():
    import paper_2305_04966_gb300 as nacc
    g = _grid(nacc)
    g.ema = None
    h = nacc.OccupancyGrid.from_state_dict(g.state_dict(), device="cpu")
    assert h.ema is None and torch.equal(h.bits, g.bits)


@pytest.mark.parametrize("bad", ["bits_shape", "bits_dtype", "ema_shape", "geometry"])
def test_malformed_grid_states_are_refused(bad):
    import paper_2305_04966_gb300 as nacc
    st = _grid(nacc).state_dict()
    if bad == "bits_shape":
        st["bits"] = st["bits"][:-1]
    elif bad == "bits_dtype":
        st["bits"] = st["bits"].to(torch.int64)
    elif bad == "ema_shape":
        st["ema"] = st["ema"][:100]
    else:
        st["res"] = 3  # 3 levels of 3^3 cells: not a whole number of 32-bit words
    with pytest.raises(ValueError):
        nacc.OccupancyGrid.from_state_dict(st)
