"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks the oracle against a closed form, an invariant, a textbook
special case, brute force written in float64 from the geometry, finite
differences, or a published generator output.  None of them re-types the
oracle's own formula in the same arithmetic.
"""
import math
import os

import numpy as np
import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# helpers: independent float64 geometry
# --------------------------------------------------------------------------

def slab64(o, d, lo, hi, t_min, t_max):
    """float64 slab clip of rays [n][3] against box [lo, hi]."""
    o = o.astype(np.float64)
    d = d.astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        ta = (np.asarray(lo) - o) / d
        tb = (np.asarray(hi) - o) / d
    near = np.where(d == 0, -np.inf, np.minimum(ta, tb))
    far = np.where(d == 0, np.inf, np.maximum(ta, tb))
    outside = (d == 0) & ((o < np.asarray(lo)) | (o > np.asarray(hi)))
    tn = np.maximum(near.max(axis=1), t_min)
    tf = np.minimum(far.min(axis=1), t_max)
    hit = (tn < tf) & ~outside.any(axis=1)
    return tn, tf, hit


def cell_of64(x, amin, amax, res, L, margin_cells=2e-3, margin_box=1e-5):
    """float64 (level, flat cell index, ambiguous) of points x [..., 3]."""
    amin = np.asarray(amin, np.float64)
    amax = np.asarray(amax, np.float64)
    cen = (amin + amax) / 2
    half = (amax - amin) / 2
    level = np.full(x.shape[:-1], -1, np.int64)
    amb = np.zeros(x.shape[:-1], bool)
    dev = np.abs(x - cen)
    for l in range(L):
        h = half * 2.0 ** l
        inside = (dev <= h).all(-1)
        near_face = (np.abs(dev - h) < margin_box).any(-1)
        amb |= near_face & (level < 0)
        level = np.where((level < 0) & inside, l, level)
    idx = np.full(x.shape[:-1], -1, np.int64)
    for l in range(L):
        m = level == l
        if not m.any():
            continue
        h = half * 2.0 ** l
        lo = cen - h
        w = 2 * h / res
        u = (x[m] - lo) / w
        fr = u - np.floor(u)
        amb_m = ((fr < margin_cells) | (fr > 1 - margin_cells)).any(-1)
        i = np.clip(np.floor(u).astype(np.int64), 0, res - 1)
        idx[m] = l * res ** 3 + (i[:, 0] * res + i[:, 1]) * res + i[:, 2]
        amb[m] |= amb_m
    return level, idx, amb


def lattice_check(orc, o, d, amin, amax, res, L, bits, step, max_steps, t_min, t_max):
    """Brute force: every unambiguous lattice point is emitted iff its float64
    midpoint lies in an occupied cell; every emitted sample is a lattice point."""
    out = orc.march(o, d, amin, amax, res, L, bits, step, max_steps, t_min, t_max)
    occ = workloads.unpack_bits(bits)
    outer_lo = np.asarray(amin, np.float64) - (np.asarray(amax) - np.asarray(amin)) / 2 * (2 ** (L - 1) - 1)
    outer_hi = np.asarray(amax, np.float64) + (np.asarray(amax) - np.asarray(amin)) / 2 * (2 ** (L - 1) - 1)
    tn, tf, hit = slab64(o, d, outer_lo, outer_hi, t_min, t_max)
    off = out["offsets"]
    checked = 0
    for r in range(o.shape[0]):
        s, e = off[r], off[r + 1]
        if not hit[r]:
            # a grazing miss may still be a float32 hit; only exact misses are pinned
            continue
        k = np.arange(max_steps)
        t0 = tn[r] + k * step
        valid = t0 < tf[r]
        amb_t = np.abs(t0 - tf[r]) < 1e-5
        tm = t0 + step / 2
        x = o[r].astype(np.float64) + d[r].astype(np.float64) * tm[:, None]
        lev, idx, amb = cell_of64(x, amin, amax, res, L)
        expect = valid & (lev >= 0) & occ[np.maximum(idx, 0)] & (idx >= 0)
        amb = amb | amb_t
        got = np.zeros(max_steps, bool)
        ks = np.rint((out["t_starts"][s:e].astype(np.float64) - tn[r]) / step).astype(np.int64)
        assert np.all(np.abs(out["t_starts"][s:e] - (tn[r] + ks * step)) < 1e-4), "not on the lattice"
        assert np.all(np.abs(out["t_ends"][s:e] - out["t_starts"][s:e] - step) < 1e-5)
        assert np.all(out["ray_indices"][s:e] == r)
        assert np.all(np.diff(ks) > 0), "samples of a ray must be in increasing t"
        got[ks] = True
        bad = (got != expect) & ~amb
        assert not bad.any(), f"ray {r}: lattice points {np.nonzero(bad)[0][:10]} disagree"
        checked += int((~amb).sum())
    assert checked > 0
    return out


# --------------------------------------------------------------------------
# RNG
# --------------------------------------------------------------------------

def test_splitmix64_published_vector(orc):
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    assert [orc.splitmix64_at(1234567, k) for k in range(5)] == vals


# --------------------------------------------------------------------------
# lattice march
# --------------------------------------------------------------------------

def test_level_geometry_is_box_scaled_about_centre(orc):
    amin, amax = (-1.0, -2.0, 0.5), (3.0, 2.0, 1.5)
    g = orc.level_geometry(amin, amax, 16, 4)
    cen = (np.array(amin) + np.array(amax)) / 2
    half = (np.array(amax) - np.array(amin)) / 2
    for l in range(4):
        np.testing.assert_allclose(g[l, 0], cen - half * 2 ** l, rtol=0, atol=1e-6)
        np.testing.assert_allclose(g[l, 1], cen + half * 2 ** l, rtol=0, atol=1e-6)
        np.testing.assert_allclose(g[l, 2] * g[l, 3], 1.0, rtol=1e-6)
        np.testing.assert_allclose(g[l, 3], half * 2 ** (l + 1) / 16, rtol=1e-6)


def test_uniform_special_case(orc):
    """Sec. 3.1 "Uniform": with every cell occupied the estimator is uniform and the
    samples are the regular lattice t_n + k*dt over [t_n, t_f]."""
    w = workloads.c1_forward(512)
    res = 8
    bits = np.full(res ** 3 // 32, 0xFFFFFFFF, np.uint32)
    step = 0.01
    out = orc.march(w.rays_o, w.rays_d, (-1.5,) * 3, (1.5,) * 3, res, 1, bits, step, 4096, 0.0, 1e10)
    tn, tf, hit = slab64(w.rays_o, w.rays_d, (-1.5,) * 3, (1.5,) * 3, 0.0, 1e10)
    n = np.diff(out["offsets"])
    for r in range(512):
        if not hit[r]:
            continue
        span = (tf[r] - tn[r]) / step
        # lattice points whose midpoint is inside the box: t_n + (k+1/2) dt <= t_f
        expect = int(np.floor(span + 0.5))
        if abs((span + 0.5) - round(span + 0.5)) < 1e-3:
            assert abs(n[r] - expect) <= 1
            continue
        assert n[r] == expect, (r, n[r], expect)
        t0 = out["t_starts"][out["offsets"][r]:out["offsets"][r + 1]]
        np.testing.assert_allclose(t0, tn[r] + np.arange(n[r]) * step, rtol=0, atol=2e-5)
    assert (n[~hit] == 0).all()


def test_max_steps_caps_lattice_index(orc):
    w = workloads.c1_forward(64)
    bits = np.full(8 ** 3 // 32, 0xFFFFFFFF, np.uint32)
    out = orc.march(w.rays_o, w.rays_d, (-1.5,) * 3, (1.5,) * 3, 8, 1, bits, 0.01, 17, 0.0, 1e10)
    assert np.diff(out["offsets"]).max() <= 17


def test_single_occupied_cell(orc):
    """Only one cell occupied: exactly the lattice points whose midpoints fall in that
    cell's box (float64 geometry) are emitted."""
    res = 8
    occ = np.zeros(res ** 3, bool)
    i0, i1, i2 = 3, 4, 2
    occ[(i0 * res + i1) * res + i2] = True
    bits = workloads.pack_bits(occ)
    g = workloads.rng(90)
    w = 3.0 / res
    centre = -1.5 + (np.array([i0, i1, i2]) + 0.5) * w
    o = workloads._normalise(g.standard_normal((300, 3))) * 4.0
    p = centre + g.uniform(-0.6 * w, 0.6 * w, size=(300, 3))
    d = workloads._normalise(p - o)
    lattice_check(orc, o.astype(np.float32), d.astype(np.float32), (-1.5,) * 3, (1.5,) * 3, res, 1,
                  bits, 0.004, 2048, 0.0, 1e10)


def test_brute_force_random_grids(orc):
    """Random tiny grids (1-3 levels): the emitted set equals the float64 brute force."""
    for seed, (res, L) in enumerate([(4, 1), (8, 2), (16, 3), (12, 2)]):
        bits = workloads.random_bitfield(L, res, 100 + seed, p_block=0.5, block=2, p_cell=0.5)
        g = workloads.rng(100 + seed, 1)
        n = 120
        o = workloads._normalise(g.standard_normal((n, 3))) * g.uniform(0.5, 6.0, size=(n, 1))
        p = g.uniform(-1.5, 1.5, size=(n, 3))
        d = workloads._normalise(p - o)
        # axis-parallel rays and rays with a zero component
        d[:10] = 0.0
        d[np.arange(10), np.arange(10) % 3] = np.where(np.arange(10) % 2 == 0, 1.0, -1.0)
        d[10:20, 1] = 0.0
        d[10:20] = workloads._normalise(d[10:20])
        lattice_check(orc, o.astype(np.float32), d.astype(np.float32), (-1.5,) * 3, (1.5,) * 3,
                      res, L, bits, 0.02, 1024, 0.1, 1e10)


def test_cascade_selects_finest_level(orc):
    """Level 0 empty, level 1 full: samples exist only outside the level-0 box."""
    res, L = 8, 2
    occ = np.zeros(L * res ** 3, bool)
    occ[res ** 3:] = True
    bits = workloads.pack_bits(occ)
    w = workloads.c1_forward(200)
    o, d = w.rays_o * 1.5, w.rays_d  # origins at radius 6, outside level 1 ([-3,3]^3)
    out = lattice_check(orc, o, d, (-1.5,) * 3, (1.5,) * 3, res, L, bits, 0.01, 2048, 0.0, 1e10)
    m = 0.5 * (out["t_starts"].astype(np.float64) + out["t_ends"])
    x = o[out["ray_indices"]].astype(np.float64) + d[out["ray_indices"]] * m[:, None]
    dev = np.abs(x).max(axis=1)
    assert (dev > 1.5 - 1e-5).all() and (dev < 3.0 + 1e-5).all()
    assert out["offsets"][-1] > 1000


def test_level_box_is_closed(orc):
    """A midpoint exactly on the face of level 0's box belongs to level 0 (the
    finest level whose closed box holds it).  Axis-parallel ray from x = 1/8
    with step 1/4: midpoints x = (k+1)/4 exactly in FP32, k = 5 on the face
    x = 3/2.  Level 0 full, level 1 empty: k = 0..5 emitted, 6 samples, both
    for the upper face (+x) and the lower face (-x)."""
    res, L = 4, 2
    occ = np.zeros(L * res ** 3, bool)
    occ[:res ** 3] = True
    bits = workloads.pack_bits(occ)
    o = np.array([[0.125, 0.3, 0.2], [-0.125, 0.3, 0.2]], np.float32)
    d = np.array([[1.0, 0.0, 0.0], [-1.0, 0.0, 0.0]], np.float32)
    out = orc.march(o, d, (-1.5,) * 3, (1.5,) * 3, res, L, bits, 0.25, 64, 0.0, 1e10)
    np.testing.assert_array_equal(np.diff(out["offsets"]), [6, 6])
    np.testing.assert_array_equal(out["t_starts"][:6], 0.25 * np.arange(6))


def test_miss_and_inside_origin(orc):
    bits = np.full(8 ** 3 // 32, 0xFFFFFFFF, np.uint32)
    o = np.array([[5.0, 5.0, 5.0], [0.0, 0.0, 0.0], [0.0, 3.0, 0.0]], np.float32)
    d = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]], np.float32)
    out = orc.march(o, d, (-1.5,) * 3, (1.5,) * 3, 8, 1, bits, 0.01, 4096, 0.0, 1e10)
    n = np.diff(out["offsets"])
    assert n[0] == 0 and n[2] == 0
    assert n[1] == 150  # from the origin (t_near = t_min = 0) to the face at 1.5
    assert out["t_starts"][0] == 0.0


def test_ray_clip_matches_float64_slab(orc):
    """The clip range [t_near, t_far] of the outermost level's box (Sec. 3.1's
    bounded range) equals the float64 slab intersection: random rays from outside
    and inside, rays with zero direction components, misses, a t_min / t_max window."""
    g = workloads.rng(95)
    n = 400
    o = g.uniform(-4.0, 4.0, size=(n, 3))
    o[:50] = g.uniform(-1.0, 1.0, size=(50, 3))  # origins inside the box
    d = workloads._normalise(g.standard_normal((n, 3)))
    d[50:80, 0] = 0.0  # one zero component, some of these miss
    d[80:90, :2] = 0.0
    d[80:90, 2] = np.where(np.arange(10) % 2 == 0, 1.0, -1.0)
    d[50:80] = workloads._normalise(d[50:80])
    o, d = o.astype(np.float32), d.astype(np.float32)
    for L, (t_min, t_max) in ((1, (0.0, 1e10)), (3, (0.0, 1e10)), (2, (1.0, 4.5))):
        half = 1.5 * 2 ** (L - 1)
        tn, tf, hit = orc.ray_clip(o, d, (-1.5,) * 3, (1.5,) * 3, 16, L, t_min, t_max)
        etn, etf, ehit = slab64(o, d, (-half,) * 3, (half,) * 3, t_min, t_max)
        grazing = np.abs(etf - etn) < 1e-4
        np.testing.assert_array_equal(hit[~grazing], ehit[~grazing])
        assert ehit.sum() > 60 and (L == 3 or (~ehit).sum() > 20)  # level 2's box holds every origin
        m = ehit & ~grazing
        np.testing.assert_allclose(tn[m], etn[m], rtol=1e-6, atol=1e-6)
        np.testing.assert_allclose(tf[m], etf[m], rtol=1e-6, atol=1e-6)


def test_exp_steps_against_float64_exp(orc):
    """The early-stop density's exponential (Cody-Waite reduction + degree-7
    Taylor polynomial, FP32 steps) is within 2 units in the last place of the
    float64 exponential on [-86, 0] (every 7th float of [-1, 0] and [-86, -80],
    a dense sweep of [-86, 0], random arguments), exactly 1 at 0, and 0 below
    -86 (its stated cut)."""
    g = workloads.rng(9001)
    parts = [np.linspace(-86.0, 0.0, 400_001).astype(np.float32),
             (-np.abs(g.standard_normal(200_000)) * 20.0).astype(np.float32)]
    for lo, hi in ((-1.0, 0.0), (-86.0, -80.0)):
        b_hi = np.array([hi if hi != 0.0 else -0.0], np.float32).view(np.uint32)[0]
        b_lo = np.array([lo], np.float32).view(np.uint32)[0]
        parts.append(np.arange(b_hi, b_lo + 1, 7, dtype=np.uint32).view(np.float32))
    a = np.concatenate(parts)
    a = a[a >= -86.0]
    e = orc.exp_steps(a)
    ref = np.exp(a.astype(np.float64))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    err = np.abs(e.astype(np.float64) - ref) / ulp
    assert err.max() <= 2.0, (a[np.argmax(err)], err.max())
    assert orc.exp_steps(np.array([0.0, -0.0], np.float32)).tolist() == [1.0, 1.0]
    below = np.array([-86.0001, -87.0, -100.0, -1e30, -np.inf, np.nan], np.float32)
    assert np.all(orc.exp_steps(below) == 0.0)
    # e^(-k ln 2) lands within the bound of 2^-k at every reduction boundary
    k = np.arange(0, 124)
    got = orc.exp_steps((-k * math.log(2)).astype(np.float32)).astype(np.float64)
    exact = np.exp((-k * math.log(2)).astype(np.float32).astype(np.float64))
    assert np.all(np.abs(got - exact) <= 2.0 * np.spacing(exact.astype(np.float32)))


def test_early_termination_cut(orc):
    """No-gradient filtering (Sec. 4.2): the field-given march emits a prefix of the
    field-less march, cut where the float64 optical depth of the emitted samples
    first exceeds -ln(1e-4)."""
    w = workloads.c1_forward(400)
    bits, _ = orc.density_grid(w.grid, w.blobs)
    m, g = w.march, w.grid
    full = orc.march(w.rays_o, w.rays_d, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, m.step,
                     m.max_steps, m.t_min, m.t_max)
    cut = orc.march(w.rays_o, w.rays_d, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, m.step,
                    m.max_steps, m.t_min, m.t_max, blobs=w.blobs, eps=1e-4)
    thr = -math.log(1e-4)
    sig, _ = orc.field_samples(w.rays_o, w.rays_d, full["ray_indices"], full["t_starts"],
                               full["t_ends"], w.blobs)
    tau = sig * (full["t_ends"].astype(np.float64) - full["t_starts"])
    n_cut_total = 0
    for r in range(400):
        fs, fe = full["offsets"][r], full["offsets"][r + 1]
        cs, ce = cut["offsets"][r], cut["offsets"][r + 1]
        nc = ce - cs
        assert nc <= fe - fs
        np.testing.assert_array_equal(cut["t_starts"][cs:ce], full["t_starts"][fs:fs + nc])
        P = np.concatenate([[0.0], np.cumsum(tau[fs:fe])])  # P[i] = depth before sample i
        if nc > 0:
            assert P[nc - 1] <= thr * (1 + 1e-5)
        if nc < fe - fs:
            n_cut_total += 1
            assert P[nc] > thr * (1 - 1e-5)
    assert n_cut_total > 10


# --------------------------------------------------------------------------
# compositing (Eq. 2) and gradient
# --------------------------------------------------------------------------

def test_homogeneous_slab_closed_form(orc):
    """Constant sigma0 over N equal intervals: T_i = exp(-sigma0 dt i), opacity =
    1 - exp(-sigma0 dt N), colour = c (1 - T_N) + bg T_N, depth = sum_i w_i m_i."""
    N, dt, s0, t0 = 200, 0.01, 7.0, 2.0
    k = np.arange(N)
    ts = (t0 + k * dt).astype(np.float32)
    te = (ts.astype(np.float64) + dt).astype(np.float32)
    dts = te.astype(np.float64) - ts
    c = np.array([0.2, 0.5, 0.9])
    bg = np.array([0.7, 0.1, 0.4])
    out = orc.render_fwd(np.array([0, N]), ts, te, np.full(N, s0), np.tile(c, (N, 1)), bg=tuple(bg))
    L = dts.sum()
    TN = math.exp(-s0 * L)
    assert out["trans"][0] == pytest.approx(TN, rel=1e-12)
    assert out["opacity"][0] == pytest.approx(1 - TN, rel=1e-12)
    np.testing.assert_allclose(out["rgb"][0], c * (1 - TN) + TN * bg, rtol=1e-12)
    Ti = np.exp(-s0 * np.concatenate([[0.0], np.cumsum(dts)[:-1]]))
    wi = Ti * (1 - np.exp(-s0 * dts))
    np.testing.assert_allclose(out["weights"], wi, rtol=1e-11)
    m = 0.5 * (ts.astype(np.float64) + te)
    assert out["depth"][0] == pytest.approx((wi * m).sum(), rel=1e-12)


def test_weights_sum_to_one_minus_transmittance(orc):
    """Eq. 3: F(t) = 1 - T(t), i.e. sum of weights = 1 - T_N; T non-increasing."""
    p = workloads.random_packed(500, 20)
    out = orc.render_fwd(p["offsets"], p["t_starts"], p["t_ends"], p["sigmas"], p["rgbs"])
    np.testing.assert_allclose(out["opacity"], 1 - out["trans"], rtol=0, atol=1e-13)
    off = p["offsets"]
    for r in range(500):
        w = out["weights"][off[r]:off[r + 1]]
        T = 1 - np.concatenate([[0.0], np.cumsum(w)])
        assert np.all(np.diff(T) <= 1e-15)
    empty = np.diff(off) == 0
    assert empty.any()
    np.testing.assert_array_equal(out["rgb"][empty], 1.0)
    np.testing.assert_array_equal(out["opacity"][empty], 0.0)
    np.testing.assert_array_equal(out["depth"][empty], 0.0)
    np.testing.assert_array_equal(out["trans"][empty], 1.0)


def test_line_integral_of_gaussian_blob(orc):
    """T_N converges to exp(-int sigma dt) with the erf closed form of a Gaussian's
    line integral as dt -> 0 (Eq. 2)."""
    blobs = workloads.Blobs(mu=np.array([[0.1, -0.2, 0.05]], np.float32),
                            std=np.array([0.25], np.float32), peak=np.array([3.0], np.float32),
                            rgb=np.array([[0.3, 0.6, 0.9]], np.float32))
    o = np.array([[-3.0, 0.1, 0.3]], np.float32)
    d = workloads._normalise(np.array([[1.0, -0.05, -0.02]])).astype(np.float32)
    tn, tf = 1.0, 5.0
    # closed form: sigma along the ray is a 1-D Gaussian in t
    mu, s, pk = blobs.mu[0].astype(np.float64), float(blobs.std[0]), float(blobs.peak[0])
    oo, dd = o[0].astype(np.float64), d[0].astype(np.float64)
    dd2 = dd @ dd
    tstar = (mu - oo) @ dd / dd2
    perp2 = np.sum((oo + tstar * dd - mu) ** 2)
    sl = s / math.sqrt(dd2)
    integral = pk * math.exp(-perp2 / (2 * s * s)) * sl * math.sqrt(math.pi / 2) * (
        math.erf((tf - tstar) / (sl * math.sqrt(2))) - math.erf((tn - tstar) / (sl * math.sqrt(2))))
    for step, tol in [(0.01, 2e-4), (0.002, 1e-5)]:
        N = int(round((tf - tn) / step))
        ts = (tn + np.arange(N) * step).astype(np.float32)
        te = np.append(ts[1:], np.float32(tf))
        sig, rgb = orc.field_samples(o, d, np.zeros(N, np.int32), ts, te, blobs)
        out = orc.render_fwd(np.array([0, N]), ts, te, sig, rgb)
        assert out["trans"][0] == pytest.approx(math.exp(-integral), rel=tol)
        np.testing.assert_allclose(out["rgb"][0], blobs.rgb[0] * (1 - math.exp(-integral)) + math.exp(-integral), rtol=tol)


def test_mask_mode_zeroes_weights_below_eps(orc):
    """Samples whose transmittance fell below eps get w = 0 (Sec. 4.2 filtering);
    T_N is the transmittance at the first masked sample."""
    N, dt, s0 = 400, 0.01, 5.0
    ts = (np.arange(N) * dt).astype(np.float32)
    te = (ts.astype(np.float64) + dt).astype(np.float32)
    out = orc.render_fwd(np.array([0, N]), ts, te, np.full(N, s0), np.full((N, 3), 0.5), eps=1e-4)
    P = s0 * np.concatenate([[0.0], np.cumsum(te.astype(np.float64) - ts)])
    first_masked = int(np.argmax(P[:N] > -math.log(1e-4)))
    assert first_masked > 0
    assert np.all(out["weights"][first_masked:] == 0)
    assert np.all(out["weights"][:first_masked] > 0)
    assert out["trans"][0] == pytest.approx(math.exp(-P[first_masked]), rel=1e-12)
    assert out["trans"][0] < 1e-4


def _fd_check(orc, p, eps, rays):
    g = workloads.rng(31)
    n = len(p["offsets"]) - 1
    gC = g.standard_normal((n, 3))
    gA = g.standard_normal(n)
    gD = g.standard_normal(n)
    sig = p["sigmas"].astype(np.float64)
    rgb = p["rgbs"].astype(np.float64)
    bg = (0.2, 0.5, 0.9)  # a coloured background, so each channel's term is checked on its own
    gs, gr = orc.render_bwd(p["offsets"], p["t_starts"], p["t_ends"], sig, rgb, gC, gA, gD, bg=bg, eps=eps)

    def loss(s, c):
        o = orc.render_fwd(p["offsets"], p["t_starts"], p["t_ends"], s, c, bg=bg, eps=eps)
        return (o["rgb"] * gC).sum() + (o["opacity"] * gA).sum() + (o["depth"] * gD).sum()

    off = p["offsets"]
    n_checked = 0
    for r in rays:
        for i in range(off[r], off[r + 1]):
            h = 1e-6 * max(1.0, abs(sig[i]))
            sp, sm = sig.copy(), sig.copy()
            sp[i] += h
            sm[i] -= h
            fd = (loss(sp, rgb) - loss(sm, rgb)) / (2 * h)
            assert gs[i] == pytest.approx(fd, rel=1e-5, abs=1e-8), (r, i)
            ch = i % 3
            cp, cm = rgb.copy(), rgb.copy()
            cp[i, ch] += 1e-6
            cm[i, ch] -= 1e-6
            fdc = (loss(sig, cp) - loss(sig, cm)) / 2e-6
            assert gr[i, ch] == pytest.approx(fdc, rel=1e-5, abs=1e-8)
            n_checked += 1
    return n_checked


def test_gradient_matches_finite_differences(orc):
    """The adjoint equals central differences of the FP64 compositing (64 rays)."""
    p = workloads.random_packed(64, 32, max_len=12, sigma_hi=30.0)
    assert _fd_check(orc, p, 0.0, range(64)) > 100


def test_gradient_mask_mode_finite_differences(orc):
    """Mask mode: away from the cut the adjoint still equals central differences."""
    p = workloads.random_packed(32, 33, max_len=40, sigma_hi=200.0, p_empty=0.0)
    out = orc.render_fwd(p["offsets"], p["t_starts"], p["t_ends"], p["sigmas"], p["rgbs"], eps=1e-4)
    assert (out["weights"] == 0).sum() > 50  # the mask is active
    # skip rays whose depth prefix is within 1e-3 of the threshold at any sample
    thr = -math.log(1e-4)
    off = p["offsets"]
    tau = p["sigmas"].astype(np.float64) * (p["t_ends"].astype(np.float64) - p["t_starts"])
    rays = []
    for r in range(32):
        P = np.cumsum(tau[off[r]:off[r + 1]])
        if P.size and np.min(np.abs(P - thr)) > 1e-3:
            rays.append(r)
    assert len(rays) > 10
    _fd_check(orc, p, 1e-4, rays)


# --------------------------------------------------------------------------
# estimator update (Eq. 4) and its sample points
# --------------------------------------------------------------------------

def test_grid_points_centres_and_jitter(orc):
    amin, amax, res, L = (-1.5,) * 3, (1.5,) * 3, 8, 2
    c = orc.grid_points(amin, amax, res, L, jitter=False)
    for l in range(L):
        w = 3.0 * 2 ** l / res
        lo = -1.5 * 2 ** l
        idx = np.arange(res ** 3)
        i = np.stack([idx // (res * res), (idx // res) % res, idx % res], -1)
        np.testing.assert_allclose(c[l * res ** 3:(l + 1) * res ** 3], lo + (i + 0.5) * w, rtol=0, atol=1e-6)
    j = orc.grid_points(amin, amax, res, L, seed=7, step=3, jitter=True)
    for l in range(L):
        w = 3.0 * 2 ** l / res
        dev = (j[l * res ** 3:(l + 1) * res ** 3] - c[l * res ** 3:(l + 1) * res ** 3]) / w
        assert dev.min() >= -0.5 - 1e-5 and dev.max() < 0.5 + 1e-5
        assert abs(dev.mean()) < 0.02 and 0.08 < dev.var() < 0.093  # U(-1/2,1/2): var 1/12
    j2 = orc.grid_points(amin, amax, res, L, seed=7, step=4, jitter=True)
    assert not np.array_equal(j, j2)
    np.testing.assert_array_equal(j, orc.grid_points(amin, amax, res, L, seed=7, step=3, jitter=True))
    # the jitter of cell 0, axis 0 is the first published SplitMix64 output of the stream
    u0 = (orc.splitmix64_at(7 ^ (3 << 32), 0) >> 40) / 2 ** 24
    assert j[0, 0] == pytest.approx(-1.5 + u0 * 3.0 / res, abs=1e-6)


def _blob_density64(x, blobs):
    """float64 blob density at points x [n][3], written from the field's definition."""
    d2 = ((x[:, None, :] - blobs.mu.astype(np.float64)[None]) ** 2).sum(-1)
    s = blobs.std.astype(np.float64)[None]
    return (blobs.peak.astype(np.float64)[None] * np.exp(-d2 / (2 * s * s))).sum(1)


def test_density_grid_cells_and_bit_layout(orc):
    """Initial grid (cells occupied where the density at the cell centre exceeds
    0.01): float64 centres from the level geometry, float64 density, and the bit
    layout (cell c is bit c % 32 of word c // 32), away from threshold ties."""
    blobs = workloads.blob_field(4, 91)
    spec = workloads.GridSpec((-1.5,) * 3, (1.5,) * 3, 8, 2)
    bits, sig = orc.density_grid(spec, blobs, 0.01)
    res, L = spec.res, spec.n_levels
    idx = np.arange(res ** 3)
    i = np.stack([idx // (res * res), (idx // res) % res, idx % res], -1)
    x = np.concatenate([-1.5 * 2 ** l + (i + 0.5) * (3.0 * 2 ** l / res) for l in range(L)])
    dens = _blob_density64(x, blobs)
    np.testing.assert_allclose(sig, dens, rtol=1e-5, atol=1e-30)
    occ = workloads.unpack_bits(bits).astype(bool)
    clear = np.abs(dens - 0.01) > 1e-6 * 0.01
    np.testing.assert_array_equal(occ[clear], (dens > 0.01)[clear])
    assert 0 < occ.sum() < occ.size


def test_density_grid_contracted_cells(orc):
    """Grid over the contracted cube: a cell is occupied where the density at the
    scene point of its centre (the inverse contraction, float64 closed form
    x = c / (m'(2 - m')) for m' = max|c_a| > 1) exceeds 0.01."""
    blobs = workloads.Blobs(mu=np.array([[3.0, 0.5, -1.0], [0.2, 0.1, 0.0], [-6.0, 2.0, 1.0]], np.float32),
                            std=np.array([0.8, 0.2, 1.5], np.float32), peak=np.array([5.0, 8.0, 3.0], np.float32),
                            rgb=np.zeros((3, 3), np.float32))
    spec = workloads.GridSpec((-0.5,) * 3, (0.5,) * 3, 8, 3)  # level 2 covers [-2, 2]^3
    bits, sig = orc.density_grid_contracted(spec, blobs, 0.01)
    res, L = spec.res, spec.n_levels
    idx = np.arange(res ** 3)
    i = np.stack([idx // (res * res), (idx // res) % res, idx % res], -1)
    c = np.concatenate([-0.5 * 2 ** l + (i + 0.5) * (1.0 * 2 ** l / res) for l in range(L)])
    mp = np.abs(c).max(1)
    x = np.where((mp > 1)[:, None], c / (mp * (2 - mp))[:, None], c)
    dens = _blob_density64(x, blobs)
    occ = workloads.unpack_bits(bits).astype(bool)
    clear = np.abs(dens - 0.01) > 1e-4 * 0.01
    np.testing.assert_array_equal(occ[clear], (dens > 0.01)[clear])
    outer = mp > 1
    assert occ[outer].sum() > 5 and (~occ[outer]).sum() > 5  # the far blobs are found through the inverse


def test_update_grid_ema_closed_form(orc):
    """EMA of Sec. 3.1 (Eq. 4): constant input d gives e_k = g^k e_0 + (1-g^k) d."""
    n = 64 * 32
    g = workloads.rng(40)
    e0 = g.uniform(0, 1, n).astype(np.float32)
    d = g.uniform(0, 1, n).astype(np.float32)
    e = e0
    for _ in range(5):
        e, bits, mean = orc.update_grid(e, d, 0.95, 0.01)
    expect = 0.95 ** 5 * e0.astype(np.float64) + (1 - 0.95 ** 5) * d
    np.testing.assert_allclose(e, expect, rtol=1e-5)
    assert mean == pytest.approx(e.astype(np.float64).mean(), rel=1e-12)
    e1, _, _ = orc.update_grid(e0, d, 0.0, 0.01)
    np.testing.assert_array_equal(e1, d)


def test_update_grid_threshold_and_bit_layout(orc):
    """Binarisation 1[sigma > tau] (Table 1) with tau = 0.01 * mean, and the bit
    layout: element c is bit c % 32 of word c // 32."""
    n = 8 ** 3 * 2
    dens = np.zeros(n, np.float32)
    dens[[0, 33, 511, 700, 900]] = [5.0, 1.0, 0.00005, 2.0, 0.001]
    e, bits, mean = orc.update_grid(np.zeros(n, np.float32), dens, 0.0, 0.01)
    assert mean == pytest.approx(8.00105 / n, rel=1e-6)
    thr = 0.01 * 8.00105 / n
    assert thr > 0.00005  # cell 511 falls below 0.01 * mean
    assert thr < 0.001 < mean  # cell 900 lies above 0.01 * mean but below the mean
    assert bits[0] == 1 and bits[1] == 2 and bits[15] == 0 and bits[21] == 1 << (700 % 32)
    assert bits[28] == 1 << (900 % 32)
    assert workloads.unpack_bits(bits).sum() == 4
    _, bits_abs, _ = orc.update_grid(np.zeros(n, np.float32), dens, 0.0, 0.0, 1.5)
    assert workloads.unpack_bits(bits_abs).sum() == 2


# --------------------------------------------------------------------------
# inverse transform sampling (Eq. 1 with F = 1 - T, Eq. 3)
# --------------------------------------------------------------------------

def test_sample_pdf_uniform_weights_give_linspace(orc):
    """Sec. 3.1 "Uniform": constant PDF -> t_i = t_n + (t_f - t_n) u_i."""
    n, nb, no = 50, 64, 32
    g = workloads.rng(50)
    tn = g.uniform(1, 2, n)
    tf = tn + g.uniform(1, 3, n)
    edges = (tn[:, None] + (tf - tn)[:, None] * np.linspace(0, 1, nb + 1)[None]).astype(np.float32)
    out = orc.sample_pdf(edges, np.ones((n, nb), np.float32), no)
    expect = tn[:, None] + (tf - tn)[:, None] * np.linspace(0, 1, no + 1)[None]
    np.testing.assert_allclose(out, expect, rtol=0, atol=2e-6)
    out0 = orc.sample_pdf(edges, np.zeros((n, nb), np.float32), no)
    np.testing.assert_allclose(out0, expect, rtol=0, atol=2e-6)


def test_sample_pdf_piecewise_constant_inverse(orc):
    """Random piecewise-constant PDFs: outputs equal the analytic inverse CDF at
    u = k/N, and are non-decreasing."""
    n, nb, no = 40, 16, 24
    g = workloads.rng(51)
    edges = np.sort(g.uniform(0, 10, (n, nb + 1)), axis=1).astype(np.float32)
    w = g.uniform(0, 1, (n, nb)).astype(np.float32)
    w[g.random((n, nb)) < 0.3] = 0.0
    w[:, 0] = np.maximum(w[:, 0], 0.1)
    w[:, -1] = np.maximum(w[:, -1], 0.1)
    out = orc.sample_pdf(edges, w, no)
    for r in range(n):
        e = edges[r].astype(np.float64)
        F = np.concatenate([[0.0], np.cumsum(w[r].astype(np.float64))])
        F /= F[-1]
        for k in range(no + 1):
            u = k / no
            j = min(int(np.searchsorted(F, u, side="right")) - 1, nb - 1)
            t = e[j] + (u - F[j]) / (F[j + 1] - F[j]) * (e[j + 1] - e[j])
            if np.min(np.abs(F[1:-1] - u)) < 1e-6:
                continue  # tie with a flat region boundary
            assert out[r, k] == pytest.approx(t, rel=1e-5, abs=1e-5)
        assert np.all(np.diff(out[r]) >= 0)


def test_sample_pdf_single_bin_mass(orc):
    """All mass in one bin: every sample lies in that bin, evenly spaced (Eq. 1)."""
    nb, no = 10, 8
    edges = np.linspace(0, 10, nb + 1, dtype=np.float32)[None]
    w = np.zeros((1, nb), np.float32)
    w[0, 4] = 2.5
    out = orc.sample_pdf(edges, w, no)
    np.testing.assert_allclose(out[0], np.linspace(4, 5, no + 1), atol=1e-6)


def test_sample_pdf_stratified(orc):
    n, nb, no = 200, 8, 16
    edges = np.tile(np.linspace(0, 1, nb + 1, dtype=np.float32), (n, 1))
    out = orc.sample_pdf(edges, np.ones((n, nb), np.float32), no, stratified=True, seed=5)
    k = np.arange(no + 1)
    assert np.all(out[:, 0] == 0) and np.all(out[:, -1] == 1)
    inner = out[:, 1:-1] * no - k[None, 1:-1]  # = U_r, constant per ray, in [0, 1)
    assert np.all(inner >= -1e-4) and np.all(inner < 1 + 1e-4)
    assert np.allclose(inner, inner[:, :1], atol=1e-4)
    assert 0.4 < inner[:, 0].mean() < 0.6


# ---------------------------------------------------------------------------
# density-proposal network oracle (oracle/proposal.py)
# ---------------------------------------------------------------------------

def test_proposal_encoding_closed_forms():
    from oracle import proposal as P
    e = P.encode(np.array([[0.0, 0.5, 1.0 / 3.0]]))[0]
    assert e.shape == (64,) and np.all(e[51:] == 0.0)
    np.testing.assert_allclose(e[0:3], [0.0, 0.5, 1.0 / 3.0], rtol=0, atol=0)
    s3 = math.sqrt(3.0) / 2.0
    for k in range(8):
        sx, cx, sy, cy, sz, cz = e[3 + 6 * k: 9 + 6 * k]
        assert sx == 0.0 and cx == 1.0                                   # x = 0
        # y = 1/2: angle 2^k pi/2 -> (1, 0) for k = 0, (0, -1) for k = 1, (0, 1) after
        np.testing.assert_allclose([sy, cy], [(1, 0), (0, -1)][k] if k < 2 else (0, 1), atol=1e-12)
        # z = 1/3: angle 2^k pi/3; 2^k mod 6 cycles 1, 2, 4, 2, 4, ... (sin = +-sqrt3/2, cos = +-1/2)
        m = (2 ** k) % 6
        exp = {1: (s3, 0.5), 2: (s3, -0.5), 4: (-s3, -0.5)}[m]
        np.testing.assert_allclose([sz, cz], exp, atol=1e-12)


def test_proposal_forward_hand_built_network():
    """W1 copies x, y, z, b1 = 1/2, W2 = identity, b2 = -1/4, w3 sums the first
    three units, b3 = -1: density = softplus(sum_j relu(relu(x_j + 1/2) - 1/4) - 1)."""
    from oracle import proposal as P
    W1 = np.zeros((64, 64), np.float32)
    W1[0, 0] = W1[1, 1] = W1[2, 2] = 1.0
    w3 = np.zeros(64, np.float32)
    w3[:3] = 1.0
    p = {"W1": W1, "b1": np.full(64, 0.5, np.float32), "W2": np.eye(64, dtype=np.float32),
         "b2": np.full(64, -0.25, np.float32), "w3": w3, "b3": np.array([-1.0], np.float32)}
    x = np.array([[0.25, -0.5, 1.0], [-1.0, -0.75, 0.0], [0.5, 0.5, 0.5]])  # exact in bfloat16
    z = np.maximum(np.maximum(x + 0.5, 0.0) - 0.25, 0.0).sum(1) - 1.0
    np.testing.assert_allclose(P.forward(p, x)["sigma"], np.log1p(np.exp(z)), rtol=1e-15)


def test_bf16_rounding_matches_torch_bfloat16():
    """The network's operand precision: round to the nearest bfloat16, ties to
    even, bit for bit the same as torch's float32 -> bfloat16 conversion (an
    independent library routine), on random values and on hand-picked ties."""
    torch = pytest.importorskip("torch")
    from oracle import proposal as P
    g = workloads.rng(97)
    x = np.concatenate([g.standard_normal(200_000) * 10.0 ** g.integers(-6, 6, 200_000),
                        1.0 + np.array([2.0 ** -8, 3 * 2.0 ** -8, 2.0 ** -8 + 2.0 ** -20, -2.0 ** -9]),
                        np.array([0.0, -0.0, 1e-40, 3.0e38])]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    got = P.bf16(x).astype(np.float32)
    np.testing.assert_array_equal(got.view(np.uint32), ref.view(np.uint32))
    assert P.bf16(np.float32(1.0 + 2.0 ** -8)) == 1.0  # tie -> even mantissa
    assert P.bf16(np.float32(1.0 + 3 * 2.0 ** -8)) == 1.0 + 2.0 ** -6


def test_proposal_forward_rounds_every_operand():
    """Inputs, weights and both hidden layers enter the products as bfloat16
    (biases FP32): a hand-built network whose values are not representable in
    bfloat16, against the same network evaluated with torch's bfloat16
    conversion at each operand."""
    torch = pytest.importorskip("torch")
    from oracle import proposal as P

    def tb(v):
        return torch.tensor(np.asarray(v, np.float64), dtype=torch.float32).to(torch.bfloat16).double().numpy()

    W1 = np.zeros((64, 64), np.float32)
    W1[0, 0], W1[1, 1], W1[2, 2] = 1.0 + 2.0 ** -10, 0.7, 1.3
    W2 = np.eye(64, dtype=np.float32) * np.float32(0.9)
    w3 = np.zeros(64, np.float32)
    w3[:3] = [1.1, 0.6, 0.85]
    p = {"W1": W1, "b1": np.full(64, 1.0 / 3.0, np.float32), "W2": W2, "b2": np.full(64, -0.1, np.float32),
         "w3": w3, "b3": np.array([-0.2], np.float32)}
    x = np.array([[0.1234, -0.05, 0.77], [0.3, 0.3001, -0.2], [0.91, 0.42, 0.05]])
    e = tb(x)  # the first three encoding entries are the coordinates
    z1 = e * tb(np.diag(W1)[:3])[None] + np.float32(1.0 / 3.0)
    h1 = tb(np.maximum(z1, 0.0))
    z2 = h1 * tb(np.float32(0.9)) + np.float32(-0.1)
    h2 = tb(np.maximum(z2, 0.0))
    z3 = h2 @ tb(w3[:3]) + np.float32(-0.2)
    np.testing.assert_allclose(P.forward(p, x)["sigma"], np.log1p(np.exp(z3)), rtol=1e-12)


def test_proposal_gradients_match_finite_differences():
    from oracle import proposal as P
    g0 = np.random.default_rng(11)
    x = g0.uniform(-1.5, 1.5, (64, 3))
    t = g0.uniform(0.0, 5.0, 64)
    p = P.init_params(3)
    p["b1"] = g0.uniform(-0.2, 0.2, 64).astype(np.float32)
    p["b2"] = g0.uniform(-0.2, 0.2, 64).astype(np.float32)
    _, g = P.loss_and_grads(p, x, t, round_bf16=False)
    # in every parameter group the three entries with the largest gradient (so
    # no check is vacuous on a dead unit) and two random ones
    picks = []
    for name in ("W1", "b1", "W2", "b2", "w3", "b3"):
        a = np.abs(np.asarray(g[name]))
        flat = list(np.argsort(a.reshape(-1))[::-1][:3]) + list(g0.integers(0, a.size, 2))
        assert a.max() > 1e-3, name
        picks += [(name, np.unravel_index(int(i), a.shape)) for i in flat]
    for name, idx in picks:
        q = {k: v.astype(np.float64) for k, v in p.items()}
        h = 1e-6
        q[name][idx] += h
        lp = P.loss_and_grads(q, x, t, round_bf16=False)[0]
        q[name][idx] -= 2 * h
        lm = P.loss_and_grads(q, x, t, round_bf16=False)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[name][idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, g[name][idx])


def test_proposal_adam_first_step_closed_form():
    """First step: m_hat = g, v_hat = g^2, so p -= lr g / (|g| + eps)."""
    from oracle import proposal as P
    p = {"b1": np.array([1.0, -2.0, 0.5], np.float32)}
    g = {"b1": np.array([0.3, -0.01, 0.0])}
    st = {}
    P.adam_step(p, g, st, lr=0.01)
    exp = np.array([1.0, -2.0, 0.5]) - 0.01 * g["b1"] / (np.abs(g["b1"]) + 1e-8)
    np.testing.assert_allclose(p["b1"], exp.astype(np.float32), rtol=0, atol=0)


def test_exact_optical_depth_matches_fine_quadrature(orc):
    """The closed-form line integral of the 8-blob field equals the oracle's
    FP64 compositing of a fine lattice (Eq. 2, dt -> 0) on a few rays; every
    other ray's direction is scaled to length 1.7 (the integral is over t, not
    arc length)."""
    from oracle import proposal as P
    w = workloads.c1_forward(6)
    rd = w.rays_d.copy()
    rd[::2] *= np.float32(1.7)
    tn, tf, hit = orc.ray_clip(w.rays_o, rd, (-1.5,) * 3, (1.5,) * 3, 128, 1, 0.0, 1e10)
    exact = P.exact_optical_depth(w.rays_o, rd, tn.astype(np.float64), tf.astype(np.float64),
                                  w.blobs.mu, w.blobs.std, w.blobs.peak)
    for r in np.nonzero(hit)[0]:
        N = 40000
        ts = np.linspace(tn[r], tf[r], N + 1)
        t0, t1 = ts[:-1].astype(np.float32), ts[1:].astype(np.float32)
        sig, rgb = orc.field_samples(w.rays_o[r:r + 1], rd[r:r + 1], np.zeros(N, np.int32), t0, t1, w.blobs)
        out = orc.render_fwd(np.array([0, N]), t0, t1, sig, rgb)
        assert -math.log(out["trans"][0]) == pytest.approx(exact[r], rel=2e-4, abs=1e-6)
    assert hit.sum() >= 3


# ---------------------------------------------------------------------------
# estimator-update variants (oracle/grid_variants.py)
# ---------------------------------------------------------------------------

def test_sample_cells_of_cell_centres_and_of_march_samples(orc):
    """A sample whose ray does not move (d = 0) sits at o: at a cell centre
    its cell is that cell.  Every sample the oracle march emits lies in an
    occupied cell (the lattice definition both share)."""
    from oracle import grid_variants as G
    res, L = 16, 3
    geom = orc.level_geometry((-1.5,) * 3, (1.5,) * 3, res, L)
    centres = orc.grid_points((-1.5,) * 3, (1.5,) * 3, res, L, jitter=False)
    n = centres.shape[0]
    cells = G.sample_cells(centres, np.zeros((n, 3), np.float32), np.arange(n), np.zeros(n, np.float32),
                           np.ones(n, np.float32), geom, res)
    # a centre belongs to the finest level whose box (half-width 1.5 * 2^l) holds it:
    # its own cell when that is its own level, else a cell of that finer level
    lvl = np.arange(n) // res ** 3
    finest = np.argmax(np.abs(centres).max(1)[:, None] <= 1.5 * 2.0 ** np.arange(L)[None, :], axis=1)
    own = cells == np.arange(n)
    assert own[finest == lvl].all()
    assert np.array_equal(cells[finest < lvl] // res ** 3, finest[finest < lvl]) and (finest < lvl).sum() > 100
    bits = workloads.random_bitfield(L, res, 31, p_block=0.5, block=4, p_cell=0.5)
    w = workloads.c1_forward(500)
    ex = orc.march(w.rays_o, w.rays_d, (-1.5,) * 3, (1.5,) * 3, res, L, bits, 0.02, 1024, 0.0, 1e10)
    c = G.sample_cells(w.rays_o, w.rays_d, ex["ray_indices"], ex["t_starts"], ex["t_ends"], geom, res)
    occ = workloads.unpack_bits(bits)
    assert len(c) > 1000 and (c >= 0).all() and occ[c].all()


def test_density_scatter_is_the_adjoint_of_lookup():
    """<lookup(density), g> = <density, backward(g)> for any density and g."""
    from oracle import grid_variants as G
    g0 = np.random.default_rng(5)
    cells = g0.integers(-1, 50, 400)
    dens = g0.standard_normal(50)
    gs = g0.standard_normal(400)
    lhs = float(G.density_lookup(dens, cells).astype(np.float64) @ gs)
    rhs = float(dens.astype(np.float32).astype(np.float64) @ G.density_backward(gs, cells, 50))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_sgd_step_and_frames_max_hand_examples():
    from oracle import grid_variants as G
    d, b = G.sgd_step(np.array([1.0, 0.5, 0.02, 3.0], np.float32), np.array([0.5, 2.0, -0.25, 0.0]), 0.5, 0.1)
    np.testing.assert_array_equal(d, np.array([0.75, 0.0, 0.145, 3.0], np.float32))
    np.testing.assert_array_equal(b, [True, False, True, True])
    np.testing.assert_array_equal(G.frames_max([[1.0, 5.0, 0.0], [2.0, -1.0, 0.0], [0.5, 4.0, 3.0]]), [2.0, 5.0, 3.0])


# ---------------------------------------------------------------------------
# unbounded scenes: contraction, s -> t, s-lattice march
# ---------------------------------------------------------------------------

def test_contraction_closed_forms(orc):
    g0 = np.random.default_rng(7)
    inner = g0.uniform(-1.0, 1.0, (200, 3)).astype(np.float32)
    np.testing.assert_array_equal(orc.contract(inner), inner)  # identity inside the unit cube
    v = g0.uniform(-1.0, 1.0, (200, 3))
    v /= np.abs(v).max(1, keepdims=True)  # max|v_a| = 1
    lam = g0.uniform(1.0, 1e4, 200)
    x = (v * lam[:, None]).astype(np.float32)
    c = orc.contract(x).astype(np.float64)
    lam32 = np.abs(x).max(1).astype(np.float64)
    np.testing.assert_allclose(c, x * ((2.0 - 1.0 / lam32) / lam32)[:, None], rtol=3e-7, atol=1e-7)
    assert np.all(np.abs(c) < 2.0) and np.all(np.abs(c).max(1) >= 1.0)
    # the FP64 inverse of the FP32 image: 2 - 1/lam carries a rounding of ~1e-7,
    # amplified by lam in the inverse
    err = np.abs(orc.uncontract(c) - x).max(1) / lam32
    assert np.all(err <= 3e-7 * lam32 + 1e-6), err.max()


def test_uncontract32_inverts_the_contraction(orc):
    """The FP32 inverse against the FP64 closed form y * (1 / (2 - m')) / m',
    the identity inside the unit cube, the clamp at m' >= 2 and a round trip."""
    g0 = np.random.default_rng(8)
    inner = g0.uniform(-1.0, 1.0, (100, 3)).astype(np.float32)
    np.testing.assert_array_equal(orc.uncontract32(inner), inner)
    v = g0.uniform(-1.0, 1.0, (300, 3))
    v /= np.abs(v).max(1, keepdims=True)
    mp = g0.uniform(1.0, 1.999, 300)
    c = (v * mp[:, None]).astype(np.float32)
    m32 = np.abs(c).max(1).astype(np.float64)
    x = orc.uncontract32(c).astype(np.float64)
    ref = c * ((1.0 / (2.0 - m32)) / m32)[:, None]
    # three FP32 roundings, the first (2 - m') exact by Sterbenz
    np.testing.assert_allclose(x, ref, rtol=4e-7, atol=0)
    assert np.all(np.abs(x).max(1) >= 1.0)
    np.testing.assert_allclose(orc.contract(x.astype(np.float32)), c, rtol=0, atol=2e-6)
    edge = np.array([[2.0, 0.5, -1.0], [-3.0, 0.0, 0.0]], np.float32)
    xe = orc.uncontract32(edge).astype(np.float64)
    big = 1.0 / (2.0 - np.float64(np.float32(1.99999988)))  # 2^23
    assert big == 2.0 ** 23
    np.testing.assert_allclose(xe[0], edge[0] * (big / 2.0), rtol=1e-7)
    np.testing.assert_allclose(xe[1], edge[1] * (big / 3.0), rtol=1e-7)


def test_s_to_t_is_disparity_linear(orc):
    tn, tf = 0.2, 1000.0
    s = np.linspace(0.0, 1.0, 257)
    t = orc.s_to_t(s, tn, tf).astype(np.float64)
    assert t[0] == pytest.approx(tn, rel=2e-7) and t[-1] == pytest.approx(tf, rel=2e-7)
    assert np.all(np.diff(t) > 0)
    np.testing.assert_allclose(1.0 / t, (1 - s) / tn + s / tf, rtol=1e-6)


def test_unbounded_march_full_grid_emits_every_lattice_point(orc):
    w = workloads.c5_unbounded(n_cams=1, width=16, height=8, res=16)
    bits = np.full(w.grid.n_cells // 32, 0xFFFFFFFF, np.uint32)
    K = 64
    ex = orc.march_unbounded(w.rays_o, w.rays_d, w.grid.aabb_min, w.grid.aabb_max, 16, 4, bits, K, 0.2, 1000.0)
    assert np.all(np.diff(ex["offsets"]) == K)
    s = (np.arange(K, dtype=np.float32) / np.float32(K)).astype(np.float32)
    np.testing.assert_array_equal(ex["t_starts"][:K], orc.s_to_t(s, 0.2, 1000.0))


def test_unbounded_march_matches_fp64_geometry(orc):
    """Samples away from cell faces: emitted iff the FP64 contracted midpoint
    falls in an occupied cell of the finest level holding it."""
    w = workloads.c5_unbounded(n_cams=2, width=24, height=8, res=16)
    res, L, K = 16, 4, 128
    bits = workloads.random_bitfield(L, res, 77, p_block=0.5, block=4, p_cell=0.5)
    occ = workloads.unpack_bits(bits)
    ex = orc.march_unbounded(w.rays_o, w.rays_d, w.grid.aabb_min, w.grid.aabb_max, res, L, bits, K, 0.2, 1000.0)
    geom = orc.level_geometry(w.grid.aabb_min, w.grid.aabb_max, res, L).astype(np.float64)
    s = np.arange(K + 1) / K
    tt = 1.0 / ((1 - s) / 0.2 + s / 1000.0)
    got = set(zip(ex["ray_indices"].tolist(), ex["t_starts"].tolist()))
    t0s = orc.s_to_t(s[:-1], 0.2, 1000.0)
    checked = 0
    for r in range(w.n_rays):
        o, d = w.rays_o[r].astype(np.float64), w.rays_d[r].astype(np.float64)
        for k in range(K):
            x = o + d * 0.5 * (tt[k] + tt[k + 1])
            m = np.abs(x).max()
            c = x if m <= 1 else x * (2 - 1 / m) / m
            lv = next((l for l in range(L) if np.all(c >= geom[l, 0]) and np.all(c <= geom[l, 1])), None)
            if lv is None:
                assert (r, float(t0s[k])) not in got
                continue
            u = (c - geom[lv, 0]) * geom[lv, 2]
            if np.min(np.abs(u - np.round(u))) < 1e-3:
                continue  # within rounding of a face
            ic = np.clip(np.floor(u).astype(int), 0, res - 1)
            idx = lv * res ** 3 + (ic[0] * res + ic[1]) * res + ic[2]
            assert bool(occ[idx]) == ((r, float(t0s[k])) in got), (r, k)
            checked += 1
    assert checked > 5000


def test_unbounded_early_termination_cut(orc):
    """The unbounded march with the field emits a prefix of its field-less
    march, cut where the float64 optical depth of the emitted samples first
    exceeds -ln(1e-4) (Sec. 4.2 filtering on the s-lattice of Sec. 3.2)."""
    w = workloads.c5_unbounded(n_cams=2, width=32, height=8, res=32)
    bits, _ = orc.density_grid_contracted(w.grid, w.blobs)
    g, m = w.grid, w.march
    K = 512
    full = orc.march_unbounded(w.rays_o, w.rays_d, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, K,
                               m.t_min, m.t_max)
    cut = orc.march_unbounded(w.rays_o, w.rays_d, g.aabb_min, g.aabb_max, g.res, g.n_levels, bits, K,
                              m.t_min, m.t_max, blobs=w.blobs, eps=1e-4)
    thr = -math.log(1e-4)
    sig, _ = orc.field_samples(w.rays_o, w.rays_d, full["ray_indices"], full["t_starts"], full["t_ends"], w.blobs)
    tau = sig * (full["t_ends"].astype(np.float64) - full["t_starts"])
    n_cut = 0
    for r in range(w.n_rays):
        fs, fe = full["offsets"][r], full["offsets"][r + 1]
        cs, ce = cut["offsets"][r], cut["offsets"][r + 1]
        nc = ce - cs
        assert nc <= fe - fs
        np.testing.assert_array_equal(cut["t_starts"][cs:ce], full["t_starts"][fs:fs + nc])
        P = np.concatenate([[0.0], np.cumsum(tau[fs:fe])])
        if nc > 0:
            assert P[nc - 1] <= thr * (1 + 1e-5)
        if nc < fe - fs:
            n_cut += 1
            assert P[nc] > thr * (1 - 1e-5)
    assert n_cut > 100
