"""Planted mistakes in the oracle: each must fail at least one of its pins.

The pins in ``test_oracle_pins.py`` only prove the oracle right if they can
tell it from a plausible wrong version of itself.  Each case below plants one
such mistake -- a dropped term, a wrong sign, an off-by-one lattice index, a
transposed cell index, the wrong end of an interval, a swapped EMA weight, a
left-side CDF search -- in a copy of the oracle (a one-line edit of
``oracle.c`` compiled into a temporary library, or of a numpy module loaded
under a temporary name), points the oracle package at the copy, runs the pins
that cover the edited function, and requires at least one of them to fail.
Nothing here touches the CUDA library; every mistake is planted on the CPU.
"""
import inspect
import os
import subprocess
import types

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# (name, function whose body is edited, text replaced, replacement, pins that must catch it)
C_MUTANTS = [
    ("march: occupancy tested at t0, not the midpoint", "static int64_t orc_march_ray(",
     "float tm = (t0 + t1) * 0.5f;", "float tm = t0;",
     ["test_single_occupied_cell", "test_brute_force_random_grids"]),
    ("march: lattice starts one step late", "static int64_t orc_march_ray(",
     "float t0 = tn + (float)k * step;", "float t0 = tn + (float)(k + 1) * step;",
     ["test_uniform_special_case", "test_brute_force_random_grids"]),
    ("march: interval end not advanced by one step", "static int64_t orc_march_ray(",
     "float t1 = t0 + step;", "float t1 = t0 + 0.5f * step;",
     ["test_uniform_special_case", "test_brute_force_random_grids"]),
    ("march: early-stop depth drops dt", "static int64_t orc_march_ray(",
     "tau = tau + s * dt;", "tau = tau + s;", ["test_early_termination_cut"]),
    ("march: early stop tests the depth after the sample", "static int64_t orc_march_ray(",
     "if (fld && tau > fld->thr) break;",
     "if (fld && tau + orc_sigma_f32(x, fld->n_blobs, fld->mu, fld->stdv, fld->peak) * (t1 - t0) > fld->thr) break;",
     ["test_early_termination_cut"]),
    ("clip: near plane of the box ignored", "static int orc_clip(",
     "if (lo > near) near = lo;", "if (0) near = lo;",
     ["test_uniform_special_case", "test_miss_and_inside_origin", "test_ray_clip_matches_float64_slab"]),
    ("clip: far plane of the box ignored", "static int orc_clip(",
     "if (hi < far) far = hi;", "if (0) far = hi;",
     ["test_ray_clip_matches_float64_slab"]),
    ("clip: zero direction component treated as a hit", "static int orc_clip(",
     "if (o[a] < outer->lmin[a] || o[a] > outer->lmax[a]) return 0;", "if (0) return 0;",
     ["test_ray_clip_matches_float64_slab"]),
    ("occupancy: cell index axes transposed", "static int orc_occupied(",
     "(i[0] * res + i[1]) * res + i[2]", "(i[2] * res + i[1]) * res + i[0]",
     ["test_single_occupied_cell", "test_brute_force_random_grids"]),
    ("occupancy: coarsest level searched first", "static int orc_occupied(",
     "for (int l = 0; l < L; ++l) {", "for (int l = L - 1; l >= 0; --l) {",
     ["test_cascade_selects_finest_level"]),
    ("occupancy: half-open level box", "static int orc_occupied(",
     "if (!(x[a] >= lv[l].lmin[a] && x[a] <= lv[l].lmax[a])) inside = 0;",
     "if (!(x[a] >= lv[l].lmin[a] && x[a] < lv[l].lmax[a])) inside = 0;", ["test_level_box_is_closed"]),
    ("occupancy: cell from the box width, not its scale", "static int orc_occupied(",
     "float u = (x[a] - lv[l].lmin[a]) * lv[l].scale[a];", "float u = (x[a] - lv[l].lmin[a]) * lv[l].width[a];",
     ["test_single_occupied_cell", "test_brute_force_random_grids"]),
    ("levels: boxes not scaled by 2^l", "static void orc_levels(",
     "float hs = half * f;", "float hs = half;",
     ["test_level_geometry_is_box_scaled_about_centre", "test_cascade_selects_finest_level"]),
    ("render: background dropped", "void orc_render_fwd(",
     "rgb_out[3 * r + a] = acc[a] + TN * bg[a];", "rgb_out[3 * r + a] = acc[a];",
     ["test_homogeneous_slab_closed_form", "test_weights_sum_to_one_minus_transmittance"]),
    ("render: first background channel for all three", "void orc_render_fwd(",
     "for (int a = 0; a < 3; ++a) rgb_out[3 * r + a] = acc[a] + TN * bg[a];",
     "for (int a = 0; a < 3; ++a) rgb_out[3 * r + a] = acc[a] + TN * bg[0];",
     ["test_homogeneous_slab_closed_form"]),
    ("adjoint: first background channel for all three", "void orc_render_bwd(",
     "g += gC[a] * (Tn * rgbs[3 * i + a] - Sc[a] - TN * bg[a]);",
     "g += gC[a] * (Tn * rgbs[3 * i + a] - Sc[a] - TN * bg[0]);",
     ["test_gradient_matches_finite_differences"]),
    ("render: inclusive instead of exclusive transmittance", "void orc_render_fwd(",
     "double T = exp(-P);", "double T = exp(-(P + tau));",
     ["test_homogeneous_slab_closed_form", "test_weights_sum_to_one_minus_transmittance"]),
    ("render: alpha from the density without the interval length", "void orc_render_fwd(",
     "double tau = sigmas[i] * dt;", "double tau = sigmas[i];",
     ["test_homogeneous_slab_closed_form", "test_line_integral_of_gaussian_blob"]),
    ("render: depth at t0 instead of the midpoint", "void orc_render_fwd(",
     "dep += w * 0.5 * ((double)t0[i] + (double)t1[i]);", "dep += w * (double)t0[i];",
     ["test_homogeneous_slab_closed_form"]),
    ("render: mask threshold never reached", "void orc_render_fwd(",
     "if (!masked && P > thr) masked = 1;", "if (!masked && P > 2.0 * thr) masked = 1;",
     ["test_mask_mode_zeroes_weights_below_eps"]),
    ("adjoint: background term with the wrong sign", "void orc_render_bwd(",
     "- Sc[a] - TN * bg[a]);", "- Sc[a] + TN * bg[a]);",
     ["test_gradient_matches_finite_differences"]),
    ("adjoint: T_i in place of T_{i+1}", "void orc_render_bwd(",
     "g += gC[a] * (Tn * rgbs[3 * i + a]", "g += gC[a] * (Ti * rgbs[3 * i + a]",
     ["test_gradient_matches_finite_differences"]),
    ("adjoint: depth suffix sum never accumulated", "void orc_render_bwd(",
     "Sm += w * m;", "Sm += 0.0 * m;", ["test_gradient_matches_finite_differences"]),
    ("adjoint: opacity term dropped", "void orc_render_bwd(",
     "g += gA * TN;", "g += 0.0 * gA;", ["test_gradient_matches_finite_differences"]),
    ("adjoint: masked samples' cut ignored", "void orc_render_bwd(",
     "if (acc > thr) { cut = j; break; }", "if (0) { cut = j; break; }",
     ["test_gradient_mask_mode_finite_differences"]),
    ("SplitMix64: wrong mixing constant", "uint64_t orc_splitmix64_at(",
     "0xBF58476D1CE4E5B9ull", "0xBF58476D1CE4E5B1ull", ["test_splitmix64_published_vector"]),
    ("SplitMix64: stream starts at element 0 instead of 1", "uint64_t orc_splitmix64_at(",
     "(counter + 1u)", "counter", ["test_splitmix64_published_vector"]),
    ("grid points: centre offset 0 instead of 1/2", "void orc_grid_points(",
     ": 0.5f;", ": 0.0f;", ["test_grid_points_centres_and_jitter"]),
    ("grid points: one jitter for all three axes", "void orc_grid_points(",
     "(uint64_t)(3 * c + a)", "(uint64_t)(3 * c)", ["test_grid_points_centres_and_jitter"]),
    ("EMA: decay and its complement swapped", "void orc_update_grid(",
     "float a = decay * ema[c];", "float a = omd * ema[c];",
     ["test_update_grid_ema_closed_form"]),
    ("EMA: threshold at the mean, not a fraction of it", "void orc_update_grid(",
     "double thr = (double)thresh_frac * mean;", "double thr = mean;",
     ["test_update_grid_threshold_and_bit_layout"]),
    ("EMA: bits packed most significant first", "void orc_update_grid(",
     "bits_out[c >> 5] |= 1u << (c & 31);", "bits_out[c >> 5] |= 1u << (31 - (c & 31));",
     ["test_update_grid_threshold_and_bit_layout"]),
    ("inverse CDF: left-side bin search", "void orc_sample_pdf(",
     "if (F[jj] <= u && F[jj] < 1.0f) j = jj;", "if (F[jj] < u && F[jj] < 1.0f) j = jj;",
     ["test_sample_pdf_single_bin_mass", "test_sample_pdf_piecewise_constant_inverse",
      "test_sample_pdf_uniform_weights_give_linspace"]),
    ("inverse CDF: position inside the bin not normalised", "void orc_sample_pdf(",
     "t = e[j] + ((u - F[j]) / den) * (e[j + 1] - e[j]);", "t = e[j] + (u - F[j]) * (e[j + 1] - e[j]);",
     ["test_sample_pdf_piecewise_constant_inverse", "test_sample_pdf_uniform_weights_give_linspace"]),
    ("inverse CDF: stratified offset not applied", "void orc_sample_pdf(",
     "u = ((float)k + U) / (float)n_out;", "u = (float)k / (float)n_out;",
     ["test_sample_pdf_stratified"]),
    ("contraction: 2 + 1/m instead of 2 - 1/m", "void orc_contract(",
     "float f = 2.0f - inv;", "float f = 2.0f + inv;", ["test_contraction_closed_forms"]),
    ("inverse contraction: divides by 2 + m'", "void orc_uncontract_points(",
     "float den = 2.0f - mc;", "float den = 2.0f + mc;", ["test_uncontract32_inverts_the_contraction"]),
    ("Phi: ends of the disparity map swapped", "float orc_s_to_t(",
     "float den = a * (1.0f - s) + b * s;", "float den = a * s + b * (1.0f - s);",
     ["test_s_to_t_is_disparity_linear"]),
    ("unbounded march: occupancy of the uncontracted point", "static int64_t orc_march_unb_ray(",
     "if (!orc_occupied(c, lv, L, res, bits)) continue;", "if (!orc_occupied(x, lv, L, res, bits)) continue;",
     ["test_unbounded_march_matches_fp64_geometry"]),
    ("unbounded march: s-lattice of K + 1 points", "static int64_t orc_march_unb_ray(",
     "float s0 = (float)k / (float)K, s1 = (float)(k + 1) / (float)K;",
     "float s0 = (float)k / (float)(K + 1), s1 = (float)(k + 1) / (float)(K + 1);",
     ["test_unbounded_march_full_grid_emits_every_lattice_point"]),
    ("unbounded march: early-stop depth drops dt", "static int64_t orc_march_unb_ray(",
     "tau = tau + sg * dt;", "tau = tau + sg;", ["test_unbounded_early_termination_cut"]),
    ("field: Gaussian exponent without the factor 2", "static void orc_field_f64(",
     "exp(-r2 / (2.0 * sd * sd))", "exp(-r2 / (sd * sd))",
     ["test_line_integral_of_gaussian_blob"]),
    ("field: colour not normalised by the density", "static void orc_field_f64(",
     "c[a] = s > 0.0 ? acc[a] / s : 0.0;", "c[a] = acc[a];",
     ["test_line_integral_of_gaussian_blob"]),
    ("march field: FP32 Gaussian exponent without the 1/2", "static float orc_sigma_f32(",
     "float coef = -0.5f / sd2;", "float coef = -1.0f / sd2;", ["test_early_termination_cut"]),
    ("defined exponential: degree-6 Taylor polynomial", "float orc_exp_steps(",
     "float p = c[7];", "float p = 0.0f;", ["test_exp_steps_against_float64_exp"]),
    ("defined exponential: low part of ln 2 dropped", "float orc_exp_steps(",
     "r = r - n * lo;", "r = r - 0.0f * lo;", ["test_exp_steps_against_float64_exp"]),
    ("defined exponential: reduction by truncation, not rounding", "float orc_exp_steps(",
     "float n = rintf(a * l2e);", "float n = truncf(a * l2e);", ["test_exp_steps_against_float64_exp"]),
    ("defined exponential: scale off by one binade", "float orc_exp_steps(",
     "uint32_t sb = (uint32_t)((int)n + 127) << 23;", "uint32_t sb = (uint32_t)((int)n + 126) << 23;",
     ["test_exp_steps_against_float64_exp"]),
    ("defined exponential: no cut below -86", "float orc_exp_steps(",
     "if (!(a >= -86.0f)) return 0.0f;", "if (!(a >= -200.0f)) return 0.0f;",
     ["test_exp_steps_against_float64_exp"]),
    ("render: alpha linearised (tau instead of 1 - exp(-tau))", "void orc_render_fwd(",
     "double w = T * -expm1(-tau);", "double w = T * tau;",
     ["test_homogeneous_slab_closed_form", "test_weights_sum_to_one_minus_transmittance"]),
    ("grid points: every level placed on level 0's lattice", "void orc_grid_points(",
     "xyz_out[3 * c + a] = lv[l].lmin[a] + q * lv[l].width[a];",
     "xyz_out[3 * c + a] = lv[0].lmin[a] + q * lv[0].width[a];", ["test_grid_points_centres_and_jitter"]),
    ("EMA: mean over n - 1 cells", "void orc_update_grid(",
     "double mean = n_cells > 0 ? sum / (double)n_cells : 0.0;",
     "double mean = n_cells > 1 ? sum / (double)(n_cells - 1) : 0.0;",
     ["test_update_grid_threshold_and_bit_layout"]),
    ("inverse CDF: last CDF value not forced to 1", "void orc_sample_pdf(",
     "F[n_bins] = 1.0f;", "F[n_bins] = F[n_bins - 1];",
     ["test_sample_pdf_uniform_weights_give_linspace", "test_sample_pdf_piecewise_constant_inverse"]),
    ("inverse CDF: zero total weight gives a degenerate CDF", "void orc_sample_pdf(",
     "for (int j = 0; j <= n_bins; ++j) F[j] = (float)j / (float)n_bins;",
     "for (int j = 0; j <= n_bins; ++j) F[j] = 0.0f;",
     ["test_sample_pdf_uniform_weights_give_linspace"]),
    ("inverse contraction: no clamp below m' = 2", "void orc_uncontract_points(",
     "float mc = mp < mmax ? mp : mmax;", "float mc = mp;", ["test_uncontract32_inverts_the_contraction"]),
]

# mistakes planted in one function of the oracle package's numpy wrappers
# (function, text replaced, replacement, pins that must catch it)
WRAPPER_MUTANTS = [
    ("density_grid", "words = occ.reshape(-1, 32).astype(np.uint64) << np.arange(32, dtype=np.uint64)",
     "words = occ.reshape(-1, 32).astype(np.uint64) << (31 - np.arange(32, dtype=np.uint64))",
     ["test_density_grid_cells_and_bit_layout"]),
    ("density_grid", "occ = sig > thresh", "occ = sig > 10.0 * thresh", ["test_density_grid_cells_and_bit_layout"]),
    ("density_grid_contracted", "sig = field_points(uncontract32(pts), blobs, n_threads)",
     "sig = field_points(pts, blobs, n_threads)", ["test_density_grid_contracted_cells"]),
    ("update_grid", "e = np.array(ema, dtype=np.float32, copy=True)", "e = np.zeros_like(np.asarray(ema, np.float32))",
     ["test_update_grid_ema_closed_form"]),
]

PY_MUTANTS = [
    ("proposal", "encoding: sin and cos swapped",
     "e[:, 3 + 6 * k + 2 * a] = np.sin(ang[:, a])", "e[:, 3 + 6 * k + 2 * a] = np.cos(ang[:, a])",
     ["test_proposal_encoding_closed_forms"]),
    ("proposal", "encoding: bands at k pi instead of 2^k pi",
     "ang = (2.0 ** k) * np.pi * x", "ang = (k + 1.0) * np.pi * x",
     ["test_proposal_encoding_closed_forms"]),
    ("proposal", "network: second ReLU dropped",
     "h2 = r(np.maximum(z2, 0.0))", "h2 = r(z2)", ["test_proposal_forward_hand_built_network"]),
    ("proposal", "network: bias of the first layer dropped",
     "z1 = e @ W1.T + b1", "z1 = e @ W1.T", ["test_proposal_forward_hand_built_network",
                                            "test_proposal_gradients_match_finite_differences"]),
    ("proposal", "adjoint: softplus derivative with the wrong sign",
     "/ (1.0 + np.exp(-f[\"z3\"]))", "/ (1.0 + np.exp(f[\"z3\"]))",
     ["test_proposal_gradients_match_finite_differences"]),
    ("proposal", "adjoint: bias gradient of the second layer averaged instead of summed",
     'g["W2"], g["b2"] = d2.T @ f["h1"], d2.sum(0)', 'g["W2"], g["b2"] = d2.T @ f["h1"], d2.mean(0)',
     ["test_proposal_gradients_match_finite_differences"]),
    ("proposal", "adjoint: ReLU mask of the first layer missing",
     "d1 = (d2 @ W2) * (f[\"z1\"] > 0)", "d1 = (d2 @ W2)",
     ["test_proposal_gradients_match_finite_differences"]),
    ("proposal", "Adam: no bias correction",
     "mh, vh = m / (1 - b1 ** t), v / (1 - b2 ** t)", "mh, vh = m, v",
     ["test_proposal_adam_first_step_closed_form"]),
    ("proposal", "BF16: ties rounded away from zero",
     "u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16", "u = ((u + 0x8000) >> 16) << 16",
     ["test_bf16_rounding_matches_torch_bfloat16"]),
    ("proposal", "BF16: truncation instead of rounding",
     "u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16", "u = (u >> 16) << 16",
     ["test_bf16_rounding_matches_torch_bfloat16", "test_proposal_forward_rounds_every_operand"]),
    ("proposal", "network: first hidden layer not rounded to BF16",
     "h1 = r(np.maximum(z1, 0.0))", "h1 = np.maximum(z1, 0.0)", ["test_proposal_forward_rounds_every_operand"]),
    ("proposal", "network: weights not rounded to BF16",
     'W1, W2, w3 = r(params["W1"]), r(params["W2"]), r(params["w3"])',
     'W1, W2, w3 = (np.asarray(params[k], np.float64) for k in ("W1", "W2", "w3"))',
     ["test_proposal_forward_rounds_every_operand"]),
    ("proposal", "exact depth: closest approach without the 1/|d|^2",
     "ts = (m @ d[i]) / dd", "ts = (m @ d[i])", ["test_exact_optical_depth_matches_fine_quadrature"]),
    ("grid_variants", "sample cells: the coarsest level wins",
     "for l in range(L - 1, -1, -1):", "for l in range(L):",
     ["test_sample_cells_of_cell_centres_and_of_march_samples"]),
    ("grid_variants", "sample cells: cell index axes transposed",
     "(ic[:, 0] * res + ic[:, 1]) * res + ic[:, 2]", "(ic[:, 2] * res + ic[:, 1]) * res + ic[:, 0]",
     ["test_sample_cells_of_cell_centres_and_of_march_samples"]),
    ("grid_variants", "density adjoint: samples of one cell overwrite instead of adding up",
     "np.add.at(g, cells[ok], np.asarray(g_sigma, np.float64)[ok])",
     "g[cells[ok]] = np.asarray(g_sigma, np.float64)[ok]",
     ["test_density_scatter_is_the_adjoint_of_lookup"]),
    ("grid_variants", "SGD: step up the gradient",
     "(np.asarray(density, f) - (f(lr)", "(np.asarray(density, f) + (f(lr)",
     ["test_sgd_step_and_frames_max_hand_examples"]),
    ("grid_variants", "dynamic grid: mean over frames instead of the maximum",
     "return np.max(np.asarray(densities, np.float32), axis=0)",
     "return np.mean(np.asarray(densities, np.float32), axis=0)",
     ["test_sgd_step_and_frames_max_hand_examples"]),
]


def _edit(src, anchor, old, new):
    """Replace the first ``old`` after ``anchor`` (one function's body)."""
    a = src.index(anchor)
    i = src.index(old, a)
    return src[:i] + new + src[i + len(old):]


def _expect_caught(names, orc):
    """Run the named pins; return the ones that failed."""
    failed = []
    for name in names:
        fn = getattr(pins, name)
        try:
            if "orc" in fn.__code__.co_varnames[:fn.__code__.co_argcount]:
                fn(orc)
            else:
                fn()
        except AssertionError:
            failed.append(name)
    return failed


@pytest.fixture(scope="module")
def orc_built():
    oracle.build()
    return oracle


def test_unmutated_oracle_passes_every_listed_pin(orc_built):
    names = sorted({n for m in C_MUTANTS for n in m[4]} | {n for m in PY_MUTANTS for n in m[4]}
                   | {n for m in WRAPPER_MUTANTS for n in m[3]})
    assert _expect_caught(names, orc_built) == []


@pytest.mark.parametrize("case", C_MUTANTS, ids=[m[0] for m in C_MUTANTS])
def test_planted_mistake_in_oracle_c_is_caught(case, orc_built, tmp_path, monkeypatch):
    name, anchor, old, new, names = case
    src = open(SRC).read()
    mutated = _edit(src, anchor, old, new)
    assert mutated != src
    c = tmp_path / "oracle_mutant.c"
    so = tmp_path / "liboracle_mutant.so"
    c.write_text(mutated)
    r = subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                        str(c), "-o", str(so), "-lm"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    monkeypatch.setattr(oracle, "_lib", oracle.load(str(so)))
    failed = _expect_caught(names, oracle)
    assert failed, f"planted mistake '{name}' passes every pin in {names}"


@pytest.mark.parametrize("case", WRAPPER_MUTANTS, ids=[f"{m[0]}: {m[2][:40]}" for m in WRAPPER_MUTANTS])
def test_planted_mistake_in_oracle_wrapper_is_caught(case, orc_built, monkeypatch):
    fname, old, new, names = case
    src = inspect.getsource(getattr(oracle, fname))
    assert src.count(old) == 1, f"edit site in {fname} is not unique"
    ns = dict(vars(oracle))
    exec(compile(src.replace(old, new), oracle.__file__, "exec"), ns)
    monkeypatch.setattr(oracle, fname, ns[fname])
    failed = _expect_caught(names, oracle)
    assert failed, f"planted mistake in {fname} passes every pin in {names}"


@pytest.mark.parametrize("case", PY_MUTANTS, ids=[m[1] for m in PY_MUTANTS])
def test_planted_mistake_in_numpy_oracle_is_caught(case, orc_built, monkeypatch):
    modname, name, old, new, names = case
    path = os.path.join(os.path.dirname(oracle.__file__), modname + ".py")
    src = open(path).read()
    assert src.count(old) == 1, f"edit site of '{name}' is not unique"
    mod = types.ModuleType(f"oracle.{modname}")
    mod.__file__ = path
    exec(compile(src.replace(old, new), path, "exec"), mod.__dict__)
    monkeypatch.setattr(oracle, modname, mod)
    failed = _expect_caught(names, oracle)
    assert failed, f"planted mistake '{name}' passes every pin in {names}"
