"""The pins catch plausible mistakes: each case plants one mistake in a copy of the oracle's C
source (a dropped term, a wrong sign, index or constant, a transposed operand, a reversed order),
builds that copy apart from the real oracle, and checks that at least one of the named pins fails
against it. The real oracle passes every one of those pins in the rest of the suite.
"""
import importlib.util
import os
import subprocess

import pytest

import test_oracle_bc1 as T_BC1
import test_oracle_bc7 as T_BC7
import test_oracle_geometry as T_GEO
import test_oracle_layouts as T_LAY
import test_oracle_pipeline as T_PIPE
import test_oracle_rate as T_RATE
import test_oracle_render as T_REN
import test_oracle_reorder as T_REO
import test_oracle_scales_quant as T_SQ
import test_oracle_sh as T_SH

ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

# name: ([(text of the oracle, planted replacement)], [pins, at least one of which must fail])
MUTANTS = {
    "scale rank off by one (the -1 dropped)": (
        [("int64_t r = ((int64_t)permille * m + 999) / 1000 - 1;", "int64_t r = ((int64_t)permille * m + 999) / 1000;")],
        [T_SQ.test_scale_is_exact_order_statistic, T_SQ.test_scale_hand_fixture]),
    "quantiser truncates instead of rounding": (
        [("long r = lrintf(t);", "long r = (long)t;")],
        [T_SQ.test_quantise_against_double_precision, T_SQ.test_quantise_ties_round_half_even]),
    "quantiser rounds half away from zero": (
        [("long r = lrintf(t);", "long r = lroundf(t);")],
        [T_SQ.test_quantise_ties_round_half_even, T_SQ.test_quantise_against_double_precision]),
    "colour key with R and B exchanged": (
        [("k |= ((r >> i) & 1u) << (3 * i + 2);", "k |= ((b >> i) & 1u) << (3 * i + 2);"),
         ("k |= ((b >> i) & 1u) << (3 * i);", "k |= ((r >> i) & 1u) << (3 * i);")],
        [T_REO.test_colour_key_hand_values]),
    "Morton code with x and z exchanged": (
        [("m |= ((x >> i) & 1u) << (3 * i + 2);", "m |= ((z >> i) & 1u) << (3 * i + 2);"),
         ("m |= ((z >> i) & 1u) << (3 * i);", "m |= ((x >> i) & 1u) << (3 * i);")],
        [T_REO.test_morton_hand_values]),
    "BC1 two-thirds entry with its operands transposed": (
        [("if (bits == 5) return ((2 * a + b) * 11) >> 2;", "if (bits == 5) return ((a + 2 * b) * 11) >> 2;")],
        [T_BC1.test_hand_built_four_colour_block, T_BC1.test_interpolation_reading_properties]),
    "BC1 three-colour mode's fourth entry opaque": (
        [("pal[3 * 4 + 3] = (c0 > c1) ? 255 : 0;", "pal[3 * 4 + 3] = 255;")],
        [T_BC1.test_hand_built_three_colour_block]),
    "BC7 interpolation without its rounding bias": (
        [("static int interp7(int e0, int e1, int w) { return ((64 - w) * e0 + w * e1 + 32) >> 6; }",
          "static int interp7(int e0, int e1, int w) { return ((64 - w) * e0 + w * e1) >> 6; }")],
        [T_BC7.test_hand_built_mode6_gradient, T_BC7.test_hand_built_mode1_membership,
         T_BC7.test_hand_built_mode4_rotation]),
    "BC7 endpoint expansion without bit replication": (
        [("static int expand_bits(int v, int n) { return n >= 8 ? v : ((v << (8 - n)) | (v >> (2 * n - 8))); }",
          "static int expand_bits(int v, int n) { return n >= 8 ? v : (v << (8 - n)); }")],
        [T_BC7.test_hand_built_mode1_membership, T_BC7.test_hand_built_mode4_rotation, T_BC7.test_constant_colours_round_trip_wherever_reachable]),
    "SH without the Condon-Shortley phase": (
        [("for (int i = 1; i <= m; i++) pmm *= -(2.0 * i - 1.0) * s;",
          "for (int i = 1; i <= m; i++) pmm *= (2.0 * i - 1.0) * s;")],
        [T_SH.test_matches_scipy_complex_sh, T_SH.test_closed_form_values]),
    "SH view direction p - f instead of f - p": (
        [("for (int a = 0; a < 3; a++) d[a] = (double)cams[3 * v + a] - (double)pos[3 * i + a];",
          "for (int a = 0; a < 3; a++) d[a] = (double)pos[3 * i + a] - (double)cams[3 * v + a];")],
        [T_SH.test_camera_directions]),
    "renderer blends far to near": (
        [("if (a->depth_bits != b->depth_bits) return a->depth_bits < b->depth_bits ? -1 : 1;",
          "if (a->depth_bits != b->depth_bits) return a->depth_bits < b->depth_bits ? 1 : -1;")],
        [T_REN.test_two_splats_blend_front_to_back]),
    "renderer transmittance without the opacity": (
        [("T *= 1.0 - mu * gv;", "T *= 1.0 - gv;")],
        [T_REN.test_head_on_isotropic_splat_closed_form, T_REN.test_two_splats_blend_front_to_back]),
    "rate control: a budget met exactly counts as over": (
        [("if (choose_all(D, ng, mid, NULL) <= budget) hi = mid; else lo = mid + 1;",
          "if (choose_all(D, ng, mid, NULL) < budget) hi = mid; else lo = mid + 1;")],
        [T_RATE.test_budget_met_exactly]),
    "rotation codes over 1023 steps while the decoder uses 1022": (
        [("code |= quant_unit(t, 1022.0f) << sh;", "code |= quant_unit(t, 1023.0f) << sh;")],
        [T_GEO.test_rotation_smallest_three]),
    "chunk test without the scale margin": (
        [("float g = 6.0f * e[6];", "float g = 0.0f * e[6];")],
        [T_GEO.test_culling_never_drops_a_drawn_gaussian]),
    "splat cross term with the wrong sign": (
        [("float a = c00 + 0.3f, b = c01, c = c11 + 0.3f;", "float a = c00 + 0.3f, b = -c01, c = c11 + 0.3f;")],
        [T_REN.test_oblique_splat_points_along_its_axis]),
    "splat without the low-pass": (
        [("float a = c00 + 0.3f, b = c01, c = c11 + 0.3f;", "float a = c00, b = c01, c = c11;")],
        [T_REN.test_head_on_isotropic_splat_closed_form]),
    "rotation matrix with one entry's sign flipped": (
        [("r[1] = 2.0f * (qx * qy - qw * qz);", "r[1] = 2.0f * (qx * qy + qw * qz);")],
        [T_REN.test_oblique_splat_points_along_its_axis]),
    "dequantisation centred on 127": (
        [("double x = ((double)texels[(i * OR_SH + k) * 3 + c] - 128.0) / 255.0 * (double)scales[k];",
          "double x = ((double)texels[(i * OR_SH + k) * 3 + c] - 127.0) / 255.0 * (double)scales[k];")],
        [T_SH.test_degree_zero_and_dequantisation, T_SH.test_camera_directions]),
    "position codes over 65536 steps while the decoder uses 65535": (
        [("qpos[3 * s + a] = (uint16_t)quant_unit(t, 65535.0f);", "qpos[3 * s + a] = (uint16_t)quant_unit(t, 65536.0f);")],
        [T_GEO.test_position_codes_within_half_a_step_of_the_chunk_box]),
    "padding repeats the first valid slot of its group": (
        [("    if (o >= 0) last = o;\n    for (int k = 0; k < OR_SH; k++)\n      for (int c = 0; c < 3; c++) tex[(k * 16 + t) * 3 + c]",
          "    if (o >= 0 && last < 0) last = o;\n    for (int k = 0; k < OR_SH; k++)\n      for (int c = 0; c < 3; c++) tex[(k * 16 + t) * 3 + c]")],
        [T_REO.test_stage_layout_d]),
    "rate weights without the square of the scale": (
        [("double v = rint((s * s * 65536.0) / mx);", "double v = rint((s * 65536.0) / mx);")],
        [T_RATE.test_distortion_table_is_dequantised_squared_error]),
    "distortion table charges BC1 errors to BC7 blocks": (
        [("uint64_t e = k < MODE_J[m] ? e7[k] : (k < MODE_B[m] ? e1[k] : e0[k]);",
          "uint64_t e = k < MODE_J[m] ? e1[k] : (k < MODE_B[m] ? e1[k] : e0[k]);")],
        [T_RATE.test_distortion_table_is_dequantised_squared_error]),
    "dropped coefficients charged as zero error": (
        [("for (int u = 0; u < 48; u++) e0[k] += (uint64_t)sq(tk[u] - 128);",
          "for (int u = 0; u < 48; u++) e0[k] += 0;")],
        [T_RATE.test_distortion_table_is_dequantised_squared_error]),
    "BC7 encoder keeps the last of equal errors": (
        [("if (s < best) { best = s; best_e = e; }", "if (s <= best) { best = s; best_e = e; }")],
        [T_BC7.test_encoder_is_the_first_minimum]),
    "BC1 indices take the last of equal palette errors": (
        [("if (best < 0 || e < best) { best = e; bj = j; }", "if (best < 0 || e <= best) { best = e; bj = j; }")],
        [T_BC1.test_encoder_output_is_canonical_and_consistent, T_BC1.test_hand_built_four_colour_block,
         T_BC1.test_encoder_against_local_brute_force]),
    "bfloat16 scales truncated instead of rounded": (
        [("u += 0x7FFFu + ((u >> 16) & 1u);", "u += 0u;")],
        [T_GEO.test_scale_and_opacity_codes]),
    "layout B with rows and columns exchanged": (
        [("*u = 4 * v + i; *c = 4 * b + j;", "*u = 4 * v + j; *c = 4 * b + i;")],
        [T_LAY.test_layout_b_placement_rows_are_gaussians]),
    "layout A block read as layout D": (
        [("if (layout == OR_LAYOUT_A) { *u = k; *c = t; }", "if (layout == OR_LAYOUT_A) { *u = t; *c = k; }")],
        [T_LAY.test_layout_a_block_is_one_gaussian]),
    "colour sort ignores the spatial chunks": (
        [("k[r].a = group_size ? (uint64_t)(r / group_size) : 0;", "k[r].a = 0;")],
        [lambda O: T_REO.test_plan_matches_independent_restatement(O, 1000, 256)]),
    "colour ties broken by original index instead of spatial rank": (
        [("k[r].c = (uint64_t)r;", "k[r].c = (uint64_t)i;")],
        [T_REO.test_colour_ties_keep_spatial_order]),
    "pixel centres at integer coordinates": (
        [("double dx = (px + 0.5) - (double)g->u, dy = (py + 0.5) - (double)g->v;",
          "double dx = (double)px - (double)g->u, dy = (double)py - (double)g->v;")],
        [T_REN.test_head_on_isotropic_splat_closed_form]),
    "splat rectangle of 2 sigma": (
        [("float rad = ceilf(3.0f * sqrtf(lam));", "float rad = ceilf(2.0f * sqrtf(lam));")],
        [T_REN.test_tile_rectangle_is_three_sigma]),
    "chunk scale bound from the last axis only": (
        [("if ((!any && a == 0) || sv > e[6]) e[6] = sv;", "if (a == 2 && (!any || sv > e[6])) e[6] = sv;")],
        [T_GEO.test_chunk_table_and_byte_count]),
    "BC7 rotation swaps alpha with the wrong channel": (
        [("if (rot) { int tmp = px[3]; px[3] = px[rot - 1]; px[rot - 1] = tmp; }",
          "if (rot) { int tmp = px[3]; px[3] = px[rot % 3]; px[rot % 3] = tmp; }")],
        [T_BC7.test_hand_built_mode4_rotation]),
    "BC7 index selection bit ignored": (
        [("if (isb) { ci = sec[t]; cbits = M->ib2; ai = pri[t]; abits = M->ib; }",
          "if (0) { ci = sec[t]; cbits = M->ib2; ai = pri[t]; abits = M->ib; }")],
        [T_BC7.test_hand_built_mode4_rotation, T_BC7.test_every_candidate_packs_losslessly]),
    "BC7 secondary index stream without its anchor bit": (
        [("for (int t = 0; t < 16; t++) sec[t] = M->ib2 ? (int)br_get(&r, M->ib2 - (t == 0)) : 0;",
          "for (int t = 0; t < 16; t++) sec[t] = M->ib2 ? (int)br_get(&r, M->ib2) : 0;")],
        [T_BC7.test_hand_built_mode4_rotation, T_BC7.test_every_candidate_packs_losslessly]),
    "BC7 shared p-bit applied to one endpoint only": (
        [("for (int s = 0; s < M->ns; s++) p[s][0] = p[s][1] = (int)br_get(&r, 1);",
          "for (int s = 0; s < M->ns; s++) p[s][0] = (int)br_get(&r, 1);")],
        [T_BC7.test_hand_built_mode1_shared_pbits_and_weights]),
    "BC7 three-subset anchors exchanged": (
        [("return s == 1 ? ANCH3A[part] : ANCH3B[part];", "return s == 1 ? ANCH3B[part] : ANCH3A[part];")],
        [T_BC7.test_partition_and_anchor_invariants]),
    "BC7 opaque modes decode alpha 0": (
        [("ev[s][e][3] = M->ab ? expand_bits(M->epb ? (code[s][e][3] << 1) | p[s][e] : code[s][e][3], M->ab + M->epb) : 255;",
          "ev[s][e][3] = M->ab ? expand_bits(M->epb ? (code[s][e][3] << 1) | p[s][e] : code[s][e][3], M->ab + M->epb) : 0;"),
         ("px[3] = M->ab ? interp7(ev[s][0][3], ev[s][1][3], wtab(abits)[ai]) : 255;",
          "px[3] = M->ab ? interp7(ev[s][0][3], ev[s][1][3], wtab(abits)[ai]) : 0;")],
        [T_BC7.test_hand_built_mode1_membership, T_BC7.test_reserved_mode_decodes_to_zero]),
    "BC1 5-bit expansion without replication": (
        [("static int ex5(int x) { return (x << 3) | (x >> 2); }", "static int ex5(int x) { return x << 3; }")],
        [T_BC1.test_hand_built_four_colour_block, T_BC1.test_exact_565_colours_round_trip]),
    "BC1 three-colour mode's fourth entry white": (
        [("      pal[3 * 4 + c] = 0;", "      pal[3 * 4 + c] = 255;")],
        [T_BC1.test_hand_built_three_colour_block]),
    "SH direction of a camera on the Gaussian is -z": (
        [("if (nn == 0.0) { d[0] = 0.0; d[1] = 0.0; d[2] = 1.0; }", "if (nn == 0.0) { d[0] = 0.0; d[1] = 0.0; d[2] = -1.0; }")],
        [T_SH.test_camera_directions]),
    "opacity logit decoded over 256 steps": (
        [("*t = ((float)qlogit[s] / 255.0f) * 16.0f - 8.0f;", "*t = ((float)qlogit[s] / 256.0f) * 16.0f - 8.0f;")],
        [T_GEO.test_scale_and_opacity_codes]),
    "scales ignore the coverage parameter": (
        [("int64_t r = ((int64_t)permille * m + 999) / 1000 - 1;", "int64_t r = ((int64_t)995 * m + 999) / 1000 - 1;")],
        [T_SQ.test_scale_is_exact_order_statistic, T_SQ.test_scale_coverage_property, T_SQ.test_scale_hand_fixture]),
    "quantiser wraps 256 to 0": (
        [("if (q > 255) q = 255;", "if (q > 256) q = 255;")],
        [T_SQ.test_quantise_special_values, T_SQ.test_quantise_against_double_precision]),
    "BC7 fit ignores anti-correlated channels": (
        [("int flip = (i != ref) && ((int64_t)n * s2[ref][i] - s1[ref] * s1[i] < 0);", "int flip = 0;")],
        [T_BC7.test_two_subset_partitions_exact, T_BC7.test_three_subset_partitions_exact]),
    "BC7 fit tries only the first p-bit combination": (
        [("int ncombo = ptype == 0 ? 1 : (ptype == 1 ? 4 : 2);", "int ncombo = 1;")],
        [T_BC7.test_constant_colours_round_trip_wherever_reachable, T_BC7.test_two_subset_partitions_exact,
         T_BC7.test_three_subset_partitions_exact]),
    "decode places a texel with its neighbour slot's Gaussian": (
        [("          int32_t o = perm[16 * g + u];\n          if (o < 0) continue;",
          "          int32_t o = perm[16 * g + (u ^ 1)];\n          if (o < 0) continue;")],
        [lambda O: T_PIPE.test_forced_format_blocks_are_layout_d(O, 1), T_PIPE.test_rate_streams_random_access_and_dropped_bands,
         lambda O: T_LAY.test_bc7_round_trip_is_lossless_when_blocks_are_constant(O, 1)]),
    "fixed codings write BC1 blocks before BC7 blocks": (
        [("    for (int k = 0; k < OR_SH; k++)\n      if (or_layout_bc7(layout, j, k)) { or_bc7_encode(tex + 48 * k, dst); dst += 16; }\n"
          "    for (int k = 0; k < OR_SH; k++)\n      if (!or_layout_bc7(layout, j, k)) { or_bc1_encode(tex + 48 * k, dst); dst += 8; }\n",
          "    for (int k = 0; k < OR_SH; k++)\n      if (!or_layout_bc7(layout, j, k)) { or_bc1_encode(tex + 48 * k, dst); dst += 8; }\n"
          "    for (int k = 0; k < OR_SH; k++)\n      if (or_layout_bc7(layout, j, k)) { or_bc7_encode(tex + 48 * k, dst); dst += 16; }\n")],
        [T_LAY.test_mixed_b_decodes_each_block_with_its_format]),
    "rate streams assembled in reverse mode order": (
        [("    for (int m = 0; m < OR_MODES; m++) {\n      int64_t gbytes",
          "    for (int m = OR_MODES - 1; m >= 0; m--) {\n      int64_t gbytes")],
        [T_PIPE.test_rate_streams_random_access_and_dropped_bands,
         lambda O: T_RATE.test_rate_targets_respect_budget(O, 24)]),
    "rotation code picks the largest component without its absolute value": (
        [("for (int a = 1; a < 4; a++) if (fabsf(u[a]) > fabsf(u[m])) m = a;",
          "for (int a = 1; a < 4; a++) if (u[a] > u[m]) m = a;")],
        [T_GEO.test_rotation_smallest_three]),
    "rotation code without making the largest component positive": (
        [("float sg = u[m] < 0.0f ? -1.0f : 1.0f;", "float sg = 1.0f;")],
        [T_GEO.test_rotation_smallest_three]),
    "opacity as the sigmoid of -t": (
        [("double mu = 1.0 / (1.0 + exp(-(double)logit[i]));", "double mu = 1.0 / (1.0 + exp((double)logit[i]));")],
        [T_REN.test_head_on_isotropic_splat_closed_form, T_REN.test_two_splats_blend_front_to_back]),
    "chunk box grown on its high side only": (
        [("for (int a = 0; a < 3; a++) c[a] = ((k >> a) & 1) ? e[3 + a] + g : e[a] - g;",
          "for (int a = 0; a < 3; a++) c[a] = ((k >> a) & 1) ? e[3 + a] + g : e[a];")],
        [T_GEO.test_culling_keeps_adversarial_chunks]),
    "chunk corners from one bit of the corner index": (
        [("for (int a = 0; a < 3; a++) c[a] = ((k >> a) & 1) ? e[3 + a] + g : e[a] - g;",
          "for (int a = 0; a < 3; a++) c[a] = ((k >> 1) & 1) ? e[3 + a] + g : e[a] - g;")],
        [T_GEO.test_culling_keeps_adversarial_chunks]),
    "chunks straddling the camera plane culled by the side test": (
        [("if (front && (left || right || top || bottom)) return 0;", "if (left || right || top || bottom) return 0;")],
        [T_GEO.test_culling_keeps_adversarial_chunks]),
    "chunk side margin of 0 px": (
        [("    if (!(u < -64.0f)) left = 0;\n    if (!(u > W + 64.0f)) right = 0;",
          "    if (!(u < 0.0f)) left = 0;\n    if (!(u > W + 0.0f)) right = 0;")],
        [T_GEO.test_culling_keeps_adversarial_chunks]),
    "BC7 nearest endpoint code keeps the last of equal distances": (
        [("    if (be < 0 || d < be) { be = d; best = code; }\n  }\n  return best;",
          "    if (be < 0 || d <= be) { be = d; best = code; }\n  }\n  return best;")],
        [T_BC7.test_nearest_code_ties_go_to_the_lower_code]),
    "BC7 fit without its least-squares step": (
        [("  if (det != 0)\n    for (int i = 0; i < nch; i++) {\n      e0[i] = clampi(",
          "  if (0)\n    for (int i = 0; i < nch; i++) {\n      e0[i] = clampi(")],
        [T_BC7.test_mode6_fit_least_squares_by_hand]),
    "BC1 encoder without its least-squares refinements": (
        [("  for (int it = 0; it < 2; it++) {\n    static const int A3[4]", "  for (int it = 0; it < 0; it++) {\n    static const int A3[4]")],
        [T_BC1.test_tiny_blocks_global_brute_force]),
    "BC1 encoder without its neighbourhood search": (
        [("  for (int round = 0; round < 4; round++) {\n    bc1_sol nb;", "  for (int round = 0; round < 0; round++) {\n    bc1_sol nb;")],
        [T_BC1.test_tiny_blocks_global_brute_force, T_BC1.test_encoder_against_local_brute_force]),
    "SH tolerance sum of the coefficients without the basis": (
        [("aa += fabs(x * Y[k]);", "aa += fabs(x);")],
        [T_SH.test_tolerance_sum_is_the_sum_of_absolute_terms]),
    "render tolerance sum without the transmittance": (
        [("ab[ch] += fabs(term);", "ab[ch] += fabs(gv * colour[3 * i + ch]);")],
        [T_REN.test_two_splats_blend_front_to_back]),
}

def _build(path, patches):
    src = open(os.path.join(ORACLE, "gsc_oracle.c")).read()
    for old, new in patches:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    c = path / "gsc_oracle_mutant.c"
    c.write_text(src)
    so = path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-pthread", "-fPIC",
                           "-shared", "-I", ORACLE, "-o", str(so), str(c), "-lm"])
    return str(so)


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    """Every planted copy, compiled in parallel once for the module."""
    from concurrent.futures import ThreadPoolExecutor
    jobs = {name: patches for name, (patches, _) in MUTANTS.items()}
    dirs = {name: tmp_path_factory.mktemp("mutant") for name in jobs}
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        futs = {name: ex.submit(_build, dirs[name], jobs[name]) for name in jobs}
        return {name: f.result() for name, f in futs.items()}


def _mutant_oracle(so):
    spec = importlib.util.spec_from_file_location("oracle_mutant_%d" % abs(hash(so)), os.path.join(ORACLE, "oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.LIB_OVERRIDE = so
    mod.lib()
    return mod


@pytest.mark.parametrize("name", list(MUTANTS))
def test_a_planted_mistake_fails_a_pin(mutant_libs, name):
    _, pins = MUTANTS[name]
    M = _mutant_oracle(mutant_libs[name])
    failed = []
    for pin in pins:
        try:
            pin(M)
        except AssertionError:
            failed.append(getattr(pin, "__name__", "pin"))
    assert failed, "no pin caught: " + name
