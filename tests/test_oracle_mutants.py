"""The oracle's pins against planted mistakes (mutation check, CPU only).

Each case copies ``oracle/lobe_oracle.c`` (or the oracle's Python module, for the parts
written in Python: Adam, back-projection and coverage, densification, the KD partition),
plants one plausible mistake in it -- a dropped term, a wrong sign, index or constant, a
transposed operand, a threshold rule read the other way -- builds or loads the copy and runs
the pins that should catch it against it: at least one of them must fail. The planted copies
live in a temporary directory or a throwaway module and never replace the oracle; the
``oracle`` module is pointed at a copy for one case and restored afterwards.
Mistakes that leave every result unchanged (reordering a product of symmetric matrices) are
not cases.
"""
import concurrent.futures
import inspect
import os
import subprocess
import sys
import types

import pytest

import oracle
import tests.test_oracle_branches as branches
import tests.test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "lobe_oracle.c")

# (name, the mistake, text of lobe_oracle.c, planted text, pins expected to catch it)
MUTANTS = [
    ('dilation', 'the 0.3 low-pass dropped on one axis',
     '    c00 += 0.3;\n',
     '    c00 += 0.0;\n',
     ['test_depth_composite_on_axis_closed_form', 'test_depth_of_two_layers_weights_front_and_back']),
    ('conic_sign', 'conic b with the wrong sign',
     'P->conic[1] = -c01 / det;',
     'P->conic[1] = c01 / det;',
     ['test_off_axis_cov2d_equals_numerical_jacobian', 'test_rotation_about_optical_axis_rotates_conic']),
    ('jacobian_index', 'J02 uses y instead of x',
     'J[2] = -k->fx * x / (z * z);',
     'J[2] = -k->fx * y / (z * z);',
     ['test_off_axis_cov2d_equals_numerical_jacobian', 'test_backward_matches_finite_differences_all_params_64']),
    ('radius', 'lambda_max with + det',
     'double lam = mid + sqrt(fmax(0.1, mid * mid - det));',
     'double lam = mid + sqrt(fmax(0.1, mid * mid + det));',
     ['test_isotropic_on_axis_closed_form']),
    ('radius_factor', 'radius 2 sqrt(lambda)',
     'double r3 = 3.0 * sqrt(lam);',
     'double r3 = 2.0 * sqrt(lam);',
     ['test_isotropic_on_axis_closed_form']),
    ('mean2d_cx', 'u without the principal point',
     'P->mean2d[0] = k->fx * x / z + k->cx;',
     'P->mean2d[0] = k->fx * x / z + k->cy;',
     ['test_principal_point_is_the_image_of_the_optical_axis']),
    ('rect_floor', 'tile rectangle end rounded down',
     'rect[2] = (int)clampd(ceil((u + r) / tw), 0, gx);',
     'rect[2] = (int)clampd(floor((u + r) / tw), 0, gx);',
     ['test_alpha_clamp_and_one_pixel_adjoint_closed_form', 'test_depth_composite_on_axis_closed_form']),
    ('guard', 'fov guard 1.5 instead of 1.3',
     'double limx = 1.3 * (0.5 * k->W) / k->fx,',
     'double limx = 1.5 * (0.5 * k->W) / k->fx,',
     ['test_fov_guard_is_1_3_times_the_half_field_of_view']),
    ('near', 'near plane ignored',
     'if (!(z >= k->near_plane && z <= k->far_plane)) return;',
     'if (!(z >= 0.0 && z <= k->far_plane)) return;',
     ['test_culling_rules']),
    ('depth_raylength', 'depth = ray length',
     'P->depth = z;',
     'P->depth = sqrt(x * x + y * y + z * z);',
     ['test_depth_key_is_float32_z', 'test_sort_breaks_depth_ties_by_index']),
    ('rotation_sign', 'rotation R01 sign',
     'R[1] = 2 * (x * y - w * z);',
     'R[1] = 2 * (x * y + w * z);',
     ['test_isotropic_on_axis_closed_form', 'test_rotation_about_optical_axis_rotates_conic']),
    ('scale_exp', 'scales not exponentiated',
     'P->s[i] = exp(ls[i]);',
     'P->s[i] = exp(0.5 * ls[i]);',
     ['test_depth_composite_on_axis_closed_form', 'test_depth_of_two_layers_weights_front_and_back']),
    ('sh_phase', 'Condon-Shortley phase dropped for m > 0',
     'A = re; dAx = drx; dAy = dry; pre = sqrt(2.0) * K * ((m & 1) ? -1.0 : 1.0);',
     'A = re; dAx = drx; dAy = dry; pre = sqrt(2.0) * K;',
     ['test_sh_matches_scipy', 'test_sh_textbook_closed_forms']),
    ('sh_norm', 'SH normalisation without 4 pi',
     'double K = sqrt((2 * l + 1) / (4.0 * ORC_PI) * factorial(l - m) / factorial(l + m));',
     'double K = sqrt((2 * l + 1) / (2.0 * ORC_PI) * factorial(l - m) / factorial(l + m));',
     ['test_alpha_clamp_and_one_pixel_adjoint_closed_form', 'test_degree0_colour_is_constant']),
    ('colour_offset', 'colour without the 0.5 offset',
     'P->color_raw[ch] = s + 0.5;',
     'P->color_raw[ch] = s;',
     ['test_alpha_clamp_and_one_pixel_adjoint_closed_form', 'test_degree0_colour_is_constant']),
    ('colour_clamp', 'colour not clamped at 0',
     'P->color[ch] = P->color_raw[ch] < 0.0 ? 0.0 : P->color_raw[ch];',
     'P->color[ch] = P->color_raw[ch];',
     ['test_negative_colour_is_clamped_and_passes_no_gradient']),
    ('opacity', 'opacity = logit',
     'P->opacity = 1.0 / (1.0 + exp(-logit));',
     'P->opacity = 1.0 / (1.0 + exp(-2.0 * logit));',
     ['test_depth_composite_on_axis_closed_form', 'test_depth_of_two_layers_weights_front_and_back']),
    ('sigma_cross', 'sigma cross term halved',
     'double sigma = 0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) + cn[1] * dx * dy;',
     'double sigma = 0.5 * (cn[0] * dx * dx + cn[2] * dy * dy + cn[1] * dx * dy);',
     ['test_backward_matches_finite_differences_all_params_64', 'test_backward_matches_finite_differences_sampled_1k_posed_camera']),
    ('alpha_clamp', 'no 0.99 clamp',
     'int clamped = araw >= 0.99;',
     'int clamped = araw >= 1.5;',
     ['test_alpha_clamp_and_one_pixel_adjoint_closed_form']),
    ('alpha_skip', '1/255 skip dropped',
     'if (alpha < 1.0 / 255.0) continue;',
     'if (alpha < 0.0) continue;',
     ['test_depth_composite_on_axis_closed_form', 'test_isotropic_on_axis_closed_form']),
    ('stop_threshold', 'stop at 1e-3',
     'if (Tn < 1e-4) break;',
     'if (Tn < 1e-3) break;',
     ['test_stop_rule_on_a_stack_closed_form']),
    ('stop_included', 'the stopping Gaussian still blended',
     '        if (Tn < 1e-4) break;\n        double w = alpha * T;\n',
     '        double w = alpha * T;\n',
     ['test_stop_rule_on_a_stack_closed_form']),
    ('transmittance', 'T update with alpha / 2',
     'double Tn = T * (1.0 - alpha);',
     'double Tn = T * (1.0 - 0.5 * alpha);',
     ['test_alpha_clamp_and_one_pixel_adjoint_closed_form', 'test_depth_composite_on_axis_closed_form']),
    ('sort_tiebreak', 'ties by descending index',
     'if (p->tile != q->tile) return p->tile < q->tile ? -1 : 1;\n    if (p->dbits != q->dbits) return p->dbits < q->dbits ? -1 : 1;\n    return p->g < q->g ? -1 : (p->g > q->g);',
     'if (p->tile != q->tile) return p->tile < q->tile ? -1 : 1;\n    if (p->dbits != q->dbits) return p->dbits < q->dbits ? -1 : 1;\n    return p->g > q->g ? -1 : (p->g < q->g);',
     ['test_sort_breaks_depth_ties_by_index']),
    ('bwd_background', 'adjoint without the colour behind',
     'dalpha += r->T * (c[ch] - B[ch]) * gC[ch];',
     'dalpha += r->T * c[ch] * gC[ch];',
     ['test_alpha_clamp_and_one_pixel_adjoint_closed_form', 'test_backward_matches_finite_differences_all_params_64']),
    ('bwd_conic_b', 'd conic b with a factor 1/2',
     'd_conic[3 * g + 1] += dsig * r->dx * r->dy;',
     'd_conic[3 * g + 1] += dsig * 0.5 * r->dx * r->dy;',
     ['test_backward_matches_finite_differences_all_params_64', 'test_backward_matches_finite_differences_sampled_1k_posed_camera']),
    ('bwd_opacity', 'd opacity with alpha for G',
     'd_opacity[g] += dalpha * r->G;',
     'd_opacity[g] += dalpha * r->alpha;',
     ['test_alpha_clamp_and_one_pixel_adjoint_closed_form']),
    ('bwd_mean_index', 'd mean2d v uses cn[0]',
     'd_mean2d[2 * g + 1] += dsig * (cn[1] * r->dx + cn[2] * r->dy);',
     'd_mean2d[2 * g + 1] += dsig * (cn[1] * r->dx + cn[0] * r->dy);',
     ['test_backward_matches_finite_differences_all_params_64', 'test_backward_matches_finite_differences_sampled_1k_posed_camera']),
    ('bwd_clamp', 'gradient through the clamp',
     '                if (r->clamped) continue;\n',
     '',
     ['test_alpha_clamp_and_one_pixel_adjoint_closed_form']),
    ('pbwd_logit', 'logit gradient without (1 - o)',
     'g_logits[g] += d_opacity[g] * P.opacity * (1.0 - P.opacity);',
     'g_logits[g] += d_opacity[g] * P.opacity;',
     ['test_backward_matches_finite_differences_all_params_64']),
    ('pbwd_viewdir', 'view direction gradient not projected',
     'for (int i = 0; i < 3; ++i) gmu[i] += (dn[i] - P.n[i] * ndn) / P.dirlen;',
     'for (int i = 0; i < 3; ++i) gmu[i] += dn[i] / P.dirlen;',
     ['test_backward_matches_finite_differences_all_params_64', 'test_backward_matches_finite_differences_sampled_1k_posed_camera']),
    ('pbwd_colour_clamp', 'SH gradient through a clamped colour',
     '            if (clamped) continue;\n            double dc = d_color[3 * g + ch];',
     '            double dc = d_color[3 * g + ch];',
     ['test_negative_colour_is_clamped_and_passes_no_gradient']),
    ('pbwd_duv', 'd z with + dv term',
     'dpc[2] += -du * fx * x / (z * z) - dv * fy * y / (z * z);',
     'dpc[2] += -du * fx * x / (z * z) + dv * fy * y / (z * z);',
     ['test_backward_matches_finite_differences_all_params_64', 'test_backward_matches_finite_differences_sampled_1k_posed_camera']),
    ('pbwd_dJ', 'dL/dJ without the factor 2',
     'dJ[3 * i + b] = 2.0 * s;',
     'dJ[3 * i + b] = s;',
     ['test_backward_matches_finite_differences_all_params_64', 'test_backward_matches_finite_differences_sampled_1k_posed_camera']),
    ('pbwd_world', 'dL/dSigma = W dSc W^T',
     'mat3_mul(Wt, dSc, T1);\n        mat3_mul(T1, W, dS);',
     'mat3_mul(W, dSc, T1);\n        mat3_mul(T1, Wt, dS);',
     ['test_backward_matches_finite_differences_sampled_1k_posed_camera']),
    ('pbwd_quat_norm', 'quaternion gradient not projected',
     'for (int c = 0; c < 4; ++c) g_quats[4 * g + c] += (dqn[c] - P.qn[c] * qd) / P.qnorm;',
     'for (int c = 0; c < 4; ++c) g_quats[4 * g + c] += dqn[c] / P.qnorm;',
     ['test_backward_matches_finite_differences_all_params_64']),
    ('pbwd_rot_grad', 'dR/dx entry',
     'double Dx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};',
     'double Dx[9] = {0, 2 * y, 2 * z, 2 * y, -2 * x, -2 * w, 2 * z, 2 * w, -4 * x};',
     ['test_backward_matches_finite_differences_all_params_64']),
    ('pbwd_scale', 'log-scale gradient without s',
     'g_log_scales[3 * g + j] += ds * P.s[j];',
     'g_log_scales[3 * g + j] += ds;',
     ['test_backward_matches_finite_differences_all_params_64']),
    ('sd_height', 'SD statistic scales v by W',
     'double a = du * 0.5 * k.W, b = dv * 0.5 * k.H;',
     'double a = du * 0.5 * k.W, b = dv * 0.5 * k.W;',
     ['test_sd_statistic_scales_by_half_width_and_height']),
    ('sd_block', 'SD statistic ignores the block',
     'if (!(mu[i] >= aabb[i] && mu[i] < aabb[3 + i])) inside = 0;',
     'if (!(mu[i] >= aabb[i] || mu[i] < aabb[3 + i])) inside = 0;',
     ['test_sd_statistic_is_scaled_mean2d_gradient_norm']),
    ('crop_overwrite', 'the visibility crop keeps only the last camera',
     '        if (P.visible) mask[g] = 1;',
     '        mask[g] = P.visible ? 1 : 0;',
     ['test_visibility_crop_is_the_union_over_the_block_cameras']),
    # the enumeration of admissible branches (the leaves of a pixel and their adjoints)
    ('walk_skip', 'the skipped outcome of a used pair never followed',
     '    if (order[0] != 0 && skip_ok) order[no++] = 0;\n',
     '    if (0 && skip_ok) order[no++] = 0;\n',
     [('branches', 'test_leaves_equal_exhaustive_filter', (0,))]),
    ('walk_clamp', 'the other side of a marginal clamp never followed',
     '        int clamp_ok = c == cl_fp || cl_m;\n',
     '        int clamp_ok = c == cl_fp;\n',
     [('branches', 'test_leaves_equal_exhaustive_filter', (0,))]),
    ('walk_stop', 'the other side of a marginal stop never followed',
     '    for (int b = 0; b < 1 + marg; ++b) {\n        int st = b == 0 ? stop : !stop;',
     '    for (int b = 0; b < 1; ++b) {\n        int st = b == 0 ? stop : !stop;',
     [('branches', 'test_leaves_equal_exhaustive_filter', (2,)), ('branches', 'test_leaves_equal_exhaustive_filter', (3,))]),
    ('walk_plain_stop', 'a marginal stop on the plain path taken as certain',
     '        if (fabs(Tn - 1e-4) < mg[M_REL] * 1e-4) {\n            pair_stop(w, &q, S, alpha, q.araw >= 0.99, NULL);',
     '        if (0) {\n            pair_stop(w, &q, S, alpha, q.araw >= 0.99, NULL);',
     [('branches', 'test_a_marginal_stop_alone_gives_both_outcomes', ())]),
    ('walk_member', 'uncertain members never flipped',
     '    int mem_fp = u != 1, mem_m = u != 0;',
     '    int mem_fp = u != 1, mem_m = 0;',
     [('branches', 'test_leaves_equal_exhaustive_filter', (3,)), ('branches', 'test_leaves_equal_exhaustive_filter', (4,))]),
    ('walk_clamped_record', 'a clamped pair recorded as unclamped on the plain path',
     '        r->dx = q.dx; r->dy = q.dy; r->clamped = q.araw >= 0.99;',
     '        r->dx = q.dx; r->dy = q.dy; r->clamped = 0;',
     [('branches', 'test_single_leaf_envelope_with_clamped_pairs_is_the_plain_adjoint', ())]),
    ('walk_fp_first', 'leaf 0 not the FP64 outcome',
     '    order[no++] = fp_used ? 1 + cl_fp : 0;',
     '    order[no++] = 0;',
     [('branches', 'test_leaves_equal_exhaustive_filter', (0,))]),
    ('walk_sigma', 'sigma margin ignored',
     '        int m_sig = fabs(q.sigma) < mg[M_SIG];\n',
     '        int m_sig = 0;\n',
     [('branches', 'test_leaves_equal_exhaustive_filter', (0,))]),
    # the extended tile lists (members a marginal projection decision may add or remove)
    ('ext_outer', 'uncertain members only up to radius r, not r + 1',
     '    int outer[4], inner[4] = {0, 0, 0, 0};\n    tile_rect(mean2d[2 * g], mean2d[2 * g + 1], radius_all[g] + 1, tw, th, gx, gy, outer);',
     '    int outer[4], inner[4] = {0, 0, 0, 0};\n    tile_rect(mean2d[2 * g], mean2d[2 * g + 1], radius_all[g], tw, th, gx, gy, outer);',
     [('branches', 'test_extended_lists_cover_every_allowed_radius', ())]),
    ('ext_inner', 'certain core of radius r instead of r - 1',
     'radius_all[g] > 1)\n        tile_rect(mean2d[2 * g], mean2d[2 * g + 1], radius_all[g] - 1, tw, th, gx, gy, inner);\n    if (tx',
     'radius_all[g] > 1)\n        tile_rect(mean2d[2 * g], mean2d[2 * g + 1], radius_all[g], tw, th, gx, gy, inner);\n    if (tx',
     [('branches', 'test_extended_lists_cover_every_allowed_radius', ())]),
    ('ext_guard', 'a marginal guard decision not uncertain',
     '    if (flags & F_GUARD) return 1;\n',
     '    if (flags & F_GUARD) return 0;\n',
     [('branches', 'test_a_marginal_guard_makes_every_tile_of_the_outer_rectangle_uncertain', ())]),
    ('ext_rect_flag', 'a marginal rectangle edge not uncertain',
     '    return (flags & (F_RADIUS | F_RECT)) != 0;',
     '    return (flags & F_RADIUS) != 0;',
     [('branches', 'test_extended_lists_cover_every_allowed_radius', ())]),
    ('ext_inside_code', 'uncertain inside / outside codes swapped',
     '    return in_own ? 2 : 1;',
     '    return in_own ? 1 : 2;',
     [('branches', 'test_extended_lists_cover_every_allowed_radius', ())])
]


@pytest.fixture(scope="module")
def planted(tmp_path_factory):
    """name -> shared library of the oracle with that mistake planted (built in parallel)."""
    src = open(SRC).read()
    root = tmp_path_factory.mktemp("planted")

    def build(m):
        name, _, old, new, _ = m
        assert name == "unchanged" or src.count(old) == 1, f"{name}: the planted text must occur exactly once"
        c = root / f"{name}.c"
        c.write_text(src.replace(old, new))
        so = root / f"lib{name}.so"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                               str(c), "-lm"])
        return name, str(so)

    with concurrent.futures.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        return dict(ex.map(build, MUTANTS + [("unchanged", "", "", "", [])]))


@pytest.mark.parametrize("name, mistake, old, new, catchers", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_a_planted_mistake(planted, monkeypatch, name, mistake, old, new, catchers):
    so = planted[name]
    monkeypatch.setattr(oracle, "_LIB", so)
    monkeypatch.setattr(oracle, "build", lambda force=False: so)
    monkeypatch.setattr(oracle, "_lib", None)
    failed = run_catchers(catchers)
    assert failed, f"no pin caught the planted mistake ({mistake}); ran {catchers}"


# the same for the oracle's Python functions: (name, the mistake, text of oracle/__init__.py,
# planted text, pins expected to catch it)
PY_MUTANTS = [
    ('adam_bias2', 'second-moment bias correction with t + 1',
     'bc2 = 1.0 - beta2 ** t',
     'bc2 = 1.0 - beta2 ** (t + 1)',
     ['test_adam_constant_gradient_closed_form']),
    ('adam_m', 'first moment mixed with beta2',
     'm = beta1 * np.asarray(exp_avg[key], np.float64) + (1.0 - beta1) * g',
     'm = beta1 * np.asarray(exp_avg[key], np.float64) + (1.0 - beta2) * g',
     ['test_adam_constant_gradient_closed_form', 'test_adam_matches_torch_optim']),
    ('adam_eps', 'eps inside the square root',
     'p_new = p - rate * (m / bc1) / (np.sqrt(v / bc2) + eps)',
     'p_new = p - rate * (m / bc1) / np.sqrt(v / bc2 + eps)',
     ['test_adam_constant_gradient_closed_form', 'test_adam_matches_torch_optim']),
    ('adam_sh_dc', 'SH DC at the rest rate',
     'rate[0, :] = float(lr["sh_dc"])',
     'rate[0, :] = float(lr["sh_rest"])',
     ['test_adam_matches_torch_optim', 'test_adam_constant_gradient_closed_form']),
    ('adam_sparse_moments', 'sparse step still decays the moments of unseen rows',
     '            m = np.where(keep, np.asarray(exp_avg[key], np.float64), m)\n',
     '',
     ['test_adam_sparse_rows_leave_the_others_untouched']),
    ('backproject_centre', 'pixel corner instead of centre',
     '(px + 0.5 - c["cx"]) / c["fx"] * d',
     '(px - c["cx"]) / c["fx"] * d',
     ['test_backprojection_inverts_the_pinhole']),
    ('backproject_normalize', 'normalisation by 1 - T dropped',
     'd = D / np.where(mask, 1.0 - T, 1.0) if normalize else D',
     'd = D',
     ['test_backprojection_inverts_the_pinhole']),
    ('backproject_inverse', 'world = viewmat applied, not its inverse',
     'Vinv = np.linalg.inv(np.asarray(c["viewmat"], np.float64).reshape(4, 4))',
     'Vinv = np.asarray(c["viewmat"], np.float64).reshape(4, 4)',
     ['test_backprojection_inverts_the_pinhole']),
    ('fcs_halfopen', 'boxes closed at hi',
     'inside = mask & np.all((pts >= lo) & (pts < hi), axis=-1)',
     'inside = mask & np.all((pts >= lo) & (pts <= hi), axis=-1)',
     ['test_coverage_boxes_are_half_open']),
    ('fcs_mask', 'pixels no Gaussian reached counted',
     'inside = mask & np.all((pts >= lo) & (pts < hi), axis=-1)',
     'inside = np.all((pts >= lo) & (pts < hi), axis=-1)',
     ['test_coverage_of_a_wall_split_by_a_block_boundary']),
    ('densify_threshold', 'strict gradient threshold',
     'mean_grad >= f32(grad_threshold)',
     'mean_grad > f32(grad_threshold)',
     ['test_densify_thresholds_and_sd_views']),
    ('densify_clone', 'clone test on the smallest scale',
     'clone = dens & (ls.max(axis=1) <= f32(max_clone_log_scale))',
     'clone = dens & (ls.min(axis=1) <= f32(max_clone_log_scale))',
     ['test_densify_branches_and_order']),
    ('densify_prune', 'prune at or below the logit',
     'prune = lg < f32(prune_logit)',
     'prune = lg <= f32(prune_logit)',
     ['test_densify_thresholds_and_sd_views']),
    ('densify_cnt', 'densify without SD views',
     'dens = ~prune & (cnt > 0) & (mean_grad',
     'dens = ~prune & (cnt >= 0) & (mean_grad',
     ['test_densify_thresholds_and_sd_views']),
    ('densify_shrink', 'split children grow',
     'out["log_scales"][child] = np.asarray(params["log_scales"], np.float64)[g] - split_log_shrink',
     'out["log_scales"][child] = np.asarray(params["log_scales"], np.float64)[g] + split_log_shrink',
     ['test_densify_branches_and_order']),
    ('densify_rotation', 'split offset with R transposed',
     'np.einsum("nij,nj->ni", R, s * zk)',
     'np.einsum("nji,nj->ni", R, s * zk)',
     ['test_split_child_is_the_rotated_scaled_draw', 'test_split_children_follow_the_gaussian']),
    ('densify_clone_count', 'a clone makes three',
     'k_out = np.where(prune, 0, np.where(clone, 2, np.where(split, n_split, 1)))',
     'k_out = np.where(prune, 0, np.where(clone, 3, np.where(split, n_split, 1)))',
     ['test_densify_branches_and_order', 'test_densify_thresholds_and_sd_views']),
    ('kd_tau', 'camera kept only above tau',
     'if len(pts) and inside(pts, lo, hi).sum() / len(pts) >= tau:',
     'if len(pts) and inside(pts, lo, hi).sum() / len(pts) > tau:',
     ['test_kd_partition_keeps_a_camera_at_exactly_tau']),
    ('kd_axis', 'split along the shorter extent',
     'a = 0 if ext[0] >= ext[1] else 1',
     'a = 1 if ext[0] >= ext[1] else 0',
     ['test_kd_partition_bisection_closed_form', 'test_kd_partition_keeps_a_camera_at_exactly_tau']),
    ('kd_bisect', 'bisection toward the heavier side',
     'qhi, q = q, 0.5 * (qlo + q)',
     'qhi, q = q, 0.5 * (qhi + q)',
     ['test_kd_partition_bisection_closed_form']),
    ('kd_leaf_tie', 'latest leaf first among equals',
     '(len(leaves[i][2]) == len(leaves[best][2]) and leaves[i][3] < leaves[best][3])',
     '(len(leaves[i][2]) == len(leaves[best][2]) and leaves[i][3] > leaves[best][3])',
     ['test_kd_partition_splits_the_heaviest_leaf_earliest_first']),
    ('kd_heaviest', 'lightest leaf split',
     'if len(leaves[i][2]) > len(leaves[best][2]) or',
     'if len(leaves[i][2]) < len(leaves[best][2]) or',
     ['test_kd_partition_splits_the_heaviest_leaf_earliest_first']),
    ('kd_halfopen', 'KD boxes closed at hi',
     '        return np.all((pts >= lo) & (pts < hi), axis=-1)\n',
     '        return np.all((pts >= lo) & (pts <= hi), axis=-1)\n',
     ['test_kd_partition_bisection_closed_form', 'test_kd_partition_splits_the_heaviest_leaf_earliest_first']),
    ('depth_colour', 'the depth composite blends colours',
     'q = Projection(p.mean2d, p.conic, np.repeat(p.depth[:, None], 3, axis=1), p.opacity,',
     'q = Projection(p.mean2d, p.conic, p.color, p.opacity,',
     ['test_depth_composite_on_axis_closed_form'])
]


def run_catchers(catchers):
    """Runs each catcher: a pin's name (tests/test_oracle_pins.py, no arguments) or
    (module, name, arguments) with module "branches" (tests/test_oracle_branches.py) or
    "pins". Returns the ones that failed."""
    failed = []
    for c in catchers:
        mod, name, args = (pins, c, ()) if isinstance(c, str) else ({"pins": pins, "branches": branches}[c[0]], c[1],
                                                                    tuple(c[2]))
        fn = getattr(mod, name)
        assert len(inspect.signature(fn).parameters) == len(args), f"{name}: wrong number of arguments"
        try:
            fn(*args)
        except Exception:  # an assertion, or arithmetic the planted mistake broke
            failed.append(c)
    return failed


@pytest.mark.parametrize("name, mistake, old, new, catchers", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_pins_catch_a_planted_mistake_in_python(monkeypatch, name, mistake, old, new, catchers):
    src = open(oracle.__file__).read()
    assert src.count(old) == 1, f"{name}: the planted text must occur exactly once"
    mod = types.ModuleType("oracle_planted")
    mod.__file__ = oracle.__file__
    monkeypatch.setitem(sys.modules, "oracle_planted", mod)  # dataclasses look their module up
    exec(compile(src.replace(old, new), oracle.__file__, "exec"), mod.__dict__)
    for k, v in vars(mod).items():
        if isinstance(v, types.FunctionType):
            monkeypatch.setattr(oracle, k, v)
    failed = run_catchers(catchers)
    assert failed, f"no pin caught the planted mistake ({mistake}); ran {catchers}"


def _unique(catchers):
    seen, out = set(), []
    for c in catchers:
        key = c if isinstance(c, str) else (c[0], c[1], tuple(c[2]))
        if key not in seen:
            seen.add(key)
            out.append(c)
    return out


def test_every_catcher_passes_on_an_unchanged_copy(planted, monkeypatch):
    """The control: built from the unchanged source (and the unchanged Python module loaded
    the same way as the planted ones), every pin named above passes, so a failure above is the
    planted mistake's doing and not the harness's."""
    so = planted["unchanged"]
    monkeypatch.setattr(oracle, "_LIB", so)
    monkeypatch.setattr(oracle, "build", lambda force=False: so)
    monkeypatch.setattr(oracle, "_lib", None)
    assert run_catchers(_unique([c for m in MUTANTS for c in m[4]])) == []
    mod = types.ModuleType("oracle_planted")
    mod.__file__ = oracle.__file__
    monkeypatch.setitem(sys.modules, "oracle_planted", mod)
    exec(compile(open(oracle.__file__).read(), oracle.__file__, "exec"), mod.__dict__)
    for k, v in vars(mod).items():
        if isinstance(v, types.FunctionType):
            monkeypatch.setattr(oracle, k, v)
    assert run_catchers(_unique([c for m in PY_MUTANTS for c in m[4]])) == []
