"""The oracle's pins against planted mistakes (mutation check, CPU only).

Each case copies ``oracle/lobe_oracle.c``, plants one plausible mistake in it -- a dropped
term, a wrong sign, index or constant, a transposed operand, a threshold rule read the other
way -- builds the copy and runs the pins that should catch it against that build: at least
one of them must fail. The planted copies live in a temporary directory and never replace
the oracle; ``oracle._lib`` is pointed at a copy for one case and restored afterwards.
Mistakes that leave every result unchanged (reordering a product of symmetric matrices) are
not cases.
"""
import concurrent.futures
import inspect
import os
import subprocess

import pytest

import oracle
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
]


@pytest.fixture(scope="module")
def planted(tmp_path_factory):
    """name -> shared library of the oracle with that mistake planted (built in parallel)."""
    src = open(SRC).read()
    root = tmp_path_factory.mktemp("planted")

    def build(m):
        name, _, old, new, _ = m
        assert src.count(old) == 1, f"{name}: the planted text must occur exactly once"
        c = root / f"{name}.c"
        c.write_text(src.replace(old, new))
        so = root / f"lib{name}.so"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                               str(c), "-lm"])
        return name, str(so)

    with concurrent.futures.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        return dict(ex.map(build, MUTANTS))


@pytest.mark.parametrize("name, mistake, old, new, catchers", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_a_planted_mistake(planted, monkeypatch, name, mistake, old, new, catchers):
    so = planted[name]
    monkeypatch.setattr(oracle, "_LIB", so)
    monkeypatch.setattr(oracle, "build", lambda force=False: so)
    monkeypatch.setattr(oracle, "_lib", None)
    failed = []
    for pin in catchers:
        fn = getattr(pins, pin)
        assert not inspect.signature(fn).parameters, f"{pin} takes arguments"
        try:
            fn()
        except Exception:  # an assertion, or arithmetic the planted mistake broke
            failed.append(pin)
    assert failed, f"no pin caught the planted mistake ({mistake}); ran {catchers}"
