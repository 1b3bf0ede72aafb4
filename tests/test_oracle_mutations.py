"""The oracle's pins against planted mistakes.

Each case plants one plausible mistake in a copy of the oracle's C source (a
dropped term, a wrong sign, constant, index or order, a transposed operand,
the other reading of an open point) and runs the pin file that must catch
it: that run has to fail.  A control case runs every pin file against an
unmodified copy, which has to pass, so a caught mistake is never an artefact
of the copying.  The mistakes live only in the temporary copy; the oracle
itself is not touched.

A representative case per area runs by default; TURBOGS_ALL_MUTATIONS=1
runs all of them (a few minutes).
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")

# (name, pin file that catches it, text in the oracle's source, planted text)
MUTATIONS = [
    ('no_dilation', 'test_oracle_projection.py',
     'g->A = S2[0] + 0.3; g->B = S2[1]; g->C = S2[3] + 0.3;',
     'g->A = S2[0]; g->B = S2[1]; g->C = S2[3];'),
    ('conic_b_sign', 'test_oracle_loss_grad.py',
     'g->conic[1] = -g->B / g->det;',
     'g->conic[1] = g->B / g->det;'),
    ('radius_2sigma', 'test_oracle_render.py',
     'g->radius_f = 3.0 * sqrt(g->lam);',
     'g->radius_f = 2.0 * sqrt(g->lam);'),
    ('opacity_sign', 'test_oracle_loss_grad.py',
     'g->opac = 1.0 / (1.0 + exp(-ol));',
     'g->opac = 1.0 / (1.0 + exp(ol));'),
    ('sh_no_offset', 'test_oracle_projection.py',
     '    double s = 0.5;\n    for (int k = 0; k < nb; ++k) s += sh[k * 3 + c] * Y[k];',
     '    double s = 0.0;\n    for (int k = 0; k < nb; ++k) s += sh[k * 3 + c] * Y[k];'),
    ('sh_no_clamp', 'test_oracle_loss_grad.py',
     'g->rgb[c] = s > 0.0 ? s : 0.0;',
     'g->rgb[c] = s;'),
    ('alpha_cap', 'test_oracle_render.py',
     'double alpha = araw < 0.99 ? araw : 0.99;',
     'double alpha = araw < 0.999 ? araw : 0.999;'),
    ('alpha_min', 'test_oracle_render.py',
     'if (alpha < 1.0 / 255.0) continue;',
     'if (alpha < 1.0 / 128.0) continue;'),
    ('T_stop', 'test_oracle_render.py',
     'if (Tn < 1e-4) break;',
     'if (Tn < 1e-3) break;'),
    ('power_b', 'test_oracle_loss_grad.py',
     'double power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;',
     'double power = -0.5 * (a * dx * dx + c * dy * dy) - 0.5 * b * dx * dy;'),
    ('pixel_centre', 'test_oracle_render.py',
     'double cxp = px + 0.5, cyp = py + 0.5;',
     'double cxp = px, cyp = py;'),
    ('composite_T', 'test_oracle_loss_grad.py',
     'acc += p.T[j] * p.alpha[j] * rgb[3 * p.acc_id[j] + c];',
     'acc += p.T[j] * (1.0 - p.alpha[j]) * rgb[3 * p.acc_id[j] + c];'),
    ('bwd_dalpha', 'test_oracle_loss_grad.py',
     'dalpha += T * (c[ch] - S[ch]) * g[ch];',
     'dalpha += T * (c[ch] + S[ch]) * g[ch];'),
    ('bwd_dx', 'test_oracle_loss_grad.py',
     'grad2d[9 * i + 0] += dpow * (a * dx + b * dy);',
     'grad2d[9 * i + 0] += dpow * (a * dx - b * dy);'),
    ('bwd_dconic_b', 'test_oracle_loss_grad.py',
     'grad2d[9 * i + 3] += dpow * (-dx * dy);',
     'grad2d[9 * i + 3] += dpow * (-0.5 * dx * dy);'),
    ('bwd_S_order', 'test_oracle_loss_grad.py',
     'for (int ch = 0; ch < 3; ++ch) S[ch] = al * c[ch] + (1.0 - al) * S[ch];',
     'for (int ch = 0; ch < 3; ++ch) S[ch] = al * c[ch] + al * S[ch];'),
    ('stats_D', 'test_oracle_render.py',
     'double q = a * dx * dx + 2.0 * b * dx * dy + c * dy * dy;',
     'double q = a * dx * dx + b * dx * dy + c * dy * dy;'),
    ('stats_w', 'test_oracle_render.py',
     'double w = p.T[j] * p.alpha[j];\n      double dx = p.dx[j], dy = p.dy[j];\n      double a = conic[3 * i], b = conic[3 * i + 1], c = conic[3 * i + 2];\n      double q',
     'double w = p.alpha[j];\n      double dx = p.dx[j], dy = p.dy[j];\n      double a = conic[3 * i], b = conic[3 * i + 1], c = conic[3 * i + 2];\n      double q'),
    ('ncc_eps', 'test_oracle_loss_grad.py',
     'D[c] = sqrt(vx[c] * vy[c] + eps_n);',
     'D[c] = sqrt(vx[c] * vy[c]) + eps_n;'),
    ('lambda_no_clip', 'test_oracle_loss_grad.py',
     'lam = clampd(lam, 0.0, 1.0);',
     'lam = lam;'),
    ('ema_swap', 'test_oracle_loss_grad.py',
     'err_map[k] = orc_double_to_half((1.0 - beta) * old + beta * err_pix[s]);',
     'err_map[k] = orc_double_to_half(beta * old + (1.0 - beta) * err_pix[s]);'),
    ('loss_grad_sign', 'test_oracle_loss_grad.py',
     'dL_drgb[3 * s + c] = d / r / (double)P - lam / (3.0 * n_active) * dncc;',
     'dL_drgb[3 * s + c] = d / r / (double)P + lam / (3.0 * n_active) * dncc;'),
    ('err_charb', 'test_oracle_loss_grad.py',
     'e += fabs(d);',
     'e += r;'),
    ('age_no_sat', 'test_oracle_loss_grad.py',
     'if (age_map[k] < 65535) age_map[k]++;',
     'age_map[k]++;'),
    ('adam_no_bc2', 'test_oracle_hybrid.py',
     'p[k] -= lr[k] * (mi[k] / bc1) / (sqrt(vi[k] / bc2) + eps);',
     'p[k] -= lr[k] * (mi[k] / bc1) / (sqrt(vi[k]) + eps);'),
    ('lm_sign', 'test_oracle_hybrid.py',
     'for (int a = 0; a < d; ++a) p[ix[a]] += lr[ix[a]] * D[a];',
     'for (int a = 0; a < d; ++a) p[ix[a]] -= lr[ix[a]] * D[a];'),
    ('lm_damp', 'test_oracle_hybrid.py',
     'A[a * d + a] += sqrt(vi[ix[a]]) + eps_lm;',
     'A[a * d + a] += vi[ix[a]] + eps_lm;'),
    ('v_update', 'test_oracle_hybrid.py',
     'vi[k] = b2 * vi[k] + (1.0 - b2) * g[k] * g[k];',
     'vi[k] = b2 * vi[k] + (1.0 - b2) * fabs(g[k]);'),
    ('hard_key_inv', 'test_oracle_sampling.py',
     'return w ? (double)L / (double)w : ldexp((double)L, 900);',
     'return w ? (double)w / (double)L : ldexp((double)L, 900);'),
    ('tile_age_max', 'test_oracle_sampling.py',
     'if (a < amin) amin = a;',
     'if (amin == 0xFFFFFFFFu || a > amin) amin = a;'),
    ('age_order', 'test_oracle_sampling.py',
     'if (x->age != y->age) return x->age > y->age ? -1 : 1;',
     'if (x->age != y->age) return x->age < y->age ? -1 : 1;'),
    ('view_anchor_min', 'test_oracle_views.py',
     'if (stack[v] && (anchor < 0 || sums[v] > sums[anchor])) anchor = v;',
     'if (stack[v] && (anchor < 0 || sums[v] < sums[anchor])) anchor = v;'),
    ('view_key_sign', 'test_oracle_views.py',
     'cand[m].key = (lg + s * 1.4426950408889634) + 0.0;',
     'cand[m].key = (lg - s * 1.4426950408889634) + 0.0;'),
    ('view_refill', 'test_oracle_views.py',
     '  if (on_stack < k)\n',
     '  if (on_stack < 1)\n'),
    ('mlp_relu2', 'test_oracle_mlp.py',
     'double d = h2[k] > 0.0 ? dy * w3 : 0.0;',
     'double d = dy * w3;'),
    ('rect_hi_no_plus1', 'test_oracle_loss_grad.py',
     'float b = floorf((cf + rf) * 0.0625f) + 1.0f;',
     'float b = floorf((cf + rf) * 0.0625f);'),
    ('rect_lo_minus', 'test_oracle_loss_grad.py',
     'float a = floorf((cf - rf) * 0.0625f);',
     'float a = floorf((cf - rf) * 0.0625f) + 1.0f;'),
    ('J_clamp_13', 'test_oracle_render.py',
     'double limx = 1.3 * (0.5 * cam->width / cam->fx), limy = 1.3 * (0.5 * cam->height / cam->fy);',
     'double limx = 1e9, limy = 1e9;'),
    ('split_floor', 'test_oracle_sampling.py',
     'int h = (hard_pm * n + 500) / 1000;',
     'int h = (hard_pm * n) / 1000;'),
    ('split_no_clamp', 'test_oracle_sampling.py',
     'if (s > n - h) s = n - h;',
     'if (0) s = n - h;'),
    ('hard_not_first', 'test_oracle_sampling.py',
     '  qsort(tmp, (size_t)m, sizeof(item_t), cmp_hard);\n  for (int i = 0; i < kh; ++i) it[tmp[i].idx].taken = 1;',
     '  qsort(tmp, (size_t)m, sizeof(item_t), cmp_unif);\n  for (int i = 0; i < kh; ++i) it[tmp[i].idx].taken = 1;'),
    ('ncc_mean_no_div', 'test_oracle_loss_grad.py',
     'for (int c = 0; c < 3; ++c) { mx[c] /= nn; my[c] /= nn; }',
     'for (int c = 0; c < 3; ++c) { mx[c] /= nn; my[c] /= (nn + 1); }'),
    ('ncc_sample_var', 'test_oracle_loss_grad.py',
     'vx[c] /= nn; vy[c] /= nn; cv[c] /= nn;',
     'vx[c] /= nn - 1; vy[c] /= nn - 1; cv[c] /= nn;'),
    ('sncc_no_avg', 'test_oracle_loss_grad.py',
     'double sncc = 1.0 - (ncc[0] + ncc[1] + ncc[2]) / 3.0;',
     'double sncc = 1.0 - (ncc[0] + ncc[1] + ncc[2]);'),
    ('loss_tile_norm', 'test_oracle_loss_grad.py',
     'loss += lam * sncc / n_active;',
     'loss += lam * sncc;'),
    ('l1_norm', 'test_oracle_loss_grad.py',
     'loss += r / (double)P;',
     'loss += r;'),
    ('bg_term', 'test_oracle_render.py',
     'out_rgb[3 * s + c] = acc + p.T_final * bg[c];',
     'out_rgb[3 * s + c] = acc + bg[c];'),
    ('stats_e', 'test_oracle_render.py',
     'stats[3 * i] += err[s] * w;',
     'stats[3 * i] += err[s];'),
    ('app_block_order', 'test_oracle_hybrid.py',
     'static const int app[4] = {11, 12, 13, 10};',
     'static const int app[4] = {10, 11, 12, 13};'),
    ('lr_groups', 'test_oracle_hybrid.py',
     'int grp = k < 3 ? 0 : k < 6 ? 1 : k < 10 ? 2 : k == 10 ? 3 : k < 14 ? 4 : 5;',
     'int grp = k < 3 ? 0 : k < 6 ? 1 : k < 10 ? 2 : k == 10 ? 3 : k < 13 ? 4 : 5;'),
    ('mlp_bias1', 'test_oracle_mlp.py',
     'double s = b1[j];',
     'double s = 0.0;'),
    ('mlp_relu1_fwd', 'test_oracle_mlp.py',
     '      s = s > 0.0 ? s : 0.0;\n      h1[j] = bf16 ? orc_round_bf16(s) : s;',
     '      h1[j] = bf16 ? orc_round_bf16(s) : s;'),
    ('obs_mean_T', 'test_oracle_predictor.py',
     'mem[4 * t + 1] = st / n;',
     'mem[4 * t + 1] = st;'),
    ('obs_target', 'test_oracle_predictor.py',
     'if (target) target[j] = log1p(se / n) - prev;',
     'if (target) target[j] = log1p(se / n);'),
    ('feat_age', 'test_oracle_predictor.py',
     'f[4] = log1p(age);',
     'f[4] = age;'),
    ('feat_centre', 'test_oracle_predictor.py',
     'double u = ((t % tx) * 16 + 8 - cx) / fx, v = ((t / tx) * 16 + 8 - cy) / fy;',
     'double u = ((t % tx) * 16 - cx) / fx, v = ((t / tx) * 16 - cy) / fy;'),
    ('refresh_expm1', 'test_oracle_predictor.py',
     'double want = expm1(p > 0.0 ? p : 0.0);',
     'double want = exp(p > 0.0 ? p : 0.0);'),
    ('view_stack_keep', 'test_oracle_views.py',
     '    if (drawn[u] || u == anchor) stack[u] = 0;',
     '    if (drawn[u]) stack[u] = 0;'),
    ('view_pose_dir', 'test_oracle_views.py',
     '  double f0 = M[8], f1 = M[9], f2 = M[10];',
     '  double f0 = M[2], f1 = M[6], f2 = M[10];'),
    ('view_log2_frac', 'test_oracle_views.py',
     '    if (hi >> 63) { frac |= 1; m = hi; }\n    else m = hi << 1;\n  }\n  return ((uint64_t)ip << 32) | frac;',
     '    if (hi >> 63) { frac |= 1; m = hi; }\n    else m = hi << 1;\n  }\n  return ((uint64_t)ip << 32);'),
    ('znear_cull', 'test_oracle_render.py',
     'if (!(z > cam->znear)) return;',
     'if (!(z > 0.0)) return;'),
    ('bwd_clamp_dz', 'test_oracle_loss_grad.py',
     'dpc[2] += dJ[2] * (cam.fx * lim / (z * z));',
     'dpc[2] += 0.0 * dJ[2];'),
    ('bwd_scale', 'test_oracle_loss_grad.py',
     'out[3 + c] = ds * g.s[c];',
     'out[3 + c] = ds;'),
    ('bwd_dS2_sign', 'test_oracle_loss_grad.py',
     'for (int k = 0; k < 4; ++k) dS2[k] = -dS2[k];',
     ''),
    ('bwd_dT2', 'test_oracle_loss_grad.py',
     'for (int k = 0; k < 6; ++k) dT[k] = 2.0 * dS2TS[k];',
     'for (int k = 0; k < 6; ++k) dT[k] = dS2TS[k];'),
    ('bin_id_order', 'test_oracle_render.py',
     'return x->id < y->id ? -1 : (x->id > y->id);',
     'return x->id > y->id ? -1 : (x->id < y->id);'),
    ('bf16_ties', 'test_oracle_mlp.py',
     'u += 0x7fffu + lsb;',
     'u += 0x8000u;'),
    ('fp16_subnormal', 'test_oracle_basics.py',
     'double q = rint(a * 16777216.0);',
     'double q = floor(a * 16777216.0);'),
    ('chol_index', 'test_oracle_hybrid.py',
     'for (int k = i + 1; k < d; ++k) s -= L[k * d + i] * x[k];',
     'for (int k = i + 1; k < d; ++k) s -= L[i * d + k] * x[k];'),
    ('neglog2_int', 'test_oracle_basics.py',
     'return ((uint64_t)(64 - ip) << 32) - frac;',
     'return ((uint64_t)(63 - ip) << 32) - frac;'),
    ('err_weight_sub', 'test_oracle_basics.py',
     'if (e == 0) return (uint64_t)m;',
     'if (e == 0) return (uint64_t)m << 1;'),
    ('refresh_mean0', 'test_oracle_predictor.py',
     'err[k] = orc_double_to_half(mean > 0.0 ? e * (want / mean) : want);',
     'err[k] = orc_double_to_half(mean > 0.0 ? e * (want / mean) : 0.0);'),
    ('mlp_bwd_dW2', 'test_oracle_mlp.py',
     'for (int k = 0; k < MLP_H; ++k) dW2[j * MLP_H + k] += dh2[j] * h1[k];',
     'for (int k = 0; k < MLP_H; ++k) dW2[k * MLP_H + j] += dh2[j] * h1[k];'),
    ('mlp_bwd_loss', 'test_oracle_mlp.py',
     'double dy = e / (double)R;',
     'double dy = e;'),
    ('sh_dir_grad', 'test_oracle_loss_grad.py',
     'for (int a = 0; a < 3; ++a) dmu[a] += (ddir[a] - g.dir[a] * dot) / g.vlen;',
     'for (int a = 0; a < 3; ++a) dmu[a] += ddir[a] / g.vlen;'),
    ('score_fade_dir', 'test_oracle_density.py',
     'double lambda_eff = lambda_base * (1.0 - rho);',
     'double lambda_eff = lambda_base * rho;'),
    ('score_no_norm', 'test_oracle_density.py',
     'double e = r[0] / (r[1] + eps);',
     'double e = r[0];'),
    ('score_swap_ed', 'test_oracle_density.py',
     '    s_out[i] = e + lambda_eff * d;',
     '    s_out[i] = d + lambda_eff * e;'),
    ('score_d_by_e', 'test_oracle_density.py',
     'double d = r[2] / (r[1] + eps);',
     'double d = r[2] / (r[0] + eps);'),
    ('ssim_cov_sign', 'test_oracle_ssim.py',
     'a2[c] = 2.0 * cv[c] + C2;',
     'a2[c] = -2.0 * cv[c] + C2;'),
    ('ssim_C1', 'test_oracle_ssim.py',
     'const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;',
     'const double C1 = 0.03 * 0.03, C2 = 0.03 * 0.03;'),
    ('ssim_C2', 'test_oracle_ssim.py',
     'const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;',
     'const double C1 = 0.01 * 0.01, C2 = 0.01 * 0.01;'),
    ('ssim_grad_factor', 'test_oracle_ssim.py',
     'double dss = 2.0 * ((my[c] * a2[c]',
     'double dss = 1.0 * ((my[c] * a2[c]'),
    ('ssim_grad_b2', 'test_oracle_ssim.py',
     'ss[c] * (mx[c] / b1[c] + (xv - mx[c]) / b2[c])) / nn;',
     'ss[c] * (mx[c] / b1[c] + (xv - mx[c]) / b1[c])) / nn;'),
    ('ssim_luminance_mean', 'test_oracle_ssim.py',
     'b1[c] = mx[c] * mx[c] + my[c] * my[c] + C1;',
     'b1[c] = 2.0 * mx[c] * my[c] + C1;'),
]

DEFAULT = {"ssim_cov_sign", "no_dilation", "T_stop", "stats_D", "bwd_dalpha", "ncc_sample_var", "ema_swap", "lm_damp",
           "split_floor", "hard_key_inv", "view_key_sign", "mlp_relu2", "feat_centre", "bwd_clamp_dz"}
ALL = os.environ.get("TURBOGS_ALL_MUTATIONS") == "1"
CASES = [m for m in MUTATIONS if ALL or m[0] in DEFAULT]


def _oracle_copy(tmp_path, src):
    d = tmp_path / "oracle"
    d.mkdir()
    (d / "turbogs_oracle.c").write_text(src)
    shutil.copy(os.path.join(ORACLE, "__init__.py"), d / "__init__.py")
    return tmp_path


def _run_pins(tmp_path, files):
    # run from the copy's directory, so the copy comes first on the path; the
    # repository root is on the path too, so the test configuration does not
    # put the original oracle in front of it
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([str(tmp_path), ROOT]))
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
    cmd += [os.path.join(ROOT, "tests", f) for f in files]
    return subprocess.run(cmd, cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=1200)


def test_unmodified_copy_passes_every_pin_file(tmp_path):
    src = open(os.path.join(ORACLE, "turbogs_oracle.c")).read()
    files = sorted({m[1] for m in MUTATIONS})
    r = _run_pins(_oracle_copy(tmp_path, src), files)
    assert r.returncode == 0, r.stdout[-2000:]
    probe = subprocess.run([sys.executable, "-c", "import oracle; print(oracle.__file__)"], cwd=str(tmp_path),
                           env=dict(os.environ, PYTHONPATH=os.pathsep.join([str(tmp_path), ROOT])),
                           capture_output=True, text=True)
    assert probe.stdout.strip().startswith(str(tmp_path))


@pytest.mark.parametrize("name,pins,old,new", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_is_caught(tmp_path, name, pins, old, new):
    src = open(os.path.join(ORACLE, "turbogs_oracle.c")).read()
    assert old in src, "the planted site is gone from the oracle: update the case"
    r = _run_pins(_oracle_copy(tmp_path, src.replace(old, new)), [pins])
    # 1: the pins ran and one failed; < 0: the mistake made the oracle itself
    # crash (a draw past the end of its candidates), which the pins surface too
    assert r.returncode == 1 or r.returncode < 0, (name, r.returncode, r.stdout[-1500:])
