"""Plants one plausible slip at a time into a copy of an oracle (or of the
parity gate, tests/parity.py) and checks that its pins fail with it.  CPU
only, run by hand:

    python tests/plant_slips.py [c|proposal|scfv|resize|parity ...] [--only NAME ...]

A slip is one exact text replacement in the oracle's source.  The C oracle's
copy is built with gcc into a temporary folder and loaded, in a child
process, in place of the real library; a numpy oracle's copy is loaded, in a
child process, in place of the real module.  The child runs the oracle's pin
file and the slip counts as caught when a pin fails.

Prints CAUGHT or SURVIVED per slip and exits 1 when a slip survives that is
not listed in EXPECTED_SURVIVORS (each with the reason it cannot be caught).
"""
from __future__ import annotations

import argparse
import os
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Slips no pin can catch, and why.
EXPECTED_SURVIVORS = {
    # Equivalent: with det H = 0 the edge ratio tr^2 / det is infinite (or NaN),
    # so the next test rejects the point anyway.
    ("c", "ref_det_ge"),
    # Equivalent: an exact double root of dp/dsigma (D = 0) has p'' = 0 exactly
    # there, which the next test rejects.
    ("c", "D_lt"),
    # Equivalent: with D > 0 the two roots are distinct and p'' is not 0 at
    # either; in the near-quadratic branch p'' is 2 a2 + O(a3), and a2 != 0.
    ("c", "pdd_zero_kept"),
    # Equivalent: a square image takes the other branch to the same size.
    ("resize", "ge_to_gt"),
    # Equivalent: an image whose larger side equals the limit is "resized" to
    # its own size, which copies it.
    ("resize", "no_resize_equal"),
}


def _run_child(code: str) -> bool:
    """True when the child's pytest run failed (the slip was caught)."""
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=1800)
    return r.returncode != 0


def check_c(slips, tmpd):
    src = open(os.path.join(ROOT, "oracle", "cdvs_oracle.c")).read()
    for name, old, new in slips:
        if src.count(old) != 1:
            raise SystemExit(f"c/{name}: the text to replace occurs {src.count(old)} times")
        cpath = os.path.join(tmpd, f"{name}.c")
        lib = os.path.join(tmpd, f"{name}.so")
        with open(cpath, "w") as f:
            f.write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-I", os.path.join(ROOT, "oracle"), cpath, "-o", lib, "-lm"])
        code = ("import sys; sys.path.insert(0, '.'); import oracle.oracle as O; "
                f"O.LIB_PATH = {lib!r}; O.build = lambda force=False: {lib!r}; import pytest; "
                "sys.exit(pytest.main(['-q', '-x', '-p', 'no:cacheprovider', 'tests/test_oracle_pins.py']))")
        yield name, _run_child(code)


def check_py(module: str, test_file: str, slips, tmpd, path=None):
    """Slips in a Python module: oracle/<module>.py, or the module at `path`
    imported under the name `module`."""
    path = path or os.path.join(ROOT, "oracle", f"{module}.py")
    src = open(path).read()
    for name, old, new in slips:
        if src.count(old) != 1:
            raise SystemExit(f"{module}/{name}: the text to replace occurs {src.count(old)} times")
        mpath = os.path.join(tmpd, f"{module.replace('.', '_')}_{name}.py")
        with open(mpath, "w") as f:
            f.write(src.replace(old, new))
        parent = module.rsplit(".", 1)[0] if "." in module else None
        code = ("import sys, types; sys.path.insert(0, '.'); sys.path.insert(0, 'tests'); "
                + (f"import {parent}; " if parent else "")
                + f"m = types.ModuleType({module!r}); m.__file__ = {path!r}; "
                f"exec(compile(open({mpath!r}).read(), {path!r}, 'exec'), m.__dict__); "
                f"sys.modules[{module!r}] = m; "
                + (f"{parent}.{module.rsplit('.', 1)[1]} = m; " if parent else "")
                + f"import pytest; sys.exit(pytest.main(['-q', '-x', '-p', 'no:cacheprovider', {test_file!r}]))")
        yield name, _run_child(code)


# ---- slips of the C oracle (S1-S11): name, text, replacement
C_SLIPS = [
    ('scale_den',
     '(double)k / (double)(p->scales_per_octave - 1)',
     '(double)k / (double)(p->scales_per_octave)'),
    ('tau_base_swap',
     '(o == 0) ? p->sigma_in : p->sigma0',
     '(o == 0) ? p->sigma0 : p->sigma_in'),
    ('taps_3sigma',
     '(int)ceil(4.0 * tau)',
     '(int)ceil(3.0 * tau)'),
    ('decimate_odd',
     'top[(size_t)(2 * y) * Wo[o - 1] + 2 * x]',
     'top[(size_t)(2 * y + 1) * Wo[o - 1] + 2 * x + 1]'),
    ('lap_no_s2',
     'L[(size_t)y * W + x] = s * s * (',
     'L[(size_t)y * W + x] = s * ('),
    ('lap_sign',
     '(l + r + u + d - 4.0 * c)',
     '(4.0 * c - l - r - u - d)'),
    ('ext_type_flip',
     'int t = pdd < 0.0 ? +1 : -1;',
     'int t = pdd < 0.0 ? -1 : +1;'),
    ('ext_tie_larger_s',
     '(fabs(v) == fabs(best_v) && s < best_s)',
     '(fabs(v) == fabs(best_v) && s > best_s)'),
    ('ext_first_wins',
     'if (best_t == 0 || fabs(v) > fabs(best_v) ||',
     'if (best_t == 0 || fabs(v) < fabs(best_v) ||'),
    ('ref_hxy_sign',
     '0.25 * (q[8] - q[6] - q[2] + q[0])',
     '0.25 * (q[8] - q[6] + q[2] - q[0])'),
    ('ref_dx_sign',
     'double dx = -(hyy * gx - hxy * gy) / det;',
     'double dx = (hyy * gx - hxy * gy) / det;'),
    ('ref_resp_full',
     'q[4] + 0.5 * (gx * dx + gy * dy)',
     'q[4] + (gx * dx + gy * dy)'),
    ('edge_lim_no_div',
     '(p->edge_r + 1.0) * (p->edge_r + 1.0) / p->edge_r',
     '(p->edge_r + 1.0) * (p->edge_r + 1.0)'),
    ('nbr_nonstrict',
     't > 0 ? !(pn < v + m * fabs(v)) : !(pn > v - m * fabs(v))',
     't > 0 ? !(pn <= v + m * fabs(v)) : !(pn >= v - m * fabs(v))'),
    ('kp_scale_oct',
     'const double scale = ldexp(1.0, o);',
     'const double scale = ldexp(1.0, o + 1);'),
    ('dd_window_half',
     'double win = ldexp(1.0, oc) * (1.0 - m);',
     'double win = ldexp(1.0, oc - 1) * (1.0 - m);'),
    ('dd_keep_lower',
     'if (rb > ra * (1.0 + m) ||',
     'if (rb < ra * (1.0 - m) ||'),
    ('dd_tie_finer',
     '(m == 0.0 && rb == ra && c[b].octave < c[a].octave)',
     '(m == 0.0 && rb == ra && c[b].octave > c[a].octave)'),
    ('sel_y_desc',
     'if (a->y != b->y) return a->y < b->y ? -1 : 1;',
     'if (a->y != b->y) return a->y < b->y ? 1 : -1;'),
    ('sel_x_before_y',
     'if (a->y != b->y) return a->y < b->y ? -1 : 1;\n    if (a->x != b->x) return a->x < b->x ? -1 : 1;',
     'if (a->x != b->x) return a->x < b->x ? -1 : 1;\n    if (a->y != b->y) return a->y < b->y ? -1 : 1;'),
    ('desc_level_floor',
     '(int)lround((double)(K - 1) * log2(so / p->sigma0))',
     '(int)floor((double)(K - 1) * log2(so / p->sigma0))'),
    ('grad_gy_sign',
     '*gy = G[(size_t)clampi(v + 1, 0, H - 1) * W + u] - G[(size_t)clampi(v - 1, 0, H - 1) * W + u];',
     '*gy = G[(size_t)clampi(v - 1, 0, H - 1) * W + u] - G[(size_t)clampi(v + 1, 0, H - 1) * W + u];'),
    ('ori_disc_le',
     'if (!(d2 < R2)) continue;',
     'if (!(d2 <= R2)) continue;'),
    ('ori_w_no_half',
     'exp(-d2 / (2.0 * sw * sw))',
     'exp(-d2 / (sw * sw))'),
    ('ori_peak_ge',
     'if (!(c > l && c > r)) continue;',
     'if (!(c >= l && c >= r)) continue;'),
    ('ori_parab_sign',
     'double off = 0.5 * (l - r) / (l - 2.0 * c + r);',
     'double off = 0.5 * (r - l) / (l - 2.0 * c + r);'),
    ('ori_centre_no_half',
     '((double)b + 0.5 + off) / 36.0',
     '((double)b + off) / 36.0'),
    ('desc_rot_sign',
     'double xr = (ct * du + st * dv) / cs;\n            double yr = (-st * du + ct * dv) / cs;',
     'double xr = (ct * du - st * dv) / cs;\n            double yr = (st * du + ct * dv) / cs;'),
    ('desc_rel_plus',
     'double rel = atan2(gy, gx) - theta;',
     'double rel = atan2(gy, gx) + theta;'),
    ('desc_cell_offset_2',
     'double cx = xr + 1.5, cy = yr + 1.5;',
     'double cx = xr + 2.0, cy = yr + 2.0;'),
    ('desc_xy_swap',
     'd[(yy * 4 + xx) * 8 + oo]',
     'd[(xx * 4 + yy) * 8 + oo]'),
    ('desc_clamp_03',
     'if (d[i] > 0.2) d[i] = 0.2;',
     'if (d[i] > 0.3) d[i] = 0.3;'),
    ('desc_no_renorm',
     '    inv = 1.0 / sqrt(n2);\n    for (int i = 0; i < 128; ++i) d[i] *= inv;\n}',
     '    inv = 1.0;\n    for (int i = 0; i < 128; ++i) d[i] *= inv;\n}'),
    ('oct_floor_half',
     'w = (w + 1) / 2; /* ceil(W/2): decimation keeps the even coordinates */',
     'w = w / 2;'),
    ('oct_min_size',
     'if (w < 3 || h < 3) break;',
     'if (w < 2 || h < 2) break;'),
    ('desc_disc_le',
     'if (!(du * du + dv * dv < R2)) continue;',
     'if (!(du * du + dv * dv <= R2)) continue;'),
    ('tr_a_v2',
     'v[2] = (h[0] - h[1]) / 2.0;\n    v[3] = (h[2] - h[3]) / 2.0;',
     'v[2] = (h[1] - h[0]) / 2.0;\n    v[3] = (h[2] - h[3]) / 2.0;'),
    ('tr_b_v7_div4',
     'v[7] = ((h[0] + h[1] + h[2] + h[3]) - (h[4] + h[5] + h[6] + h[7])) / 8.0;',
     'v[7] = ((h[0] + h[1] + h[2] + h[3]) - (h[4] + h[5] + h[6] + h[7])) / 4.0;'),
    ('tr_checker_swap',
     'if (((cx + cy) & 1) == 0) transform_set_a',
     'if (((cx + cy) & 1) == 1) transform_set_a'),
    ('tern_le',
     'q[j] = (int8_t)(v[j] < t_lo[j] ? -1 : (v[j] > t_hi[j] ? 1 : 0));',
     'q[j] = (int8_t)(v[j] <= t_lo[j] ? -1 : (v[j] >= t_hi[j] ? 1 : 0));'),
    ('dd_dlog_no_abs',
     'if (!(fabs(log2(c[a].sigma / c[b].sigma)) <= p->dedupe_dlog2 * (1.0 - m))) continue;',
     'if (!(log2(c[a].sigma / c[b].sigma) <= p->dedupe_dlog2 * (1.0 - m))) continue;'),
    ('sel_no_cap',
     'int N = m < p->max_keypoints ? m : p->max_keypoints;',
     'int N = m;'),
    ('ori_max_ori',
     'int n = np < p->max_orientations ? np : p->max_orientations;',
     'int n = np;'),
    ('ori_bin_round',
     'double fl = floor(f);',
     'double fl = floor(f + 0.5);'),
    ('contrast_strict',
     'if (!(fabs(v) >= T)) continue;',
     'if (!(fabs(v) > T)) continue;'),
    ('offset_lt',
     'if (!(fabs(dx) <= omax && fabs(dy) <= omax)) return 0;',
     'if (!(fabs(dx) < omax && fabs(dy) < omax)) return 0;'),
    ('sigma_range_open',
     'if (!(s >= lo && s <= hi)) continue;',
     'if (!(s > lo && s < hi)) continue;'),
    ('dd_any_octaves',
     'if (d != 1 && d != -1) continue;',
     'if (d == 0) continue;'),
    ('ref_det_ge',
     'if (!(det > 0.0)) return 0;',
     'if (!(det >= 0.0)) return 0;'),
    ('sel_resp_asc',
     'if (ra != rb) return ra > rb ? -1 : 1;',
     'if (ra != rb) return ra < rb ? -1 : 1;'),
    ('sel_sigma_desc',
     'if (a->sigma != b->sigma) return a->sigma < b->sigma ? -1 : 1;',
     'if (a->sigma != b->sigma) return a->sigma < b->sigma ? 1 : -1;'),
    ('sel_oct_desc',
     'if (a->octave != b->octave) return a->octave < b->octave ? -1 : 1;',
     'if (a->octave != b->octave) return a->octave < b->octave ? 1 : -1;'),
    ('peak_ratio_ge',
     'if (!(c > p->ori_peak_ratio * mx * (1.0 - m))) continue;',
     'if (!(c >= p->ori_peak_ratio * mx * (1.0 - m))) continue;'),
    ('peaks_tie_bin_desc',
     '(pv[j] == pv[j - 1] && pb[j] < pb[j - 1])',
     '(pv[j] == pv[j - 1] && pb[j] > pb[j - 1])'),
    ('taps_no_norm',
     'for (int i = 0; i < 2 * r + 1; ++i) taps[i] /= sum;',
     ''),
    ('base_from_level2',
     'const double *top = levels + off - (size_t)Wo[o - 1] * Ho[o - 1];',
     'const double *top = levels + off - 2 * (size_t)Wo[o - 1] * Ho[o - 1];'),
    ('kp_no_offset',
     'k.xo = x + r[0];',
     'k.xo = x;'),
    ('p_ss_factor',
     'k.p_ss = 6.0 * a[3] * ss + 2.0 * a[2];',
     'k.p_ss = 3.0 * a[3] * ss + 2.0 * a[2];'),
    ('tr_a_v6_half',
     'v[6] = ((h[0] + h[4]) - (h[2] + h[6])) / 4.0;',
     'v[6] = ((h[0] + h[4]) - (h[2] + h[6])) / 2.0;'),
    ('ori_margin_dir',
     'if (p->ori_margin > 0.0 && frac > 1.0 - p->ori_margin) b += 1;',
     'if (p->ori_margin > 0.0 && frac > 1.0 - p->ori_margin) b -= 1;'),
    ('desc_w_sigma',
     'const double ws2 = 2.0 * p->desc_weight_sigma * p->desc_weight_sigma;',
     'const double ws2 = p->desc_weight_sigma * p->desc_weight_sigma;'),
    ('describe_level0',
     'const double *G = levels + oracle_level_offset(W, H, p, o, k);',
     'const double *G = levels + oracle_level_offset(W, H, p, o, 0);'),
    ('extract_unordered',
     'for (int i = 0; i < N; ++i) sel[i] = cand[order[i]];',
     'for (int i = 0; i < N; ++i) sel[i] = cand[i];'),
    ('quad_root_sign',
     'if (B != 0.0) roots[nr++] = -C / B;',
     'if (B != 0.0) roots[nr++] = C / B;'),
    ('detect_border_2',
     'for (int y = 1; y < H - 1; ++y)',
     'for (int y = 2; y < H - 1; ++y)'),
    ('filter_zero_pad',
     'for (int q = -r; q <= r; ++q) acc += in[(size_t)clampi(i + q, 0, H - 1) * W + j] * taps[q + r];',
     'for (int q = -r; q <= r; ++q) if (i + q >= 0 && i + q < H) acc += in[(size_t)(i + q) * W + j] * taps[q + r];'),
    ('lap_zero_left',
     'double l = G[(size_t)y * W + clampi(x - 1, 0, W - 1)];',
     'double l = x > 0 ? G[(size_t)y * W + x - 1] : 0.0;'),
    ('D_lt',
     'if (D <= 0.0) return 0;',
     'if (D < 0.0) return 0;'),
    ('pdd_zero_kept',
     'if (pdd == 0.0) continue;',
     ''),
    ('ref_gy_sign',
     'double gy = 0.5 * (q[7] - q[1]);',
     'double gy = 0.5 * (q[1] - q[7]);'),
    ('ref_hyy_wrong',
     'double hyy = q[7] - 2.0 * q[4] + q[1];',
     'double hyy = q[7] - 2.0 * q[4] + q[3];'),
]

# ---- slips of the proposal-network oracle
PROPOSAL_SLIPS = [
    ('no_bf16_a1',
     'a1 = rnd(np.maximum(z1, 0.0))',
     'a1 = np.maximum(z1, 0.0)'),
    ('w_not_rounded',
     'w1, w2, w3, wh = rnd(p["W1"]), rnd(p["W2"]), rnd(p["W3"]), rnd(p["Wh"])',
     'w1, w2, w3, wh = p["W1"], p["W2"], p["W3"], p["Wh"]'),
    ('conv1_stride1',
     'z1 = conv3x3(x, w1, p["b1"], 2)',
     'z1 = conv3x3(x, w1, p["b1"], 1)'),
    ('pool_cells_2',
     'cell = a3[:, 4 * ty:min(4 * ty + 4, H2), 4 * tx:min(4 * tx + 4, W2)]',
     'cell = a3[:, 2 * ty:min(2 * ty + 2, H2), 2 * tx:min(2 * tx + 2, W2)]'),
    ('b2_dropped',
     'z2 = conv3x3(a1, w2, p["b2"], 2)',
     'z2 = conv3x3(a1, w2, 0 * p["b2"], 2)'),
    ('bce_no_log1p',
     '+ np.log1p(np.exp(-np.abs(z)))',
     '+ 0.0'),
    ('input_shift_127',
     '(np.asarray(img, np.float64) - 128.0) / 64.0',
     '(np.asarray(img, np.float64) - 127.0) / 64.0'),
    ('no_relu_a3',
     'a3 = np.maximum(z3, 0.0)',
     'a3 = z3'),
    ('pool_sum_over_16',
     'cell.mean(axis=(1, 2)) if cell.size else 0.0',
     'cell.sum(axis=(1, 2)) / 16.0 if cell.size else 0.0'),
    ('head_bias_sign',
     '+ p["bh"][0]',
     '- p["bh"][0]'),
    ('no_bf16_a2',
     'a2 = rnd(np.maximum(z2, 0.0))',
     'a2 = np.maximum(z2, 0.0)'),
    ('conv3_stride2',
     'z3 = conv3x3(a2, w3, p["b3"], 1)',
     'z3 = conv3x3(a2, w3, p["b3"], 2)'),
    ('bce_sign',
     '- y * z +',
     '+ y * z +'),
    ('blocks_of_8',
     'th, tw = -(-H // 16), -(-W // 16)',
     'th, tw = -(-H // 8), -(-W // 8)'),
    ('bw_sigmoid_sign',
     'dz = (1.0 / (1.0 + np.exp(-z)) - y) / n_blocks',
     'dz = (y - 1.0 / (1.0 + np.exp(-z))) / n_blocks'),
    ('bw_no_relu_mask_2',
     'dz2 = da2 * (c["z2"] > 0)',
     'dz2 = da2'),
    ('bw_pool_div_16',
     'da3[:, ys, xs] = dP[:, ty, tx][:, None, None] / n',
     'da3[:, ys, xs] = dP[:, ty, tx][:, None, None] / 16'),
    ('bw_dw_transposed',
     'dw[:, :, ky, kx] = np.einsum("ohw,chw->oc", dz, pad[sl])',
     'dw[:, :, ky, kx] = np.einsum("ohw,chw->co", dz, pad[sl])'),
    ('bw_da_w_transposed',
     'dpad[sl] += np.einsum("oc,ohw->chw", w[:, :, ky, kx], dz)',
     'dpad[sl] += np.einsum("co,ohw->chw", w[:, :, ky, kx], dz)'),
    ('bw_bh_mean',
     'g["bh"] += dz.sum()',
     'g["bh"] += dz.mean()'),
    ('bw_per_image_mean',
     'dz = (1.0 / (1.0 + np.exp(-z)) - y) / n_blocks',
     'dz = (1.0 / (1.0 + np.exp(-z)) - y) / len(imgs)'),
    ('labels_floor',
     'bx = min(max(int(np.floor(x + 0.5)) // 16, 0), tw - 1)',
     'bx = min(max(int(np.floor(x)) // 16, 0), tw - 1)'),
    ('layout_w2_w3_swapped',
     'SHAPES = [("W1", (C, 1, 3, 3)), ("b1", (C,)), ("W2", (C, C, 3, 3)), ("b2", (C,)),\n          ("W3", (C, C, 3, 3)), ("b3", (C,)), ("Wh", (C,)), ("bh", (1,))]',
     'SHAPES = [("W1", (C, 1, 3, 3)), ("b1", (C,)), ("W3", (C, C, 3, 3)), ("b2", (C,)),\n          ("W2", (C, C, 3, 3)), ("b3", (C,)), ("Wh", (C,)), ("bh", (1,))]'),
    ('bf16_ties_away',
     'b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000',
     'b = (b + 0x8000) & 0xFFFF0000'),
    ('bf16_truncate',
     'b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000',
     'b = b & 0xFFFF0000'),
]

# ---- slips of the SCFV oracle
SCFV_SLIPS = [
    ('bits_ge',
     'if g_mu[i, k] > 0:',
     'if g_mu[i, k] >= 0:'),
    ('bits_reversed',
     'word |= 1 << k',
     'word |= 1 << (31 - k)'),
    ('pca_plus_mean',
     '(np.asarray(X, np.float64) - np.asarray(mean, np.float64))',
     '(np.asarray(X, np.float64) + np.asarray(mean, np.float64))'),
    ('logjoint_no_logw',
     'l[:, i] = math.log(w[i]) - 0.5',
     'l[:, i] = 0.0 - 0.5'),
    ('logjoint_no_norm',
     '+ np.log(2 * math.pi * var[i]).sum())',
     '+ 0.0)'),
    ('gmu_w_not_sqrt',
     '/ (K * math.sqrt(w[i]))',
     '/ (K * w[i])'),
    ('gsig_no_sqrt2',
     '/ (K * math.sqrt(2.0 * w[i]))',
     '/ (K * math.sqrt(w[i]))'),
    ('gsig_minus_half',
     '(d * d - 1.0)',
     '(d * d - 0.5)'),
    ('d_over_var',
     'd = (Y - means[i]) / sd[i]',
     'd = (Y - means[i]) / var[i]'),
    ('delta_no_center',
     '((g_mu - g_mu.mean(axis=1, keepdims=True)) ** 2)',
     '(g_mu ** 2)'),
    ('ranking_ties_high',
     'key=lambda i: (-delta[i], i)',
     'key=lambda i: (-delta[i], -i)'),
    ('ranking_ascending',
     'key=lambda i: (-delta[i], i)',
     'key=lambda i: (delta[i], i)'),
]

# ---- slips of the S0 resize oracle
RESIZE_SLIPS = [
    ('round_half_up',
     'if 2 * r > den or (2 * r == den and q % 2 == 1):',
     'if 2 * r >= den:'),
    ('round_floor',
     '    if 2 * r > den or (2 * r == den and q % 2 == 1):\n        q += 1\n',
     ''),
    ('size_floor',
     'return max_side, max(1, round_half_even_div(height * max_side, width))',
     'return max_side, max(1, (height * max_side) // width)'),
    ('size_swap',
     'return max(1, round_half_even_div(width * max_side, height)), max_side',
     'return max_side, max(1, round_half_even_div(width * max_side, height))'),
    ('ge_to_gt',
     'if width >= height:',
     'if width > height:'),
    ('xs_off_by_one',
     'xs = range((x2 * W) // W2, min(-(-((x2 + 1) * W) // W2), W))',
     'xs = range((x2 * W) // W2, min(-(-((x2 + 1) * W) // W2), W - 1))'),
    ('overlap_swapped',
     'return max(0, min((o + 1) * n_in, (i + 1) * n_out) - max(o * n_in, i * n_out))',
     'return max(0, min((o + 1) * n_out, (i + 1) * n_in) - max(o * n_out, i * n_in))'),
    ('no_resize_equal',
     'if max_side <= 0 or max(width, height) <= max_side:',
     'if max_side <= 0 or max(width, height) < max_side:'),
]


# ---- slips of the parity gate (tests/parity.py), checked by tests/test_parity_helpers.py
PARITY_SLIPS = [
    ('window_1px',
     '(np.abs(bx - ax[i]) < 0.5) & (np.abs(by - ay[i]) < 0.5)',
     '(np.abs(bx - ax[i]) < 1.0) & (np.abs(by - ay[i]) < 1.0)'),
    ('dlog_wide',
     '(np.abs(np.log(bsg / asg[i])) < 0.01)',
     '(np.abs(np.log(bsg / asg[i])) < 0.1)'),
    ('no_octave_test',
     '(b["octave"] == a["octave"][i]) & ',
     ''),
    ('dup_record_margin',
     'bad += 1  # a duplicate of oracle records already paired',
     'margin += 1  # a duplicate of oracle records already paired'),
    ('dup_points_ignored',
     '(extra & ~extra_margin).sum() + dup.sum())',
     '(extra & ~extra_margin).sum())'),
    ('extra_always_margin',
     'extra_margin = extra & g_in_loose',
     'extra_margin = extra'),
    ('miss_margin_or',
     'miss_margin = miss & ~(e_in_loose & e_in_strict)',
     'miss_margin = miss & ~(e_in_loose | e_in_strict)'),
    ('theta_tol_10x',
     'if ang(ek["theta"][j], gk["theta"][i]) <= THETA_TOL and rel_l2(gd[i], ed[j]) <= DESC_TOL])',
     'if ang(ek["theta"][j], gk["theta"][i]) <= 10 * THETA_TOL and rel_l2(gd[i], ed[j]) <= DESC_TOL])'),
    ('desc_tol_10x',
     'if ang(ek["theta"][j], gk["theta"][i]) <= THETA_TOL and rel_l2(gd[i], ed[j]) <= DESC_TOL])',
     'if ang(ek["theta"][j], gk["theta"][i]) <= THETA_TOL and rel_l2(gd[i], ed[j]) <= 10 * DESC_TOL])'),
    ('ang_no_wrap',
     'return min(d, 2 * np.pi - d)',
     'return d'),
    ('greedy_matching',
     'if k not in seen_left:',
     'if False:'),
    ('perturbed_runs_ignored',
     '                hit = True\n',
     '                hit = False\n'),
    ('at_point_ignored',
     'if not hit and at_point is not None:',
     'if False:'),
]

def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("oracles", nargs="*", help="c, proposal, scfv, resize and/or parity (default: all five)")
    ap.add_argument("--only", nargs="*", default=None, help="slip names to run (default: all)")
    args = ap.parse_args()
    args.oracles = args.oracles or ["c", "proposal", "scfv", "resize", "parity"]
    for o in args.oracles:
        if o not in ("c", "proposal", "scfv", "resize", "parity"):
            ap.error(f"unknown oracle {o!r}")

    def pick(slips):
        return [s for s in slips if args.only is None or s[0] in args.only]

    unexpected = []
    with tempfile.TemporaryDirectory(prefix="slips_") as tmpd:
        for oracle in args.oracles:
            if oracle == "c":
                runs = check_c(pick(C_SLIPS), tmpd)
            elif oracle == "proposal":
                runs = check_py("oracle.proposal_oracle", "tests/test_proposal_oracle.py", pick(PROPOSAL_SLIPS), tmpd,
                                os.path.join(ROOT, "oracle", "proposal_oracle.py"))
            elif oracle == "scfv":
                runs = check_py("oracle.scfv_oracle", "tests/test_scfv_oracle.py", pick(SCFV_SLIPS), tmpd,
                                os.path.join(ROOT, "oracle", "scfv_oracle.py"))
            elif oracle == "resize":
                runs = check_py("oracle.resize_oracle", "tests/test_resize_oracle.py", pick(RESIZE_SLIPS), tmpd,
                                os.path.join(ROOT, "oracle", "resize_oracle.py"))
            else:
                runs = check_py("parity", "tests/test_parity_helpers.py", pick(PARITY_SLIPS), tmpd,
                                os.path.join(ROOT, "tests", "parity.py"))
            for name, caught in runs:
                expected = (oracle, name) in EXPECTED_SURVIVORS
                tag = "CAUGHT" if caught else ("SURVIVED (expected)" if expected else "SURVIVED")
                print(f"{oracle:9s} {name:22s} {tag}", flush=True)
                if not caught and not expected:
                    unexpected.append(f"{oracle}/{name}")
    if unexpected:
        print("unexpected survivors:", " ".join(unexpected))
        sys.exit(1)


if __name__ == "__main__":
    main()
