"""Planted mistakes in a copy of oracle.c must each fail at least one pin.

Every mutant is a plausible slip (a dropped term, a wrong sign or index, a
transposed operand, truncation instead of floor). The copy is compiled to a
temporary library on the CPU and the pins of tests/oracle_pins.py are run
against it; a mutant that passes every pin would mean the pins leave that
part of the oracle unchecked.
"""
import os

import pytest

import oracle
from tests import oracle_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = [
    ("drop_weight", "double w = f * f;", "double w = 1.0;"),
    ("weight_f_not_f2", "double w = f * f;", "double w = f;"),
    ("truncate_not_floor", "double fx = floor(x), fy = floor(y);\n    long n = (long)fx, m = (long)fy;\n    double a = x - fx, b = y - fy;\n    double s0",
     "double fx = (double)(long)x, fy = (double)(long)y;\n    long n = (long)fx, m = (long)fy;\n    double a = x - fx, b = y - fy;\n    double s0"),
    ("mix_swapped", "return x * (1.0 - a) + y * a;", "return x * a + y * (1.0 - a);"),
    ("taps_transposed", "double s0 = mix(tap(img, nu, nv, m, n), tap(img, nu, nv, m, n + 1), a);",
     "double s0 = mix(tap(img, nu, nv, m, n), tap(img, nu, nv, m + 1, n), a);"),
    ("eu_sign", "double r0[4] = {-sn * mu + cu * r2[0], c * mu + cu * r2[1], 0.0, cu};",
     "double r0[4] = {sn * mu + cu * r2[0], c * mu + cu * r2[1], 0.0, cu};"),
    ("centre_half_pixel", "const double cu = 0.5 * (nu - 1) + u_off;\n    const double cv = 0.5 * (nv - 1) + v_off;\n    const double x0",
     "const double cu = 0.5 * nu + u_off;\n    const double cv = 0.5 * (nv - 1) + v_off;\n    const double x0"),
    ("depth_sign", "double r2[4] = {-c / sid, -sn / sid, 0.0, 1.0};", "double r2[4] = {c / sid, sn / sid, 0.0, 1.0};"),
    ("voxel_origin", "const double z0 = oz - 0.5 * (nz - 1) * sz;", "const double z0 = oz - 0.5 * nz * sz;"),
    ("bp_skip_last_view", "vol[((long)k * ny + j) * nx + i] += val * w;", "if (s + 1 < np) vol[((long)k * ny + j) * nx + i] += val * w;"),
    ("fp_weights_swapped", "double ww[4] = {(1 - a) * (1 - b), a * (1 - b), (1 - a) * b, a * b};",
     "double ww[4] = {(1 - a) * (1 - b), (1 - a) * b, a * (1 - b), a * b};"),
    ("fp_missing_weight", "double val = vol[((long)k * ny + j) * nx + i] * f * f * scale;",
     "double val = vol[((long)k * ny + j) * nx + i] * f * scale;"),
    ("ramlak_odd_sign", "else v = -1.0 / (M_PI * M_PI", "else v = 1.0 / (M_PI * M_PI"),
    ("ramlak_even_terms", "else if (n % 2 == 0) v = 0.0;", "else if (n % 2 == 0) v = -0.5 / (M_PI * M_PI * (double)n * (double)n * dp * dp);"),
    ("filter_no_cosine", "g[m] = src[m] * sdd / sqrt(sdd * sdd + um * um + vm * vm);", "g[m] = src[m];"),
    ("filter_no_dp", "dst[n] = dp * acc;", "dst[n] = acc;"),
    ("filter_pitch_not_scaled", "const double dp = du * sid / sdd;", "const double dp = du;"),
    ("phantom_rotation_transposed",
     "pb[a] = (R[0 * 3 + a] * p[0] + R[1 * 3 + a] * p[1] + R[2 * 3 + a] * p[2]) / E[3 + a];\n                    db[a] = (R[0 * 3 + a] * dir[0] + R[1 * 3 + a] * dir[1] + R[2 * 3 + a] * dir[2]) / E[3 + a];",
     "pb[a] = (R[a * 3 + 0] * p[0] + R[a * 3 + 1] * p[1] + R[a * 3 + 2] * p[2]) / E[3 + a];\n                    db[a] = (R[a * 3 + 0] * dir[0] + R[a * 3 + 1] * dir[1] + R[a * 3 + 2] * dir[2]) / E[3 + a];"),
    ("conv_tap_sign", "int zi = z + t / 9 - 1, yi = yy + (t / 3) % 3 - 1, xi = xx + t % 3 - 1;\n                            if (zi < 0 || zi >= D || yi < 0 || yi >= H || xi < 0 || xi >= W) continue;\n                            const double *xp",
     "int zi = z - t / 9 + 1, yi = yy + (t / 3) % 3 - 1, xi = xx + t % 3 - 1;\n                            if (zi < 0 || zi >= D || yi < 0 || yi >= H || xi < 0 || xi >= W) continue;\n                            const double *xp"),
    ("conv_no_bias", "double acc = b ? b[co] : 0.0;", "double acc = 0.0;"),
    ("conv_dgrad_transposed_w", "acc += w[((long)co * 27 + t) * cin + ci] * gp[co];", "acc += w[((long)co * 27 + (26 - t)) * cin + ci] * gp[co];"),
    ("conv_wgrad_bias_sum", "for (long v = 0; v < (long)N * D * H * W; ++v) bsum += dy[v * cout + co];", "for (long v = 1; v < (long)N * D * H * W; ++v) bsum += dy[v * cout + co];"),
    ("phantom_chord_half", "if (disc > 0.0) sum += E[15] * sqrt(disc) / A * L;", "if (disc > 0.0) sum += E[15] * sqrt(disc) / (2.0 * A) * L;"),
    ("mlem_no_sensitivity", "if (sens[j] > eps) x[j] = x[j] * b[j] / sens[j];", "if (sens[j] > eps) x[j] = x[j] * b[j];"),
    ("mlem_ratio_inverted", "y[i] = (y[i] > eps) ? pt[i] / y[i] : 0.0;", "y[i] = (y[i] > eps) ? y[i] / pt[i] : 0.0;"),
    ("sart_no_ray_norm", "(pt[i] - y[i]) / ray[i] : 0.0;", "(pt[i] - y[i]) : 0.0;"),
    ("slab_slice_offset", "const int k = k0 + kk;", "const int k = kk;"),
    ("slab_weight_f", "bilinear(im, nu, nv, x, y) * f * f;", "bilinear(im, nu, nv, x, y) * f;"),
    ("points_no_scale", "out[t] = acc * scale;", "out[t] = acc;"),
    ("points_ij_swapped", "double i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];",
     "double j = ijk[3 * t], i = ijk[3 * t + 1], k = ijk[3 * t + 2];"),
    ("sart_sign", "if (sens[j] > eps) x[j] += lambda * b[j] / sens[j];", "if (sens[j] > eps) x[j] -= lambda * b[j] / sens[j];"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mpath = tmp_path / f"{name}.c"
    mpath.write_text(src.replace(old, new))
    so = oracle.compile_source(str(mpath), str(tmp_path / f"lib{name}.so"))
    failed = []
    with oracle.using(so):
        for pin in oracle_pins.ALL:
            try:
                pin()
            except AssertionError:
                failed.append(pin.__name__)
                break
    assert failed, f"mutant {name} passed every pin"
