"""The pins are sensitive: each plausible mistake planted in a copy of the
oracle (a dropped term, a wrong sign, index or operand, a swapped field) makes
at least one pin test fail.  Mutants are compiled on the CPU into a temporary
directory; the committed oracle is never modified."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "tmd_oracle.c")

MUTANTS = {
    "drop_h2_term_in_c00": ("s->c00 = fmaf(h2, a2, fmaf(dx, a1, a0));", "s->c00 = fmaf(dx, a1, a0);"),
    "rotation_sign": ("float b = s->ty * ca - sa;", "float b = s->ty * ca + sa;"),
    "rotation_transposed": ("float ny = s->y * ca - s->x * sa;", "float ny = s->x * ca - s->y * sa;"),
    "drop_process_noise": ("s->c11 = fmaf(m->qty, adx, fmaf(dx, b2, b1));", "s->c11 = fmaf(dx, b2, b1);"),
    "wrong_gain_operand": ("k1 = s->c01 * inv", "k1 = s->c02 * inv"),
    "no_slope_propagation": ("s->ty = fmaf(s->c, dx, s->ty);", "s->ty = s->ty;"),
    "missing_half": ("float h = (0.5f * s->c) * dx;", "float h = s->c * dx;"),
    "cov_update_index": ("s->c12 = fmaf(-k1, c02, s->c12);", "s->c12 = fmaf(-k1, c01, s->c12);"),
    "time_cov_gain": ("s->d11 = fmaf(-g1, d01, s->d11);", "s->d11 = fmaf(-g0, d01, s->d11);"),
    "rotation_curvature_power": ("s->c = s->c * ((ia * ia) * ia);", "s->c = s->c * (ia * ia);"),
    "no_side_flip": ("if ((s->sec < 18) != (nsec < 18)) {", "if (0) {"),
    "unattached_no_running_sum": ("padq = (padq + f->pad_diff_u[u]) & 0xFFFFu;",
                                  "padq = f->pad_diff_u[u];"),
    "record_sigma_swap": ("dst[6] = sig_time; dst[7] = sig_pad;", "dst[6] = sig_pad; dst[7] = sig_time;"),
    "quant_truncates": ("return (uint32_t)floorf(v + 0.5f);", "return (uint32_t)floorf(v);"),
    "seed_slope_no_curvature": ("s->ty = s->y / s->x + (s->c * s->x) * 0.5f;", "s->ty = s->y / s->x;"),
    "pad_to_y_inverse_width": ("0.015625f, -g_halfnp[r]) * g_w[r];",
                               "0.015625f, -g_halfnp[r]) * g_invw[r];"),
    "unattached_sort_pad_first": ("if (T->time_u[a] != T->time_u[b]) return T->time_u[a] < T->time_u[b] ? -1 : 1;",
                                  "if (T->pad_u[a] != T->pad_u[b]) return T->pad_u[a] < T->pad_u[b] ? -1 : 1;"),
    "time_residual_sign": ("o->time_res[d] = T->time[j] - ptime;", "o->time_res[d] = ptime - T->time[j];"),
    "row_key_mod": ("sec = (sec + f->slice_leg_diff[d] % O_NSEC) % O_NSEC;",
                    "sec = (sec + f->slice_leg_diff[d] / O_NSEC) % O_NSEC;"),
    "xyz_rotation_sign": ("gx[i] = g_x[r] * ca - yl * sa;", "gx[i] = g_x[r] * ca + yl * sa;"),
    "xyz_sector_edge_not_centre": ("const float ca = g_ccen[s % 18], sa = g_scen[s % 18];",
                                   "const float ca = g_cos[s % 18], sa = g_sin[s % 18];"),
    "xyz_drift_speed": ("const float zabs = 250.0f - t * 0.5f;", "const float zabs = 250.0f - t;"),
    "xyz_side_sign": ("gz[i] = s < 18 ? zabs : -zabs;", "gz[i] = zabs;"),
    "rans_drop_cumulative": ("x = (x / fs) * O_R_M + c[p][s] + (x % fs);",
                             "x = (x / fs) * O_R_M + (x % fs);"),
    "rans_renorm_threshold": ("if ((uint64_t)x >= ((uint64_t)fs << 20)) {",
                              "if ((uint64_t)x >= ((uint64_t)fs << 19)) {"),
    "rans_words_not_reversed": ("words[l * (O_R_K * 4 + 1) + q] = stack[ns - 1 - q];",
                                "words[l * (O_R_K * 4 + 1) + q] = stack[q];"),
    "rans_deficit_to_symbol_zero": ("if (sum < O_R_M) f[smax] += (uint32_t)(O_R_M - sum);",
                                    "if (sum < O_R_M) f[0] += (uint32_t)(O_R_M - sum);"),
    "rans_lane_major_words": ("o_put32(out + a_words + 4u * (woff + 32u * j + l), lo | (hi << 16));",
                              "o_put32(out + a_words + 4u * (woff + maxpairs * l + j), lo | (hi << 16));"),
    "rans_high_byte_first": ("v |= s << (8 * p);\n          while (x < O_R_LOWER) {",
                             "v |= s << (8 * (w - 1 - p));\n          while (x < O_R_LOWER) {"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique/found: {old}"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-shared", "-fPIC", "-o", str(so), str(mut), "-lm"])
    env = dict(os.environ, TMD_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_xyz.py"),
                        os.path.join(ROOT, "tests", "test_oracle_rans.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
