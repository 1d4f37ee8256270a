"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake (a flipped sign, a swapped index, a dropped term, a
transposed operand, a wrong rounding or comparison) in a copy of the oracle source,
compiles it, and runs the pin suite against the broken build in a fresh process: the
suite must fail.  The planted mistakes live only in temporary copies, on the CPU."""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "psf_oracle.cpp")
PINS = ["tests/test_oracle_keys.py", "tests/test_oracle_accumulate.py", "tests/test_oracle_cv.py",
        "tests/test_oracle_levels.py", "tests/test_oracle_progressive.py", "tests/test_oracle_sh.py"]
INSERT_SCALE = ("uint32_t oracle_insert(void* h, const float* verts, uint64_t n) {\n    Oracle* o = static_cast<Oracle*>(h);\n"
                "    const Config& c = o->cfg;\n    const double scale = std::ldexp(1.0, static_cast<int>(c.frac_bits));")
PROG = "value[3 * idx + ch] = field == 0 ? Le + t[ch] * C_next[ch] : t[ch] * (Le_next[ch] + C_next[ch]);"

MUTANTS = {
    "cv_sign_of_control": ("L - c.beta * (t[ch] * C_next[ch]) + c.beta * C[ch]",
                           "L + c.beta * (t[ch] * C_next[ch]) + c.beta * C[ch]"),
    "cv_swapped_vertices": ("L - c.beta * (t[ch] * C_next[ch]) + c.beta * C[ch]",
                            "L - c.beta * (t[ch] * C[ch]) + c.beta * C_next[ch]"),
    "cv_dropped_integral": ("L - c.beta * (t[ch] * C_next[ch]) + c.beta * C[ch]",
                            "L - c.beta * (t[ch] * C_next[ch])"),
    "cv_last_vertex": ("const bool cv = (j + 1 < static_cast<int64_t>(D))", "const bool cv = (j < static_cast<int64_t>(D))"),
    "biased_range_inclusive": ("(static_cast<uint64_t>(j) < j_end)", "(static_cast<uint64_t>(j) <= j_end)"),
    "alpha_transposed": ("std::sqrt(cn / (co + cn))", "std::sqrt(co / (co + cn))"),
    "alpha_no_sqrt": ("std::sqrt(cn / (co + cn))", "(cn / (co + cn))"),
    "alpha_min_not_max": ("std::max(std::sqrt(cn / (co + cn)), c.alpha_min)",
                          "std::min(std::sqrt(cn / (co + cn)), c.alpha_min)"),
    "blend_weights_swapped": ("(1.0 - alpha) * cell.L[ch] + alpha * mean", "alpha * cell.L[ch] + (1.0 - alpha) * mean"),
    "c_old_not_cumulative": ("cell.c_old = sat_add(cell.c_old, cell.c_new);", "cell.c_old = cell.c_new;"),
    "untouched_cells_blended": ("if (cell.c_new == 0) continue;", "if (cell.c_new < 0) continue;"),
    "octahedral_fold_swapped": ("float fu = 1.0f - std::fabs(v);", "float fu = 1.0f - std::fabs(u);"),
    "no_lower_hemisphere_fold": ("if (wz < 0.0f) {", "if (wz < -2.0f) {"),
    "direction_not_reversed": ("direction_bins(-d[0], -d[1], -d[2]", "direction_bins(d[0], d[1], d[2]"),
    "cell_index_truncates": ("std::floor(static_cast<double>(p) *", "std::trunc(static_cast<double>(p) *"),
    "normal_tie_break": ("if (ax >= ay && ax >= az)", "if (ax > ay && ax >= az)"),
    "fixed_point_truncates": ("std::llrint(static_cast<double>(prod[ch]) * scale)",
                              "static_cast<int64_t>(static_cast<double>(prod[ch]) * scale)"),
    "range_bound_exclusive": ("std::fabs(prod[ch]) <= 32768.0f", "std::fabs(prod[ch]) < 32768.0f"),
    "packed_axes_swapped": ("(bx << 32) | (by << 16) | bz", "(bz << 32) | (by << 16) | bx"),
    "biased_gamma_on_approximant": ("gamma * (L - t[ch] * C_next[ch]) + C[ch]", "(L - t[ch] * C_next[ch]) + gamma * C[ch]"),
    "biased_corrector_sign": ("gamma * (L - t[ch] * C_next[ch]) + C[ch]", "gamma * (L + t[ch] * C_next[ch]) + C[ch]"),
    "level_read_one_deeper": ("return static_cast<uint32_t>(j < top ? j : top);",
                              "return static_cast<uint32_t>(j + 1 < top ? j + 1 : top);"),
    "level_coarse_truncates": ("std::floor(static_cast<double>(x) * std::ldexp(1.0, q))",
                               "std::trunc(static_cast<double>(x) * std::ldexp(1.0, q))"),
    "level_coarse_finer": ("static_cast<int>(c.pos_bits_q) - static_cast<int>(level)",
                           "static_cast<int>(c.pos_bits_q) + static_cast<int>(level)"),
    "level_bits_dropped": ("*key = CellKey(level, nb,", "*key = CellKey(0u, nb,"),
    "insert_level_zero_only": ("l < level_count(c); ++l) {  // every level's cell receives the vertex",
                               "l < 1; ++l) {  // every level's cell receives the vertex"),
    "fixed_point_ignores_frac_bits": (INSERT_SCALE, INSERT_SCALE.replace("static_cast<int>(c.frac_bits)", "24")),
    "cell_index_upper_edge_excluded": ("if (t < -32768.0 || t > 32767.0) return false;",
                                       "if (t < -32768.0 || t >= 32767.0) return false;"),
    "progressive_weight_bound_exclusive": ("(w <= 32768.0)", "(w < 32768.0)"),
    "reset_also_clears_the_approximant": ("for (auto& kv : o->cells) kv.second.c_old = 0;",
                                          "for (auto& kv : o->cells) { kv.second.c_old = 0; kv.second.L[0] = 0.0; }"),
    "counter_does_not_saturate": ("if (a > INT64_MAX - b) return INT64_MAX;", "if (a < 0) return INT64_MAX;"),
    "zero_weight_vertex_inserted": ("const int64_t cw = std::llrint(static_cast<double>(w) * scale);\n        if (cw == 0) {",
                                    "const int64_t cw = std::llrint(static_cast<double>(w) * scale);\n        if (cw < 0) {"),
    "progressive_alg1_without_emission": (PROG, PROG.replace("? Le + t[ch] * C_next[ch]", "? t[ch] * C_next[ch]")),
    "progressive_alg1_own_cell": (PROG, PROG.replace("? Le + t[ch] * C_next[ch]", "? Le + t[ch] * C[ch]")),
    "progressive_alg1_without_throughput": (PROG, PROG.replace("? Le + t[ch] * C_next[ch]", "? Le + C_next[ch]")),
    "progressive_alg2_own_emission": (PROG, PROG.replace("(Le_next[ch] + C_next[ch])", "(Le + C_next[ch])")),
    "sh_centering_sign": ('static_cast<i128>(W) * snn[idx[j][k]] - static_cast<i128>(sn[j]) * sn[k]',
                         'static_cast<i128>(W) * snn[idx[j][k]] + static_cast<i128>(sn[j]) * sn[k]'),
    "sh_cross_term_uses_chroma": ('static_cast<i128>(W) * sYn[j] - static_cast<i128>(c.s[0]) * sn[j]',
                                 'static_cast<i128>(W) * sYn[j] - static_cast<i128>(c.s[1]) * sn[j]'),
    "sh_ridge_not_scaled_by_weight": ('m[j][j] += ridge * Wd * Wd;',
                                     'm[j][j] += ridge * Wd;'),
    "sh_intercept_without_gradient": ('(static_cast<double>(c.s[0]) - (g[0] * sn[0] + g[1] * sn[1] + g[2] * sn[2])) / Wd',
                                     'static_cast<double>(c.s[0]) / Wd'),
    "sh_chroma_swapped": ('out[4] = static_cast<double>(c.s[1]) / Wd;\n    out[5] = static_cast<double>(c.s[2]) / Wd;',
                         'out[4] = static_cast<double>(c.s[2]) / Wd;\n    out[5] = static_cast<double>(c.s[1]) / Wd;'),
    "sh_inverse_blue_sign": ('out[2] = Y - coef[4] - coef[5];',
                            'out[2] = Y - coef[4] + coef[5];'),
    "sh_luminance_weights": ('float wY = 0.25f * p[0] + 0.5f * p[1];',
                            'float wY = 0.5f * p[0] + 0.25f * p[1];'),
    "sh_moment_index_transposed": ('{{0, 1, 2}, {1, 3, 4}, {2, 4, 5}}',
                                  '{{0, 1, 2}, {1, 3, 5}, {2, 5, 4}}'),
    "sh_lookup_at_direction": ('sh_rgb(it->second.coef, verts + 16 * i + 4, C);',
                              'sh_rgb(it->second.coef, verts + 16 * i + 8, C);'),
    "sh_band1_not_blended": ('for (int k = 0; k < 6; ++k) cell.coef[k] = (1.0 - alpha) * cell.coef[k] + alpha * fit[k];',
                            'for (int k = 0; k < 6; ++k) cell.coef[k] = (k >= 1 && k <= 3) ? fit[k] : (1.0 - alpha) * cell.coef[k] + alpha * fit[k];'),
    "sh_luminance_moment_uses_weight": ('fx(wY * nr[0]), fx(wY * nr[1]), fx(wY * nr[2]),',
                                       'fx(m[0]), fx(m[1]), fx(m[2]),'),
    "sh_normal_bound_exclusive": ('ok = std::fabs(nr[k]) <= 1.0009765625f;',
                                 'ok = std::fabs(nr[k]) < 1.0009765625f;'),
    "sh_cv_sign_of_control": ('(L - c.beta * (t[ch] * C[3 * (idx + P) + ch]) + c.beta * C[3 * idx + ch])',
                             '(L + c.beta * (t[ch] * C[3 * (idx + P) + ch]) + c.beta * C[3 * idx + ch])'),
    "progressive_value_not_saturated": ("prod[ch] = std::min(std::max(prod[ch], -32768.0), 32768.0);",
                                        "(void)prod[ch];"),
    "progressive_record_rule_missing": ("ok = std::isfinite(own) && std::fabs(own) <= 32768.0f && std::isfinite(v[ch == 0 ? 7 : ch == 1 ? 11 : 15]);",
                                        "ok = std::isfinite(own) || true;"),
    "sums_saturate_instead_of_wrapping": ("return static_cast<int64_t>(static_cast<uint64_t>(a) + static_cast<uint64_t>(b));",
                                          "return (b > 0 && a > INT64_MAX - b) ? INT64_MAX : (b < 0 && a < INT64_MIN - b) ? INT64_MIN : a + b;"),
    "sum_range_count_off_by_one": ("return *iter_vertices >= (uint64_t{1} << (48u - frac_bits - extra_bits)) ? ST_SUM_RANGE : 0u;",
                                   "return *iter_vertices > (uint64_t{1} << (48u - frac_bits - extra_bits)) ? ST_SUM_RANGE : 0u;"),
    "progressive_alg2_without_throughput": (PROG, PROG.replace("t[ch] * (Le_next[ch] + C_next[ch])",
                                                               "(Le_next[ch] + C_next[ch])")),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutant = tmp_path / "mutant.cpp"
    mutant.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", str(mutant), "-o", str(so)],
                   check=True)
    env = dict(os.environ, PSF_ORACLE_LIB=str(so))
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS], cwd=ROOT,
                         env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, f"the pins did not catch the planted mistake '{name}'"


def test_unmodified_copy_passes(tmp_path):
    """Control: the same mechanism with no mistake planted passes the pins."""
    so = tmp_path / "libcopy.so"
    subprocess.run(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", str(so)], check=True)
    env = dict(os.environ, PSF_ORACLE_LIB=str(so))
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS], cwd=ROOT,
                         env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout[-2000:]
