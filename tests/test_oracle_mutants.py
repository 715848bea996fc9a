"""Planted mistakes in the oracle: each case edits one expression of a copy
of ``oracle/oracle.c`` (or of ``oracle/mlp.py``) into a plausible error (a
dropped term, a wrong sign, power or index, a formula as the paper prints it
where the reading corrects it, a step of the procedure applied to the wrong
state), builds that copy into a library of its own (or imports it in place of
mlp.py) and runs one of the oracle's pin files against it in a child process.
Every such mistake must make a pin fail: the pins are not just the oracle's
formulas typed again. A control case runs unedited copies the same way, and
they must pass. The oracle's own files are never touched. CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# oracle.c: (name, pin file that must fail: tests/test_oracle_<file>.py,
# original text, planted text)
MUTANTS = [
    ('whole_restarts_from_kicked_v', 'whole',
     'memcpy(v, vpre, b3);',
     'memcpy(v, v0, b3);'),
    ('whole_keeps_second_kick', 'whole',
     'if (!whole) or_kick(rows, m, q, v, G, 0.5 * tau);',
     'or_kick(rows, m, q, v, G, 0.5 * tau);'),
    ('whole_one_planet_enough', 'whole',
     'if (np >= 2) return 1;',
     'if (np >= 1) return 1;'),
    ('whole_keeps_transition', 'whole',
     'G, INFINITY, p->eps_H, p->eta,',
     'G, rcrit[0], p->eps_H, p->eta,'),
    ('stumpff_series_factorial', 'kepler',
     'term_s *= -y / ((2.0 * k + 4.0) * (2.0 * k + 5.0));',
     'term_s *= -y / ((2.0 * k + 4.0) * (2.0 * k + 6.0));'),
    ('stumpff_S_closed_power', 'kepler',
     '*S = (sy - sin(sy)) / (sy * sy * sy);',
     '*S = (sy - sin(sy)) / (sy * sy);'),
    ('stumpff_hyperbolic_sign', 'kepler',
     '*C = (cosh(sy) - 1.0) / (-y);',
     '*C = (cosh(sy) - 1.0) / y;'),
    ('kepler_F_drops_sigma_term', 'kepler',
     '*F = -sqmu * dt + sig * x * x * C + b * x * x * x * S + r0 * x;',
     '*F = -sqmu * dt + b * x * x * x * S + r0 * x;'),
    ('kepler_Fpp_wrong', 'kepler',
     '*Fpp = sig * (1.0 - y * C) + b * x * (1.0 - y * S);',
     '*Fpp = sig * (1.0 - y * S) + b * x * (1.0 - y * S);'),
    ('fdot_as_printed', 'kepler',
     'double fdot = sqmu * x * (y * S - 1.0) / (r * r0);',
     'double fdot = sqmu * x * (y * x * S - 1.0) / (r * r0);'),
    ('gdot_uses_r0', 'kepler',
     'double gdot = 1.0 - x * x / r * C;',
     'double gdot = 1.0 - x * x / r0 * C;'),
    ('laguerre_n4', 'kepler',
     'const double n = 5.0;',
     'const double n = 4.0;'),
    ('mu_includes_body_mass', 'step',
     'const double G = p->G, m0 = m[0], mu = G * m0;',
     'const double G = p->G, m0 = m[0], mu = G * (m0 + m[1]);'),
    ('drift_not_over_m0', 'step',
     'q[3 * i + k] += dt * S[k] / m[0];',
     'q[3 * i + k] += dt * S[k];'),
    ('force_sign', 'forces',
     'for (int k = 0; k < 3; ++k) a[k] -= w * d[k];',
     'for (int k = 0; k < 3; ++k) a[k] += w * d[k];'),
    ('force_inverse_square_weight', 'forces',
     'double w = G * m[j] / (r2 * r);',
     'double w = G * m[j] / r2;'),
    ('force_uses_own_mass', 'forces',
     'double w = G * m[j] / (r2 * r);',
     'double w = G * m[i] / (r2 * r);'),
    ('energy_drops_dft_term', 'forces',
     'double E = dot3(S, S) / (2.0 * m[0]);',
     'double E = 0.0;'),
    ('energy_pair_inverse_square', 'forces',
     'row += m[j] / sqrt(dot3(d, d));',
     'row += m[j] / dot3(d, d);'),
    ('helio_to_dh_over_m0', 'forces',
     'for (int k = 0; k < 3; ++k) v[3 * i + k] -= s[k] / mt;',
     'for (int k = 0; k < 3; ++k) v[3 * i + k] -= s[k] / m[0];'),
    ('dh_to_helio_sign', 'forces',
     'for (int k = 0; k < 3; ++k) v[3 * i + k] += S[k] / m[0];',
     'for (int k = 0; k < 3; ++k) v[3 * i + k] -= S[k] / m[0];'),
    ('hill_missing_three', 'encounters',
     'rH[i] = r * cbrt(m[i] / (3.0 * m[0]));',
     'rH[i] = r * cbrt(m[i] / m[0]);'),
    ('dmin_cubic_c2', 'encounters',
     'double c2 = 3.0 * (d1 - d0) - 2.0 * s0 - s1;',
     'double c2 = 3.0 * (d1 - d0) - s0 - s1;'),
    ('dmin_slope_no_tau', 'encounters',
     'double s1 = 2.0 * dot3(dq1, dv1) * tau;',
     'double s1 = 2.0 * dot3(dq1, dv1);'),
    ('encounter_radius_single', 'encounters',
     'double R = a_E * (rH[i] + rH[j]);',
     'double R = a_E * rH[i];'),
    ('rcrit_drops_aH', 'encounters',
     'rcrit[s] = a_H * mx;',
     'rcrit[s] = mx;'),
    ('transition_argument', 'encounters',
     'double y = 1.1 * s / rcrit - 0.1;',
     'double y = s / rcrit;'),
    ('transition_Kp_chain', 'encounters',
     '*Kp = 0.5 * OR_PI * c * cos(ph);',
     '*Kp = 0.5 * OR_PI * cos(ph);'),
    ('transition_Kpp_sign', 'encounters',
     '*Kpp = -(0.5 * OR_PI * c) * (0.5 * OR_PI * c) * sin(ph);',
     '*Kpp = (0.5 * OR_PI * c) * (0.5 * OR_PI * c) * sin(ph);'),
    ('kcorr_drops_Kp', 'encounters',
     'double w = -G * m[j] / (r * r * r) * (1.0 - K + r * Kp);',
     'double w = -G * m[j] / (r * r * r) * (1.0 - K);'),
    ('hermite_jerk_drops_Kpp', 'encounters',
     'ji[c] += w * (rv * d[c] * Kpp + (dv[c] - 3.0 * rv * d[c] / s2) * br);',
     'ji[c] += w * ((dv[c] - 3.0 * rv * d[c] / s2) * br);'),
    ('hermite_star_jerk_power', 'encounters',
     'ji[c] += w * (u[3 * i + c] - 3.0 * rv * x[3 * i + c] / s2);',
     'ji[c] += w * (u[3 * i + c] - 3.0 * rv * x[3 * i + c] / s);'),
    ('hermite_predictor_jerk', 'encounters',
     'xp[id] = x[id] + h * (u[id] + h * (0.5 * a0[id] + h * j0[id] / 6.0));',
     'xp[id] = x[id] + h * (u[id] + h * (0.5 * a0[id] + h * j0[id] / 2.0));'),
    ('hermite_a3_sign', 'encounters',
     'a3[c] = (12.0 * (a0[id] - a1[id]) + 6.0 * h * (j0[id] + j1[id])) / (h * h * h);',
     'a3[c] = (12.0 * (a0[id] - a1[id]) + 6.0 * h * (j0[id] - j1[id])) / (h * h * h);'),
    ('hermite_corrector_v', 'encounters',
     'u[id] = up[id] + h * h * h * (a2[c] / 6.0 + h * a3[c] / 24.0);',
     'u[id] = up[id] + h * h * h * (a2[c] / 6.0);'),
    ('aarseth_no_sqrt', 'encounters',
     'return sqrt(eta * (na * n2 + nj * nj) / den);',
     'return eta * (na * n2 + nj * nj) / den;'),
    ('step_kcorr_full_tau', 'step',
     'or_kcorr(k, members + k0, m, q0, v0, G, rcrit[st], 0.5 * tau);',
     'or_kcorr(k, members + k0, m, q0, v0, G, rcrit[st], tau);'),
    ('step_second_kick_missing', 'step',
     'if (!whole) or_kick(rows, m, q, v, G, 0.5 * tau);',
     'if (!whole) (void)0;'),
    ('step_hermite_from_kepler_state', 'step',
     'q[3 * i + c] = q0[3 * i + c];\n                            v[3 * i + c] = v0[3 * i + c];',
     '(void)0;'),
    ('step_hill_from_end_state', 'step',
     'or_hill_radii(rows, m, q0, v0, G, rH);',
     'or_hill_radii(rows, m, q, v, G, rH);'),
    ('uf_root_not_smallest', 'encounters',
     'if (a < b) parent[b] = a; else parent[a] = b;   /* root = smallest index */',
     'parent[a] = b;'),
    ('sets_member_order', 'encounters',
     'members[set_start[s] + fill[s]++] = i;',
     'members[set_start[s + 1] - 1 - fill[s]++] = i;'),
    ('rcrit_min_not_max', 'encounters',
     'if (rH[members[k]] > mx) mx = rH[members[k]];',
     'if (mx == 0.0 || rH[members[k]] < mx) mx = rH[members[k]];'),
    ('laguerre_sign_minus', 'kepler',
     'dx = n * rf / (1.0 + sq);',
     'dx = n * rf / (1.0 - sq);'),
    ('residual_tolerance_loose', 'kepler',
     'if (fabs(F) <= 1e-14 * scale) {',
     'if (fabs(F) <= 1e-8 * scale) {'),
    ('bracket_not_widened', 'kepler',
     'double xb = sqmu * dt / rp * (1.0 + 1e-12);',
     'double xb = sqmu * dt / rp * (1.0 - 1e-9);'),
    ('standard_guess_r0_squared', 'kepler',
     'x = sqmu * dt / r0;\n    else if (guess == 1)',
     'x = sqmu * dt / (r0 * r0);\n    else if (guess == 1)'),
    ('kick_double_dt', 'encounters',
     'for (int k = 0; k < 3; ++k) v[3 * i + k] += dt * a[3 * i + k];',
     'for (int k = 0; k < 3; ++k) v[3 * i + k] += 2.0 * dt * a[3 * i + k];'),
    ('first_drift_full_tau', 'step',
     '/* item 1: drift tau/2 */\n        or_drift(rows, m, q, v, 0.5 * tau);',
     '/* item 1: drift tau/2 */\n        or_drift(rows, m, q, v, tau);'),
    ('kcorr_q1_uses_q0', 'step',
     '/* item 7: pre-remove the (1-K) part of the coming kick at q1 */\n                    or_kcorr(k, members + k0, m, q, v, G, rcrit[st], 0.5 * tau);',
     '/* item 7: pre-remove the (1-K) part of the coming kick at q1 */\n                    or_kcorr(k, members + k0, m, q0, v, G, rcrit[st], 0.5 * tau);'),
    ('kcorr_sign', 'encounters',
     'for (int k = 0; k < 3; ++k) v[3 * mem[a] + k] -= dt * dv[3 * a + k];',
     'for (int k = 0; k < 3; ++k) v[3 * mem[a] + k] += dt * dv[3 * a + k];'),
    ('hermite_smoothing_dropped', 'encounters',
     'double s2 = dot3(d, d) + eps * eps;',
     'double s2 = dot3(d, d);'),
    ('hermite_star_mass_body', 'encounters',
     'double w = -G * m0 / (s2 * s);',
     'double w = -G * (m0 + mm[i]) / (s2 * s);'),
    ('hermite_startup_eta', 'encounters',
     'double dt_c = jn > 0.0 ? eta_s * norm3(a0 + 3 * i) / jn : T;',
     'double dt_c = jn > 0.0 ? norm3(a0 + 3 * i) / jn : T;'),
    ('hermite_level_up_any_time', 'encounters',
     'kn = (tn % ((int64_t)1 << (OR_KMAX - up1)) == 0) ? up1 : lev[i];',
     'kn = up1;'),
    ('hermite_a2_j_weights', 'encounters',
     'a2[c] = (-6.0 * (a0[id] - a1[id]) - h * (4.0 * j0[id] + 2.0 * j1[id])) / (h * h);',
     'a2[c] = (-6.0 * (a0[id] - a1[id]) - h * (2.0 * j0[id] + 4.0 * j1[id])) / (h * h);'),
    ('energy_kinetic_no_half', 'forces',
     'E += 0.5 * m[i] * dot3(v + 3 * i, v + 3 * i);',
     'E += m[i] * dot3(v + 3 * i, v + 3 * i);'),
    ('energy_star_term_sign', 'forces',
     'E -= G * m[0] * m[i] / sqrt(dot3(q + 3 * i, q + 3 * i));',
     'E += G * m[0] * m[i] / sqrt(dot3(q + 3 * i, q + 3 * i));'),
    ('dmin_skips_interior_roots', 'encounters',
     'if (u[k] > 0.0 && u[k] < 1.0) {',
     'if (u[k] > 0.0 && u[k] < 0.5) {'),
    ('encounters_strict_upper_only_ij', 'step',
     'for (int64_t j = i + 1; j < rows; ++j) {\n        double dq0[3], dv0[3], dq1[3], dv1[3];\n        pair_diffs(q0, v0, q1, v1, i, j, dq0, dv0, dq1, dv1);\n        double R = a_E * (rH[i] + rH[j]);',
     'for (int64_t j = i + 2; j < rows; ++j) {\n        double dq0[3], dv0[3], dq1[3], dv1[3];\n        pair_diffs(q0, v0, q1, v1, i, j, dq0, dv0, dq1, dv1);\n        double R = a_E * (rH[i] + rH[j]);'),
    ('residual_scale_inflated', 'kepler',
     'res[i] = fabs(F) / scale;',
     'res[i] = fabs(F) / (1e6 * scale);'),
    ('residual_scale_offset', 'kepler',
     'double scale = fabs(sqmu * dt) + fabs(sig * xx * xx * C) +',
     'double scale = 1.0 + fabs(sqmu * dt) + fabs(sig * xx * xx * C) +'),
    ('accel_rows_wrong_row', 'forces',
     'for (int64_t k = 0; k < nsel; ++k) or_accel_row(rows, m, q, G, sel[k], a + 3 * k);',
     'for (int64_t k = 0; k < nsel; ++k) or_accel_row(rows, m, q, G, sel[0], a + 3 * k);'),
    ('accel_row_includes_star', 'forces',
     'for (int64_t j = 1; j < rows; ++j) {\n        if (j == i) continue;',
     'for (int64_t j = 0; j < rows; ++j) {\n        if (j == i) continue;'),
    ('encounters_rows_unordered', 'encounters',
     'int64_t a = i < j ? i : j, b = i < j ? j : i;',
     'int64_t a = i, b = j;'),
    ('encounters_rows_skips_lower', 'encounters',
     'for (int64_t j = 1; j < rows; ++j) {\n            if (j == i) continue;\n            double dq0[3]',
     'for (int64_t j = i + 1; j < rows; ++j) {\n            if (j == i) continue;\n            double dq0[3]'),
    ('guess_mode_ignores_given_x', 'kepler',
     '    else\n        x = x_guess;',
     '    else\n        x = sqmu * dt / r0;'),
    ('fallback_newton_not_laguerre', 'kepler',
     'st = or_kepler_solve_br(sqmu, dt, r0, sig, alpha, 0, max_iter, lo, hi, &x, &it2);',
     'st = or_kepler_solve_br(sqmu, dt, r0, sig, alpha, solver, 2, lo, hi, &x, &it2);'),
    ('iters_not_reported', 'kepler',
     'if (iters_out) iters_out[i] = it;',
     'if (iters_out) iters_out[i] = 0;'),
    ('hermite_ticks_off_by_one', 'encounters',
     'const int64_t TT = (int64_t)1 << OR_KMAX;      /* tau in ticks */',
     'const int64_t TT = ((int64_t)1 << OR_KMAX) - 1;      /* tau in ticks */'),
    ('hermite_backward_sign_ignored', 'encounters',
     'const double T = fabs(tau), sg = tau >= 0.0 ? 1.0 : -1.0;',
     'const double T = fabs(tau), sg = 1.0;'),
    ('hermite_steps_not_counted', 'encounters',
     '        ++steps;\n    }\n    for (int64_t i = 0; i < k; ++i)',
     '    }\n    for (int64_t i = 0; i < k; ++i)'),
    ('hermite_corrects_everyone', 'encounters',
     'if (ti[i] + dti != tn) continue;',
     'if (ti[i] + dti < tn) continue;'),
    ('step_stats_encounters_not_counted', 'step',
     'stats[0] += npairs;',
     'stats[0] += 0;'),
    ('step_records_step_index', 'step',
     'enc[3 * ne_total] = step0 + s;',
     'enc[3 * ne_total] = s;'),
    ('kepler_energy_mu_with_body', 'kepler',
     'double alpha = 2.0 / r0 - v2 / mu;',
     'double alpha = 2.0 / r0 - v2 / (mu * 1.000001);'),
    ('sets_rcrit_from_first_member', 'encounters',
     'for (int64_t k = set_start[s]; k < set_start[s + 1]; ++k)\n            if (rH[members[k]] > mx) mx = rH[members[k]];',
     'mx = rH[members[set_start[s]]];'),
]


# oracle/mlp.py, the learned guess's reference: every one of these must fail a
# pin of tests/test_oracle_mlp.py
MLP_MUTANTS = [
    ("grad_W2_transposed", "gW2, aW2 = dp2in.T @ h1in", "gW2, aW2 = h1in.T @ dp2in"),
    ("gelu_derivative_at_wrong_layer", "dp1 = dh1 * dgelu(p1)", "dp1 = dh1 * dgelu(p2)"),
    ("grad_W1_scaled_input", "gW1, aW1 = dp1.T @ fn", "gW1, aW1 = dp1.T @ (fn * 1.001)"),
    ("grad_b3_from_residual", "gb3, ab3 = np.sum(dy)", "gb3, ab3 = np.sum(r)"),
    ("gelu_derivative_sign", "(1.0 - th * th) * K0", "(1.0 + th * th) * K0"),
    ("feature_u1_scale", "u1 = rv / np.sqrt(mu * r0)", "u1 = rv / np.sqrt(mu / r0)"),
    ("target_scale_inverted", "return (z - 1.0) / sigma(q0, dt, mu)",
     "return (z - 1.0) * sigma(q0, dt, mu)"),
    ("adam_bias_correction_step", "mh = m / (1.0 - b1 ** t)", "mh = m / (1.0 - b1 ** (t + 1))"),
    ("bf16_rounds_ties_up", "u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000",
     "u = (u + 0x7FFF) & 0xFFFF0000"),
]


def _run_pins(pins, env):
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           "-m", "not gpu", os.path.join("tests", f"test_oracle_{pins}.py")],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def _build_copy(tmp_path, name, text):
    c = tmp_path / (name + ".c")
    so = tmp_path / (name + ".so")
    c.write_text(text)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-std=c11", "-o", str(so), str(c), "-lm"])
    return so


def test_unedited_copies_pass_the_pins(tmp_path):
    """The route the planted mistakes take (a library built from a copy, an
    imported copy of mlp.py, a child pytest) passes with nothing planted, so
    a failure in the cases below comes from the planted mistake."""
    so = _build_copy(tmp_path, "unedited", open(SRC).read())
    py = tmp_path / "mlp.py"
    py.write_text(open(os.path.join(ROOT, "oracle", "mlp.py")).read())
    for pins, env in (("kepler", {"QYM_ORACLE_LIB": str(so)}),
                      ("encounters", {"QYM_ORACLE_LIB": str(so)}),
                      ("mlp", {"QYM_ORACLE_MLP": str(py)})):
        r = _run_pins(pins, dict(os.environ, **env))
        assert r.returncode == 0, r.stdout[-2000:]


def _pins_fail(pins, env):
    r = _run_pins(pins, env)
    assert r.returncode == 1, f"no pin failed:\n{r.stdout[-2000:]}"
    assert "FAILED" in r.stdout


@pytest.mark.parametrize("name, pins, old, new", MUTANTS, ids=[x[0] for x in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, name, pins, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, "the text to edit must occur exactly once"
    so = _build_copy(tmp_path, name, src.replace(old, new))
    _pins_fail(pins, dict(os.environ, QYM_ORACLE_LIB=str(so)))


@pytest.mark.parametrize("name, old, new", MLP_MUTANTS, ids=[x[0] for x in MLP_MUTANTS])
def test_planted_mistake_in_guess_reference_fails_a_pin(tmp_path, name, old, new):
    src = open(os.path.join(ROOT, "oracle", "mlp.py")).read()
    assert src.count(old) == 1, "the text to edit must occur exactly once"
    py = tmp_path / "mlp.py"
    py.write_text(src.replace(old, new))
    _pins_fail("mlp", dict(os.environ, QYM_ORACLE_MLP=str(py)))
