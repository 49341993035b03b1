"""The oracle pins catch plausible mistakes: each case plants one in a copy of oracle.c.

Every mutant below is a mistake someone could make when writing the
definitions (a dropped term, a wrong sign, swapped weights, a missing factor)
and none of them can read out of bounds.  The copy is compiled into a
temporary library, the pin tests run against it, and at least one of them
must fail.
"""
import os
import subprocess

import pytest

import oracle
import test_oracle_fir_pins as fir_pins
import test_oracle_grad_pins as grad_pins
import test_oracle_iq_pins as iq_pins
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "pwi_sin_sign": ("x * sin(theta)", "-x * sin(theta)",
                     ["test_pwi_delay_closed_forms"]),
    "pwi_cos_for_sin": ("x * sin(theta) + z * cos(theta)", "x * cos(theta) + z * sin(theta)",
                        ["test_pwi_delay_closed_forms"]),
    "dropped_depth_term": ("sqrt(dx * dx + z * z)", "sqrt(dx * dx)",
                           ["test_stai_delay_closed_forms", "test_delay_under_element_is_two_way_depth"]),
    "stai_rx_twice": ("(or_dist(p, x, z, et) + or_dist(p, x, z, er))",
                      "(2.0 * or_dist(p, x, z, er))", ["test_stai_delay_closed_forms"]),
    "hann_half_missing": ("g * 0.5 * (1.0 + cos(M_PI * u))", "g * (1.0 + cos(M_PI * u))",
                          ["test_hann_closed_forms"]),
    "aperture_width": ("z / (2.0 * p->f_number)", "z / p->f_number", ["test_hann_closed_forms"]),
    "lerp_weights_swapped": ("(1.0 - f) * tr[i] + f * tr[i + 1]",
                             "f * tr[i] + (1.0 - f) * tr[i + 1]",
                             ["test_lerp_integer_half_and_range"]),
    "tx_weight_dropped": ("acc += wt * inner;", "acc += inner;", ["test_das_unit_rf_sums_weights"]),
    "element_offset": ("0.5 * (double)(p->n_elements - 1)", "0.5 * (double)(p->n_elements)",
                       ["test_element_positions_are_centred", "test_das_ramp_equals_delay"]),
    "t_start_sign": ("- t_start * p->fs;\n}\n\n/*\n * PWI", "+ t_start * p->fs;\n}\n\n/*\n * PWI",
                     ["test_stai_delay_closed_forms"]),
    "one_sided_factor": ("else if (2 * k < n) h = 2.0;", "else if (2 * k < n) h = 1.0;",
                         ["test_bin_centred_cosine_has_unit_envelope"]),
    "inverse_scale": ("if (inverse) { ar /= n; ai /= n; }", "", ["test_dft_matches_numpy_fft"]),
    "natural_log": ("20.0 * log10(e / ref)", "20.0 * log(e / ref)", ["test_logclip_closed_forms"]),
    # reverse-mode derivatives
    "adjoint_fraction_swapped": ("grad_rf[base + i] += yp * W * (1.0 - f);",
                                 "grad_rf[base + i] += yp * W * f;",
                                 ["test_adjoint_identity", "test_single_term_by_hand"]),
    "adjoint_wrong_sample": ("grad_rf[base + i + 1] += yp * W * f;",
                             "grad_rf[base + i] += yp * W * f;", ["test_adjoint_identity"]),
    "grad_g_tx_term_dropped": ("if (mode == 0) grad_g[et] += yp * at * gr * ar * v;", "",
                               ["test_weight_gradient_matches_central_difference"]),
    "grad_g_skips_zero_weight": ("if (ar == 0.0) continue;",
                                 "if (ar == 0.0 || (p->elem_weight && p->elem_weight[r] == 0.0)) continue;",
                                 ["test_weight_gradient_matches_central_difference"]),
    "grad_c_sign": ("double dsdc = -(s + t0 * p->fs) / p->c;", "double dsdc = (s + t0 * p->fs) / p->c;",
                    ["test_sound_speed_gradient_matches_central_difference", "test_single_term_by_hand"]),
    "grad_c_t_start_dropped": ("double dsdc = -(s + t0 * p->fs) / p->c;", "double dsdc = -s / p->c;",
                               ["test_sound_speed_gradient_matches_central_difference",
                                "test_single_term_by_hand"]),
    "env_bwd_missing_1_over_n": ("yr[k] *= h / (double)nz;", "yr[k] *= h;",
                                 ["test_envelope_backward_matches_central_difference"]),
    "env_bwd_imag_dropped": ("gi[iz] = m > 0.0 ? g * zi[iz] / m : 0.0;", "gi[iz] = 0.0;",
                             ["test_envelope_backward_matches_central_difference"]),
    "logclip_bwd_natural_log": ("g_env[i] = g_db[i] * 20.0 / (log(10.0) * v);",
                                "g_env[i] = g_db[i] * 20.0 / v;",
                                ["test_logclip_backward_matches_central_difference_including_the_frame_max"]),
    "logclip_bwd_ref_dropped": ("if (ref_is_max && arg >= 0) g_env[arg] += s_ref;", "",
                                ["test_logclip_backward_matches_central_difference_including_the_frame_max"]),
    "fir_correlation_for_convolution": ("int64_t i = (int64_t)n + c - k;", "int64_t i = (int64_t)n - c + k;",
                                        ["test_fir_impulse_response_is_the_taps",
                                         "test_fir_equals_same_mode_convolution"]),
    "iq_mix_sign": ("im -= h[k] * x[i] * sin(ph);", "im += h[k] * x[i] * sin(ph);",
                    ["test_iq_demod_of_a_tone_at_f0"]),
    "iq_decimation_offset": ("int64_t i = (int64_t)m * decim + c - k;", "int64_t i = (int64_t)m * decim - k;",
                             ["test_iq_demod_at_zero_frequency_is_the_fir", "test_iq_demod_of_a_tone_at_f0"]),
    "window_width": ("double half_width = 0.5 * z / p->f_number;", "double half_width = z / p->f_number;",
                     ["test_window_is_apod_without_weight", "test_adjoint_identity"]),
    # delay-and-sum of IQ data
    "iq_remod_sign": ("double c = cos(ph), sn = sin(ph);", "double c = cos(ph), sn = -sin(ph);",
                      ["test_iq_das_single_element_phase_by_hand",
                       "test_iq_das_envelope_matches_rf_envelope"]),
    "iq_decimation_ignored": ("double u = s / (double)decim;", "double u = s;",
                              ["test_iq_das_single_element_phase_by_hand",
                               "test_iq_das_focuses_point_target"]),
    "iq_imag_dropped": ("double vi = (1.0 - f) * tr[2 * i + 1] + f * tr[2 * i + 3];", "double vi = 0.0;",
                        ["test_iq_das_single_element_phase_by_hand",
                         "test_iq_das_envelope_matches_rf_envelope"]),
    "iq_phase_at_baseband_index": ("double ph = 2.0 * M_PI * f0 * s / p->fs;",
                                   "double ph = 2.0 * M_PI * f0 * u / p->fs;",
                                   ["test_iq_das_single_element_phase_by_hand",
                                    "test_iq_das_envelope_matches_rf_envelope"]),
    "iq_rx_weight_dropped": ("in_re += wr * (vr * c - vi * sn);", "in_re += (vr * c - vi * sn);",
                             ["test_iq_das_reduces_to_rf_das"]),
}


def _call(name, golden):
    if hasattr(iq_pins, name):
        getattr(iq_pins, name)()       # every mode and decimation of the pin
        return
    if hasattr(fir_pins, name):
        fn = getattr(fir_pins, name)
        if "n_taps" in fn.__code__.co_varnames[: fn.__code__.co_argcount]:
            for n_taps in (1, 7, 31):
                fn(n_taps=n_taps)
            return
        fn()
        return
    if hasattr(grad_pins, name):
        fn = getattr(grad_pins, name)
        if "k" in fn.__code__.co_varnames[: fn.__code__.co_argcount]:
            failures = []
            for k in range(len(grad_pins.CASES)):   # every case; any failure counts
                try:
                    fn(k=k)
                except AssertionError as e:
                    failures.append(e)
            if failures:
                raise failures[0]
            return
        fn()
        return
    fn = getattr(pins, name)
    params = {"test_bin_centred_cosine_has_unit_envelope": {"n": 64, "k0": 5},
              "test_dft_matches_numpy_fft": {"n": 16}}.get(name, {})
    if "golden" in fn.__code__.co_varnames[: fn.__code__.co_argcount]:
        params["golden"] = golden
    fn(**params)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, golden, tmp_path):
    find, repl, tests = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(find) == 1, f"mutation anchor not unique: {find!r}"
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(find, repl))
    so = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                           str(mut), "-o", str(so), "-lm"])
    for t in tests:  # the pins pass on the real oracle ...
        _call(t, golden)
    caught = False
    with oracle.swap_library(str(so)):  # ... and at least one fails on the mutant
        for t in tests:
            try:
                _call(t, golden)
            except AssertionError:
                caught = True
    assert caught, f"no pin caught mutant {name}"
