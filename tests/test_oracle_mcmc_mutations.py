"""Plant plausible mistakes in copies of the MCMC and network oracles and
check that their pins (tests/test_oracle_mcmc.py, tests/test_oracle_mlp.py)
reject each one.

Each mutant is one edit of the oracle's C source, compiled on the CPU and
swapped in for the oracle's library while the pins run: a wrong Philox
constant or round count, Box-Muller slips, transform and Jacobian mistakes,
prior parameter slips, and, in the network oracle, backpropagation and Adam
mistakes. The unmodified sources pass the same pins.
"""
import tempfile
from pathlib import Path

import pytest

import oracle

import tests.test_oracle_mcmc as mc
import tests.test_oracle_mlp as ml

HERE = Path(oracle.__file__).parent
MCMC_SRC = (HERE / "mcmc_oracle.c").read_text()
MLP_SRC = (HERE / "mlp_oracle.c").read_text()

MCMC_PINS = (
    mc.test_philox_known_answers,
    mc.test_uniform_and_normal_moments,
    lambda: [mc.test_transform_constraints_and_roundtrip(K) for K in (2, 3, 5)],
    lambda: [mc.test_log_density_equals_scipy_plus_jacobian(K) for K in (2, 3)],
    mc.test_mean_outside_box_has_zero_prior,
    mc.test_box_edges,
)

MLP_PINS = (
    ml.test_forward_matches_numpy,
    ml.test_gradient_matches_finite_differences,
    ml.test_loss_is_negative_log_density_without_constants,
    ml.test_adam_first_step_moves_lr_against_the_gradient_sign,
    ml.test_adam_constant_gradient_moves_lr_per_step,
    ml.test_adam_is_invariant_to_gradient_scale,
    ml.test_adam_reaches_the_minimiser_of_a_separable_quadratic,
)

MCMC_MUTANTS = {
    "philox_multiplier": ("#define PHILOX_M0 0xD2511F53u", "#define PHILOX_M0 0xD2511F55u"),
    "philox_nine_rounds": ("for (int r = 0; r < 10; ++r) {", "for (int r = 0; r < 9; ++r) {"),
    "philox_key_schedule": ("k[0] += PHILOX_W0; k[1] += PHILOX_W1;", "k[0] += PHILOX_W1; k[1] += PHILOX_W0;"),
    "philox_word_order": ("c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;",
                          "c[0] = n0; c[1] = lo0; c[2] = n2; c[3] = lo1;"),
    "box_muller_radius": ("double rad = sqrt(-2.0 * log(a));", "double rad = sqrt(-log(a));"),
    "box_muller_same_branch": ("return (index & 1) ? rad * sin(ang) : rad * cos(ang);",
                               "return rad * cos(ang);"),
    "uniform_word": ("return u01(o[0]);\n}\n\nint oracle_theta_dim", "return u01(o[0] & 0xFFFFu);\n}\n\nint oracle_theta_dim"),
    "dirichlet_without_jacobian": ("lp += pr->alpha_P * (z - lse);", "lp += (pr->alpha_P - 1.0) * (z - lse);"),
    "pi_reference_state": ("double z = k == 0 ? 0.0 : th[o + k - 1];", "double z = k == 0 ? th[o] : th[o + k - 1];"),
    "gamma_rate_inverted": ("b = m / pr->p_var;", "b = pr->p_var / m;"),
    "gamma_mean_halves_swapped": ("double m = (k < K / 2) ? pr->p_mean_lo : pr->p_mean_hi;",
                                  "double m = (k < K / 2) ? pr->p_mean_hi : pr->p_mean_lo;"),
    "logistic_jacobian_dropped": ("lp += a * lpk - b * p[k] + l1p;", "lp += a * lpk - b * p[k];"),
    "iw_exponent": ("-0.5 * (pr->iw_df + 3.0) * log(det)", "-0.5 * (pr->iw_df + 1.0) * log(det)"),
    "cov_jacobian_power": ("3.0 * u + 3.0 * v;", "2.0 * u + 2.0 * v;"),
    "correlation_scale": ("sxy = rho * sx * sy;", "sxy = rho * sx * sx;"),
    "box_bound_swapped": ("x > pr->box[1]", "x > pr->box[3]"),
}

MLP_MUTANTS = {
    "relu_derivative_dropped": ("dh2[i] = h2[i] > 0.0 ? s : 0.0;", "dh2[i] = s;"),
    "batch_mean_dropped": ("dout[i] = -r * inv / B;", "dout[i] = -r * inv;"),
    "sigma_gradient": ("(1.0 - r * r * inv) / B", "(1.0 - r * r) / B"),
    "log_sigma_term_dropped": ("loss += 0.5 * r * r * inv + s;", "loss += 0.5 * r * r * inv;"),
    "W3_backprop_transposed": ("s += dout[o] * W3[(size_t)o * H + i];", "s += dout[o] * W3[(size_t)i * 2 * d + o];"),
    "first_bias_dropped": ("double s = b1[j];", "double s = 0.0;"),
    "standardisation_inverted": ("x[i] = (theta[(size_t)b * d + i] - mean[i]) / in_scale[i];",
                                 "x[i] = (theta[(size_t)b * d + i] - mean[i]) * in_scale[i];"),
    "adam_bias_correction_dropped": ("double mh = m[i] / (1.0 - pow(b1, t));", "double mh = m[i];"),
    "adam_second_moment": ("v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];",
                           "v[i] = b2 * v[i] + (1.0 - b2) * fabs(g[i]);"),
    "adam_second_bias_correction_dropped": ("double vh = v[i] / (1.0 - pow(b2, t));", "double vh = v[i];"),
    "adam_sign": ("p[i] -= lr * mh / (sqrt(vh) + eps);", "p[i] += lr * mh / (sqrt(vh) + eps);"),
    "adam_eps_inside_sqrt": ("p[i] -= lr * mh / (sqrt(vh) + eps);", "p[i] -= lr * mh / sqrt(vh + eps);"),
    "adam_betas_swapped": ("m[i] = b1 * m[i] + (1.0 - b1) * g[i];", "m[i] = b2 * m[i] + (1.0 - b2) * g[i];"),
    "adam_first_moment_lagged": ("double mh = m[i] / (1.0 - pow(b1, t));",
                                 "double mh = m[i] / (1.0 - pow(b1, t + 1));"),
}


def _caught(pins) -> bool:
    for pin in pins:
        try:
            pin()
        except AssertionError:
            return True
    return False


def _swap_in(monkeypatch, source):
    L = oracle.compile_variant(source, tempfile.mkdtemp())
    monkeypatch.setattr(oracle, "lib", lambda: L)


def test_unmodified_sources_pass(monkeypatch):
    _swap_in(monkeypatch, MCMC_SRC + "\n" + MLP_SRC)
    assert not _caught(MCMC_PINS)
    assert not _caught(MLP_PINS)


@pytest.mark.parametrize("name", sorted(MCMC_MUTANTS))
def test_mcmc_mutant_is_caught(name, monkeypatch):
    a, b = MCMC_MUTANTS[name]
    assert MCMC_SRC.count(a) == 1, name
    _swap_in(monkeypatch, MCMC_SRC.replace(a, b) + "\n" + MLP_SRC)
    assert _caught(MCMC_PINS), f"pins did not catch mutant {name}"


@pytest.mark.parametrize("name", sorted(MLP_MUTANTS))
def test_mlp_mutant_is_caught(name, monkeypatch):
    a, b = MLP_MUTANTS[name]
    assert MLP_SRC.count(a) == 1, name
    _swap_in(monkeypatch, MCMC_SRC + "\n" + MLP_SRC.replace(a, b))
    assert _caught(MLP_PINS), f"pins did not catch mutant {name}"
