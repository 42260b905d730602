"""Plants plausible mistakes in the oracle (on the CPU, one at a time, through
monkeypatch) and checks that its pins catch each one: a dropped term, a flipped sign, a
wrong weight or normalisation, an operand that is not the transpose, an index shifted
by one, a missing projection, a skipped coarse correction or preconditioner.  Each
planted mistake must make at least one of the pin tests named beside it fail with an
AssertionError."""
import os

import numpy as np
import pytest

import test_oracle_curv as TC
import test_oracle_flat as TF
import test_oracle_grad as TG
import test_oracle_pm as TP
from oracle import curv, flat, grad, pm

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _drop_z_term(orig):
    return lambda u, h=1.0: orig(u, h) - (np.roll(u, 1, 0) + np.roll(u, -1, 0) - 2 * u) / h ** 2


def _flip_diagonal(orig):
    return lambda u, h=1.0: orig(u, h) + 12.0 * u / h ** 2


def _scale(orig, s):
    return lambda *a, **k: orig(*a, **k) * s


def _shift_x(orig):
    return lambda *a, **k: np.roll(orig(*a, **k), 1, axis=-1)


def _add_const(orig, c):
    return lambda *a, **k: orig(*a, **k) + c


def _halve_mixed_hessian(orig):
    def f(psi, h=1.0):
        H = orig(psi, h).copy()
        for a, b in ((0, 1), (1, 0)):
            H[a, b] *= 0.5
        return H
    return f


def _wrong_power_of_J(orig):
    def f(psi, h=1.0):
        J, B = orig(psi, h)
        return J, B * J[None, None]
    return f


def _not_transpose(orig):
    return lambda y, B, h=1.0: orig(y, B, h) + 0.01 * curv.at(y, 0, 1)


def _grad_T_not_transpose(orig):
    return lambda w, h=1.0: orig(w, h) + 0.01 * w[0]


def _read_shifted(orig):
    return lambda field, pos: orig(np.roll(field, 1, axis=-1), pos)


def _vjp_psi_bar_sign(orig):
    def f(*a, **k):
        dbar, pbar = orig(*a, **k)
        return dbar, -pbar
    return f


def _predict_wrong_weight(orig):
    def f(history, order, growth=1.0):
        out = orig(history, order, growth)
        return out + 0.01 * (history[0] - history[1]) if order >= 1 and len(history) > 1 else out
    return f


def _pcg_no_preconditioner(orig):
    return lambda r, steps, precond, apply: orig(r, steps, lambda v: v, apply)


def _motion_source_sign(orig):
    def f(*a, **k):
        new, psidot = orig(*a, **k)
        return -new, -psidot
    return f


def _force_sign(orig):
    def f(*a, **k):
        phi, F = orig(*a, **k)
        return phi, -F
    return f


def _sym_not_symmetric(orig):
    return lambda u, B, h=1.0: orig(u, B, h) + 0.01 * curv.at(u, 0, 1)


MUTANTS = {
    "apply_A drops the z second difference": (
        flat, "apply_A", _drop_z_term, [lambda: TF.test_plane_wave_eigenvalue((8, 12, 16))]),
    "apply_A with the diagonal sign flipped": (
        flat, "apply_A", _flip_diagonal, [lambda: TF.test_plane_wave_eigenvalue((8, 12, 16))]),
    "eigenvalues off by 0.1%": (
        flat, "eigenvalues", lambda o: _scale(o, 1.001), [lambda: TF.test_fft_solve_residual_and_gauge((16, 8, 32))]),
    "fft_solve without the gauge": (
        flat, "fft_solve", lambda o: _add_const(o, 0.5), [lambda: TF.test_fft_solve_residual_and_gauge((16, 8, 32))]),
    "restriction not normalised": (
        flat, "restrict_fw", lambda o: _scale(o, 1.01),
        [TF.test_restriction_is_prolongation_transpose_over_8, TF.test_restriction_is_27_tap_tensor_weights]),
    "prolongation shifted by one fine cell": (
        flat, "prolong", _shift_x,
        [TF.test_prolongation_exact_on_linear_functions, TF.test_restriction_is_prolongation_transpose_over_8]),
    "Chebyshev on the wrong interval": (
        flat, "chebyshev_interval", lambda o: (lambda alpha=8.0: (2.0 / alpha, 2.2)),
        [lambda: TF.test_chebyshev_plane_wave_factor(3, GOLDEN)]),
    "Jacobi with the wrong weight": (
        flat, "smooth_jacobi",
        lambda o: (lambda e, r, h, sweeps=2, omega=2.0 / 3.0: o(e, r, h, sweeps, 1.1 * omega)),
        [lambda: TF.test_jacobi_plane_wave_factor(GOLDEN)]),
    "coarse solve without the mean projection": (
        flat, "coarse_solve", lambda o: _add_const(o, 1.0), [lambda: TF.test_coarse_solve_is_pseudo_inverse((4, 4, 4), 8.0)]),
    "mixed Hessian term halved": (
        curv, "hessian", _halve_mixed_hessian, [TC.test_triad_plane_wave_closed_form, TC.test_geometry_against_linalg]),
    "B = J^2 A^-2 instead of J A^-2": (
        curv, "geometry", _wrong_power_of_J, [TC.test_geometry_against_linalg]),
    "face coefficient from one cell": (
        curv, "face_coeff", lambda o: (lambda B, a, b: B[a, b].copy()),
        [TC.test_second_order_consistency_with_continuum]),
    "M^T not the transpose of M": (
        curv, "apply_MT", _not_transpose, [TC.test_transpose_dot_product]),
    "edge coefficient from two cells": (
        curv, "edge_coeff", lambda o: (lambda B, a, b: 0.5 * (B[a, b] + curv.at(B[a, b], a, 1))),
        [TC.test_sym_second_order_consistency_and_agreement_with_literal]),
    "fourth-order gradient off by 1%": (
        grad, "grad4", lambda o: _scale(o, 1.01), [TG.test_grad_symbols]),
    "gradient transpose not the transpose": (
        grad, "grad4_T", _grad_T_not_transpose, [TG.test_grad_transposes]),
    "CIC paint shifted by one cell": (
        pm, "cic_paint", _shift_x, [TP.test_paint_conserves_mass_and_hits_nodes, TP.test_read_is_transpose_of_paint]),
    "V-cycle without the coarse correction": (
        flat, "prolong", lambda o: (lambda ec: np.zeros(tuple(2 * n for n in ec.shape))),
        [TF.test_plain_method_32_converges_to_fft, lambda: TF.test_convergence_factor_mesh_independent(GOLDEN)]),
    "predictor with a wrong extrapolation weight": (
        flat, "predict", _predict_wrong_weight, [TF.test_predictors_exact_on_their_sequences]),
    "PCG without its preconditioner": (
        flat, "pcg", _pcg_no_preconditioner, [TF.test_pcg_exact_preconditioner_converges_in_one_step]),
    "psi_bar with its sign flipped": (
        curv, "solve_vjp", _vjp_psi_bar_sign, [TC.test_vjp_against_central_differences]),
    "binomial smoothing one pass short": (
        curv, "smooth_binomial", lambda o: (lambda u, passes: o(u, max(0, passes - 1))),
        [TC.test_binomial_smoothing_plane_wave_factor]),
    "mesh-motion source with the wrong sign": (
        curv, "mesh_motion_step", _motion_source_sign, [TC.test_mesh_motion_flat_mesh_is_spectral_solve]),
    "PM force with the wrong sign": (
        pm, "pm_force", _force_sign, [TP.test_force_pipeline_is_antisymmetric_for_a_pair]),
    "Jacobi diagonal doubled": (
        curv, "diag_M", lambda o: _scale(o, 2.0), [TC.test_psi_zero_solve_equals_flat_jacobi_cycle]),
    "symmetric variant not symmetric": (
        curv, "apply_M_sym", _sym_not_symmetric, [TC.test_sym_operator_is_symmetric_with_19_points]),
    "symmetric-variant B cotangent off by 1%": (
        curv, "Bbar_from_operator_sym", lambda o: _scale(o, 1.01), [TC.test_sym_Bbar_is_the_derivative_of_the_bilinear_form]),
    "second-order gradient off by 1%": (
        grad, "grad2", lambda o: _scale(o, 1.01), [TG.test_grad_symbols]),
    "CIC read from the wrong cell": (
        pm, "cic_read", _read_shifted, [TP.test_read_is_transpose_of_paint, TP.test_read_interpolates_linear_fields_exactly]),
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_the_planted_mistake(name, monkeypatch):
    module, attr, make, pins = MUTANTS[name]
    monkeypatch.setattr(module, attr, make(getattr(module, attr)))
    caught = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            caught += 1
    assert caught > 0, f"no pin caught: {name}"
