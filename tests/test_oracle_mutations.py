"""The oracle's pins catch plausible mistakes: each case plants one mistake in a copy of
the oracle's C source (compiled apart, on the CPU; the oracle itself is untouched) and
runs the pins that must then fail.

A wrong coefficient or Bessel order in Eq. wtilde, a sign in Eq. wtilde_pair or
Eq. pe_eff_int_2, a sign of p x B in Eq. chi_exact, a Philox multiplier, the shares of
Eq. return_to_nrg given to the wrong lepton, half the optical-depth decrement of Sec. 2,
the parent tag left out of a descendant's id, the photon of an emission given the
lepton's energy or a wrong recoil split in a cascade, the pair-rate domain edge of
Sec. 4.2, another uniform map, the wrong target in the upper tail of Eq. again, the sign
of the pusher's second electric half-kick, the constant of Eq. gammaLCFA, the sign of
the projection of Eq. fl_perp, the second difference of Eq. condit, s of Eq. subs_altri,
and a created particle stepped in the step that created it: every one fails at least one
pin, and every pin passes on an unplanted copy.
"""
import importlib.util
import os
import shutil

import numpy as np
import pytest

import test_oracle_blcfa as PB
import test_oracle_cascade as PC
import test_oracle_mc as PM
import test_oracle_pins as PP
import test_oracle_push as PU
import test_surrogate_oracle as PS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")

# (name, original text, planted text, pins that must fail)
CASES = [
    ("wtilde coefficient", "(45.0 * x * x + 42.0 * x + 20.0)", "(45.0 * x * x + 24.0 * x + 20.0)",
     [PP.test_wrad_small_chi_series]),
    ("wtilde Bessel order", "return f * orc_besselk(2.0 / 3.0, v) * 3.0 * t * t;",
     "return f * orc_besselk(1.0 / 3.0, v) * 3.0 * t * t;", [PP.test_wrad_at_zero]),
    ("wtilde_pair sign", "return (9.0 - v * v) / (3.0 * om) * orc_besselk(2.0 / 3.0, eta);",
     "return (9.0 + v * v) / (3.0 * om) * orc_besselk(2.0 / 3.0, eta);",
     [PP.test_wpair_small_chi_series, PP.test_wpair_vs_scipy]),
    ("pe CDF sign", "((1.0 + ops * ops) * k23 - ops * ki13)", "((1.0 + ops * ops) * k23 + ops * ki13)",
     [lambda O: PP.test_pe_cdf_normalisation(O, 1.0)]),
    ("chi sign of p x B", "{E[0] + b[1] * B[2] - b[2] * B[1],\n                         E[1] + b[2] * B[0] - b[0] * B[2],",
     "{E[0] + b[1] * B[2] - b[2] * B[1],\n                         E[1] + b[2] * B[0] + b[0] * B[2],",
     [PP.test_chi_special_cases, PP.test_chi_covariant_form]),
    ("Philox multiplier", "(uint64_t)0xD2511F53u * c0", "(uint64_t)0xD2511F55u * c0", [PP.test_philox_known_answers]),
    ("pair shares swapped", "if (rp >= 0.0) { *xi_e = big; *xi_p = small; }",
     "if (rp < 0.0) { *xi_e = big; *xi_p = small; }", [lambda O: PP.test_pair_sampler_vs_scipy_cdf(O, 1.0, 0.3)]),
    ("half the optical-depth decrement", "const double tn = s->tau - R * P->dt;\n    if (fabs(tn) <= P->near_od * s->tau0) note_near(info, n);\n    if (!(tn < 0.0)) { s->tau = tn; return; }\n    info->n_events++;\n    const double su",
     "const double tn = s->tau - 0.5 * R * P->dt;\n    if (fabs(tn) <= P->near_od * s->tau0) note_near(info, n);\n    if (!(tn < 0.0)) { s->tau = tn; return; }\n    info->n_events++;\n    const double su",
     [PM.test_soft_photon_counts_are_poisson]),
    ("child id without the parent tag", "0x100u | ((parent_tag & 3u) << 2) | member", "0x100u | member",
     [PC.test_child_ids_are_philox_words]),
    ("emitted photon with the lepton's energy", "collinear(nh, gph, pph);", "collinear(nh, gnew, pph);",
     [lambda O: PC.test_cascade_conserves_energy(PC.make_cascade(O, n=16, nsteps=40))]),
    ("recoil split", "const double gnew = gamma / (1.0 + su);", "const double gnew = gamma / (1.0 + 2.0 * su);",
     [lambda O: PC.test_cascade_conserves_energy(PC.make_cascade(O, n=16, nsteps=40))]),
    ("pair-rate domain edge", "if (chi < 0.01) return 0.0;", "if (chi < 0.001) return 0.0;",
     [PP.test_pair_rate_cutoff_and_prefactor]),
    ("uniform map", "((double)(w >> 9) + 0.5) * 0x1p-23", "((double)(w >> 8) + 0.5) * 0x1p-24",
     [PP.test_uniform_map]),
    ("photon sampler upper-tail target", "rctx c = {chi, (1.0 - r) * W};", "rctx c = {chi, r * W};",
     [lambda O: PP.test_photon_sampler_vs_scipy_cdf(O, 1.0, 0.97)]),
    ("Boris second half-kick sign", "for (int k = 0; k < 3; ++k) u[k] = up[k] + 0.5 * q * dt * E[k];",
     "for (int k = 0; k < 3; ++k) u[k] = up[k] - 0.5 * q * dt * E[k];", [PU.test_electric_kick]),
    ("BLCFA threshold constant", "return 0.7 * gamma /", "return 0.75 * gamma /",
     [PP.test_blcfa_threshold_triple_angle]),
    ("sign of the projection in Eq. fl_perp", "for (int k = 0; k < 3; ++k) F[k] = FL[k] - fp * pL[k];",
     "for (int k = 0; k < 3; ++k) F[k] = FL[k] + fp * pL[k];", [PP.test_blcfa_perpendicular_force_projection]),
    ("second difference in Eq. condit", "Fdd[k] = (d1[k] - dF[k]) / (dt * dt);", "Fdd[k] = (d1[k] + dF[k]) / (dt * dt);",
     [PM.test_blcfa_delta_of_a_plane_wave]),
    ("s of Eq. subs_altri", "return 1.5 * chi * w * w * w;", "return 1.0 * chi * w * w * w;",
     [lambda O: PP.test_photon_sampler_vs_scipy_cdf(O, 1.0, 0.3)]),
    ("Eq. pe_dp integral term dropped",
     "((1.0 + opu * opu) * orc_besselk(2.0 / 3.0, x) - opu * orc_besselk_int(1.0 / 3.0, x));",
     "((1.0 + opu * opu) * orc_besselk(2.0 / 3.0, x));",
     [lambda O: PB.test_spectrum_integrates_to_the_rate(O, 2000.0, 1.0), PB.test_spectrum_soft_photon_end]),
    ("Eq. pe_dp sign of the integral term", "orc_besselk(2.0 / 3.0, x) - opu * orc_besselk_int(1.0 / 3.0, x));",
     "orc_besselk(2.0 / 3.0, x) + opu * orc_besselk_int(1.0 / 3.0, x));",
     [lambda O: PB.test_spectrum_integrates_to_the_rate(O, 2000.0, 1.0), PB.test_spectrum_radiated_power_small_chi]),
    ("Eq. pe_dp without 1/(1 + u)", "return pref / (ge * ge) / opu *", "return pref / (ge * ge) *",
     [lambda O: PB.test_spectrum_integrates_to_the_rate(O, 2000.0, 1.0)]),
    ("Eq. rej_cond reversed", "if (!(u[2] * Sb <= SL)) { info->n_rejected++; return; }",
     "if (!(u[2] * Sb >= SL)) { info->n_rejected++; return; }",
     [lambda O: PB.test_rejection_law_of_accepted_photons(O, 0.1, n=1000)]),
    ("rejection applied above the threshold", "if (!(gbar > gL)) {", "if (!(gbar < gL)) {",
     [lambda O: PB.test_rejection_law_of_accepted_photons(O, 0.1, n=1000)]),
    ("no-emission rule reversed", "if (!(gL < 0.75 * g)) { info->n_no_emission++; return; }",
     "if (!(gL > 0.75 * g)) { info->n_no_emission++; return; }",
     [lambda O: PB.test_threshold_below_the_rule_still_emits(O, n=600)]),
    ("no-emission constant below 0.7", "if (!(gL < 0.75 * g)) { info->n_no_emission++; return; }",
     "if (!(gL < 0.6 * g)) { info->n_no_emission++; return; }",
     [lambda O: PB.test_threshold_below_the_rule_still_emits(O, n=600)]),
    ("gate with zeta for zeta^2", "delta / (ORC_ZETA * ORC_ZETA) > out->chi", "delta / ORC_ZETA > out->chi",
     [PB.test_gate_boundary_delta]),
    ("gate without chi > zeta", "(out->chi > ORC_ZETA);", "(out->chi > 0.0);", [PB.test_gate_boundary_chi]),
    ("created particle stepped in its own step", "for (int c = 0; c < nk; ++c) {\n                orc_state t",
     "for (int c = 0; c < kids.n; ++c) {\n                orc_state t",
     [lambda O: PC.test_created_particles_evolve_as_primaries_of_their_own(PC.make_cascade(O), O)]),
]


def _mutant(tmp, orig, planted):
    with open(os.path.join(ORACLE, "sfq_oracle.c")) as fh:
        src = fh.read()
    assert src.count(orig) == 1, orig
    d = str(tmp)
    shutil.copy(os.path.join(ORACLE, "oracle.py"), os.path.join(d, "oracle.py"))
    with open(os.path.join(d, "sfq_oracle.c"), "w") as fh:
        fh.write(src.replace(orig, planted))
    spec = importlib.util.spec_from_file_location("oracle_mutant_" + os.path.basename(d), os.path.join(d, "oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    assert mod._SRC == os.path.join(d, "sfq_oracle.c")        # builds and loads the planted copy
    return mod


# a planted mistake may leave scipy's reference quadrature in a pin without convergence
@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
@pytest.mark.parametrize("name,orig,planted,pins", CASES, ids=[c[0] for c in CASES])
def test_pins_catch_the_planted_mistake(tmp_path, name, orig, planted, pins):
    mut = _mutant(tmp_path, orig, planted)
    for pin in pins:
        with pytest.raises(AssertionError):
            pin(mut)


def test_unplanted_copy_passes_every_pin(tmp_path):
    """Control: every pin of every case passes on a copy compiled the same way without a
    planted mistake, so each case above fails for its mistake and nothing else."""
    mut = _mutant(tmp_path, "(45.0 * x * x + 42.0 * x + 20.0)", "(45.0 * x * x + 42.0 * x + 20.0)")
    for name, _, _, pins in CASES:
        for pin in pins:
            pin(mut)
    assert np.isfinite(mut.wtilde_rad([1.0])[0])


# The surrogate's oracle (oracle/surrogate.py, numpy): the same test on a planted copy.
SURROGATE_CASES = [
    ("SiLU derivative", "return s * (1.0 + z * (1.0 - s))", "return s * (1.0 + z * s)",
     [PS.test_gradient_matches_finite_differences]),
    ("bfloat16 ties", "b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000", "b = (b + 0x8000) & 0xFFFF0000",
     [PS.test_bf16_rounding_matches_torch]),
    ("backpropagation through a layer", "d = d @ Wq", "d = d @ Wq * 0.5", [PS.test_gradient_matches_finite_differences]),
]


def _surrogate_mutant(tmp, orig, planted):
    with open(os.path.join(ORACLE, "surrogate.py")) as fh:
        src = fh.read()
    assert src.count(orig) == 1, orig
    path = os.path.join(str(tmp), "surrogate_planted.py")
    with open(path, "w") as fh:
        fh.write(src.replace(orig, planted))
    spec = importlib.util.spec_from_file_location("oracle.surrogate_planted_" + os.path.basename(str(tmp)), path)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "oracle"                                 # its relative import finds the oracle
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name,orig,planted,pins", SURROGATE_CASES, ids=[c[0] for c in SURROGATE_CASES])
def test_surrogate_pins_catch_the_planted_mistake(tmp_path, name, orig, planted, pins):
    mut = _surrogate_mutant(tmp_path, orig, planted)
    for pin in pins:
        with pytest.raises(AssertionError):
            pin(mut)


def test_unplanted_surrogate_copy_passes_every_pin(tmp_path):
    mut = _surrogate_mutant(tmp_path, "d = d @ Wq", "d = d @ Wq")
    for name, _, _, pins in SURROGATE_CASES:
        for pin in pins:
            pin(mut)

