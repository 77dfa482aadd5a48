"""Planted mistakes in the oracle.

Each case compiles a copy of the oracle (rv_oracle.c) with one plausible
mistake: a transposed operand, a wrong sign, a reversed tie order, a dropped
term, the wrong threshold, swapped axes, or a wrong radius. It then runs the
pins that guard that part and checks that at least one of them fails. This is
evidence that the pins would catch such a mistake in the oracle itself.

The copies are built in a temporary directory with the oracle's own compiler
flags. The oracle's source and its regular build are not touched.
"""
import inspect
import os
import subprocess

import pytest

import oracle
from oracle import build as oracle_build
from tests import test_oracle_alg1_pins as alg1_pins
from tests import test_oracle_pins as pins
from tests import test_oracle_pose_pins as pose_pins
from tests import test_oracle_stereo_pins as stereo_pins

CASES = [
    ("App. A product M = L(a)^T L'(b) with L(a) not transposed",
     "acc += La[k * 4 + r] * Lb[k * 4 + c];", "acc += La[r * 4 + k] * Lb[k * 4 + c];",
     [pins.test_M_eigenvalues_are_pm1, pins.test_quad_equals_residual_over_4,
      pins.test_S_is_projector_and_vanishes_at_true_q]),
    ("threshold sin^2(delta - r) instead of sin^2(delta + r)",
     "const double s = sin_d * cr + cos_d * sr; /* sin(delta + r) */",
     "const double s = sin_d * cr - cos_d * sr; /* sin(delta + r) */",
     [pins.test_tau_closed_form]),
    ("ties ranked to the larger index",
     "    if (a->idx < b->idx) return -1;\n    if (a->idx > b->idx) return 1;",
     "    if (a->idx > b->idx) return -1;\n    if (a->idx < b->idx) return 1;",
     [pins.test_rank_fixtures]),
    ("the last entry of the fit's 4x4 sum dropped",
     "for (int k = 0; k < 16; ++k) A[k] += S[16 * i + k];", "for (int k = 0; k < 15; ++k) A[k] += S[16 * i + k];",
     [pins.test_fit_equals_svd_closed_form, pins.test_noise_free_fit_recovers_truth]),
    ("refit membership by the winning cell's threshold instead of sin^2(delta)",
     "const double thr = sd * sd; /* sin^2(delta) */", "const double thr = win_tau;",
     [pins.test_refit_each_step_follows_the_rule, pins.test_refit_converges_to_a_fixed_point]),
    ("Alg. 1 cell index with the x and z axes swapped",
     "    return (i[2] * n + i[1]) * n + i[0];\n}\n\n/* The whole of Alg. 1",
     "    return (i[0] * n + i[1]) * n + i[2];\n}\n\n/* The whole of Alg. 1",
     [alg1_pins.test_projection_of_the_lower_half_lands_in_the_unit_ball_and_inverts,
      alg1_pins.test_counts_sum_to_samples_and_noise_free_argmax_finds_the_rotation]),
    ("Alg. 1 basis q_b2 = [0, b] q_b1 with one cross-product term of the wrong sign",
     "    q2[1] = w * b0 + (b1 * vz - b2 * vy);", "    q2[1] = w * b0 - (b1 * vz - b2 * vy);",
     [alg1_pins.test_every_sample_lies_on_the_pairs_quaternion_circle,
      alg1_pins.test_basis_is_orthonormal_and_q_b1_is_the_minimal_rotation]),
    ("peak suppression by cos(theta) instead of cos(theta / 2)",
     "    const double cth = cos(theta / 2.0);", "    const double cth = cos(theta);",
     [alg1_pins.test_peaks_obey_the_greedy_suppression_invariants]),
    ("rigid-pose length check without the absolute value",
     "fabs(lm - ln) <= mu", "(lm - ln) <= mu",
     [pose_pins.test_kept_pairs_equal_a_direct_evaluation]),
    ("stereographic inverse projection with w of the wrong sign",
     "    q[3] = (c2 - 1.0) / den;\n    *chord = sqrt(3.0) * h / sqrt((1.0 + minv2) * den);",
     "    q[3] = (1.0 - c2) / den;\n    *chord = sqrt(3.0) * h / sqrt((1.0 + minv2) * den);",
     [stereo_pins.test_stereo_centre_is_the_inverse_projection]),
    ("stereographic cell radius from the centre's conformal factor instead of the box's largest",
     "    *chord = sqrt(3.0) * h / sqrt((1.0 + minv2) * den);", "    *chord = sqrt(3.0) * h / sqrt((1.0 + c2) * den);",
     [stereo_pins.test_stereo_radius_covers_the_box_and_is_not_loose]),
]


def _build_mutant(tmp_path, old, new):
    src = open(oracle_build.SRC).read()
    assert src.count(old) == 1, "the planted text must name one place"
    path_c = os.path.join(tmp_path, "rv_oracle_planted.c")
    with open(path_c, "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(tmp_path, "librvoracle_planted.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", lib,
                    path_c, "-lm", "-lpthread"], check=True)
    return lib


def _fails(pin):
    args = [oracle] if inspect.signature(pin).parameters else []
    try:
        pin(*args)
    except Exception:  # an assertion, or arithmetic that breaks the pin's own checks
        return True
    return False


@pytest.mark.parametrize("what,old,new,guards", CASES, ids=[c[0] for c in CASES])
def test_a_pin_catches_the_planted_mistake(tmp_path, what, old, new, guards):
    lib = _build_mutant(str(tmp_path), old, new)
    with oracle.using_library(lib):
        caught = [g.__name__ for g in guards if _fails(g)]
    assert caught, f"no pin caught: {what}"
    # the regular oracle passes the same pins
    for g in guards:
        assert not _fails(g), g.__name__
