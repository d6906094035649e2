"""The oracle's pins catch plausible mistakes: each case plants one mistake in a copy
of the C oracle (compiled to a temporary directory, on the CPU) and checks that at
least one pin fails against it.  CPU only."""
import contextlib
import subprocess

import pytest

from oracle import oracle as O
import tests.test_oracle_grad as TG
import tests.test_oracle_preprocess as TP
import tests.test_oracle_render as TR

SRC = O._SRC.read_text()

MUTATIONS = [
    # (original, mistake, pins expected to catch it)
    ("GTm[i] *= 2.0", "GTm[i] *= 1.0",
     [lambda: TG.test_backward_matches_central_fd(*TG.FD_CASES[0])]),
    ("(S[4 * (k + 1) + ch] + T * bg[ch]) / (1.0 - a)", "(S[4 * (k + 1) + ch]) / (1.0 - a)",
     [lambda: TG.test_backward_matches_central_fd(*TG.FD_CASES[1])]),
    ("dY[12][0] = -6 * d3 * x * z;", "dY[12][0] = 6 * d3 * x * z;",
     [lambda: TP.test_sh_basis_gradient_fd()]),
    ("term[1] = dLdp * (-(r[4] * dy + r[3] * dx));", "term[1] = dLdp * (-(r[4] * dy - r[3] * dx));",
     [lambda: TG.test_backward_matches_central_fd(*TG.FD_CASES[2])]),
    ("o->a = cov[0] + 0.3;", "o->a = cov[0] + 0.03;",
     [TP.test_isotropic_on_axis_closed_form]),
    ("o->J[2] = -fx * xc / (tz * tz);", "o->J[2] = fx * xc / (tz * tz);",
     [lambda: TP.test_ewa_covariance_matches_numeric_jacobian(0)]),
    ("R[1] = 2 * (x * y - w * z);", "R[1] = 2 * (x * y + w * z);",
     [TP.test_rotation_about_z_swaps_axes,
      lambda: TP.test_ewa_covariance_matches_numeric_jacobian(1)]),
    ("Y[11] = -d2 * y * (4 * zz - xx - yy);", "Y[11] = d2 * y * (4 * zz - xx - yy);",
     [lambda: TP.test_sh_basis_matches_scipy(0)]),
    ("*D += r[9] * alpha * T;", "*D += r[9] * alpha;",
     [TR.test_stack_transmittance_and_early_stop]),
    ("if (testT < 1e-4) {", "if (testT < 1e-3) {",
     [TR.test_stack_transmittance_and_early_stop]),
    ("if (a->slot != b->slot) return a->slot < b->slot ? -1 : 1;",
     "if (a->slot != b->slot) return a->slot > b->slot ? -1 : 1;",
     [lambda: TR.test_bin_lists_brute_force(0)]),
    ("rect[1] = clampi(floordiv(fu + r + B - 1, B), 0, Tx);",
     "rect[1] = clampi(floordiv(fu + r, B), 0, Tx);",
     [lambda: TR.test_bin_lists_brute_force(1)]),
    ("double gx = slot_grads[NREC * s] * 0.5 * W", "double gx = slot_grads[NREC * s] * W",
     [TG.test_densify_stats_hand_example]),
    ("if (acc < 0.0) { acc = 0.0;", "if (0) { acc = 0.0;",
     [TP.test_sh_degree0_colour_is_view_independent_and_clamped]),
    ("rect[2] = clampi(floordiv(fv - r, B), 0, Ty);", "rect[2] = clampi(floordiv(fv - r + 1, B), 0, Ty);",
     [lambda: TR.test_bin_lists_brute_force(2), lambda: TR.test_tiled_render_matches_brute_force(3)]),
    ("if (a->z != b->z) return a->z < b->z ? -1 : 1;", "if (a->z != b->z) return a->z > b->z ? -1 : 1;",
     [lambda: TR.test_tiled_render_matches_brute_force(3)]),
]


@contextlib.contextmanager
def mutated_oracle(tmp_path, original, mistake):
    assert SRC.count(original) == 1, original
    src = tmp_path / "m.c"
    so = tmp_path / "m.so"
    src.write_text(SRC.replace(original, mistake))
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                    "-o", str(so), str(src), "-lm"], check=True)
    saved = (O._lib, O._SO, O._SRC)
    O._lib, O._SO, O._SRC = None, so, src
    try:
        yield
    finally:
        O._lib, O._SO, O._SRC = saved


@pytest.mark.parametrize("case", range(len(MUTATIONS)))
def test_planted_mistake_is_caught(tmp_path, case):
    original, mistake, pins = MUTATIONS[case]
    with mutated_oracle(tmp_path, original, mistake):
        caught = False
        for pin in pins:
            try:
                pin()
            except AssertionError:
                caught = True
        assert caught, f"no pin caught: {mistake}"
    # and the unmutated oracle passes the same pins
    for pin in pins:
        pin()
