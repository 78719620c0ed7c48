"""The representative pins must fail on a wrong oracle (CPU only).

Each case plants one plausible mistake in a copy of the oracle's C source --
Eq. 13's weights taken as the signed s_i instead of |s_i|, or its
normalisation by sum |nu_j| dropped, in the paper's treecode or in the group
treecode's rep_mode 0; a sign or factor of the first-order far-field terms or
of their transpose; a sign or factor of the local expansions, of their
transpose, or their cut-off decision; the clusters' centre, sums or count --
compiles the copy, swaps it in for the
real oracle and checks that the pins of tests/test_oracle_paper_tree.py,
tests/test_oracle_dipole.py and tests/test_oracle_local.py then fail.  The copy
lives in pytest's temporary directory; the real oracle is untouched.
"""
import os

import pytest

import oracle
from oracle import OP_A, OP_AT, OP_G

import test_oracle_dipole as dpins     # the pin modules, on sys.path as test files
import test_oracle_local as lpins
import test_oracle_paper_tree as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "wnnc_oracle.c")

# (name, text in the source, replacement, pins that must fail)
MUTATIONS = [
    ("paper tree: signed weights",
     "            a = sqrt(a);\n            sw += a;\n            for (int q = 0; q < 3; ++q) { sx[q] += a * P->x",
     "            a = (dim == 1) ? nu[i] : sqrt(a);\n            sw += a;\n"
     "            for (int q = 0; q < 3; ++q) { sx[q] += a * P->x",
     [lambda: pins.test_paper_tree_worked_far_node(OP_AT),
      lambda: pins.test_representative_ignores_the_sign_of_nu("paper")]),
    ("paper tree: no normalisation",
     "rep[3 * b + q] = sw > 0.0 ? sx[q] / sw : sc[q] / (double)P->count[b];",
     "rep[3 * b + q] = sw > 0.0 ? sx[q] : sc[q] / (double)P->count[b];",
     [lambda: pins.test_paper_tree_worked_far_node(OP_A),
      lambda: pins.test_paper_tree_worked_far_node(OP_G),
      lambda: pins.test_paper_tree_worked_far_node(OP_AT)]),
    ("group tree rep_mode 0: signed weights",
     "            a = sqrt(a);\n            sw += a;\n            for (int k = 0; k < 3; ++k) sx[k] += a * t->x",
     "            a = (dim == 1) ? nu[i] : sqrt(a);\n            sw += a;\n"
     "            for (int k = 0; k < 3; ++k) sx[k] += a * t->x",
     [lambda: pins.test_group_tree_worked_far_node(OP_AT, 0),
      lambda: pins.test_representative_ignores_the_sign_of_nu("group")]),
    ("group tree rep_mode 0: no normalisation",
     "rep[3 * b + k] = (rep_mode == 0 && sw > 0.0) ? sx[k] / sw : t->cent[3 * b + k];",
     "rep[3 * b + k] = (rep_mode == 0 && sw > 0.0) ? sx[k] : t->cent[3 * b + k];",
     [lambda: pins.test_group_tree_worked_far_node(OP_A, 0),
      lambda: pins.test_group_tree_worked_far_node(OP_G, 0),
      lambda: pins.test_group_tree_worked_far_node(OP_AT, 0)]),
    ("first-order far field: sign of A's term",
     "out[0] = tr / (4.0 * OR_PI * r3) - 3.0 * dSd / (4.0 * OR_PI * r5);",
     "out[0] = -(tr / (4.0 * OR_PI * r3) - 3.0 * dSd / (4.0 * OR_PI * r5));",
     [lambda: dpins.test_far_error_order(OP_A)]),
    ("first-order far field: factor of G's S d term",
     "out[k] = (6.0 * Sd[k] + 3.0 * tr * d[k])",
     "out[k] = (3.0 * Sd[k] + 3.0 * tr * d[k])",
     [lambda: dpins.test_far_error_order(OP_G)]),
    ("first-order far field: sign of the transposed push-down",
     "for (int k = 0; k < 3; ++k) far[k] -= hd[k];",
     "for (int k = 0; k < 3; ++k) far[k] += hd[k];",
     [lambda: dpins.test_far_error_order_of_the_transpose()]),
    ("local expansion: sign of A's first-order term",
     "out[0] = ce[0] - (dl[0] * ce[1] + dl[1] * ce[2] + dl[2] * ce[3]);",
     "out[0] = ce[0] + (dl[0] * ce[1] + dl[1] * ce[2] + dl[2] * ce[3]);",
     [lambda: lpins.test_local_error_order(OP_A)]),
    ("local expansion: factor of J's trace term",
     "const double diag = a == c ? 3.0 * dm : 0.0;",
     "const double diag = a == c ? dm : 0.0;",
     [lambda: lpins.test_local_error_order(OP_G)]),
    ("local expansion: sign of the transposed HPhi term",
     "out[k] = -S * D[k] / (4.0 * OR_PI * r3) + (3.0 * D[k] * dd - r2 * Dg[k]) / (4.0 * OR_PI * r5);",
     "out[k] = -S * D[k] / (4.0 * OR_PI * r3) - (3.0 * D[k] * dd - r2 * Dg[k]) / (4.0 * OR_PI * r5);",
     [lambda: lpins.test_local_error_order_of_the_transpose()]),
    ("local expansion: the cut-off bound compared with w^2 unsquared",
     "return m > 0.0 && m2 >= w2;",
     "return m > 0.0 && m >= w2;",
     [lambda: lpins.test_groups_fall_back_to_pairs_at_wide_cutoffs()]),
    ("cluster expansion: taken about the group's centre",
     "if (loc && LC->K >= 2) L[2] = cluster_frame(T, g / LC->K, LC->K);",
     "if (loc && LC->K >= 2) L[2] = group_frame(T, g);",
     [lambda: lpins.test_cluster_error_order(OP_A), lambda: lpins.test_cluster_error_order(OP_G)]),
    ("cluster expansion: its transpose from the first member's sums only",
     "const double* sd = cl == 2 ? SDC + 6 * (g / K) : SD + 6 * g;",
     "const double* sd = SD + 6 * g;",
     [lambda: lpins.test_cluster_error_order_of_the_transpose()]),
    ("cluster expansion: its transpose counted once per member",
     "if (cl == 2 && g % K != 0) continue;",
     "if (cl == 2 && g % K != 0 && 0) continue;",
     [lambda: lpins.test_cluster_error_order_of_the_transpose()]),
    ("local expansion: the cut-off bound without the group radius",
     "const double m = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]) - rho;",
     "const double m = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);",
     [lambda: lpins.test_groups_fall_back_to_pairs_at_wide_cutoffs()]),
]


@pytest.mark.parametrize("case", range(len(MUTATIONS)), ids=[m[0] for m in MUTATIONS])
def test_pins_fail_on_a_mutated_representative(case, tmp_path, monkeypatch):
    name, old, new, must_fail = MUTATIONS[case]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site of '{name}' not found once in the oracle source"
    src = tmp_path / "mutant.c"
    src.write_text(text.replace(old, new))
    mutant = oracle.load(oracle.compile_source(str(src), str(tmp_path / "libmutant.so")))
    # the unmutated oracle passes these pins (they run in the pin file too)
    for pin in must_fail:
        pin()
    monkeypatch.setattr(oracle, "_lib", mutant)
    for pin in must_fail:
        with pytest.raises(AssertionError):
            pin()
